"""Host-side sharding of a scene batch over ranks (one process per GPU).

Independent scenes need no exchange: every rank builds and projects its own
share and only the timing is reduced (max over ranks).  Shares are balanced
by the work estimate N^3 (background cells), longest first onto the least
loaded rank (ties by rank), so the batch time is set by the heaviest share.
"""


def shard_scenes(sizes, world):
    """sizes: background resolution N of every scene.  Returns, per rank, the
    sorted list of scene indices it owns; every scene is owned exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    share = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]) ** 3, i)):
        r = min(range(world), key=lambda r: (load[r], r))
        share[r].append(i)
        load[r] += int(sizes[i]) ** 3
    return [sorted(s) for s in share]
