"""Helper of the GPU tests: build a solver with the coarsest-level CG pinned
to one of its forms through the tuner's decision file (FVEM_TUNE_FILE)."""
import os

# fields of the tune file's last line
SEQ64, PERSIST64, PERSIST32, COOP32 = 0, 12, 13, 8


def pinned_solver(fv, sc, tune_file, mode64=None, mode32=None, **kw):
    """mode64: "seq" (kernel sequence), "coop" (cooperative launch) or
    "persist" (persistent launch, matrix in shared memory); mode32: "persist"
    or "other" (the tuner's choice among the others).  Builds once to let the
    tuner write the file, then rebuilds with the edited decisions."""
    os.environ["FVEM_TUNE_FILE"] = tune_file
    try:
        if not os.path.exists(tune_file):
            fv.Solver(levels=5, **kw).build(sc.N, sc.tris)
        lines = [x for x in open(tune_file).read().split("\n") if x.strip()]
        last = lines[-1].split()
        if mode64 is not None:
            last[SEQ64] = "0" if mode64 == "coop" else "1"
            last[PERSIST64] = "1" if mode64 == "persist" else "0"
        if mode32 is not None:
            last[PERSIST32] = "1" if mode32 == "persist" else "0"
        lines[-1] = " ".join(last)
        open(tune_file, "w").write("\n".join(lines) + "\n")
        S = fv.Solver(levels=5, **kw)
        S.build(sc.N, sc.tris)
    finally:
        del os.environ["FVEM_TUNE_FILE"]
    return S
