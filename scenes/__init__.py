"""Seeded synthetic inputs for the cut-cell VEM pressure projection.

This module only *generates inputs*: obstacle triangle meshes, the background
resolution, and the intermediate velocity field u'.  It holds none of the
method's arithmetic (no cutting, no VEM, no multigrid), so both the CPU oracle
and the CUDA library may be fed from it.

Random numbers come from one hand-written SplitMix64 generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014); normal
draws use the Box-Muller transform on (0,1]-mapped 53-bit uniforms.

The scenes stand in for the paper's workloads (Sec. 6: 128^3 background grids,
narrow gaps, thin sheets, 5 levels); the paper's own meshes are not used.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele et al. 2014): 64-bit state, golden-gamma increment."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform on [0,1): top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_open0(self) -> float:
        """Uniform on (0,1]."""
        return ((self.next_u64() >> 11) + 1) * (1.0 / 9007199254740992.0)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)

    def normal(self) -> float:
        """Box-Muller; one of the pair is used per call (simple and reproducible)."""
        u1 = self.uniform_open0()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------
# obstacle meshes (closed, outward oriented triangle soups)
# --------------------------------------------------------------------------

def icosphere(center, radius, subdiv):
    """Icosahedron subdivided `subdiv` times, vertices pushed to the sphere."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}
        nf = []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts) * radius + np.asarray(center, dtype=np.float64)
    F = np.array(faces, dtype=np.int64)
    return _orient_outward(V[F])     # (T,3,3)


def icosphere_level(radius, n):
    """Smallest subdivision whose edge (about 1.0515 r / 2^s) is <= h = 1/n."""
    h = 1.0 / n
    s = 0
    while 1.0515 * radius / (2 ** s) > h:
        s += 1
    return s


def rot_z(deg):
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_x(deg):
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def rot_axis(axis, ang):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    x, y, z = axis
    c, s = math.cos(ang), math.sin(ang)
    C = 1.0 - c
    return np.array([[c + x * x * C, x * y * C - z * s, x * z * C + y * s],
                     [y * x * C + z * s, c + y * y * C, y * z * C - x * s],
                     [z * x * C - y * s, z * y * C + x * s, c + z * z * C]])


def _orient_outward(tris):
    """Flip triangles of a convex piece so that normals point away from its
    vertex centroid."""
    tris = np.array(tris, dtype=np.float64)
    c = tris.reshape(-1, 3).mean(axis=0)
    n = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    flip = np.einsum("ij,ij->i", n, tris.mean(axis=1) - c) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris


_BOX_QUADS = [(0, 2, 3, 1), (4, 5, 7, 6),      # -x, +x
              (0, 1, 5, 4), (2, 6, 7, 3),      # -y, +y
              (0, 4, 6, 2), (1, 3, 7, 5)]      # -z, +z


def box(center, size, R):
    """Closed box: local corners (+-size/2) rotated by R about `center`."""
    center = np.asarray(center, dtype=np.float64)
    half = np.asarray(size, dtype=np.float64) / 2.0
    corners = []
    for i in range(8):
        sx = half[0] if (i & 4) else -half[0]
        sy = half[1] if (i & 2) else -half[1]
        sz = half[2] if (i & 1) else -half[2]
        corners.append(center + R @ np.array([sx, sy, sz]))
    C = np.array(corners)
    tris = []
    for (a, b, c, d) in _BOX_QUADS:
        tris.append([C[a], C[b], C[c]])
        tris.append([C[a], C[c], C[d]])
    return _orient_outward(np.array(tris))


def convex_prism(points_2d, z0, z1, frame_origin, ex, ey, ez):
    """Closed convex prism over a CCW polygon in a local (ex,ey) frame,
    extruded from ez*z0 to ez*z1."""
    o = np.asarray(frame_origin, dtype=np.float64)
    bot = [o + p[0] * ex + p[1] * ey + z0 * ez for p in points_2d]
    top = [o + p[0] * ex + p[1] * ey + z1 * ez for p in points_2d]
    n = len(points_2d)
    tris = []
    for i in range(1, n - 1):
        tris.append([bot[0], bot[i + 1], bot[i]])
        tris.append([top[0], top[i], top[i + 1]])
    for i in range(n):
        j = (i + 1) % n
        tris.append([bot[i], bot[j], top[j]])
        tris.append([bot[i], top[j], top[i]])
    return _orient_outward(np.array(tris))


def holed_sheet(thickness=1e-5, tilt_deg=30.0, hole=0.2, extent=1.2):
    """Plane y=0.5 rotated by `tilt_deg` about x through the domain centre,
    `thickness` thick, with a hole x hole square hole at the centre.  Built as
    four convex slabs around the hole (a closed thin shell as a union of convex
    pieces; the slabs extend past the unit box)."""
    R = rot_x(tilt_deg)
    ex, ey = R @ np.array([1.0, 0, 0]), R @ np.array([0, 0, 1.0])
    ez = np.cross(ex, ey)
    c = np.array([0.5, 0.5, 0.5])
    a, e = hole / 2.0, extent
    strips = [
        [(-e, -e), (e, -e), (e, -a), (-e, -a)],     # below the hole
        [(-e, a), (e, a), (e, e), (-e, e)],         # above the hole
        [(-e, -a), (-a, -a), (-a, a), (-e, a)],     # left of the hole
        [(a, -a), (e, -a), (e, a), (a, a)],         # right of the hole
    ]
    parts = [convex_prism(s, -thickness / 2, thickness / 2, c, ex, ey, ez) for s in strips]
    return parts


# --------------------------------------------------------------------------
# velocity: sum of random Fourier modes
# --------------------------------------------------------------------------

@dataclass
class Fourier:
    k: np.ndarray      # (M,3) integer wavevectors in {1..4}^3
    a: np.ndarray      # (M,3) amplitudes ~ N(0,1)
    theta: np.ndarray  # (M,)  phases ~ U[0, 2pi)

    def __call__(self, x):
        """u(x) = sum_m a_m cos(2 pi k_m . x + theta_m), x: (n,3) -> (n,3)."""
        x = np.asarray(x, dtype=np.float64)
        ph = 2.0 * math.pi * (x @ self.k.T.astype(np.float64)) + self.theta[None, :]
        return np.cos(ph) @ self.a


def fourier_modes(rng: SplitMix64, M: int) -> Fourier:
    k = np.zeros((M, 3), dtype=np.int64)
    a = np.zeros((M, 3))
    th = np.zeros(M)
    for m in range(M):
        for c in range(3):
            k[m, c] = rng.randint(1, 4)
        for c in range(3):
            a[m, c] = rng.normal()
        th[m] = 2.0 * math.pi * rng.uniform()
    return Fourier(k, a, th)


# --------------------------------------------------------------------------
# scene presets
# --------------------------------------------------------------------------

@dataclass
class Scene:
    name: str
    N: int                       # background resolution (h = 1/N)
    tris: np.ndarray             # (T,3,3) float64, closed outward-oriented obstacle triangles
    comp: np.ndarray             # (T,) int32 obstacle component id (union = inside any one)
    velocity: Fourier
    order_k: int = 1
    tol: float = 1e-6
    u_inflow: float = 0.0        # uniform inflow speed on the x=0 face (0 = wall)
    levels: int = 5
    extra: dict = field(default_factory=dict)


def _pack(parts):
    tris = np.concatenate(parts, axis=0)
    comp = np.concatenate([np.full(len(p), i, dtype=np.int32) for i, p in enumerate(parts)])
    return tris, comp


def sphere_scene(N, seed, modes, name, tol, radius=0.23, center=(0.47, 0.52, 0.49), **kw):
    rng = SplitMix64(seed)
    vel = fourier_modes(rng, modes)
    s = icosphere_level(radius, N)
    tris, comp = _pack([icosphere(center, radius, s)])
    return Scene(name, N, tris, comp, vel, tol=tol, **kw)


def two_boxes_scene(N=128, seed=1001, modes=32, gap_cells=0.3):
    rng = SplitMix64(seed)
    vel = fourier_modes(rng, modes)
    R = rot_z(17.0)
    xh = R @ np.array([1.0, 0.0, 0.0])
    g = gap_cells / N
    c = np.array([0.5, 0.5, 0.5])
    off = (0.15 + g / 2.0) * xh
    size = (0.3, 0.5, 0.3)
    tris, comp = _pack([box(c - off, size, R), box(c + off, size, R)])
    return Scene("two_boxes_gap", N, tris, comp, vel, tol=1e-6, extra={"gap": g})


def random_scene(s_index, seed=None):
    seed = 2000 + s_index if seed is None else seed
    rng = SplitMix64(seed)
    N = [32, 48, 64, 80, 96][rng.randint(0, 4)]
    nobs = rng.randint(1, 4)
    parts = []
    for _ in range(nobs):
        is_sphere = rng.uniform() < 0.5
        if is_sphere:
            r = 0.08 + (0.25 - 0.08) * rng.uniform()
            cen = [rng.uniform(), rng.uniform(), rng.uniform()]
            parts.append(icosphere(cen, r, icosphere_level(r, N)))
        else:
            size = [0.08 + (0.25 - 0.08) * rng.uniform() for _ in range(3)]
            cen = [rng.uniform(), rng.uniform(), rng.uniform()]
            axis = [rng.normal(), rng.normal(), rng.normal()]
            ang = 2.0 * math.pi * rng.uniform()
            parts.append(box(cen, size, rot_axis(axis, ang)))
    vel = fourier_modes(rng, 32)
    tris, comp = _pack(parts)
    return Scene(f"random_{s_index}", N, tris, comp, vel, tol=1e-6)


def sheet_scene(N=128, seed=1004, modes=32):
    rng = SplitMix64(seed)
    vel = fourier_modes(rng, modes)
    tris, comp = _pack(holed_sheet())
    return Scene("holed_sheet", N, tris, comp, vel, order_k=2, tol=1e-6)


def config(i: int, N: int | None = None) -> Scene:
    """The five workloads: 0 sphere 16^3 (tol 1e-10), 1 two boxes with a
    0.3-cell gap at 128^3, 2 sphere 64^3 with inflow, 3 first random scene of
    the batch, 4 holed 1e-5 sheet at 128^3 (second order)."""
    if i == 0:
        return sphere_scene(N or 16, 1000, 8, "sphere16", 1e-10)
    if i == 1:
        return two_boxes_scene(N or 128)
    if i == 2:
        return sphere_scene(N or 64, 1002, 32, "sphere_inflow", 1e-6, u_inflow=1.0)
    if i == 3:
        return random_scene(0)
    if i == 4:
        return sheet_scene(N or 128)
    raise ValueError(i)


def batch_scenes(n=32):
    return [random_scene(s) for s in range(n)]


def mesh_volume(tris):
    """Signed volume enclosed by a closed triangle soup (divergence theorem)."""
    a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
    return float(np.sum(np.einsum("ij,ij->i", a, np.cross(b, c))) / 6.0)


def empty_scene(N, seed=7, modes=4):
    """No obstacle: the whole unit box is fluid."""
    rng = SplitMix64(seed)
    vel = fourier_modes(rng, modes)
    return Scene(f"empty{N}", N, np.zeros((0, 3, 3)), np.zeros(0, dtype=np.int32), vel, tol=1e-10)


# --------------------------------------------------------------------------
# particles
# --------------------------------------------------------------------------

def splitmix64_uniforms(seed: int, start: int, n: int) -> np.ndarray:
    """Uniforms number start .. start+n-1 of SplitMix64(seed).uniform(),
    computed in closed form (the generator's state after k steps is
    seed + k * gamma mod 2^64), vectorised with wrapping uint64 arithmetic."""
    k = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def particles(N: int, per_axis: int = 2, seed: int = 4242) -> np.ndarray:
    """Stratified jittered particles: every background cube of the N^3 grid
    split into per_axis^3 sub-cubes, one uniform point in each (the usual
    8-per-cell FLIP seeding at per_axis = 2).  Returns (3, n) SoA positions,
    n = (N * per_axis)^3, ordered by sub-cube (x fastest); points inside
    obstacles are kept (the solver marks them with cell -1)."""
    M = N * per_axis
    n = M ** 3
    out = np.empty((3, n))
    chunk = M * M
    for z0 in range(M):
        u = splitmix64_uniforms(seed, 3 * z0 * chunk, 3 * chunk).reshape(chunk, 3)
        j = np.arange(chunk)
        ix, iy = j % M, j // M
        s = slice(z0 * chunk, (z0 + 1) * chunk)
        out[0, s] = (ix + u[:, 0]) / M
        out[1, s] = (iy + u[:, 1]) / M
        out[2, s] = (z0 + u[:, 2]) / M
    return out
