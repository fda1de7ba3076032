"""Pins of the oracle's VEM element quality indicator (Eq. 18, App. C):
closed forms on the unit cube and the regular tetrahedron, the kernel factor
on a non-convex (L-shaped) prism, invariance under scaling and translation,
and rho1 = 1 on the convex cells of a real cut-cell mesh."""
import numpy as np
import pytest

from oracle.quality import cell_kernel_volume, cell_quality, face_kernel_area, is_cut


def _outward(V, faces):
    """Orient every face cycle counter-clockwise about the outward normal
    (normal away from the vertex centroid of the solid; convex-enough test
    shapes only)."""
    c = V.mean(axis=0)
    out = []
    for cyc in faces:
        P = V[cyc]
        n = np.cross(P[1] - P[0], P[2] - P[0])
        out.append(list(cyc) if np.dot(n, P.mean(axis=0) - c) > 0 else list(cyc)[::-1])
    return out


def _cube(a=1.0, x0=(0.0, 0.0, 0.0)):
    V = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], dtype=float) * a + np.array(x0)
    idx = lambda i, j, k: i + 2 * j + 4 * k
    faces = [[idx(0, 0, 0), idx(0, 1, 0), idx(0, 1, 1), idx(0, 0, 1)],
             [idx(1, 0, 0), idx(1, 1, 0), idx(1, 1, 1), idx(1, 0, 1)],
             [idx(0, 0, 0), idx(1, 0, 0), idx(1, 0, 1), idx(0, 0, 1)],
             [idx(0, 1, 0), idx(1, 1, 0), idx(1, 1, 1), idx(0, 1, 1)],
             [idx(0, 0, 0), idx(1, 0, 0), idx(1, 1, 0), idx(0, 1, 0)],
             [idx(0, 0, 1), idx(1, 0, 1), idx(1, 1, 1), idx(0, 1, 1)]]
    return V, _outward(V, faces)


def test_unit_cube_closed_form():
    """Convex, so rho1 = 1; |E|^(1/3) = 1 < h_f = sqrt(2), h_E = sqrt(3);
    each face: sqrt(|f|) = 1 = shortest edge, h_f = sqrt(2); 6 faces of 4
    edges."""
    V, F = _cube()
    rho, r1, r2, r3 = cell_quality(V, F)
    e2 = 1.0 / np.sqrt(3.0) + 1.0 / np.sqrt(2.0)
    e3 = 4.0 / 6.0 + 3.0 / 4.0
    assert abs(r1 - 1.0) <= 1e-12 and abs(r2 - e2) <= 1e-14 and abs(r3 - e3) <= 1e-14
    assert abs(rho - np.sqrt(e2 + e3) / 2.0) <= 1e-14
    assert not is_cut(V, F)


def test_regular_tetrahedron_closed_form():
    """Edge a: |E| = a^3 / (6 sqrt 2), every diameter a, |f| = sqrt(3) a^2 / 4;
    4 triangular faces."""
    V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
    F = _outward(V, [[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]])
    a = 2.0 * np.sqrt(2.0)
    vol = a ** 3 / (6.0 * np.sqrt(2.0))
    area = np.sqrt(3.0) / 4.0 * a * a
    e2 = min(np.cbrt(vol), a) / a + min(np.sqrt(area), a) / a
    e3 = 4.0 / 4.0 + 3.0 / 3.0
    rho, r1, r2, r3 = cell_quality(V, F)
    assert abs(r1 - 1.0) <= 1e-12 and abs(r2 - e2) <= 1e-14 and abs(r3 - e3) <= 1e-14
    assert abs(rho - np.sqrt(e2 + e3) / 2.0) <= 1e-14
    assert is_cut(V, F)


def test_l_prism_kernel_factor():
    """L-shaped polygon [0,2]x[0,1] u [0,1]x[0,2] (area 3): its kernel is the
    unit square at the reflex corner (area 1), and the prism over it (height
    1, volume 3) has the unit cube as kernel; rectangles are their own
    kernels, so rho1 = (1/3) (1/3)^2 = 1/27."""
    L = [(0, 0), (2, 0), (2, 1), (1, 1), (1, 2), (0, 2)]
    V = np.array([(x, y, 0.0) for x, y in L] + [(x, y, 1.0) for x, y in L], dtype=float)
    n = len(L)
    bottom = list(range(n))[::-1]          # outward normal -z
    top = [n + i for i in range(n)]        # outward normal +z
    sides = [[i, (i + 1) % n, n + (i + 1) % n, n + i] for i in range(n)]
    F = [bottom, top] + sides              # sides of a CCW base are outward as listed
    assert abs(face_kernel_area(V, top) - 1.0) <= 1e-9
    assert abs(cell_kernel_volume(V, F) - 1.0) <= 1e-9
    rho, r1, r2, r3 = cell_quality(V, F)
    assert abs(r1 - 1.0 / 27.0) <= 1e-9
    assert abs(r3 - (4.0 / 8.0 + (2 * 3.0 / 6.0 + 6 * 3.0 / 4.0) / 8.0)) <= 1e-14


@pytest.mark.parametrize("scale,shift", [(1e-3, (0.3, -2.0, 5.0)), (7.0, (0.0, 0.0, 0.0))])
def test_invariant_under_scaling_and_translation(scale, shift):
    V, F = _cube()
    W = V * np.array([1.0, 2.0, 0.5])                      # a box, not a cube
    r0 = cell_quality(W, F)
    r1 = cell_quality(W * scale + np.array(shift), F)
    # rho2 and rho3 are closed-form in the geometry; the kernel factor rho1
    # carries the linear program's and the hull's tolerances (about 1e-9)
    assert np.allclose(r0[2:], r1[2:], rtol=1e-12, atol=0.0)
    assert np.allclose(r0[:2], r1[:2], rtol=1e-8, atol=0.0)
    assert is_cut(W, F)


def test_sphere_cells_are_convex(sphere8):
    """The cells of the 8^3 sphere scene's cut-cell mesh (every 7th, for
    time) are convex: each kernel is the cell and each face's kernel the
    face, so rho1 = 1 (to the kernel computation's tolerance)."""
    M = sphere8.meshes[0]
    for cf in M.cell_faces[::7]:
        r = cell_quality(M.V, [f[2] for f in cf])
        assert abs(r[1] - 1.0) <= 1e-8
        assert 0.0 < r[0] <= 1.0
