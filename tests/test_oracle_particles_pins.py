"""Pins of the oracle's particle transfers (Sec. 3.2 P2G, Sec. 3.3 G2P and
advection): the radial kernel's closed form; P2G reproduces constants, and
linear fields at a vertex whose particles are placed symmetrically about it;
hand-worked two-particle averages; located cells contain their points by an
independent test (signed pyramid volumes) and the located fraction matches
the fluid volume; G2P at alpha = 1 and 0 and on linear fields; the midpoint
rule in closed form on a linear field; mirror reflection at a wall and at an
obstacle face."""
import numpy as np
import pytest

import scenes
from oracle import particles as P


def test_kernel_closed_form():
    q = np.array([0.0, 0.25, 0.5, 1.0, 1.5])
    assert np.array_equal(P.kernel_weight(q), np.array([1.0, 0.421875, 0.125, 0.0, 0.0]))


def test_p2g_constant_and_single_particle():
    rng = np.random.default_rng(3)
    V = rng.uniform(0.2, 0.8, (20, 3))
    xp = rng.uniform(0.0, 1.0, (400, 3))
    f = np.full((400, 2), [1.5, -0.25])
    out = P.p2g(V, xp, f, 0.2)
    hit = np.array([(((xp - v) ** 2).sum(1) < 0.04).any() for v in V])
    assert hit.all()
    assert np.allclose(out, [1.5, -0.25], rtol=0, atol=1e-15)
    # one particle inside the ball gives its value; one on or outside it, 0
    V1 = np.array([[0.5, 0.5, 0.5]])
    assert abs(P.p2g(V1, [[0.55, 0.5, 0.5]], [[3.0]], 0.1)[0, 0] - 3.0) <= 1e-15
    assert P.p2g(V1, [[0.75, 0.5, 0.5]], [[3.0]], 0.25)[0, 0] == 0.0   # q = 1 exactly
    assert P.p2g(V1, [[0.61, 0.5, 0.5]], [[3.0]], 0.1)[0, 0] == 0.0


def test_p2g_two_particles_by_hand():
    """|d1|^2 = R^2/4 -> w1 = 27/64; |d2|^2 = R^2/2 -> w2 = 1/8."""
    R = 0.2
    V = np.array([[0.5, 0.5, 0.5]])
    xp = np.array([[0.6, 0.5, 0.5], [0.5, 0.5 + R / np.sqrt(2.0), 0.5]])
    f = np.array([[2.0], [10.0]])
    w1, w2 = 27.0 / 64.0, 1.0 / 8.0
    assert abs(P.p2g(V, xp, f, R)[0, 0] - (2.0 * w1 + 10.0 * w2) / (w1 + w2)) <= 1e-14


def test_p2g_linear_field_symmetric_particles():
    """Particles at the 8 corners and 6 axis points of a cube about the vertex
    (every pair symmetric): the average of a linear field is its value at the
    vertex, whatever the weights."""
    x0 = np.array([0.41, 0.53, 0.47])
    a = 0.03
    pts = [x0 + a * np.array(s) for s in np.array(np.meshgrid([-1, 1], [-1, 1], [-1, 1])).reshape(3, -1).T]
    pts += [x0 + 0.05 * s * e for e in np.eye(3) for s in (-1, 1)]
    xp = np.array(pts)
    A = np.array([[1.0, -2.0, 0.5], [0.3, 0.0, 4.0], [-1.0, 2.5, 1.0]])
    b = np.array([0.2, -0.7, 1.1])
    f = xp @ A.T + b
    out = P.p2g(x0[None], xp, f, 0.08)
    assert np.allclose(out[0], A @ x0 + b, rtol=0, atol=1e-14)


def _pyramid_inside(mesh, c, x, tol=1e-12):
    """x inside convex cell c: every face's pyramid with apex x has volume
    >= 0 and together they make the cell's volume."""
    V = mesh.V
    vols = []
    for (_, _, cyc) in mesh.cell_faces[c]:
        a = V[cyc[0]]
        v = 0.0
        for m in range(1, len(cyc) - 1):
            v += float(np.dot(a - x, np.cross(V[cyc[m]] - x, V[cyc[m + 1]] - x))) / 6.0
        vols.append(v)
    ref = []
    c0 = V[mesh.cell_verts[c]].mean(axis=0)
    for (_, _, cyc) in mesh.cell_faces[c]:
        a = V[cyc[0]]
        for m in range(1, len(cyc) - 1):
            ref.append(float(np.dot(a - c0, np.cross(V[cyc[m]] - c0, V[cyc[m + 1]] - c0))) / 6.0)
    return min(vols) >= -tol and abs(sum(vols) - sum(ref)) <= 1e-12


def test_locate_against_pyramid_volumes(sphere8):
    M = sphere8.meshes[0]
    planes = P.face_planes(M)
    # each cell's vertex mean is interior to it and to no other cell
    means = np.array([M.V[v].mean(axis=0) for v in M.cell_verts])
    assert np.array_equal(P.locate(M, means[::5], planes), np.arange(len(means))[::5])
    # random points: located ones lie in their cell; unlocated ones in no cell
    pts = scenes.particles(8, per_axis=1, seed=11).T[::3]
    c = P.locate(M, pts, planes)
    for x, ci in zip(pts, c):
        if ci >= 0:
            assert _pyramid_inside(M, int(ci), x)
        else:
            assert not any(_pyramid_inside(M, k, x, tol=-1e-12) for k in range(len(M.cell_faces)))
    # the sphere's centre is inside the obstacle
    assert P.locate(M, [[0.47, 0.52, 0.49]], planes)[0] == -1


def test_located_fraction_is_fluid_volume(sphere8):
    sc = scenes.config(0, 8)
    M = sphere8.meshes[0]
    pts = scenes.particles(8, per_axis=2, seed=5).T[::2]
    frac = float((P.locate(M, pts) >= 0).mean())
    fluid = 1.0 - scenes.mesh_volume(sc.tris.reshape(-1, 3, 3))
    sd = np.sqrt(fluid * (1 - fluid) / len(pts))
    assert abs(frac - fluid) <= 4 * sd


def test_g2p_limits_and_linear_fields(sphere8):
    M, cells = sphere8.meshes[0], sphere8.cells
    A = np.array([[0.5, -1.0, 2.0], [1.5, 0.25, -0.5], [-2.0, 1.0, 0.75]])
    b = np.array([0.1, -0.2, 0.3])
    u_lin = M.V @ A.T + b
    pts = scenes.particles(8, per_axis=1, seed=9).T[::4]
    cell = P.locate(M, pts)
    live = cell >= 0
    up = np.random.default_rng(1).normal(size=pts.shape)
    # Pi_1 reproduces linears: the new field evaluates to A x + b
    new = P.cell_linear(cells, u_lin)
    pic = P.g2p(cells, pts, cell, u_lin, new, 0.0, up)
    assert np.allclose(pic[live], pts[live] @ A.T + b, rtol=0, atol=1e-12)
    assert np.array_equal(pic[~live], up[~live])
    # unchanged grid field: FLIP leaves particle velocities as they are
    flip = P.g2p(cells, pts, cell, u_lin, new, 1.0, up)
    assert np.allclose(flip, up, rtol=0, atol=1e-12)
    # FLIP increment: new = old + constant (0, 0, 1) adds exactly that
    shifted = new.copy()
    shifted[:, 2, 0] += 1.0
    flip2 = P.g2p(cells, pts, cell, u_lin, shifted, 1.0, up)
    assert np.allclose(flip2[live], up[live] + [0.0, 0.0, 1.0], rtol=0, atol=1e-12)
    # PIC with an increment: the new field alone (the increment sits inside
    # the FLIP weight), and the blend at alpha = 0.25
    pic2 = P.g2p(cells, pts, cell, u_lin, shifted, 0.0, up)
    assert np.allclose(pic2[live], pts[live] @ A.T + b + [0.0, 0.0, 1.0], rtol=0, atol=1e-12)
    mix = P.g2p(cells, pts, cell, u_lin, shifted, 0.25, up)
    assert np.allclose(mix[live], 0.25 * (up[live] + [0.0, 0.0, 1.0]) + 0.75 * pic2[live], rtol=0, atol=1e-12)


def _constant_poly(cells, v):
    c = np.zeros((len(cells), 3, 4))
    c[:, :, 0] = v
    return c


def test_advect_midpoint_rule_on_a_linear_field(empty4):
    """Empty box: v = A x + b; one midpoint step from x is
    x + dt (A (x + dt/2 (A x + b)) + b)."""
    M, cells = empty4.meshes[0], empty4.cells
    A = np.array([[0.0, -1.0, 0.2], [1.0, 0.0, 0.0], [-0.2, 0.0, 0.1]])
    b = np.array([0.05, -0.02, 0.01])
    poly = P.cell_linear(cells, M.V @ A.T + b)
    x = np.array([[0.4, 0.45, 0.52], [0.61, 0.3, 0.35], [0.55, 0.55, 0.6]])
    cell = P.locate(M, x)
    dt = 0.05
    X, C = P.advect(M, cells, np.zeros((0, 3, 3)), poly, dt, x, cell)
    ref = x + dt * ((x + 0.5 * dt * (x @ A.T + b)) @ A.T + b)
    assert np.allclose(X, ref, rtol=0, atol=1e-14)
    assert np.array_equal(C, P.locate(M, ref))


def test_advect_is_the_midpoint_rule(empty4):
    """Cells left of x = 0.5 move at 1, the others at 3 (h = 1/4).  From
    x = 0.45 with dt = 0.12 the midpoint 0.51 is in the fast half, so the
    step ends at 0.45 + 0.12 * 3 = 0.81 (Heun's rule would give 0.69)."""
    M, cells = empty4.meshes[0], empty4.cells
    poly = _constant_poly(cells, [1.0, 0.0, 0.0])
    for c, cv in enumerate(cells):
        if cv.xE[0] > 0.5:
            poly[c, 0, 0] = 3.0
    x = np.array([[0.45, 0.3, 0.6]])
    X, _ = P.advect(M, cells, np.zeros((0, 3, 3)), poly, 0.12, x, P.locate(M, x))
    assert np.allclose(X, [[0.81, 0.3, 0.6]], rtol=0, atol=1e-15)


def test_advect_wall_mirror(empty4):
    M, cells = empty4.meshes[0], empty4.cells
    poly = _constant_poly(cells, [2.0, 0.0, 0.0])
    x = np.array([[0.95, 0.5, 0.5]])
    X, C = P.advect(M, cells, np.zeros((0, 3, 3)), poly, 0.05, x, P.locate(M, x))
    assert np.allclose(X, [[2.0 - 1.05, 0.5, 0.5]], rtol=0, atol=1e-15) and C[0] >= 0


def test_advect_obstacle_mirror():
    """Axis-aligned box obstacle [0.3, 0.7]^3 on a 6^3 grid: a particle at
    x = 0.25 moving +x at speed 1 for dt = 0.08 reaches 0.33 (inside), which
    mirrors across the face x = 0.3 to 0.27; its midpoint 0.29 is still
    outside, so both stages see the constant field."""
    from oracle.pipeline import build_system
    tris = scenes.box([0.5, 0.5, 0.5], [0.4, 0.4, 0.4], np.eye(3))
    sc = scenes.Scene("box6", 6, tris, np.zeros(len(tris), dtype=np.int32), scenes.empty_scene(6).velocity)
    S = build_system(sc, L=2)
    M, cells = S.meshes[0], S.cells
    poly = _constant_poly(cells, [1.0, 0.0, 0.0])
    x = np.array([[0.25, 0.5, 0.45]])
    X, C = P.advect(M, cells, tris, poly, 0.08, x, P.locate(M, x))
    assert np.allclose(X, [[0.27, 0.5, 0.45]], rtol=0, atol=1e-14) and C[0] >= 0
    # without the obstacle the same step ends inside the box: no fluid cell there
    assert P.locate(M, [[0.33, 0.5, 0.45]])[0] == -1


def test_particle_generator_stream_and_stratification():
    """The closed-form SplitMix64 stream equals the scalar generator's draws
    (from any start), and the particles put exactly one point in every
    sub-cube."""
    r = scenes.SplitMix64(4242)
    ref = np.array([r.uniform() for _ in range(40)])
    assert np.array_equal(scenes.splitmix64_uniforms(4242, 0, 40), ref)
    assert np.array_equal(scenes.splitmix64_uniforms(4242, 17, 23), ref[17:])
    X = scenes.particles(3, per_axis=2, seed=8)
    M = 6
    sub = np.floor(X * M).astype(np.int64)
    key = (sub[2] * M + sub[1]) * M + sub[0]
    assert X.shape == (3, M ** 3) and np.array_equal(np.sort(key), np.arange(M ** 3))
    assert (X >= 0).all() and (X < 1).all()
