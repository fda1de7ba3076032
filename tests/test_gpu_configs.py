"""GPU parity on the benchmark configurations' own scenes and settings,
through the C ABI, against the FP64 CPU oracle:

* the sphere scene at 16^3 in FP64 against the oracle's dense solve;
* the two-box scene at 32^3 in the FP32 V-cycle with the level-0 stencil
  slices on (the form the benchmark runs), against the oracle's pressure
  stored by tests/golden/make_two_boxes_32.py;
* the torch.autograd.Function against the hand-written adjoint and the
  oracle's dense adjoint;
* the differentiable configuration's loss (squared projected velocity inside
  [0.6, 0.9]^3, integrated exactly per cell) by central differences at 64^3
  and against the dense adjoint at 12^3;
* a batch of scenes against the oracle, scene by scene;
* the failure statuses FVEM_ENOCONV and FVEM_EBREAKDOWN.
"""
import hashlib
import os

import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_17725_b300 import build
    build.build()
    import paper_2607_17725_b300 as m
    return m


def _solver(fv, scene, **kw):
    S = fv.Solver(**kw)
    S.build(scene.N, scene.tris)
    return S


def _vel(sc, S):
    return torch.tensor(sc.velocity(S.export_level(0)["V"]).T.copy(), device="cuda")


def test_sphere_16_fp64_matches_dense_solve(fv):
    from oracle.pipeline import build_system, dense_solve
    sc = scenes.config(0)
    assert sc.N == 16 and sc.tol == 1e-10
    O = build_system(sc)
    S = _solver(fv, sc, rel_tol=1e-10)
    u = sc.velocity(O.meshes[0].V)
    p, _, st = S.project(torch.tensor(u.T.copy(), device="cuda"))
    pd = dense_solve(O, u)
    assert st["rel_res"] <= 1e-10
    assert np.linalg.norm(p.cpu().numpy() - pd) / np.linalg.norm(pd) <= 1e-8


@pytest.mark.parametrize("coarse_iters", [80, 160])
def test_two_boxes_32_fp32_stencil_vcycle_matches_oracle(fv, coarse_iters):
    """The FP32 V-cycle with stencil slices on level 0 inside FP64 CG at
    1e-6: pressure within 1e-5 of the oracle's direct solve (relative L2);
    the FP64 mode at 1e-10 within 1e-8; with the default coarsest CG and with
    the benchmark's 160 iterations.  The stored pressure belongs to the same
    level-0 vertices (their coordinates' SHA-256 is stored with it)."""
    g = np.load(os.path.join(HERE, "golden", "two_boxes_32.npz"))
    sc = scenes.config(1, 32)
    S = _solver(fv, sc, precision="fp32", rel_tol=1e-6, coarse_iters=coarse_iters)
    V = S.export_level(0)["V"]
    assert hashlib.sha256(np.ascontiguousarray(V).tobytes()).digest() == g["v_sha256"].tobytes()
    q = S.query()
    assert q["n_dofs"][0] == int(g["n_free"]) and q["stencil_slices32"][0] > 0
    S.set_stencil(0, True)
    assert S.query()["stencil_used32"][0] == 1
    u = _vel(sc, S)
    p, _, st = S.project(u)
    pref = g["p"]
    assert st["rel_res"] <= 1e-6
    assert np.linalg.norm(p.cpu().numpy() - pref) / np.linalg.norm(pref) <= 1e-5
    S.set_precision("fp64")
    S.set_tolerance(1e-10, 500)
    p, _, st = S.project(u)
    assert np.linalg.norm(p.cpu().numpy() - pref) / np.linalg.norm(pref) <= 1e-8


def test_autograd_gradients_equal_adjoint_and_dense_oracle(fv, sphere8):
    from oracle.pipeline import dense_adjoint
    S = _solver(fv, sphere8.scene, rel_tol=1e-13, max_iters=1000)
    Fn = fv.projection_function()
    V = sphere8.meshes[0].V
    nc = len(sphere8.cells)
    w = np.random.default_rng(11).standard_normal(12 * nc)
    wd = torch.tensor(w.reshape(nc, 3, 4), device="cuda")
    u = torch.tensor(sphere8.scene.velocity(V).T.copy(), device="cuda", requires_grad=True)
    uin = torch.tensor(0.3, dtype=torch.float64, device="cuda", requires_grad=True)
    cp = Fn.apply(S, u, uin)
    (cp * wd).sum().backward()
    gu, gin, _ = S.adjoint(wd)
    assert torch.equal(u.grad, gu)
    assert float(uin.grad) == gin
    gu_ref, gin_ref = dense_adjoint(sphere8, w)
    assert np.linalg.norm(u.grad.cpu().numpy() - gu_ref) / np.linalg.norm(gu_ref) <= 1e-8
    assert abs(gin - gin_ref) <= 1e-8 * max(1.0, abs(gin_ref))


def _box_loss_weights(S, lo=0.6, hi=0.9):
    """Per level-0 cell, the 4x4 mass matrix of its scaled monomials (1, x, y,
    z about the centroid, over the diameter) when the centroid lies inside
    [lo, hi]^3, else 0.  The loss is sum_E sum_c c_E,c^T M_E c_E,c, i.e. the
    integral of |u_new|^2 over those cells (reading S7: the cell velocity is
    the linear polynomial Pi_1 u_new)."""
    from oracle.vem import mass_moments
    E = S.export_level(0)
    vol, cen, h, _ = S.export_cells()
    nc = len(vol)
    M = np.zeros((nc, 4, 4))
    inside = np.nonzero(np.all((cen >= lo) & (cen <= hi), axis=1))[0]
    for c in inside:
        faces = [E["face_v"][E["face_vptr"][f]:E["face_vptr"][f + 1]] for f in
                 range(E["cell_fptr"][c], E["cell_fptr"][c + 1])]
        M[c] = mass_moments(E["V"], faces, cen[c], h[c])
    return M, inside


def _loss_and_grad(cp, Md):
    """L = sum_E sum_c c^T M_E c and dL/dc = 2 M_E c (cp: (nc, 3, 4))."""
    Mc = torch.einsum("eab,ecb->eca", Md, cp)
    return float((cp * Mc).sum()), 2.0 * Mc


def test_config2_box_loss_adjoint_by_central_differences_64(fv):
    """Sphere with inflow on x = 0 at 64^3, the loss of the differentiable
    configuration.  L is quadratic in (u', U_in), so central differences are
    exact up to the solve and rounding; they are taken with FP64 solves at
    1e-13 along 20 SplitMix64 (seed 3002) directions over u' and U_in and
    compared at 1e-4 with the adjoint gradient evaluated in the FP32-V-cycle
    mode (solve to 1e-10)."""
    sc = scenes.config(2)
    assert sc.N == 64 and sc.u_inflow == 1.0
    S = _solver(fv, sc, precision="fp32", rel_tol=1e-10, max_iters=1000)
    M, inside = _box_loss_weights(S)
    assert len(inside) > 1000
    Md = torch.tensor(M, device="cuda")
    u0 = _vel(sc, S)
    _, cp, _ = S.project(u0, sc.u_inflow)
    _, g = _loss_and_grad(cp, Md)
    gu, gin, _ = S.adjoint(g.contiguous())
    gu = gu.cpu().numpy()
    S.set_precision("fp64")
    S.set_tolerance(1e-13, 2000)
    u0 = u0.cpu().numpy()

    def loss(u, uin):
        return _loss_and_grad(S.project(torch.tensor(u, device="cuda"), uin)[1], Md)[0]

    rng = scenes.SplitMix64(3002)
    h = 1e-6
    for _ in range(20):
        du = np.array([rng.normal() for _ in range(u0.size)]).reshape(u0.shape)
        dq = rng.normal()
        fd = (loss(u0 + h * du, sc.u_inflow + h * dq) - loss(u0 - h * du, sc.u_inflow - h * dq)) / (2 * h)
        ad = float((gu * du).sum()) + gin * dq
        assert abs(fd - ad) <= 1e-4 * max(1.0, abs(fd)), (fd, ad)


def test_config2_box_loss_adjoint_matches_dense_oracle_12(fv):
    """The same loss on the config's sphere at 12^3 with inflow: the adjoint
    (FP32 V-cycle, solve to 1e-12) against the oracle's dense adjoint J^T g
    (explicit solve), within 1e-8."""
    from oracle.pipeline import build_system, dense_adjoint
    sc = scenes.config(2, 12)
    O = build_system(sc)
    S = _solver(fv, sc, precision="fp32", rel_tol=1e-12, max_iters=2000)
    M, inside = _box_loss_weights(S)
    assert len(inside) > 10
    Md = torch.tensor(M, device="cuda")
    u = _vel(sc, S)
    _, cp, _ = S.project(u, sc.u_inflow)
    _, g = _loss_and_grad(cp, Md)
    gu, gin, _ = S.adjoint(g.contiguous())
    gu_ref, gin_ref = dense_adjoint(O, g.cpu().numpy().ravel())
    assert np.linalg.norm(gu.cpu().numpy() - gu_ref) / np.linalg.norm(gu_ref) <= 1e-8
    assert abs(gin - gin_ref) <= 1e-8 * max(1.0, abs(gin_ref))


def test_batched_scenes_match_oracle(fv):
    """Three scenes of uneven size (the sphere at 12^3, the two boxes at 16^3,
    random scene 2 at 16^3), each on its own stream, projected in one batched
    call in FP64 to 1e-10: every pressure within 1e-8 of the oracle's dense
    solve."""
    from oracle.pipeline import build_system, dense_solve
    r2 = scenes.random_scene(2)
    scs = [scenes.config(0, 12), scenes.config(1, 16), scenes.Scene(r2.name, 16, r2.tris, r2.comp, r2.velocity)]
    solvers, us, refs, keep = [], [], [], []
    for sc in scs:
        O = build_system(sc)
        st = torch.cuda.Stream()
        keep.append(st)
        S = fv.Solver(rel_tol=1e-10, stream=st.cuda_stream)
        S.build(sc.N, sc.tris)
        u = sc.velocity(O.meshes[0].V)
        us.append(torch.tensor(u.T.copy(), device="cuda"))
        refs.append(dense_solve(O, u))
        solvers.append(S)
    torch.cuda.synchronize()
    ps, _, stats = fv.project_batched(solvers, us)
    torch.cuda.synchronize()
    for p, pd, st in zip(ps, refs, stats):
        assert st["rel_res"] <= 1e-10
        assert np.linalg.norm(p.cpu().numpy() - pd) / np.linalg.norm(pd) <= 1e-8


def test_failure_statuses_noconv_and_breakdown(fv, sphere8):
    """max_iters = 1 at a 1e-10 tolerance returns FVEM_ENOCONV; a Chebyshev
    bound of a tenth of the level-0 spectrum makes the V-cycle indefinite
    (the smoothing polynomial grows like T_5 outside its interval), so CG
    stops with FVEM_EBREAKDOWN.  The context stays usable after both."""
    S = _solver(fv, sphere8.scene, rel_tol=1e-10, max_iters=1)
    u = torch.tensor(sphere8.scene.velocity(sphere8.meshes[0].V).T.copy(), device="cuda")
    with pytest.raises(fv.FastVEMError) as e:
        S.project(u)
    assert e.value.status == 4
    S.set_tolerance(1e-10, 500)
    lm = S.query()["lmax"][0]
    S.set_cheb_lmax(0, 0.1 * lm)
    with pytest.raises(fv.FastVEMError) as e:
        S.project(u)
    assert e.value.status == 5
    S.set_cheb_lmax(0, lm)
    _, _, st = S.project(u)
    assert st["rel_res"] <= 1e-10


@pytest.mark.parametrize("graphs", [True, False])
def test_persistent_abort_path_reports_timeout_and_recovers(fv, tmp_path, graphs):
    """The persistent coarsest CG's bounded-wait exit, taken on purpose: with
    its abort word armed by the host, the next launch leaves before its first
    copy (no GPU fault or hang), the projection reports FVEM_ETIMEOUT, the
    context is reset, and the next projection converges to the same pressure
    as before."""
    from tune_pin import pinned_solver
    sc = scenes.config(0, 8)
    S = pinned_solver(fv, sc, str(tmp_path / "tune.txt"), mode64="persist", rel_tol=1e-10)
    assert S.query()["coarse_mode"] == "persistent"
    S.set_graphs(graphs)
    u = torch.tensor(sc.velocity(S.export_level(0)["V"]).T.copy(), dtype=torch.float64, device="cuda")
    p0, _, st0 = S.project(u)
    p0 = p0.clone()
    S.arm_coarse_abort()
    with pytest.raises(fv.FastVEMError) as e:
        S.project(u)
    assert e.value.status == 9  # FVEM_ETIMEOUT
    p1, _, st1 = S.project(u)
    assert st1["rel_res"] <= 1e-10 and st1["iters"] == st0["iters"]
    assert torch.equal(p0, p1)
