"""C-ABI library on the host (no GPU): symbols, and bit-exact integer topology
against the oracle."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def fv():
    from paper_2607_17725_b300 import build
    build.build()
    import paper_2607_17725_b300 as m
    return m


def test_library_exports_every_declared_symbol(fv):
    hdr = open(os.path.join(ROOT, "include", "fastvem.h")).read()
    names = sorted(set(re.findall(r"^(?:fvem_status|void|const char\*)\s+(fvem_[a-z_0-9]+)\s*\(", hdr, re.M)))
    assert len(names) >= 20
    L = fv.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing
    assert set(fv.EXPORTS) <= set(names)


def _lib_solver(fv, scene, balance=True):
    S = fv.Solver(levels=5, balance=balance)
    S.build_topology(scene.N, scene.tris)
    return S


def _compare_topology(S, meshes):
    for l, M in enumerate(meshes):
        E = S.export_level(l)
        assert np.array_equal(E["V"], M.V), l                     # coordinates bit-exact
        assert np.array_equal(np.diff(E["cell_vptr"]), [len(v) for v in M.cell_verts])
        assert np.array_equal(E["cell_v"], np.concatenate([np.array(v) for v in M.cell_verts]))
        faces = []
        for c in range(len(M.cell_faces)):
            for f in range(E["cell_fptr"][c], E["cell_fptr"][c + 1]):
                faces.append((int(E["face_pid"][f]), int(E["face_sg"][f]),
                              tuple(E["face_v"][E["face_vptr"][f]:E["face_vptr"][f + 1]])))
        ref = [(p, s, tuple(cyc)) for cf in M.cell_faces for (p, s, cyc) in cf]
        assert faces == ref, l
        if M.parent is not None:
            assert np.array_equal(E["parent"], M.parent)


def test_topology_bitexact_sphere8(fv, sphere8):
    S = _lib_solver(fv, sphere8.scene)
    _compare_topology(S, sphere8.meshes)


def test_topology_bitexact_box_scene_of_the_greedy_pin(fv):
    """The hand-worked box scene of the cut-order and greedy-removal pins
    (tests/test_oracle_hierarchy_pins.py): the library's levels equal the
    oracle's bit for bit, so the library removes the same cuts."""
    import test_oracle_hierarchy_pins as pins
    from oracle.cutcell import build_cut_grid
    from oracle.hierarchy import build_hierarchy
    from oracle.mesh import build_meshes
    sc = scenes.Scene("box", 4, pins.box_tris(), None, None)
    G = build_cut_grid(4, sc.tris)
    _compare_topology(_lib_solver(fv, sc), build_meshes(G, build_hierarchy(G, 5)))


@pytest.mark.parametrize("balance", [True, False])
def test_topology_bitexact_sphere12_balance_switch(fv, balance):
    """Aggregation with and without 2:1 balance (balance=False is the rule as
    Sec. 5.2 prints it): the library follows the oracle bit for bit either
    way, and the two settings differ on this scene."""
    from oracle.cutcell import build_cut_grid
    from oracle.hierarchy import build_hierarchy
    from oracle.mesh import build_meshes
    sc = scenes.config(0, 12)
    G = build_cut_grid(sc.N, sc.tris)
    meshes = build_meshes(G, build_hierarchy(G, 5, balance))
    _compare_topology(_lib_solver(fv, sc, balance), meshes)
    other = build_hierarchy(G, 5, not balance)
    assert any(len(a.cells) != len(b.cells) for a, b in zip(build_hierarchy(G, 5, balance), other))


def test_dofs_and_patterns_match_oracle(fv, sphere8):
    S = _lib_solver(fv, sphere8.scene)
    for l in range(len(sphere8.meshes)):
        d = S.export_dofs(l)
        assert np.array_equal(np.nonzero(d >= 0)[0], sphere8.free[l])
        # A pattern = clique union of the level's cells over free DOFs
        _, rp, col, _ = S.export_matrix(0, l, values=False)
        pos = -np.ones(len(d), dtype=np.int64)
        pos[sphere8.free[l]] = np.arange(len(sphere8.free[l]))
        rows = [set() for _ in range(len(sphere8.free[l]))]
        for vs in sphere8.meshes[l].cell_verts:
            loc = [pos[v] for v in vs if pos[v] >= 0]
            for a in loc:
                rows[a].update(loc)
        ref_rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])])
        ref_col = np.concatenate([sorted(r) for r in rows])
        assert np.array_equal(rp, ref_rp) and np.array_equal(col, ref_col)
    for l in range(len(sphere8.meshes) - 1):
        (nr, nc), rp, col, _ = S.export_matrix(1, l, values=False)
        Pref = sphere8.Pfull[l][sphere8.free[l]][:, sphere8.free[l + 1]].tocsr()
        Pref.sort_indices()
        got = sp.csr_matrix((np.ones(len(col)), col, rp), shape=(nr, nc))
        got.sort_indices()
        assert np.array_equal(got.indptr, Pref.indptr) and np.array_equal(got.indices, Pref.indices)


def test_naive_prolongation_patterns_match_oracle(fv):
    """The naive prolongation of Eq. 16 (the Ours^np ablation), host plan of
    the 8^3 sphere: its P pattern equals the oracle's naive P structure on
    every level; every coarse operator pattern holds the oracle's P^T A P
    nonzeros and more entries than the diffusion-free pattern (the coupling
    spreads across coarse cells)."""
    from oracle.pipeline import build_system
    sc = scenes.config(0, 8)
    O = build_system(sc, naive_prolongation=True)
    S = fv.Solver(levels=5, naive_prolongation=True)
    S.build_topology(sc.N, sc.tris)
    D = _lib_solver(fv, sc)
    for l in range(len(O.meshes) - 1):
        (nr, nc), rp, col, _ = S.export_matrix(1, l, values=False)
        Pref = O.Pfull[l][O.free[l]][:, O.free[l + 1]].tocsr()
        Pref.sort_indices()
        got = sp.csr_matrix((np.ones(len(col)), col, rp), shape=(nr, nc))
        got.sort_indices()
        assert np.array_equal(got.indptr, Pref.indptr) and np.array_equal(got.indices, Pref.indices), l
    for l in range(1, len(O.meshes)):
        (n, _), rp, col, _ = S.export_matrix(0, l, values=False)
        pat = sp.csr_matrix((np.ones(len(col)), col, rp), shape=(n, n))
        ref = O.H.A[l].tocoo()
        assert all(pat[i, j] for i, j in zip(ref.row, ref.col)), l
        (_, _), rpd, _, _ = D.export_matrix(0, l, values=False)
        assert rp[-1] > rpd[-1], l


def test_naive_k2_prolongation_pattern_matches_oracle(fv):
    """Second order with the naive prolongation of Eq. 16 (sphere at 4^3, two
    levels): the library's k = 2 prolongation pattern equals the structure of
    the oracle's naive k = 2 P bit for bit, and differs from the
    diffusion-free one."""
    from oracle.system2 import build_hierarchy2
    sc = scenes.config(0, 4)
    O = build_hierarchy2(sc, L=2, naive_prolongation=True)
    S = fv.Solver(levels=2, order_k=2, naive_prolongation=True)
    S.build_topology(sc.N, sc.tris)
    (nr, nc), rp, col = S.export_prolongation_pattern_k2(0)
    P = O.Pfull[0].tocsr()
    P.sort_indices()
    assert (nr, nc) == P.shape
    assert np.array_equal(rp, P.indptr) and np.array_equal(col, P.indices)
    D = fv.Solver(levels=2, order_k=2)
    D.build_topology(sc.N, sc.tris)
    assert D.export_prolongation_pattern_k2(0)[1][-1] < rp[-1]
    # the solver's own plan: P over the condensed free DOFs (columns of a row
    # listed in the cell's DOF order) has the oracle's pattern, and the
    # level-1 pattern holds every nonzero of the oracle's P^T A P
    (nr, nc), prp, pcol, _ = S.export_matrix(1, 0, values=False)
    Po = O.Hc.H.P[0].tocsr()
    Po.sort_indices()
    assert (nr, nc) == Po.shape and np.array_equal(prp, Po.indptr)
    assert all(np.array_equal(np.sort(pcol[prp[r]:prp[r + 1]]), Po.indices[Po.indptr[r]:Po.indptr[r + 1]])
               for r in range(nr))
    (nr, nc), arp, acol, _ = S.export_matrix(0, 1, values=False)
    pat = sp.csr_matrix((np.ones(len(acol)), acol, arp), shape=(nr, nc))
    nzo = (abs(O.Hc.H.A[1]) > 0).astype(float)
    assert (nzo - nzo.multiply(pat)).nnz == 0
    assert S.query()["nnz"][1] > 3 * D.query()["nnz"][1]


@pytest.mark.slow
@pytest.mark.parametrize("ci,N", [(0, 16), (1, 16)])
def test_topology_bitexact_16(fv, ci, N):
    from oracle.cutcell import build_cut_grid
    from oracle.hierarchy import build_hierarchy
    from oracle.mesh import build_meshes
    sc = scenes.config(ci, N)
    G = build_cut_grid(sc.N, sc.tris)
    meshes = build_meshes(G, build_hierarchy(G, 5))
    _compare_topology(_lib_solver(fv, sc), meshes)


@pytest.mark.slow
def test_topology_bitexact_random_scene_with_sliver_face(fv):
    """Random scene 1 of the batch at 32^3: overlapping obstacles leave a
    sliver face (area 1.8e-8, about 2e-5 of a cell face) whose overlay pieces
    sum to its area only up to the rounding of its long edges; both sides
    accept it and agree bit for bit."""
    from oracle.cutcell import build_cut_grid
    from oracle.hierarchy import build_hierarchy
    from oracle.mesh import build_meshes
    sc = scenes.random_scene(1)
    assert sc.N == 32
    G = build_cut_grid(sc.N, sc.tris)
    meshes = build_meshes(G, build_hierarchy(G, 1))   # the sliver face is on level 0
    _compare_topology(_lib_solver(fv, sc), meshes)


@pytest.mark.slow
def test_coarse_patterns_hold_galerkin_product_with_nonlocal_prolongation(fv):
    """Random scene 5 at 80^3: a fine vertex 1.4e-8 from a coarse vertex sits
    within the weld distance of a coarse edge of one parent cell but not of
    the other, so its prolongation row leaves that parent.  The element lists
    widen the coarse blocks and every level's pattern still holds the
    structural pattern of P^T A P (Sec. 4.3 Galerkin operator)."""
    sc = scenes.random_scene(5)
    S = fv.Solver(levels=5)
    S.build_topology(sc.N, sc.tris)
    nl = len([x for x in S.query()["n_dofs"] if x > 0])

    def pat(which, l):
        (nr, nc), rp, col, _ = S.export_matrix(which, l, values=False)
        return sp.csr_matrix((np.ones(len(col)), col, rp), shape=(nr, nc))

    for l in range(nl - 1):
        A, P, Ac = pat(0, l), pat(1, l), pat(0, l + 1)
        G = (P.T @ A @ P).tocsr()
        G.data[:] = 1.0
        assert (G - G.multiply(Ac)).count_nonzero() == 0, l


def test_degenerate_triangle_is_rejected(fv):
    S = fv.Solver()
    tris = np.zeros((1, 3, 3))
    with pytest.raises(fv.FastVEMError) as e:
        S.build_topology(8, tris)
    assert e.value.status == 3


def test_nan_geometry_is_rejected(fv):
    S = fv.Solver()
    tris = scenes.config(0, 8).tris.copy()
    tris[3, 1, 2] = np.nan
    with pytest.raises(fv.FastVEMError) as e:
        S.build_topology(8, tris)
    assert e.value.status == 6


def test_build_without_device_reports_nodev(fv):
    import torch
    if torch.cuda.is_available():
        pytest.skip("device present")
    S = fv.Solver()
    with pytest.raises(fv.FastVEMError) as e:
        S.build(8, scenes.config(0, 8).tris)
    assert e.value.status == 8


def test_batched_projection_rejects_bad_arguments(fv):
    """fvem_project_batched checks its arguments before any device work: an
    empty batch, null arrays and contexts that were not built give EINVAL."""
    import ctypes
    L = fv.lib()
    S1, S2 = fv.Solver(), fv.Solver()
    H = (ctypes.c_void_p * 2)(S1._h.value, S2._h.value)
    nul = (ctypes.c_void_p * 2)(None, None)
    assert L.fvem_project_batched(H, 0, nul, None, nul, nul, None) == 1
    assert L.fvem_project_batched(None, 2, nul, None, nul, nul, None) == 1
    assert L.fvem_project_batched(H, 2, nul, None, nul, nul, None) == 1   # not built, null buffers


def test_particle_calls_reject_unbuilt_contexts_and_bad_arguments(fv):
    """The particle entry points (Sec. 3.2-3.3) check their arguments before
    any device work: an unbuilt context, a negative count and null buffers
    give EINVAL."""
    L = fv.lib()
    S = fv.Solver()
    assert L.fvem_p2g(S._h, 0, None, None, 3, None, None) == 1
    assert L.fvem_locate(S._h, 10, None, None) == 1
    assert L.fvem_g2p(S._h, -1, None, None, None, None, 0.5, None) == 1
    assert L.fvem_advect(S._h, 0, 0.1, None, None, None) == 1
    assert L.fvem_locate(None, 0, None, None) == 1


def test_k2_dof_numbering_matches_oracle(fv, sphere8):
    """Second-order DOFs (Sec. 3.1) of every level of the 8^3 sphere scene: the
    library's global numbering, element DOF lists and Dirichlet mask equal the
    oracle's bit for bit, and on the coarsest level (the largest cells) so does
    the pattern over free DOFs of the oracle's assembled k = 2 operator."""
    from oracle.system2 import level2
    S = _lib_solver(fv, sphere8.scene)
    for l, M in enumerate(sphere8.meshes):
        with_k = l == len(sphere8.meshes) - 1     # the assembled operator on the coarsest level
        Lv = level2(M, elements=with_k)
        D = S.export_dofs_k2(l)
        assert (D["n"], D["nv"], D["ne"], D["nf"], D["nc"]) == (Lv.n, Lv.nv, Lv.ne, Lv.nf, len(Lv.dofmap)), l
        ref = np.concatenate(Lv.dofmap)
        ptr = np.concatenate([[0], np.cumsum([len(d) for d in Lv.dofmap])])
        assert np.array_equal(D["elem_ptr"], ptr) and np.array_equal(D["elem_dof"], ref), l
        assert np.array_equal(D["dirichlet"], Lv.dirichlet), l
        if not with_k:
            continue
        # pattern over free DOFs: that of the oracle's assembled k = 2 operator
        free = np.nonzero(~Lv.dirichlet)[0]
        Kf = Lv.K[free][:, free].tocsr()
        Kf.sort_indices()
        rp, col = S.export_pattern_k2(l)
        assert np.array_equal(rp, Kf.indptr) and np.array_equal(col, Kf.indices), l


def test_k2_prolongation_pattern_matches_oracle(fv):
    """Sphere scene at 4^3, two levels: the library's k = 2 prolongation pattern
    (which coarse DOFs each fine vertex, edge-midpoint, face-mean and cell-mean
    DOF uses) equals the structure of the oracle's k = 2 P bit for bit."""
    from oracle.system2 import build_hierarchy2
    sc = scenes.config(0, 4)
    O = build_hierarchy2(sc, L=2)
    S = fv.Solver(levels=2)
    S.build_topology(sc.N, sc.tris)
    (nr, nc), rp, col = S.export_prolongation_pattern_k2(0)
    P = O.Pfull[0].tocsr()
    P.sort_indices()
    assert (nr, nc) == P.shape
    assert np.array_equal(rp, P.indptr) and np.array_equal(col, P.indices)


def test_k2_condensed_plan_matches_oracle(fv):
    """Second-order plan on the sphere at 4^3 with two levels (host only):
    the unknowns of the condensed system on each level are exactly the
    oracle's free vertex, edge and face DOFs (cell means eliminated, reading
    K2; coarse DOFs kept where the prolongation uses them), and the level-0
    operator's pattern has the oracle's size."""
    from oracle.system2 import build_hierarchy2
    sc = scenes.config(0, 4)
    o = build_hierarchy2(sc, L=2)
    S = fv.Solver(order_k=2, levels=2)
    S.build_topology(sc.N, sc.tris)
    q = S.query()
    assert q["order_k"] == 2 and q["n_dofs_all"] == [Lv.n for Lv in o.levels]
    for l, Lv in enumerate(o.levels):
        d = np.zeros(Lv.cdof, np.int32)
        S._check(fv.lib().fvem_export_dofs(S._h, l, fv._ptr(d)), "export_dofs")
        ref = o.free[l][o.free[l] < Lv.cdof]
        assert np.array_equal(np.nonzero(d >= 0)[0], ref), l
    (nr, nc), rp, col, _ = S.export_matrix(0, 0, values=False)
    A = o.S0.tocsr()
    A.sort_indices()
    assert (nr, nc) == A.shape and np.array_equal(rp, A.indptr) and np.array_equal(col, A.indices)
    (nr, nc), _, _, _ = S.export_matrix(1, 0, values=False)
    assert (nr, nc) == o.Hc.H.P[0].shape
