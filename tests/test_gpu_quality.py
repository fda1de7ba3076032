"""The element quality indicator (Eq. 18, Eq. 19, App. C) on the GPU against
the oracle's, cell by cell, on every level of the 8^3 sphere scene and on
level 0 of the two-box scene at 12^3: rho(E) within 1e-8 (the oracle's kernel
factor carries its linear program's tolerance), the cut cells and rho(P)."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_17725_b300 import build
    build.build()
    import paper_2607_17725_b300 as m
    return m


def _check(S, mesh, level):
    from oracle.quality import mesh_quality
    rho_ref, cut_ref, grid_ref = mesh_quality(mesh)
    rho, grid, ncut = S.quality(level)
    rho = rho.cpu().numpy()
    assert rho.shape == rho_ref.shape
    assert np.abs(rho - rho_ref).max() <= 1e-8 * np.abs(rho_ref).max()
    assert ncut == int(cut_ref.sum())
    assert abs(grid - grid_ref) <= 1e-8 * grid_ref


def test_quality_sphere8_every_level(fv, sphere8):
    S = fv.Solver(levels=5, rel_tol=1e-6)
    S.build(sphere8.scene.N, sphere8.scene.tris)
    for l, M in enumerate(sphere8.meshes):
        _check(S, M, l)


def test_quality_two_boxes_12(fv):
    from oracle.pipeline import build_system
    sc = scenes.config(1, 12)
    O = build_system(sc, L=2)
    S = fv.Solver(levels=2, rel_tol=1e-6)
    S.build(sc.N, sc.tris)
    _check(S, O.meshes[0], 0)


def test_quality_rejects_bad_level(fv, sphere8):
    S = fv.Solver(levels=5, rel_tol=1e-6)
    S.build(sphere8.scene.N, sphere8.scene.tris)
    with pytest.raises(fv.FastVEMError):
        S.quality(99)
