"""The allocation-free V-cycle (fvem_vcycle_static) gives the same result as
fvem_vcycle, on two calls in a row, with each form of the coarsest-level
CG; it allocates no device memory; and it rejects a hierarchy whose work
vectors do not fit its static array before launching anything.  Collected
last on purpose: a failure here comes after every other test has run."""
import os

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


@pytest.mark.parametrize("mode", ["seq", "coop", "persist"])
def test_static_vcycle_matches_vcycle_twice(fv, tmp_path, mode):
    from tune_pin import pinned_solver
    sc = scenes.config(0, 8)
    S = pinned_solver(fv, sc, str(tmp_path / "tune.txt"), mode64=mode, rel_tol=1e-10)
    assert S.query()["coarse_mode"] == {"seq": "kernel sequence", "coop": "cooperative",
                                         "persist": "persistent"}[mode]
    n = S.query()["n_dofs"][0]
    rs = [torch.tensor(np.cos(np.arange(n) * (0.37 + 0.1 * k)), dtype=torch.float64, device="cuda")
          for k in range(2)]
    zs = [torch.full_like(r, np.nan) for r in rs]
    z_ref = [torch.empty_like(r) for r in rs]
    S.vcycle_static(rs[0], zs[0])           # first call on the device: looks up the array's address
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    for k in range(2):
        zs[k].fill_(np.nan)
        S.vcycle_static(rs[k], zs[k])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_reserved() == res0
    for k in range(2):
        S.vcycle(rs[k], z_ref[k])
        err = float(torch.linalg.norm(zs[k] - z_ref[k]) / torch.linalg.norm(z_ref[k]))
        # the same kernels with the same launch shapes in the same order: the
        # results agree to the last bits
        assert err <= 1e-15, (mode, k, err)


def test_static_vcycle_rejects_a_hierarchy_that_does_not_fit(fv):
    """Two-box scene at 80^3: five level vectors over all levels exceed the
    2^21 doubles of the static array; the call returns FVEM_EINVAL and
    launches nothing."""
    sc = scenes.config(1, 80)
    S = fv.Solver(levels=5, rel_tol=1e-6)
    S.build(sc.N, sc.tris)
    q = S.query()
    assert 5 * sum(q["n_dofs"]) > 2 ** 21
    n = q["n_dofs"][0]
    r = torch.ones(n, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    n0 = S.launch_count()
    with pytest.raises(fv.FastVEMError) as e:
        S.vcycle_static(r, z)
    assert e.value.status == 1
    assert S.launch_count() == n0
    assert float(z.abs().max()) == 0.0
