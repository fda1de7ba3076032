"""The allocation-free V-cycle (fvem_vcycle_static) gives the same result as
fvem_vcycle, on two calls in a row.  Collected last on purpose: a failure here
comes after every other test has run."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_static_vcycle_matches_vcycle_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_17725_b300 import build
    build.build()
    import paper_2607_17725_b300 as fv
    sc = scenes.config(0, 8)
    S = fv.Solver(levels=5, rel_tol=1e-10)
    S.build(sc.N, sc.tris)
    n = S.query()["n_dofs"][0]
    for k in range(2):
        r = torch.tensor(np.cos(np.arange(n) * (0.37 + 0.1 * k)), dtype=torch.float64, device="cuda")
        z_ref = torch.empty_like(r)
        z = torch.full_like(r, np.nan)
        S.vcycle(r, z_ref)
        S.vcycle_static(r, z)
        err = float(torch.linalg.norm(z - z_ref) / torch.linalg.norm(z_ref))
        # same kernels, same order of operations: agreement to the V-cycle parity tolerance
        assert err <= 1e-10, (k, err)
