"""Nested solves (fld_solve_params.nested): the start from successively
coarser, box-averaged problems changes the iteration path only -- the solve
must land on the oracle's fixed point like a cold one."""
import numpy as np
import pytest

import fld_inputs
import oracle

pytestmark = pytest.mark.gpu

fld = pytest.importorskip("paper_1403_8105_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

INNER = (slice(1, -1),) * 3


@pytest.mark.parametrize("shape,levels", [((32, 32, 32), 1), ((32, 32, 32), 2), ((29, 17, 23), 1), ((20, 20, 20), 3)])
def test_nested_solve_reaches_the_oracle_fixed_point(shape, levels):
    nz, ny, nx = shape
    sig, alb = fld_inputs.cloud_medium(nx, seed=5, albedo=0.95, ny=ny, nz=nz)
    h = 1.0 / max(shape)
    q = oracle.bake_directional(sig, alb, h, (0, 0, -1), 1.0).astype(np.float32)
    ref = oracle.make_problem(sig, alb, q.astype(np.float64), h, omega=1.6, local_iters=2)
    oracle.init_state(ref)
    it, rel, _ = oracle.solve(ref, tol=1e-11, max_iters=400000, check_every=20)
    assert rel <= 1e-11
    with fld.Grid(nx, ny, nz, h) as g:
        g.set_medium(sig, alb)
        g.set_source(q)
        # (1e-6: mixed precision floors near 2e-7 at 32^3 -- single-precision D)
        p = fld.params(tol=1e-6, check_every=32, max_iters=400000, nested=levels)
        r = g.solve(p)
        assert r.status == fld.FLD_OK, r.as_dict()
        phi, _ = g.get_state()
        r2 = g.solve(p)                         # the coarse chain is reused
        phi2, _ = g.get_state()
    err = np.linalg.norm(phi[INNER] - ref.phi[INNER]) / np.linalg.norm(ref.phi[INNER])
    assert err <= 1e-5
    assert np.array_equal(phi, phi2) and r2.iterations == r.iterations
    small = min(shape) // 2 < 8
    if not small:
        assert r.iterations_coarse > 0 and r.updates_coarse > 0
        assert r.ms >= r.ms_coarse > 0
    if shape == (20, 20, 20):
        # 20 -> 10 -> (5: below the minimum edge): one level is used
        assert r.updates_coarse == r.iterations_coarse * 10 ** 3
