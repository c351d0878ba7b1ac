"""Failure detection, with the failure made on the host (no GPU fault): a
non-finite value planted in the state through the public API must end the
solve as FLD_ERR_DIVERGED at the first residual check, leave the grid usable,
and -- inside a server batch -- retire that grid alone; a tolerance below the
floor of the arithmetic must end as FLD_ERR_NOT_CONVERGED by the stall rule,
long before max_iters."""
import numpy as np
import pytest

import fld_inputs

pytestmark = pytest.mark.gpu

fld = pytest.importorskip("paper_1403_8105_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def baked(n, seed):
    sig, alb = fld_inputs.cloud_medium(n, seed=seed, albedo=0.9)
    g = fld.Grid(n, n, n, 1.0 / n)
    g.set_medium(sig, alb)
    g.bake_directional((0.0, 0.0, -1.0), 1.0)
    return g


def initialised(n, seed):
    g = baked(n, seed)
    r = g.solve(fld.params(max_iters=0, check_every=1), check=False)   # the initial state only
    assert r.iterations == 0
    return g


def poison(g):
    phi, D = g.get_state()
    phi[5, 6, 7] = np.nan
    g.set_state(phi, D)


def test_nan_state_reports_divergence_and_the_grid_recovers():
    p = fld.params(tol=1e-6, check_every=32, max_iters=100000)
    with baked(20, 3) as ref:
        want = ref.solve(p)
        want_phi = ref.get_state()[0]
    with initialised(20, 3) as g:
        poison(g)
        warm = fld.params(tol=1e-6, check_every=32, max_iters=100000, warm_start=1)
        r = g.solve(warm, check=False)
        assert r.status == fld.FLD_ERR_DIVERGED and r.iterations == 0
        assert "NaN" in fld.fld_last_error()
        r2 = g.solve(p)                                  # a cold solve starts over
        assert r2.status == fld.FLD_OK and r2.iterations == want.iterations
        assert np.array_equal(g.get_state()[0], want_phi)


def test_server_retires_a_poisoned_grid_alone():
    p = fld.params(tol=1e-6, check_every=32, max_iters=100000, warm_start=1)
    solo = []
    for seed in (1, 2, 3):
        with initialised(16, seed) as g:
            r = g.solve(p)
            assert r.status == fld.FLD_OK
            solo.append((r.iterations, g.get_state()[0]))
    grids = [initialised(16, seed) for seed in (1, 2, 3)]
    poison(grids[1])
    done = {}
    try:
        with fld.Server(p) as srv:
            for tag, g in enumerate(grids):
                srv.add(g, tag)
            steps = 0
            while srv.active > 0 or len(done) < 3:
                for tag, r in srv.step():
                    done[tag] = r
                steps += 1
                assert steps < 100000
        assert done[1].status == fld.FLD_ERR_DIVERGED and done[1].iterations == 0
        for tag in (0, 2):
            assert done[tag].status == fld.FLD_OK
            assert done[tag].iterations == solo[tag][0]
            assert np.array_equal(grids[tag].get_state()[0], solo[tag][1])
    finally:
        for g in grids:
            g.close()


def test_unreachable_tolerance_stalls_instead_of_running_to_max_iters():
    with baked(24, 4) as g:
        r = g.solve(fld.params(tol=1e-13, check_every=32, max_iters=10_000_000), check=False)
        assert r.status == fld.FLD_ERR_NOT_CONVERGED
        assert r.iterations < 200_000
        assert "stalled" in fld.fld_last_error()
        assert 0 < r.rel_residual < 1e-6                 # it did converge as far as the arithmetic allows
