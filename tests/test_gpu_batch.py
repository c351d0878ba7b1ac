"""Batched solves (many grids of uneven size in shared launches): each grid's
result must be the same alone and in the mix, and match the FP64 oracle."""
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
SHAPES = [(16, 16, 16), (20, 18, 22), (12, 12, 12), (24, 24, 24), (9, 33, 17)]


def _inputs():
    out = []
    for s, shape in enumerate(SHAPES):
        nz, ny, nx = shape
        sig, alb = fld_inputs.cloud_medium(nx, seed=20 + s, albedo=0.9 + 0.02 * s, ny=ny, nz=nz)
        out.append((sig, alb, 1.0 / max(shape)))
    return out


def _grid(sig, alb, h, light):
    nz, ny, nx = sig.shape
    g = fld.Grid(nx, ny, nz, h)
    g.set_medium(sig, alb)
    if light == 0:
        g.bake_directional((0.0, 0.0, -1.0), 1.0)
    else:
        g.bake_point((0.3, 0.7, 1.3), 2.0)
    return g


def test_batch_equals_solo_solves_bitwise():
    p = fld.params(limiter="lp", precision="mixed", tol=1e-7, omega=1.7, check_every=32, max_iters=200000)
    ins = _inputs()
    solo = []
    for a, (sig, alb, h) in enumerate(ins):
        with _grid(sig, alb, h, a % 2) as g:
            r = g.solve(p)
            assert r.status == fld.FLD_OK, r.as_dict()
            solo.append((r.iterations, r.iterations_fp32, g.get_state()[0]))
    grids = [_grid(sig, alb, h, a % 2) for a, (sig, alb, h) in enumerate(ins)]
    try:
        st, rs = fld.fld_solve_batch(grids, p)
        assert st == fld.FLD_OK
        for a, g in enumerate(grids):
            assert rs[a].status == fld.FLD_OK
            assert (rs[a].iterations, rs[a].iterations_fp32) == solo[a][:2]
            phi, _ = g.get_state()
            assert np.array_equal(phi, solo[a][2]), a
    finally:
        for g in grids:
            g.close()


def test_batch_matches_oracle_fixed_points():
    p = fld.params(limiter="kershaw", precision="mixed", tol=1e-7, check_every=32, max_iters=200000)
    ins = _inputs()[:3]
    # the oracle's bake of each grid's light, given to both sides
    qs = [oracle.bake_directional(sig, alb, h, (0.0, 0.0, -1.0), 1.0).astype(np.float32).astype(np.float64)
          for sig, alb, h in ins]
    grids = []
    for (sig, alb, h), q in zip(ins, qs):
        nz, ny, nx = sig.shape
        g = fld.Grid(nx, ny, nz, h)
        g.set_medium(sig, alb)
        g.set_source(q.astype(np.float32))
        grids.append(g)
    try:
        st, rs = fld.fld_solve_batch(grids, p)
        assert st == fld.FLD_OK
        for (sig, alb, h), g, q in zip(ins, grids, qs):
            ref = oracle.make_problem(sig, alb, q, h, limiter="kershaw", omega=1.6, local_iters=2)
            oracle.init_state(ref)
            it, rel, _ = oracle.solve(ref, tol=1e-11, max_iters=400000, check_every=20)
            assert rel <= 1e-11
            phi, _ = g.get_state()
            err = np.linalg.norm(phi[INNER] - ref.phi[INNER]) / np.linalg.norm(ref.phi[INNER])
            assert err <= 1e-5, err
    finally:
        for g in grids:
            g.close()


def test_batch_rejects_fp64_and_duplicates():
    sig, alb, h = _inputs()[2]
    with _grid(sig, alb, h, 0) as g:
        with pytest.raises(fld.FldError) as e:
            fld.fld_solve_batch([g], fld.params(precision="fp64"))
        assert e.value.status == fld.FLD_ERR_INVALID_ARG
        with pytest.raises(fld.FldError) as e:
            fld.fld_solve_batch([g, g], fld.params())
        assert e.value.status == fld.FLD_ERR_INVALID_ARG


@pytest.mark.parametrize("limiter,precision,bf16,anderson", [
    ("lp", "mixed", 0, 0), ("kershaw", "mixed", 0, 0), ("lp", "pair", 1, 0), ("larsen", "fp32", 0, 0),
    ("lp", "mixed", 0, 4)])
def test_multi_grid_launches_equal_per_grid_graphs(limiter, precision, bf16, anderson):
    # batch_launch = 1 runs the grids in FP32 / hi-lo sweeps as one multi-grid
    # launch per colour pass; it must give every grid the bits, iteration
    # counts and checks of the per-grid graphs (batch_launch = 0)
    ins = _inputs()
    out = {}
    for mode in (0, 1):
        p = fld.params(limiter=limiter, precision=precision, tol=1e-7 if precision == "mixed" else 1e-6,
                       check_every=32, max_iters=200000, medium_bf16=bf16, anderson=anderson, batch_launch=mode)
        grids = [_grid(sig, alb, h, a % 2) for a, (sig, alb, h) in enumerate(ins)]
        try:
            st, rs = fld.fld_solve_batch(grids, p)
            out[mode] = [(r.status, r.iterations, r.iterations_fp32, r.iterations_mid, r.iterations_corr, r.checks,
                          r.anderson_steps, g.get_state()[0]) for r, g in zip(rs, grids)]
        finally:
            for g in grids:
                g.close()
    for a, (x, y) in enumerate(zip(out[0], out[1])):
        assert x[:7] == y[:7], (a, x[:7], y[:7])
        assert np.array_equal(x[7], y[7]), a
    if precision == "mixed":
        assert all(x[0] == fld.FLD_OK for x in out[1])
