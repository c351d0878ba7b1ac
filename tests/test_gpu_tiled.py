"""The temporally blocked red-black sweeps (fld_solve_params.temporal_depth):
TMA-staged tiles in shared memory, 2T colour passes per launch as a
z-wavefront.  Every point update is the launched passes' own arithmetic, so
the blocked iterations must give the launched passes' state bit for bit; and
through that, and directly, the oracle's."""
import numpy as np
import pytest

import fld_inputs
import oracle

pytestmark = pytest.mark.gpu

fld = pytest.importorskip("paper_1403_8105_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_parity import INNER, gpu_grid, random_case, rel_el, rel_l2  # noqa: E402

# (temporal depth, tile rows): every configuration the library offers
CONFIGS = [(1, 32), (2, 24), (4, 8)]
SHAPES = [(16, 12, 20), (6, 35, 57), (9, 33, 17), (1, 1, 1), (40, 3, 113)]


def _state_after(sig, alb, j, h, phi0, D0, precision, depth, tile_y, iters, limiter="lp", bf16=0):
    with gpu_grid(sig, alb, j, h) as g:
        g.set_state(phi0, D0)
        p = fld.params(limiter=limiter, precision=precision, omega=1.6, local_iters=2, warm_start=1,
                       temporal_depth=depth, tile_y=tile_y, medium_bf16=bf16)
        g.iterate(p, iters)
        return g.get_state()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("precision", ["fp32", "pair"])
def test_blocked_equals_launched_bit_for_bit(shape, precision):
    sig, alb, j, h = random_case(shape, 17)
    ref = oracle.make_problem(sig, alb, j.astype(np.float64), h, omega=1.6, local_iters=2, nthreads=1)
    oracle.init_state(ref)
    oracle.rb_iteration(ref, 3)
    phi0, D0 = ref.phi.copy(), ref.D.copy()
    iters = 8
    want = _state_after(sig, alb, j, h, phi0, D0, precision, -1, 0, iters)
    for depth, ty in CONFIGS:
        got = _state_after(sig, alb, j, h, phi0, D0, precision, depth, ty, iters)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), (depth, ty)


@pytest.mark.parametrize("limiter", ["kershaw", "larsen", "sum", "cda"])
@pytest.mark.parametrize("bf16", [0, 1])
def test_blocked_equals_launched_other_limiters_and_bf16(limiter, bf16):
    sig, alb, j, h = random_case((12, 19, 61), 23)
    ref = oracle.make_problem(sig, alb, j.astype(np.float64), h, limiter=limiter, omega=1.6, local_iters=2,
                              nthreads=1)
    oracle.init_state(ref)
    oracle.rb_iteration(ref, 2)
    phi0, D0 = ref.phi.copy(), ref.D.copy()
    for precision in ("fp32", "pair"):
        want = _state_after(sig, alb, j, h, phi0, D0, precision, -1, 0, 4, limiter, bf16)
        for depth, ty in CONFIGS:
            got = _state_after(sig, alb, j, h, phi0, D0, precision, depth, ty, 4, limiter, bf16)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), (precision, depth, ty)


@pytest.mark.parametrize("depth,ty", CONFIGS)
def test_blocked_iterations_match_the_oracle(depth, ty):
    # T iterations in one blocked launch (two launches: the state returns to its
    # buffers) against the oracle's FP64 Algorithm 1 from the same state
    sig, alb, j, h = random_case((16, 12, 20), 5)
    ref = oracle.make_problem(sig, alb, j.astype(np.float64), h, limiter="lp", omega=1.5, local_iters=2, nthreads=1)
    oracle.init_state(ref)
    oracle.rb_iteration(ref, 4)
    ref.phi[...] = ref.phi.astype(np.float32)
    ref.D[...] = ref.D.astype(np.float32)
    phi0, D0 = ref.phi.copy(), ref.D.copy()
    oracle.rb_iteration(ref, 2 * depth)
    with gpu_grid(sig, alb, j, h) as g:
        g.set_state(phi0, D0)
        g.iterate(fld.params(limiter="lp", precision="fp32", omega=1.5, local_iters=2, warm_start=1,
                             temporal_depth=depth, tile_y=ty), 2 * depth)
        phi, D = g.get_state()
    # single-precision arithmetic over 2T iterations (the launched passes are
    # held to 3e-6 after one)
    e_phi = rel_el(phi, ref.phi, also=phi0)
    print(f"blocked T={depth} ty={ty}: per-element phi {e_phi:.2e}")
    assert e_phi <= 3e-6 * 2 * depth


@pytest.mark.parametrize("depth", [1, 2, 4])
def test_blocked_fixed_point_matches_oracle(depth):
    shape = (23, 17, 29)
    nz, ny, nx = shape
    sig, alb = fld_inputs.cloud_medium(nx, seed=11, albedo=0.95, ny=ny, nz=nz)
    h = 1.0 / max(shape)
    q = oracle.bake_directional(sig, alb, h, (0, 0, -1), 1.0).astype(np.float32)
    ref = oracle.make_problem(sig, alb, q.astype(np.float64), h, limiter="lp", omega=1.7, local_iters=2)
    oracle.init_state(ref)
    _, rel, _ = oracle.solve(ref, tol=1e-11, max_iters=400000, check_every=20)
    assert rel <= 1e-11
    results = {}
    for d in (-1, depth):
        with gpu_grid(sig, alb, q, h) as g:
            r = g.solve(fld.params(limiter="lp", precision="mixed", tol=1e-6, omega=1.7, local_iters=2,
                                   check_every=32, max_iters=400000, temporal_depth=d))
            assert r.status == fld.FLD_OK, r.as_dict()
            results[d] = (r.iterations, g.get_state()[0])
    # same iterations, same bits as the launched passes ...
    assert results[depth][0] == results[-1][0]
    assert np.array_equal(results[depth][1], results[-1][1])
    # ... and the oracle's fixed point
    phi = results[depth][1]
    assert rel_l2(phi[INNER], ref.phi[INNER]) <= 1e-5
    assert rel_el(phi[INNER], ref.phi[INNER], floor=1e-3) <= 1e-4


def test_autotuned_solve_equals_launched_and_reports_its_choice():
    # the default (temporal_depth 0) picks a launch shape by timing; whatever it
    # picks, the solve is the launched passes' bit for bit
    n = 40
    sig, alb = fld_inputs.cloud_medium(n, seed=3, albedo=0.9)
    h = 1.0 / n
    out = {}
    for d in (-1, 0):
        with fld.Grid(n, n, n, h) as g:
            g.set_medium(sig, alb)
            g.bake_directional((0.0, 0.0, -1.0), 1.0)
            r = g.solve(fld.params(precision="mixed", tol=1e-6, check_every=64, temporal_depth=d))
            assert r.status == fld.FLD_OK
            out[d] = (r.iterations, g.get_state()[0])
    assert out[0][0] == out[-1][0] and np.array_equal(out[0][1], out[-1][1])


def test_batch_with_blocked_sweeps_equals_solo():
    p = fld.params(limiter="lp", precision="mixed", tol=1e-6, omega=1.7, check_every=32, max_iters=200000,
                   temporal_depth=2, tile_y=24)
    shapes = [(16, 16, 16), (9, 33, 17), (20, 18, 22)]
    ins = []
    for s, (nz, ny, nx) in enumerate(shapes):
        sig, alb = fld_inputs.cloud_medium(nx, seed=50 + s, albedo=0.9, ny=ny, nz=nz)
        ins.append((sig, alb, 1.0 / max(nx, ny, nz)))

    def grid(sig, alb, h):
        nz, ny, nx = sig.shape
        g = fld.Grid(nx, ny, nz, h)
        g.set_medium(sig, alb)
        g.bake_directional((0.0, 0.0, -1.0), 1.0)
        return g

    solo = []
    for sig, alb, h in ins:
        with grid(sig, alb, h) as g:
            r = g.solve(p)
            assert r.status == fld.FLD_OK, r.as_dict()
            solo.append((r.iterations, g.get_state()[0]))
    grids = [grid(*x) for x in ins]
    try:
        st, rs = fld.fld_solve_batch(grids, p)
        assert st == fld.FLD_OK
        for a, g in enumerate(grids):
            assert rs[a].iterations == solo[a][0]
            assert np.array_equal(g.get_state()[0], solo[a][1]), a
    finally:
        for g in grids:
            g.close()


def test_invalid_blocking_parameters_are_rejected():
    sig, alb, j, h = random_case((6, 6, 6), 1)
    with gpu_grid(sig, alb, j, h) as g:
        for bad in (dict(temporal_depth=3), dict(temporal_depth=-2), dict(temporal_depth=2, tile_y=16),
                    dict(tile_y=-1)):
            with pytest.raises(fld.FldError) as e:
                g.solve(fld.params(**bad))
            assert e.value.status == fld.FLD_ERR_INVALID_ARG


@pytest.mark.parametrize("shape", SHAPES + [(5, 7, 127), (3, 4, 9)])
@pytest.mark.parametrize("precision", ["fp32", "pair"])
@pytest.mark.parametrize("bf16", [0, 1])
def test_four_cells_per_thread_equals_two_bit_for_bit(shape, precision, bf16):
    # the launched passes with 128-bit loads (four unknowns per thread, ragged
    # row tails stored element by element) against the two-unknown passes
    sig, alb, j, h = random_case(shape, 29)
    ref = oracle.make_problem(sig, alb, j.astype(np.float64), h, omega=1.6, local_iters=2, nthreads=1)
    oracle.init_state(ref)
    oracle.rb_iteration(ref, 3)
    phi0, D0 = ref.phi.copy(), ref.D.copy()
    out = []
    for cells in (2, 4):
        for lim in ("lp", "kershaw"):
            with gpu_grid(sig, alb, j, h) as g:
                g.set_state(phi0, D0)
                g.iterate(fld.params(limiter=lim, precision=precision, omega=1.6, local_iters=2, warm_start=1,
                                     temporal_depth=-1, cells_per_thread=cells, medium_bf16=bf16), 5)
                out.append(g.get_state())
    for a, b in ((0, 2), (1, 3)):
        assert np.array_equal(out[a][0], out[b][0]) and np.array_equal(out[a][1], out[b][1])
