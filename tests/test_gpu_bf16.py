"""GPU parity with the bfloat16 medium (medium_bf16 = 1): sigma' and sigma_a'
rounded to 8 significant bits, read as bfloat16 by the single-precision and
hi/lo sweeps and as the same values, upcast, by every other kernel.  The
oracle solves on the identically rounded medium, so parity tests the solver;
the effect of the rounding itself on phi* is measured, not held to 1e-5."""
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


@pytest.mark.parametrize("shape", [(16, 12, 20), (9, 11, 13)])
@pytest.mark.parametrize("precision", ["fp32", "pair", "mixed"])
@pytest.mark.parametrize("limiter", ["lp", "kershaw", "larsen", "sum"])
def test_one_iteration_bf16_matches_oracle(shape, precision, limiter):
    sig, alb, j, h = random_case(shape, 5)
    ref = oracle.make_problem(sig, alb, j.astype(np.float64), h, limiter=limiter, omega=1.5, local_iters=2,
                              nthreads=1, medium_bf16=True)
    oracle.init_state(ref)
    oracle.rb_iteration(ref, 4)
    if precision == "fp32":
        ref.phi[...] = ref.phi.astype(np.float32)
    ref.D[...] = ref.D.astype(np.float32)
    phi0, D0 = ref.phi.copy(), ref.D.copy()
    oracle.rb_iteration(ref, 1)
    with gpu_grid(sig, alb, j, h) as g:
        g.set_state(phi0, D0)
        p = fld.params(limiter=limiter, precision=precision, omega=1.5, local_iters=2, warm_start=1,
                       medium_bf16=1)
        g.iterate(p, 1)
        phi, D = g.get_state()
    e_phi, e_D = rel_el(phi, ref.phi, also=phi0), rel_el(D, ref.D, also=D0)
    print(f"bf16 {precision} {limiter} {shape}: per-element phi {e_phi:.2e} D {e_D:.2e}")
    assert e_phi <= 3e-6
    assert e_D <= 3e-5


def test_residual_uses_the_rounded_medium_and_switches_back():
    sig, alb, j, h = random_case((14, 15, 16), 8)
    refs = {}
    for bf in (False, True):
        r = oracle.make_problem(sig, alb, j.astype(np.float64), h, omega=1.5, local_iters=2, nthreads=1,
                                medium_bf16=bf)
        refs[bf] = r
    oracle.init_state(refs[False])
    oracle.rb_iteration(refs[False], 30)
    state = (refs[False].phi.copy(), refs[False].D.copy())
    want = {}
    for bf, r in refs.items():
        r.phi, r.D = state[0].copy(), state[1].copy()
        want[bf] = oracle.residual(r)[0]
    assert abs(want[True] - want[False]) > 1e-6 * want[False]     # the rounding is visible
    with gpu_grid(sig, alb, j, h) as g:
        g.set_state(*state)
        for bf in (True, False, True):          # re-prepared whenever the medium mode changes
            got64 = g.residual(fld.params(precision="fp64", medium_bf16=int(bf)))
            gotf = g.residual(fld.params(precision="mixed", medium_bf16=int(bf)))
            assert abs(got64 - want[bf]) <= 1e-11 * want[bf], bf
            assert abs(gotf - want[bf]) <= 2e-5 * want[bf], bf


def test_cloud_fixed_point_bf16_mixed_and_fp64():
    n = 24
    sig, alb = fld_inputs.cloud_medium(n, seed=11, albedo=0.95)
    h = 1.0 / n
    q = oracle.bake_directional(sig, alb, h, (0, 0, -1), 1.0).astype(np.float32)
    sols = {}
    for bf in (False, True):
        ref = oracle.make_problem(sig, alb, q.astype(np.float64), h, omega=1.7, local_iters=2, medium_bf16=bf)
        oracle.init_state(ref)
        it, rel, _ = oracle.solve(ref, tol=1e-11, max_iters=400000, check_every=20)
        assert rel <= 1e-11
        sols[bf] = ref.phi[INNER].copy()
    quant = np.linalg.norm(sols[True] - sols[False]) / np.linalg.norm(sols[False])
    assert 1e-5 < quant < 2e-2          # rounding effect: measured, above the parity bound
    for precision, tol, bound, bound_el in (("mixed", 1e-6, 1e-5, 1e-4), ("fp64", 1e-10, 1e-8, 1e-7)):
        with gpu_grid(sig, alb, q, h) as g:
            p = fld.params(limiter="lp", precision=precision, tol=tol, omega=1.7, local_iters=2, check_every=32,
                           max_iters=400000, medium_bf16=1)
            r = g.solve(p)
            assert r.status == fld.FLD_OK, r.as_dict()
            assert r.rel_residual <= tol
            phi, _ = g.get_state()
        err, err_el = rel_l2(phi[INNER], sols[True]), rel_el(phi[INNER], sols[True], floor=1e-3)
        print(f"bf16 fixed point {precision}: rel L2 {err:.2e} per-element {err_el:.2e}")
        assert err <= bound, (precision, err)
        assert err_el <= bound_el, (precision, err_el)


def test_batch_with_bf16_medium_equals_solo():
    p = fld.params(limiter="kershaw", precision="mixed", tol=1e-7, omega=1.7, check_every=32, max_iters=200000,
                   medium_bf16=1)
    shapes = [(16, 16, 16), (9, 33, 17), (20, 18, 22)]
    ins = []
    for s, (nz, ny, nx) in enumerate(shapes):
        sig, alb = fld_inputs.cloud_medium(nx, seed=40 + s, albedo=0.9, ny=ny, nz=nz)
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
            assert rs[a].status == fld.FLD_OK and rs[a].iterations == solo[a][0]
            assert np.array_equal(g.get_state()[0], solo[a][1]), a
    finally:
        for g in grids:
            g.close()
