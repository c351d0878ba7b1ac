"""The oracle's Picard + aggregation-multigrid reference solver (the
nonlinear-multigrid direction; the paper names multigrid only as future work):
its lagged system is Eq. 31 itself, and it lands on the fixed point of
Algorithm 1."""
import numpy as np
import pytest

import fld_inputs
import oracle

pytest.importorskip("scipy")
INNER = (slice(1, -1),) * 3


def _cloud(shape, seed):
    nz, ny, nx = shape
    sig, alb = fld_inputs.cloud_medium(nx, seed=seed, albedo=0.95, ny=ny, nz=nz)
    h = 1.0 / max(shape)
    q = oracle.bake_directional(sig, alb, h, (0.0, 0.0, -1.0), 1.0)
    return sig, alb, q, h


def _sor_fixed_point(sig, alb, q, h):
    ref = oracle.make_problem(sig, alb, q, h, limiter="lp", local_iters=2, omega=1.6)
    oracle.init_state(ref)
    _, rel, _ = oracle.solve(ref, tol=1e-11, max_iters=200000, check_every=20)
    assert rel <= 1e-11
    return ref


def test_lagged_system_is_the_residual_of_eq37():
    # with D recomputed from phi, b - A phi of the lagged system is R_p h^2,
    # the residual field the C oracle computes (an independent assembly)
    sig, alb, q, h = _cloud((9, 11, 13), 5)
    p = oracle.make_problem(sig, alb, q, h, limiter="kershaw", local_iters=2, omega=1.5)
    oracle.init_state(p)
    oracle.rb_iteration(p, 30)   # a state away from the fixed point
    A, b = oracle.lagged_system(p, oracle.fresh_D_field(p, p.phi))
    r = b - A @ p.phi[INNER].ravel()
    _, _, _, R = oracle.residual(p, field=True)
    np.testing.assert_allclose(r, (R * h * h).ravel(), rtol=1e-9, atol=1e-12 * np.abs(b).max())


@pytest.mark.parametrize("shape,seed", [((12, 12, 12), 3), ((14, 10, 16), 7)])
def test_picard_multigrid_reaches_the_sor_fixed_point(shape, seed):
    sig, alb, q, h = _cloud(shape, seed)
    ref = _sor_fixed_point(sig, alb, q, h)
    p = oracle.make_problem(sig, alb, q, h, limiter="lp", local_iters=2)
    oracle.init_state(p)
    steps, cg_its, rel = oracle.solve_picard_mg(p, 1e-10)
    assert rel <= 1e-10 and steps < 200 and cg_its > 0
    err = np.linalg.norm(p.phi[INNER] - ref.phi[INNER]) / np.linalg.norm(ref.phi[INNER])
    assert err <= 1e-9, err
    assert np.array_equal(p.phi[0], ref.phi[0])   # the Dirichlet ghosts stay as set


def test_aggregation_multigrid_preconditions_the_jumps():
    # the coefficients jump from the vacuum floor to the cloud; Galerkin
    # coarse operators of 2x2x2 aggregates keep CG's iterations far below
    # those of a Jacobi preconditioner
    import scipy.sparse.linalg as spla
    sig, alb, q, h = _cloud((16, 16, 16), 2)
    p = oracle.make_problem(sig, alb, q, h, limiter="lp", local_iters=2, omega=1.5)
    oracle.init_state(p)
    oracle.rb_iteration(p, 100)
    A, b = oracle.lagged_system(p, oracle.fresh_D_field(p, p.phi))
    mg = oracle.AggregationMG(A, (16, 16, 16), coarsest=100)
    assert len(mg.A) >= 3
    its = {}
    for name, M in (("mg", spla.LinearOperator(A.shape, matvec=mg.vcycle)),
                    ("jacobi", spla.LinearOperator(A.shape, matvec=lambda r: r / A.diagonal()))):
        count = [0]
        x, info = spla.cg(A, b, rtol=1e-8, maxiter=5000, M=M, callback=lambda _xk: count.__setitem__(0, count[0] + 1))
        assert info == 0
        assert np.linalg.norm(b - A @ x) <= 1e-7 * np.linalg.norm(b)
        its[name] = count[0]
    assert its["mg"] * 3 < its["jacobi"], its


def test_newton_with_multigrid_preconditioning_converges_fast_to_the_same_point():
    # from Picard steps to rel. 1e-2, Newton steps (Jacobian-vector products
    # by differences of the residual of Eq. 37, the V-cycle of the lagged
    # operator as preconditioner) cut the residual at least tenfold per step
    # and land on Algorithm 1's fixed point
    sig, alb, q, h = _cloud((12, 12, 12), 3)
    ref = _sor_fixed_point(sig, alb, q, h)
    p = oracle.make_problem(sig, alb, q, h, limiter="lp", local_iters=2)
    oracle.init_state(p)
    pic, newton, vcycles, fevals, hist = oracle.solve_newton_mg(p, 1e-10)
    assert hist[-1] <= 1e-10 and newton <= 6, hist
    assert all(b <= 0.1 * a for a, b in zip(hist[1:], hist[2:])), hist
    err = np.linalg.norm(p.phi[INNER] - ref.phi[INNER]) / np.linalg.norm(ref.phi[INNER])
    assert err <= 1e-9, err


def test_smoothed_aggregation_keeps_its_strength_with_depth():
    # one damped-Jacobi step on the piecewise-constant aggregates (smoothed
    # aggregation) keeps CG's iteration count nearly flat from 16^3 to 32^3,
    # where the plain aggregates lose strength with every added level
    import scipy.sparse.linalg as spla
    its = {}
    for n in (16, 32):
        sig, alb, q, h = _cloud((n, n, n), 0)
        p = oracle.make_problem(sig, alb, q, h, limiter="lp", local_iters=2, omega=1.5)
        oracle.init_state(p)
        oracle.rb_iteration(p, 200)
        A, b = oracle.lagged_system(p, oracle.fresh_D_field(p, p.phi))
        for smooth in (False, True):
            mg = oracle.AggregationMG(A, (n, n, n), coarsest=200, smooth=smooth)
            count = [0]
            _, info = spla.cg(A, b, rtol=1e-8, maxiter=3000, M=spla.LinearOperator(A.shape, matvec=mg.vcycle),
                              callback=lambda _xk: count.__setitem__(0, count[0] + 1))
            assert info == 0
            its[(n, smooth)] = count[0]
    assert its[(32, True)] <= its[(16, True)] + 4, its
    assert its[(32, True)] < its[(32, False)], its
