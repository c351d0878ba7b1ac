"""Pins of the oracle's solve (Algorithm 1) against what the mathematics fixes.

* Brute force on tiny grids: the fixed point phi* of Eq. 31 with D from
  Eq. 33-35 is computed here independently by Picard iteration with dense
  numpy solves (freeze D(phi), assemble the linear system of Eq. 31, solve
  exactly, repeat).  The oracle's red-black SOR must land on the same phi*.
* Invariants that hold for any correct solver: the discrete energy balance
  (internal face fluxes cancel because D_ps is symmetric), the constant
  solution, the 48 cube symmetries, independence of omega, of the initial
  guess and of the per-point update path, positivity, and the flux-limiting
  constraint |E| <= phi (Eq. 14) at convergence.
"""
import itertools

import numpy as np
import pytest

import oracle

OFFS = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]


def dense_picard(p, phi_init, max_iters=3000):
    """Independent fixed-point solve of Eq. 31 (dense linear algebra)."""
    nx, ny, nz, h = p.nx, p.ny, p.nz, p.h
    ph = phi_init.copy()
    D_ghost = p.D.copy()
    N = nx * ny * nz
    idx = lambda i, j, k: (k * ny + j) * nx + i
    fl = p.eps * p.jbar
    for m in range(max_iters):
        D = D_ghost.copy()
        c = ph[1:-1, 1:-1, 1:-1]
        gx = (ph[1:-1, 1:-1, 2:] - ph[1:-1, 1:-1, :-2]) / (2 * h)
        gy = (ph[1:-1, 2:, 1:-1] - ph[1:-1, :-2, 1:-1]) / (2 * h)
        gz = (ph[2:, 1:-1, 1:-1] - ph[:-2, 1:-1, 1:-1]) / (2 * h)
        g = np.sqrt(gx ** 2 + gy ** 2 + gz ** 2)
        R = np.maximum(g, fl) / np.maximum(p.sp * c, fl)
        D[1:-1, 1:-1, 1:-1] = oracle.limiter(p.limiter, R, p.larsen_n) / p.sp
        A = np.zeros((N, N))
        b = (p.j * h * h).ravel().copy()
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    r = idx(i, j, k)
                    A[r, r] += p.sa[k, j, i] * h * h
                    for di, dj, dk in OFFS:
                        I, J, K = i + di, j + dj, k + dk
                        Dps = 0.5 * (D[k + 1, j + 1, i + 1] + D[K + 1, J + 1, I + 1])
                        A[r, r] += Dps
                        if 0 <= I < nx and 0 <= J < ny and 0 <= K < nz:
                            A[r, idx(I, J, K)] -= Dps
                        else:
                            b[r] += Dps * ph[K + 1, J + 1, I + 1]
        new = np.linalg.solve(A, b).reshape(nz, ny, nx)
        change = np.abs(new - c).max() / np.abs(new).max()
        ph[1:-1, 1:-1, 1:-1] = new
        if change < 2e-16:
            break
    return ph


def random_medium(shape, seed, vacuum=True):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    sig = rng.uniform(0.5, 30.0, shape).astype(np.float32)
    if vacuum and sig.size > 1:
        sig.ravel()[rng.integers(0, sig.size)] = 0.0
    alb = rng.uniform(0.3, 0.99, shape).astype(np.float32)
    j = rng.uniform(0.0, 5.0, shape)
    j[sig == 0] = 0.0          # no emission in vacuum (q_ri = L sigma_s T)
    return sig, alb, j, 1.0 / max(nx, ny, nz)


CASES = [((1, 1, 1), 0), ((4, 3, 2), 1), ((4, 4, 4), 2), ((5, 5, 5), 3), ((4, 5, 6), 4), ((6, 6, 6), 5)]


@pytest.mark.parametrize("shape,seed", CASES)
@pytest.mark.parametrize("limiter", ["lp", "kershaw", "larsen", "sum", "max", "cda"])
def test_rb_sor_reaches_dense_picard_fixed_point(shape, seed, limiter):
    sig, alb, j, h = random_medium(shape, seed)
    ref = oracle.make_problem(sig, alb, j, h, limiter=limiter, nthreads=1)
    oracle.init_state(ref)
    want = dense_picard(ref, ref.phi)
    # Algorithm 1 as printed (omega = 1) and with the self-consistent point
    # update under over-relaxation: both must reach the same phi*.
    for omega, local in ((1.0, 1), (1.6, 2)):
        p = oracle.make_problem(sig, alb, j, h, limiter=limiter, nthreads=1, omega=omega, local_iters=local)
        oracle.init_state(p)
        it, rel, _ = oracle.solve(p, tol=1e-14, max_iters=60000, check_every=5)
        assert rel <= 1e-13, (omega, local, rel)
        err = np.abs(p.phi - want).max() / np.abs(want).max()
        assert err <= 1e-12, (omega, local, err)


def test_no_emission_anywhere_gives_zero_without_nan():
    # jbar = 0: the floor of Eq. 35 falls back to a fixed tiny value, phi = 0.
    shape = (3, 4, 5)
    sig = np.zeros(shape, np.float32)
    sig[1, 2, 2] = 5.0
    alb = np.full(shape, 0.9, np.float32)
    p = oracle.make_problem(sig, alb, np.zeros(shape), 0.2, limiter="lp", nthreads=1)
    oracle.init_state(p)
    oracle.rb_iteration(p, 5)
    assert np.all(p.phi == 0.0) and np.all(np.isfinite(p.D))
    rel, s2, _ = oracle.residual(p)
    assert rel == 0.0


def test_single_unknown_closed_form():
    # n = 1: all six neighbours are ghosts, the central gradient is 0, so
    # R = eps*jbar / max(sigma' phi, eps*jbar) and phi solves
    # phi = (j h^2 + sum D_ps phi_b) / (sigma_a' h^2 + sum D_ps), D_ps = (D(phi) + D_b)/2.
    sig = np.array([[[7.0]]], np.float32)
    alb = np.array([[[0.625]]], np.float32)     # exact in FP32
    j = np.array([[[3.0]]])
    h = 0.25
    p = oracle.make_problem(sig, alb, j, h, limiter="lp", nthreads=1)
    oracle.init_state(p, phi_b=0.4, D_b=0.05)
    oracle.solve(p, tol=1e-15, max_iters=200, check_every=1)
    sp, sa = 7.0, 0.375 * 7.0
    fl = 1e-20 * 3.0

    def g(phi):
        R = fl / max(sp * phi, fl)
        D = (1.0 / 3.0 - R * R / 45.0) / sp
        Dps = 0.5 * (D + 0.05)
        return (3.0 * h * h + 6 * Dps * 0.4) / (sa * h * h + 6 * Dps) - phi

    lo, hi = 1e-6, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(lo) * g(mid) <= 0:
            hi = mid
        else:
            lo = mid
    assert abs(p.phi[1, 1, 1] - 0.5 * (lo + hi)) < 1e-14


def test_energy_balance_identity():
    # Summing Eq. 37 over all unknowns, internal face terms cancel in pairs
    # (D_ps = D_sp): sum_p R_p h^2 = sum_p (j_p - sigma_a' phi_p) h^2
    #                              + sum_{boundary faces} D_ps (phi_ghost - phi_p).
    # Checked with the CDA limiter, where D = 1/(3 sigma') is known.
    rng = np.random.default_rng(11)
    shape = (5, 6, 7)
    sig = rng.uniform(0.0, 20.0, shape).astype(np.float32)
    alb = rng.uniform(0.2, 0.95, shape).astype(np.float32)
    j = rng.uniform(0.0, 3.0, shape)
    h = 1.0 / 7
    p = oracle.make_problem(sig, alb, j, h, limiter="cda", nthreads=1)
    oracle.init_state(p, phi_b=0.3, D_b=0.02)
    p.phi[1:-1, 1:-1, 1:-1] = rng.uniform(0.1, 2.0, shape)
    rel, s2, cnt, R = oracle.residual(p, field=True)
    D = np.full(p.phi.shape, 0.02)
    D[1:-1, 1:-1, 1:-1] = 1.0 / (3.0 * p.sp)
    lhs = R.sum() * h * h
    rhs = ((p.j - p.sa * p.phi[1:-1, 1:-1, 1:-1]) * h * h).sum()
    nz, ny, nx = shape
    for k in range(nz):
        for jj in range(ny):
            for i in range(nx):
                for di, dj, dk in OFFS:
                    I, J, K = i + di, jj + dj, k + dk
                    if not (0 <= I < nx and 0 <= J < ny and 0 <= K < nz):
                        Dps = 0.5 * (D[k + 1, jj + 1, i + 1] + D[K + 1, J + 1, I + 1])
                        rhs += Dps * (p.phi[K + 1, J + 1, I + 1] - p.phi[k + 1, jj + 1, i + 1])
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs) + 1.0)


@pytest.mark.parametrize("limiter", ["lp", "cda", "kershaw"])
def test_constant_solution(limiter):
    # No absorption, no emission, ghost value c: phi = c is the solution.
    shape = (6, 5, 7)
    sig = np.random.default_rng(2).uniform(0.5, 10, shape).astype(np.float32)
    alb = np.ones(shape, np.float32)
    j = np.zeros(shape)
    p = oracle.make_problem(sig, alb, j, 1.0 / 7, limiter=limiter, nthreads=1, omega=1.5, local_iters=2)
    oracle.init_state(p, phi0=1.7, phi_b=1.7, D_b=0.1)
    rel, s2, cnt = oracle.residual(p)
    assert np.sqrt(s2 / cnt) <= 1e-14 * 1.7 / (3 * 0.5) * 7 ** 2   # rounding only
    oracle.init_state(p, phi0=0.2, phi_b=1.7, D_b=0.1)
    p.phi[1:-1, 1:-1, 1:-1] = np.random.default_rng(3).uniform(0.5, 3.0, shape)
    oracle.rb_iteration(p, 600)
    assert np.abs(p.phi - 1.7).max() < 1e-10


def _converged(limiter, n=9, omega=1.5, local=2, phi0=None, seed=0):
    rng = np.random.default_rng(seed)
    sig = np.full((n, n, n), 4.0, np.float32)
    alb = np.full((n, n, n), 0.8, np.float32)
    j = np.zeros((n, n, n))
    j[n // 2, n // 2, n // 2] = float(n ** 3)
    p = oracle.make_problem(sig, alb, j, 1.0 / n, limiter=limiter, nthreads=1, omega=omega, local_iters=local)
    oracle.init_state(p, phi0=phi0)
    it, rel, _ = oracle.solve(p, tol=1e-13, max_iters=20000, check_every=5)
    assert rel <= 1e-13
    return p


@pytest.mark.parametrize("limiter", ["lp", "kershaw", "cda"])
def test_cube_symmetries(limiter):
    # Odd n, centred source, homogeneous medium: phi* is invariant under all
    # 48 symmetries of the cube.
    p = _converged(limiter)
    phi = p.phi
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product((False, True), repeat=3):
            t = np.transpose(phi, perm)
            for ax, f in enumerate(flips):
                if f:
                    t = np.flip(t, axis=ax)
            assert np.abs(t - phi).max() <= 1e-11 * phi.max()


def test_fixed_point_independent_of_omega_and_initial_guess():
    a = _converged("lp", omega=1.0, local=1)
    b = _converged("lp", omega=1.7, local=2)
    c = _converged("lp", omega=1.3, local=3, phi0=5.0)
    for o in (b, c):
        assert np.abs(o.phi - a.phi).max() <= 1e-11 * a.phi.max()


def test_positivity_and_flux_limit_on_heterogeneous_medium():
    sig, alb, j, h = random_medium((7, 8, 9), 21)
    for limiter in ("lp", "kershaw", "larsen", "sum", "max"):
        p = oracle.make_problem(sig, alb, j, h, limiter=limiter, nthreads=1, omega=1.5, local_iters=2)
        oracle.init_state(p)
        it, rel, _ = oracle.solve(p, tol=1e-12, max_iters=20000, check_every=5)
        assert rel <= 1e-12
        inner = p.phi[1:-1, 1:-1, 1:-1]
        assert np.all(inner > 0)
        E = oracle.flux_magnitude(p)
        assert np.all(E <= inner * (1 + 1e-12)), limiter      # Eq. 14
