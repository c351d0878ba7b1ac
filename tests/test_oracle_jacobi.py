"""Pins of the oracle's Jacobi iteration (the order-free alternative to
Algorithm 1's red-black sweep).

* One step is the textbook damped Jacobi step of the lagged linear system:
  with D^k = F(R(phi^k))/sigma' (Eq. 33-35) the system A(D^k) phi = b of
  Eq. 31 is assembled here densely, independently, and
  phi^{k+1} = phi^k + omega diag(A)^-1 (b - A phi^k) must hold to rounding.
* Iterated, it reaches the dense Picard fixed point on tiny grids, and the
  same phi* as the red-black sweep on a small cloud.
"""
import numpy as np
import pytest

import fld_inputs
import oracle

from test_oracle_fixed_point import OFFS, dense_picard, random_medium  # noqa: E402


def numpy_D(p, ph):
    """D at the unknowns from phi (Eq. 33-35), ghost D from p.D."""
    h = p.h
    D = p.D.copy()
    c = ph[1:-1, 1:-1, 1:-1]
    gx = (ph[1:-1, 1:-1, 2:] - ph[1:-1, 1:-1, :-2]) / (2 * h)
    gy = (ph[1:-1, 2:, 1:-1] - ph[1:-1, :-2, 1:-1]) / (2 * h)
    gz = (ph[2:, 1:-1, 1:-1] - ph[:-2, 1:-1, 1:-1]) / (2 * h)
    g = np.sqrt(gx ** 2 + gy ** 2 + gz ** 2)
    fl = p.eps * p.jbar
    R = np.maximum(g, fl) / np.maximum(p.sp * c, fl)
    D[1:-1, 1:-1, 1:-1] = oracle.limiter(p.limiter, R, p.larsen_n) / p.sp
    return D


def assemble(p, ph, D):
    """Dense A, b of Eq. 31 with face coefficients (D_p + D_s)/2; ghost phi in b."""
    nx, ny, nz, h = p.nx, p.ny, p.nz, p.h
    N = nx * ny * nz
    idx = lambda i, j, k: (k * ny + j) * nx + i
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
    return A, b


@pytest.mark.parametrize("limiter", ["lp", "kershaw", "larsen", "cda"])
@pytest.mark.parametrize("omega", [1.0, 0.7])
def test_one_step_is_damped_jacobi_of_the_lagged_system(limiter, omega):
    sig, alb, j, h = random_medium((4, 5, 6), seed=9)
    p = oracle.make_problem(sig, alb, j, h, limiter=limiter, omega=1.3, local_iters=2, nthreads=1)
    oracle.init_state(p)
    oracle.rb_iteration(p, 5)              # a non-trivial state
    ph = p.phi.copy()
    D = numpy_D(p, ph)
    A, b = assemble(p, ph, D)
    x = ph[1:-1, 1:-1, 1:-1].ravel()
    want = x + omega * (b - A @ x) / np.diag(A)
    p.omega = omega
    oracle.jacobi_iteration(p, 1)
    got = p.phi[1:-1, 1:-1, 1:-1].ravel()
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)
    np.testing.assert_allclose(p.D[1:-1, 1:-1, 1:-1], D[1:-1, 1:-1, 1:-1], rtol=1e-14, atol=0)
    # ghosts unchanged
    g = p.phi.copy()
    g[1:-1, 1:-1, 1:-1] = ph[1:-1, 1:-1, 1:-1]
    np.testing.assert_array_equal(g, ph)


@pytest.mark.parametrize("limiter", ["lp", "kershaw"])
def test_jacobi_reaches_dense_picard_fixed_point(limiter):
    sig, alb, j, h = random_medium((4, 4, 5), seed=2)
    ref = oracle.make_problem(sig, alb, j, h, limiter=limiter, nthreads=1)
    oracle.init_state(ref)
    want = dense_picard(ref, ref.phi)
    p = oracle.make_problem(sig, alb, j, h, limiter=limiter, nthreads=1, omega=0.9)
    oracle.init_state(p)
    for _ in range(400):
        oracle.jacobi_iteration(p, 50)
        rel = oracle.residual(p)[0]
        if rel <= 1e-13:
            break
    assert rel <= 1e-13
    err = np.abs(p.phi - want).max() / np.abs(want).max()
    assert err <= 1e-11


def test_jacobi_and_red_black_share_the_fixed_point():
    n = 10
    sig, alb = fld_inputs.cloud_medium(n, seed=4, albedo=0.9)
    h = 1.0 / n
    q = oracle.bake_directional(sig, alb, h, (0, 0, -1), 1.0)
    rb = oracle.make_problem(sig, alb, q, h, omega=1.5, local_iters=2)
    oracle.init_state(rb)
    it, rel, _ = oracle.solve(rb, tol=1e-12, max_iters=200000, check_every=20)
    assert rel <= 1e-12
    jp = oracle.make_problem(sig, alb, q, h, omega=1.0)
    oracle.init_state(jp)
    for _ in range(2000):
        oracle.jacobi_iteration(jp, 100)
        relj = oracle.residual(jp)[0]
        if relj <= 1e-12:
            break
    assert relj <= 1e-12
    err = np.linalg.norm(jp.phi - rb.phi) / np.linalg.norm(rb.phi)
    assert err <= 1e-10
