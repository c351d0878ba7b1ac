"""Closed-form pins for a point source in a homogeneous medium (Sec. 4.1, 6.1).

* CDA with Dirichlet ghosts set from the analytic solution: the numerical
  fluence approaches the CDA Green's function of Eq. 27,
  phi(r) = P exp(-sigma_tr r) / (4 pi D r), D = 1/(3 sigma_t),
  sigma_tr = sqrt(sigma_a / D), with the error of a second-order scheme
  (about 4x smaller per halving of the voxel size).
* FLD near a source in an optically thin medium follows the transport
  limit of Eq. 29 (an inverse square law) while CDA does not.
"""
import numpy as np
import pytest

import fld_inputs
import oracle


def cda_green(r, sigma_t, sigma_s, P=1.0):
    D = 1.0 / (3.0 * sigma_t)
    sigma_tr = np.sqrt((sigma_t - sigma_s) / D)
    return P * np.exp(-sigma_tr * r) / (4.0 * np.pi * D * r)


def _cda_analytic_ghost_error(n):
    ps = fld_inputs.point_source_medium(n, 10.0, 9.0)
    h = ps.h
    c = np.array(ps.centre)
    p = oracle.make_problem(ps.sigma_t, ps.albedo, ps.j, h, limiter="cda", nthreads=4,
                            omega=oracle.omega_default(n, n, n))
    idx = np.arange(-1, n + 1)
    K, J, I = np.meshgrid(idx, idx, idx, indexing="ij")
    r = h * np.sqrt((I - c[0]) ** 2 + (J - c[1]) ** 2 + (K - c[2]) ** 2)
    oracle.init_state(p, phi0=0.0)
    ghost = np.ones(p.phi.shape, bool)
    ghost[1:-1, 1:-1, 1:-1] = False
    p.phi[ghost] = cda_green(r[ghost], 10.0, 9.0)
    p.D[ghost] = 1.0 / 30.0
    it, rel, _ = oracle.solve(p, tol=1e-12, max_iters=20000, check_every=10)
    assert rel <= 1e-12
    ri = r[1:-1, 1:-1, 1:-1]
    m = (ri >= 0.2) & (ri <= 0.4)
    err = p.phi[1:-1, 1:-1, 1:-1][m] / cda_green(ri[m], 10.0, 9.0) - 1.0
    return np.sqrt(np.mean(err ** 2)), np.abs(err).max()


def test_cda_matches_greens_function_second_order():
    e15 = _cda_analytic_ghost_error(15)
    e31 = _cda_analytic_ghost_error(31)
    e63 = _cda_analytic_ghost_error(63)
    assert e63[1] < 5e-3                   # close match at the finest grid
    assert e15[0] / e31[0] > 3.0 and e31[0] / e63[0] > 3.0


def _slope(limiter, n=31, sigma_t=1.0, albedo=0.5):
    ps = fld_inputs.point_source_medium(n, sigma_t, sigma_t * albedo)
    c = ps.centre
    p = oracle.make_problem(ps.sigma_t, ps.albedo, ps.j, ps.h, limiter=limiter, nthreads=4,
                            omega=1.7, local_iters=2)
    oracle.init_state(p)
    it, rel, _ = oracle.solve(p, tol=1e-10, max_iters=20000, check_every=10)
    assert rel <= 1e-10
    ks = np.arange(3, n // 2)
    r = ks * ps.h
    phi = p.phi[c[2] + 1, c[1] + 1, c[0] + 1 + ks]
    m = r <= 0.3
    return np.polyfit(np.log(r[m]), np.log(phi[m]), 1)[0]


@pytest.mark.parametrize("limiter", ["lp", "kershaw"])
def test_fld_inverse_square_near_source(limiter):
    # tau across the box = 1: near the source FLD is in the transport regime,
    # phi ~ exp(-(1-alpha) tau) / tau^2 (Eq. 29), slope about -2.
    s = _slope(limiter)
    assert -2.3 < s < -1.85, s


def test_cda_is_not_inverse_square():
    # CDA lacks the tau^-2 term (Sec. 4.1): its slope is much shallower.
    s = _slope("cda")
    assert s > -1.7, s


def test_paper_point_source_fld_close_to_cda_far_field():
    # C1-like setup (sigma_t = 10, sigma_s = 9, phi = 0 ghosts): FLD-LP and the
    # CDA closed form agree to within tens of percent at 0.15 <= r <= 0.3
    # (the paper reports only a rough match, Sec. 6.1); reported, loosely gated.
    n = 31
    ps = fld_inputs.point_source_medium(n, 10.0, 9.0)
    p = oracle.make_problem(ps.sigma_t, ps.albedo, ps.j, ps.h, limiter="lp", nthreads=4, omega=1.7,
                            local_iters=2)
    oracle.init_state(p, phi0=1e-6, phi_b=0.0)
    it, rel, _ = oracle.solve(p, tol=1e-10, max_iters=20000, check_every=10)
    assert rel <= 1e-10
    c = ps.centre
    ks = np.arange(5, 10)
    r = ks * ps.h
    phi = p.phi[c[2] + 1, c[1] + 1, c[0] + 1 + ks]
    ratio = phi / cda_green(r, 10.0, 9.0)
    assert np.all((ratio > 0.5) & (ratio < 1.5)), ratio
