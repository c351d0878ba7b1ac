"""Pins of the oracle's medium preparation (Algorithm 1, first steps; Sec. 5).

Each expected value below is worked out by hand from the paper's
definitions, not by calling the oracle a second way:

* sigma' = max(sigma_t, sigma_eps): a voxel with sigma_t = 0, one just below
  and one just above the floor, and a dense voxel;
* sigma_a' = (1 - albedo) sigma': albedo 1 (pure scattering) gives exactly 0,
  albedo 0 gives sigma' itself, and the vacuum floor is scaled the same way;
* sigma_eps = 1e-3 / L with L the largest grid extent in world units: a
  40-voxel edge with h = 0.01 (L = 0.4) gives 2.5e-3, an anisotropic
  40 x 80 x 20 grid with the same h gives 1e-3 / 0.8 = 1.25e-3;
* jbar = RMS of j over the unknowns: sqrt(mean(j^2)) of a multi-voxel source
  whose value is known in closed form, which a mean, a max or a sum would
  miss.

A mistake such as sigma_eps = 1e-3 * n, a floor applied to sigma_a' instead
of sigma', sigma_a' from the raw sigma_t, or jbar as a mean of |j| fails one
of these.
"""
import numpy as np
import pytest

import oracle


def _prep(sig, alb, h=1.0, sigma_eps=None):
    sig = np.asarray(sig, np.float32).reshape(1, 1, -1)
    alb = np.asarray(alb, np.float32).reshape(1, 1, -1)
    j = np.ones(sig.shape)
    return oracle.make_problem(sig, alb, j, h, sigma_eps=sigma_eps)


def test_fp64_floor_on_sigma():
    seps = 1e-3
    below = np.float32(0.999e-3)      # just under the floor
    above = np.float32(1.001e-3)      # just over it
    p = _prep([0.0, below, above, 7.5], [0.5, 0.5, 0.5, 0.5], sigma_eps=seps)
    want_sp = [1e-3, 1e-3, float(above), 7.5]
    np.testing.assert_array_equal(p.sp.ravel(), want_sp)
    # sigma_a' = (1 - albedo) sigma' uses the floored sigma (R3)
    np.testing.assert_array_equal(p.sa.ravel(), [0.5e-3, 0.5e-3, 0.5 * float(above), 3.75])


def test_albedo_one_and_zero():
    p = _prep([0.0, 3.0, 3.0, 0.0], [1.0, 1.0, 0.0, 0.0], sigma_eps=2e-3)
    np.testing.assert_array_equal(p.sp.ravel(), [2e-3, 3.0, 3.0, 2e-3])
    np.testing.assert_array_equal(p.sa.ravel(), [0.0, 0.0, 3.0, 2e-3])


@pytest.mark.parametrize("shape,h,want", [((40, 40, 40), 0.01, 2.5e-3),
                                          ((20, 80, 40), 0.01, 1.25e-3),      # (nz, ny, nx): L = 80 h
                                          ((8, 8, 8), 0.125, 1e-3),            # unit cube
                                          ((3, 5, 250), 0.002, 2e-3)])         # L = 0.5 along x
def test_sigma_eps_default_is_1e3_over_largest_extent(shape, h, want):
    nz, ny, nx = shape
    assert oracle.sigma_eps_default(nx, ny, nz, h) == pytest.approx(want, rel=1e-15)
    # and make_problem applies it: a vacuum voxel gets sigma' = sigma_eps
    sig = np.zeros(shape, np.float32)
    sig[0, 0, 0] = 5.0
    alb = np.full(shape, 0.25, np.float32)
    p = oracle.make_problem(sig, alb, np.ones(shape), h)
    assert p.sp[0, 0, 0] == 5.0
    assert p.sp[-1, -1, -1] == pytest.approx(want, rel=1e-15)
    assert p.sa[-1, -1, -1] == pytest.approx(0.75 * want, rel=1e-15)


def test_jbar_is_rms_over_unknowns():
    # j = 3 on one voxel, 4 on another, 0 on the remaining 6 of a 2x2x2 grid:
    # RMS = sqrt((9 + 16) / 8) = 5 / sqrt(8); the mean would be 7/8, the max 4
    j = np.zeros((2, 2, 2))
    j[0, 0, 0], j[1, 1, 0] = 3.0, 4.0
    sig = np.ones((2, 2, 2), np.float32)
    alb = np.full((2, 2, 2), 0.5, np.float32)
    p = oracle.make_problem(sig, alb, j, 0.5)
    assert p.jbar == pytest.approx(5.0 / np.sqrt(8.0), rel=1e-15)
    # a linear ramp 1..n has RMS sqrt((n+1)(2n+1)/6)
    n = 60
    j = np.arange(1, n + 1, dtype=np.float64).reshape(3, 4, 5)
    p = oracle.make_problem(np.ones(j.shape, np.float32), np.zeros(j.shape, np.float32), j, 0.1)
    assert p.jbar == pytest.approx(np.sqrt((n + 1) * (2 * n + 1) / 6.0), rel=1e-14)


def test_initial_state_uses_eps_jbar_dl():
    # Algorithm 1: phi = eps jbar dl and D = eps dl everywhere, ghosts included
    j = np.zeros((2, 3, 4))
    j[1, 2, 3] = 12.0                      # RMS = 12 / sqrt(24)
    p = oracle.make_problem(np.ones(j.shape, np.float32), np.full(j.shape, 0.5, np.float32), j, 0.25)
    oracle.init_state(p)
    jbar = 12.0 / np.sqrt(24.0)
    assert p.phi.shape == (4, 5, 6)
    np.testing.assert_allclose(p.phi, oracle.EPS * jbar * 0.25, rtol=1e-15)
    np.testing.assert_allclose(p.D, oracle.EPS * 0.25, rtol=1e-15)
