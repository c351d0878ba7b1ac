"""Pins of the oracle's flux limiters (Table 2) against what the paper fixes:
the limits of Eq. 19, the constraint F <= 1/R of Eq. 17, and independent
high-precision evaluations of the tabulated closed forms."""
import numpy as np
import pytest

import oracle

FLD = ["sum", "max", "kershaw", "larsen", "lp"]


@pytest.mark.parametrize("kind", FLD + ["cda"])
def test_diffusive_limit_is_one_third(kind):
    # Eq. 19: F -> 1/3 as R -> 0 (every tabulated form deviates by O(R) at most).
    assert abs(oracle.limiter(kind, 0.0) - 1.0 / 3.0) < 1e-16
    for R in (1e-12, 1e-8, 1e-4):
        assert abs(oracle.limiter(kind, R) - 1.0 / 3.0) <= R / 9.0 + 1e-16


@pytest.mark.parametrize("kind", FLD)
def test_transport_limit_R_F_to_one(kind):
    # Eq. 19: R F(R) -> 1 as R -> infinity.
    for R, tol in ((1e4, 2e-3), (1e8, 1e-7), (1e20, 1e-15)):
        assert abs(R * oracle.limiter(kind, R) - 1.0) < tol


@pytest.mark.parametrize("kind", FLD)
def test_flux_limiting_constraint_and_monotone(kind):
    # Eq. 17: F <= 1/R for every R; and F never increases with R.
    R = np.logspace(-12, 25, 4000)
    F = oracle.limiter(kind, R)
    assert np.all(R * F <= 1.0 + 4e-16)
    assert np.all(np.diff(F) <= 1e-16 * F[:-1])
    assert np.all(F > 0)


def test_cda_is_constant():
    R = np.logspace(-10, 10, 50)
    assert np.all(oracle.limiter("cda", R) == 1.0 / 3.0)


def test_max_limiter_continuous_at_3():
    a = oracle.limiter("max", 3.0 - 1e-12)
    b = oracle.limiter("max", 3.0 + 1e-12)
    assert abs(a - b) < 1e-12


def test_larsen_n2_equals_inverse_hypot():
    # Larsen-2: (9 + R^2)^(-1/2).
    R = np.logspace(-6, 6, 200)
    F = oracle.limiter("larsen", R, larsen_n=2.0)
    assert np.allclose(F, 1.0 / np.hypot(3.0, R), rtol=1e-14, atol=0)


def test_larsen_large_n_tends_to_max():
    # (3^n + R^n)^(-1/n) -> 1/max(3, R) as n -> infinity.
    R = np.array([0.1, 1.0, 2.0, 5.0, 50.0])
    F = oracle.limiter("larsen", R, larsen_n=200.0)
    assert np.allclose(F, 1.0 / np.maximum(3.0, R), rtol=6e-3)


def test_lp_small_R_series_branch_is_continuous():
    # The series branch (R < 0.2) and the closed form meet without a jump.
    lo = oracle.limiter("lp", np.nextafter(0.2, 0.0))
    hi = oracle.limiter("lp", 0.2)
    assert abs(lo - hi) < 1e-15


@pytest.mark.parametrize("kind", FLD)
def test_against_multiprecision(kind):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50

    def ref(R):
        R = mp.mpf(R)
        if kind == "sum":
            return 1 / (3 + R)
        if kind == "max":
            return 1 / max(mp.mpf(3), R)
        if kind == "kershaw":
            return 2 / (3 + mp.sqrt(9 + 4 * R * R))
        if kind == "larsen":
            return (mp.mpf(3) ** 2 + R ** 2) ** (-mp.mpf(1) / 2)
        return (mp.coth(R) - 1 / R) / R

    for R in (1e-6, 1e-3, 0.05, 0.1999, 0.2, 0.5, 1.0, 3.0, 17.0, 1e3, 1e9):
        got = oracle.limiter(kind, R, larsen_n=2.0)
        want = float(ref(R))
        assert abs(got - want) <= 5e-14 * abs(want), (R, got, want)
