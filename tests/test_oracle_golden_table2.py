"""The oracle's flux limiters against the stored 60-digit evaluations of
Table 2's closed forms (tests/golden/table2_limiters.txt, written by the
script beside it from the formulas alone).  Unlike the multiprecision test in
test_oracle_limiters.py this needs no mpmath at run time and also covers
Larsen-n for n = 1, 3 and 4.5."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_limiters.txt")


def _rows():
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            kind, n, R, F = line.split()
            yield kind, float(n), float(R), float(F)


ROWS = list(_rows())


def test_table_covers_every_limiter_and_both_limits():
    kinds = {r[0] for r in ROWS}
    assert kinds == {"cda", "sum", "max", "kershaw", "larsen", "lp"}
    assert {r[1] for r in ROWS if r[0] == "larsen"} == {1.0, 2.0, 3.0, 4.5}
    Rs = [r[2] for r in ROWS]
    assert min(Rs) == 0.0 and max(Rs) >= 1e15
    # Eq. 19 in the stored values themselves: 1/3 at R = 0, R F -> 1 at the largest R
    for kind, n, R, F in ROWS:
        if R == 0.0:
            assert F == pytest.approx(1.0 / 3.0, rel=1e-15)
        if R >= 1e15 and kind != "cda":
            assert R * F == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("kind", ["cda", "sum", "max", "kershaw", "larsen", "lp"])
def test_oracle_limiter_matches_golden(kind):
    rows = [r for r in ROWS if r[0] == kind]
    assert rows
    for _, n, R, want in rows:
        got = oracle.limiter(kind, R, larsen_n=n if kind == "larsen" else 2.0)
        assert abs(got - want) <= 5e-14 * abs(want), (kind, n, R, got, want)


def test_larsen_one_is_the_sum_limiter():
    # Larsen-1 reduces to the sum limiter: (3 + R)^(-1).
    by_key = {(k, n, R): F for k, n, R, F in ROWS}
    for (k, n, R), F in by_key.items():
        if k == "larsen" and n == 1.0:
            assert F == by_key[("sum", 0.0, R)]


# ---------------------------------------------------------------------------
# The whole Knudsen -> limiter -> D chain (Eq. 33-35) of one red pass against
# the same table: a 1 x 1 x (2m - 1) column with h = 1/2, sigma' = 1 and
# phi = 1 everywhere except the x-ghosts of red cell k, set to 1 and 1 + R_k.
# The central difference (Eq. 34) of that cell is then ((1 + R_k) - 1) / (2h)
# = R_k along x and 0 along y and z (both neighbours 1), so its Knudsen number is
# R_k / (sigma' phi_p) = R_k, and the stored D after the red pass with one
# local round is F(R_k) / sigma' = F(R_k).  A dropped 1/(2h), a wrong
# neighbour or a limiter mix-up moves D off the table.
# ---------------------------------------------------------------------------

COLUMN_R = sorted({r[2] for r in ROWS})


def column_state(Rs):
    m = len(Rs)
    nz = 2 * m - 1
    phi = np.ones((nz + 2, 3, 3))
    D = np.ones((nz + 2, 3, 3))
    for k, R in enumerate(Rs):
        phi[2 * k + 1, 1, 2] = 1.0 + R            # entry k -> red cell 2k (padded K = 2k + 1)
    return phi, D


def expected(kind, n):
    table = {(r[2]): r[3] for r in ROWS if r[0] == kind and (kind != "larsen" or r[1] == n)}
    return np.array([table[R] for R in COLUMN_R])


@pytest.mark.parametrize("kind,n", [("cda", 2.0), ("sum", 2.0), ("max", 2.0), ("kershaw", 2.0), ("larsen", 1.0),
                                    ("larsen", 2.0), ("larsen", 3.0), ("larsen", 4.5), ("lp", 2.0)])
def test_oracle_red_pass_D_matches_golden(kind, n):
    phi, D = column_state(COLUMN_R)
    nz = phi.shape[0] - 2
    shape = (nz, 1, 1)
    p = oracle.make_problem(np.ones(shape, np.float32), np.zeros(shape, np.float32), np.zeros(shape), 0.5,
                            limiter=kind, larsen_n=n, omega=1.0, local_iters=1, nthreads=1)
    p.phi, p.D = phi, D
    oracle.colour_pass(p, 0)
    got = p.D[1:-1:2, 1, 1]
    want = expected(kind, n)
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)
    # the black cells' D was not touched by the red pass
    assert np.all(p.D[2:-1:2, 1, 1] == 1.0)
