"""The GPU's Knudsen -> limiter -> D chain (Eq. 33-35) against the stored
60-digit evaluations of Table 2 (tests/golden/table2_limiters.txt).

A 1 x 1 x (2m - 1) column with h = 1/2, sigma' = 1 and phi = 1 everywhere
except the x-ghosts of red cell 2k, set to 1 and 1 + R_k: that cell's central
difference (Eq. 34) is R_k along x and 0 along y and z, so its Knudsen number
is R_k and the D it stores in the red pass of one iteration (one local round,
omega = 1) is F(R_k).  Every precision family is checked: FP64 to the table's
1e-13, the float-float pass (IEEE quotients, expf, powf) to 2e-6, and the
FP32 and hi/lo passes (approximate quotients, __expf, __powf: a few ulp each,
a few more where 1 - 1/R cancels just above R = 1) to 4e-6.  A wrong term of
a limiter or of the gradient moves D by far more.  The same column drives
the oracle's CPU-side pin of this chain.
"""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

fld = pytest.importorskip("paper_1403_8105_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_limiters.txt")


def _rows():
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            kind, n, R, F = line.split()
            yield kind, float(n), float(R), float(F)


ROWS = list(_rows())
COLUMN_R = sorted({r[2] for r in ROWS})


def column_state(Rs):
    nz = 2 * len(Rs) - 1
    phi = np.ones((nz + 2, 3, 3))
    D = np.ones((nz + 2, 3, 3))
    for k, R in enumerate(Rs):
        phi[2 * k + 1, 1, 2] = 1.0 + R            # entry k -> red cell 2k (padded K = 2k + 1)
    return phi, D


def expected(kind, n):
    table = {r[2]: r[3] for r in ROWS if r[0] == kind and (kind != "larsen" or r[1] == n)}
    return np.array([table[R] for R in COLUMN_R])


KINDS = [("cda", 2.0), ("sum", 2.0), ("max", 2.0), ("kershaw", 2.0), ("larsen", 1.0), ("larsen", 2.0),
         ("larsen", 3.0), ("larsen", 4.5), ("lp", 2.0)]


@pytest.mark.parametrize("precision,rtol,bf16", [("fp64", 1e-13, 0), ("fp32", 4e-6, 0), ("fp32", 4e-6, 1),
                                                 ("pair", 4e-6, 0), ("mixed", 2e-6, 0)])
@pytest.mark.parametrize("kind,n", KINDS)
def test_red_pass_D_matches_golden(kind, n, precision, rtol, bf16):
    phi, D = column_state(COLUMN_R)
    nz = phi.shape[0] - 2
    with fld.Grid(1, 1, nz, 0.5) as g:
        g.set_medium(np.ones((nz, 1, 1), np.float32), np.zeros((nz, 1, 1), np.float32))
        g.set_source(np.zeros((nz, 1, 1), np.float32))
        g.set_state(phi, D)
        g.iterate(fld.params(limiter=kind, larsen_n=n, precision=precision, omega=1.0, local_iters=1,
                             warm_start=1, medium_bf16=bf16), 1)
        _, Dg = g.get_state()
    got = Dg[1:-1:2, 1, 1]
    want = expected(kind, n)
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=rtol, atol=0)


@pytest.mark.parametrize("kind,n", KINDS)
def test_fp64_red_pass_equals_oracle(kind, n):
    # the same state through the oracle's red pass: every stored D of the column
    phi, D = column_state(COLUMN_R)
    nz = phi.shape[0] - 2
    shape = (nz, 1, 1)
    ref = oracle.make_problem(np.ones(shape, np.float32), np.zeros(shape, np.float32), np.zeros(shape), 0.5,
                              limiter=kind, larsen_n=n, omega=1.0, local_iters=1, nthreads=1)
    ref.phi, ref.D = phi.copy(), D.copy()
    oracle.colour_pass(ref, 0)
    with fld.Grid(1, 1, nz, 0.5) as g:
        g.set_medium(np.ones(shape, np.float32), np.zeros(shape, np.float32))
        g.set_source(np.zeros(shape, np.float32))
        g.set_state(phi, D)
        # the red pass alone: one iteration, then compare only the red cells' D
        g.iterate(fld.params(limiter=kind, larsen_n=n, precision="fp64", omega=1.0, local_iters=1,
                             warm_start=1), 1)
        _, Dg = g.get_state()
    np.testing.assert_allclose(Dg[1:-1:2, 1, 1], ref.D[1:-1:2, 1, 1], rtol=1e-13, atol=0)
