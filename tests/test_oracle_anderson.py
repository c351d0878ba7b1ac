"""The reading behind Anderson mixing of sweep blocks, checked on the oracle:
a block of red-black sweeps (Algorithm 1) is a map G whose fixed point is the
solution of Eq. 31, so starting each block from an affine combination of
earlier images G(x_i) (weights summing to 1) converges to the same phi* --
here in fewer sweeps.  The mix (`oracle.solve_anderson`, numpy on top of the
oracle's own sweeps and residual) gives the reference solutions of grids
where plain SOR takes too long; here it is pinned against the plain solve.
Nothing here touches the GPU library."""
import numpy as np
import pytest

import fld_inputs
import oracle

INNER = (slice(1, -1),) * 3


def _problem(n, seed=2):
    sig, alb = fld_inputs.cloud_medium(n, seed=seed, albedo=0.95)
    h = 1.0 / n
    q = oracle.bake_directional(sig, alb, h, (0, 0, -1), 1.0)
    p = oracle.make_problem(sig, alb, q, h, omega=1.6, local_iters=2, nthreads=2)
    oracle.init_state(p)
    return p


def _anderson_solve(p, tol, sweeps_per_block=16, m=6, max_sweeps=200000):
    return oracle.solve_anderson(p, tol, sweeps_per_block=sweeps_per_block, m=m, max_sweeps=max_sweeps)


def test_mixed_sweeps_reach_the_same_fixed_point_in_fewer_sweeps():
    n = 16
    plain = _problem(n)
    it_plain, rel_plain, _ = oracle.solve(plain, tol=1e-11, max_iters=400000, check_every=16)
    assert rel_plain <= 1e-11
    mixed = _problem(n)
    it_mixed, rel_mixed = _anderson_solve(mixed, 1e-11)
    assert rel_mixed <= 1e-11
    err = np.linalg.norm(mixed.phi[INNER] - plain.phi[INNER]) / np.linalg.norm(plain.phi[INNER])
    assert err <= 1e-9, err
    assert it_mixed < it_plain, (it_mixed, it_plain)
    # the Dirichlet ghosts are untouched by the mix
    assert np.array_equal(mixed.phi[0], plain.phi[0]) and np.array_equal(mixed.phi[:, :, -1], plain.phi[:, :, -1])


@pytest.mark.parametrize("m", [1])
def test_one_slot_is_plain_sor(m):
    # with a single slot the weight is 1 and the mix returns G(x): the same
    # iterates as the unmixed sweeps, bit for bit
    n = 10
    a = _problem(n, seed=4)
    b = _problem(n, seed=4)
    _anderson_solve(a, 0.0, sweeps_per_block=8, m=m, max_sweeps=64)
    oracle.rb_iteration(b, 64)
    assert np.array_equal(a.phi, b.phi)
