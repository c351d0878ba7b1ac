"""How far an iterate at relative residual 1e-6 is from the fixed point.

The solves of the heterogeneous clouds stop at R/jbar <= 1e-6 (Eq. 37 with
fresh D), while parity is stated on phi against the fixed point phi*.  The
oracle's own iterate at its first check with rel <= 1e-6 is compared here with
its phi* (rel <= 1e-11, the FP64 floor being far lower) on the clouds the GPU
fixed-point parity tests use.  Measured: relative L2 error 7e-8 to 4.3e-7
(omega 1.7 and 1.0), far below the 1e-5 the single-precision solves are held
to, so those tests stop at the solve target 1e-6 itself and need no tighter
stop.  Per element, relative to max(|phi*|, 1e-3 max|phi*|), the error reaches
5e-5 in the dimmest cells at omega 1.0; the bound below is 1e-4.
"""
import numpy as np
import pytest

import fld_inputs
import oracle

INNER = (slice(1, -1),) * 3


@pytest.mark.parametrize("shape,omega,check_every", [((23, 17, 29), 1.7, 1), ((23, 17, 29), 1.0, 1),
                                                     ((24, 24, 24), 1.7, 4)])
def test_iterate_at_1e6_is_within_1e5_of_fixed_point(shape, omega, check_every):
    nz, ny, nx = shape
    sig, alb = fld_inputs.cloud_medium(nx, seed=11, albedo=0.95, ny=ny, nz=nz)
    h = 1.0 / max(shape)
    q = oracle.bake_directional(sig, alb, h, (0, 0, -1), 1.0)
    p = oracle.make_problem(sig, alb, q, h, limiter="lp", omega=omega, local_iters=2)
    oracle.init_state(p)
    _, rel6, _ = oracle.solve(p, tol=1e-6, max_iters=400000, check_every=check_every)
    assert rel6 <= 1e-6
    phi6 = p.phi.copy()
    _, rel_star, _ = oracle.solve(p, tol=1e-11, max_iters=400000, check_every=20)
    assert rel_star <= 1e-11
    a, b = phi6[INNER], p.phi[INNER]
    l2 = np.linalg.norm(a - b) / np.linalg.norm(b)
    per_el = (np.abs(a - b) / np.maximum(np.abs(b), 1e-3 * np.abs(b).max())).max()
    assert l2 <= 1e-6, l2
    assert per_el <= 1e-4, per_el
