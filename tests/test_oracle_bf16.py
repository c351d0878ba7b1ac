"""Pins of the oracle's bfloat16 medium (sigma' and sigma_a' stored with 8
significant bits, the reduced-precision medium of the 256^3 runs).

* The rounding is the library's: PyTorch's CPU float32 -> bfloat16
  conversion (round to nearest, ties to even) of the same single-precision
  sigma' = max(sigma_t, sigma_eps) and sigma_a' = (1 - albedo) sigma',
  including exact ties with an even and an odd kept part.
* The rounding error is at most the unit roundoff of 8 significant bits:
  2^-8 relative.
* A medium that bfloat16 already represents is left unchanged, and the
  rounded medium's solve still lands on the dense Picard fixed point.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

from test_oracle_fixed_point import dense_picard, random_medium  # noqa: E402


def torch_bf16(x32: np.ndarray) -> np.ndarray:
    return torch.from_numpy(np.ascontiguousarray(x32)).to(torch.bfloat16).to(torch.float64).numpy()


def ties_and_edges():
    # float32 bit patterns: exact ties (low 16 bits 0x8000) with even and odd
    # kept parts, values just either side of a tie, and the largest finite
    bits = np.array([0x3F808000, 0x3F818000, 0x3F807FFF, 0x3F808001, 0x41208000, 0x41218000,
                     0x3A83126F, 0x7F7F0000, 0x00808000, 0x3F800000], dtype=np.uint32)
    return bits.view(np.float32)


def test_bf16_prep_matches_library_rounding():
    rng = np.random.default_rng(11)
    n = 4096
    sig = np.concatenate([rng.uniform(0.0, 120.0, n).astype(np.float32),
                          (10.0 ** rng.uniform(-6, 6, n)).astype(np.float32), ties_and_edges(),
                          np.zeros(7, np.float32)])
    alb = rng.uniform(0.0, 1.0, sig.size).astype(np.float32)
    alb[-len(ties_and_edges()) - 7:] = 0.0            # sigma_a' = sigma' for the tie cases
    shape = (1, 1, sig.size)
    j = np.ones(shape)
    seps = 1e-3
    p = oracle.make_problem(sig.reshape(shape), alb.reshape(shape), j, 1.0, sigma_eps=seps, medium_bf16=True)
    s32 = np.maximum(sig, np.float32(seps))
    a32 = (np.float32(1.0) - alb) * s32
    assert s32.dtype == np.float32 and a32.dtype == np.float32
    np.testing.assert_array_equal(p.sp.ravel(), torch_bf16(s32))
    np.testing.assert_array_equal(p.sa.ravel(), torch_bf16(a32))
    # the tie cases really are ties, and both directions occur
    t = ties_and_edges()[:2]
    r = torch_bf16(t)
    assert r[0] == np.float32(1.0) and r[1] > t[1]


def test_bf16_error_bound_and_plain_prep_relation():
    sig, alb, j, h = random_medium((6, 5, 7), seed=3)
    p64 = oracle.make_problem(sig, alb, j, h)
    pb = oracle.make_problem(sig, alb, j, h, medium_bf16=True)
    for a, b in ((p64.sp, pb.sp), (p64.sa, pb.sa)):
        rel = np.abs(b - a) / np.where(a > 0, a, 1.0)
        assert rel.max() <= 2.0 ** -8 * (1 + 1e-6)
        assert np.any(b != a)                       # the rounding did something
    assert pb.jbar == p64.jbar                      # the source is not rounded


def test_representable_medium_is_unchanged():
    rng = np.random.default_rng(5)
    shape = (4, 5, 6)
    sig = rng.choice(np.array([0.5, 1.0, 2.0, 4.5, 10.0, 24.0], np.float32), shape)
    alb = rng.choice(np.array([0.5, 0.75, 0.875], np.float32), shape)
    j = rng.uniform(0.0, 2.0, shape)
    p64 = oracle.make_problem(sig, alb, j, 1.0 / 6, local_iters=2)
    pb = oracle.make_problem(sig, alb, j, 1.0 / 6, local_iters=2, medium_bf16=True)
    np.testing.assert_array_equal(pb.sp, p64.sp)
    np.testing.assert_array_equal(pb.sa, p64.sa)
    for q in (p64, pb):
        oracle.init_state(q)
        oracle.rb_iteration(q, 3)
    np.testing.assert_array_equal(pb.phi, p64.phi)


@pytest.mark.parametrize("limiter", ["lp", "kershaw"])
def test_rounded_medium_reaches_dense_picard_fixed_point(limiter):
    sig, alb, j, h = random_medium((4, 4, 5), seed=7)
    ref = oracle.make_problem(sig, alb, j, h, limiter=limiter, nthreads=1, medium_bf16=True)
    oracle.init_state(ref)
    want = dense_picard(ref, ref.phi)
    p = oracle.make_problem(sig, alb, j, h, limiter=limiter, nthreads=1, omega=1.6, local_iters=2,
                            medium_bf16=True)
    oracle.init_state(p)
    it, rel, _ = oracle.solve(p, tol=1e-14, max_iters=60000, check_every=5)
    assert rel <= 1e-13
    err = np.abs(p.phi - want).max() / np.abs(want).max()
    assert err <= 1e-12
