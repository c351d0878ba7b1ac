"""Pins of the oracle's single-scatter source q_ri = L sigma_s T (Sec. 3
after Eq. 6) with the marched transmittance of Eq. 3.

* Light along -z, step h/2: samples at quarter-voxel offsets blend the two
  nearest voxel centres 3:1 and 1:3, so the march equals the trapezoid rule
  on the voxel-centre values (an exclusive cumulative sum along z) plus half
  a voxel of the top value.
* A homogeneous medium gives T = exp(-sigma d) exactly.
* The general-direction march tends to the axis case as the direction tends
  to -z, and a distant point light tends to a directional light.
* Rotating the medium and the light together rotates q.
"""
import numpy as np

import fld_inputs
import oracle


def _medium(n=12, seed=5):
    sig, alb = fld_inputs.cloud_medium(n, seed=seed, albedo=0.9)
    rng = np.random.default_rng(seed)
    sig = (sig + rng.uniform(0, 3, sig.shape)).astype(np.float32)
    alb = rng.uniform(0.5, 1.0, sig.shape).astype(np.float32)
    return sig, alb, 1.0 / n


def test_axis_light_is_trapezoid_scan():
    sig, alb, h = _medium()
    q = oracle.bake_directional(sig, alb, h, (0, 0, -1), 2.0)
    s = sig.astype(np.float64)
    seg = 0.5 * h * (s[:-1] + s[1:])                   # trapezoid between centres k, k+1
    tail = np.cumsum(seg[::-1], axis=0)[::-1]          # sum over segments above k
    tau = np.zeros_like(s)
    tau[:-1] = tail
    tau += 0.5 * h * s[-1][None]                       # top centre to the top face
    want = 2.0 * alb.astype(np.float64) * s * np.exp(-tau)
    assert np.allclose(q, want, rtol=1e-12, atol=1e-300)


def test_homogeneous_exponential_attenuation():
    n = 10
    sig = np.full((n, n, n), 3.5, np.float32)
    alb = np.full((n, n, n), 0.5, np.float32)
    h = 1.0 / n
    q = oracle.bake_directional(sig, alb, h, (0, 0, -1), 1.0)
    d = (n - (np.arange(n) + 0.5)) * h
    want = 0.5 * 3.5 * np.exp(-3.5 * d)
    assert np.allclose(q, want[:, None, None] * np.ones((1, n, n)), rtol=1e-13)
    # the same along an oblique direction in a homogeneous medium: exp(-sigma * path length)
    w = np.array([0.3, -0.2, -1.0])
    q2 = oracle.bake_directional(sig, alb, h, tuple(w), 1.0)
    u = -w / np.linalg.norm(w)
    k, j, i = np.indices(sig.shape)
    x = np.stack([(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h], -1)
    t = np.full(sig.shape, np.inf)
    for a in range(3):
        if u[a] > 0:
            t = np.minimum(t, (1.0 - x[..., a]) / u[a])
        elif u[a] < 0:
            t = np.minimum(t, (0.0 - x[..., a]) / u[a])
    assert np.allclose(q2, 0.5 * 3.5 * np.exp(-3.5 * t), rtol=1e-12)


def test_oblique_tends_to_axis():
    sig, alb, h = _medium()
    q0 = oracle.bake_directional(sig, alb, h, (0, 0, -1), 1.0)
    errs = []
    for th in (0.004, 0.002, 0.001):
        q = oracle.bake_directional(sig, alb, h, (np.sin(th), 0, -np.cos(th)), 1.0)
        errs.append(np.abs(q - q0).max() / q0.max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 6e-3                      # first order in the angle
    assert 1.6 < errs[0] / errs[1] < 2.5


def test_distant_point_light_tends_to_directional():
    sig, alb, h = _medium(n=8)
    qd = oracle.bake_directional(sig, alb, h, (0, 0, -1), 1.0)
    errs = []
    for dist in (1e2, 1e3, 1e4):
        pos = (0.5, 0.5, 0.5 + dist)
        qp = oracle.bake_point(sig, alb, h, pos, power=1.0)
        k, j, i = np.indices(sig.shape)
        r2 = ((i + 0.5) * h - 0.5) ** 2 + ((j + 0.5) * h - 0.5) ** 2 + ((k + 0.5) * h - pos[2]) ** 2
        errs.append(np.abs(qp * 4 * np.pi * r2 - qd).max() / qd.max())
    assert errs[2] < 5e-4                         # first order in 1/distance
    assert 5 < errs[0] / errs[1] < 20 and 5 < errs[1] / errs[2] < 20


def test_rotation_equivariance():
    sig, alb, h = _medium()
    q = oracle.bake_directional(sig, alb, h, (0, 0, -1), 1.0)
    # light along -x on the medium with axes (z, y, x) -> (x, y, z) swapped
    sig_t = np.ascontiguousarray(np.transpose(sig, (2, 1, 0)))
    alb_t = np.ascontiguousarray(np.transpose(alb, (2, 1, 0)))
    q_t = oracle.bake_directional(sig_t, alb_t, h, (-1, 0, 0), 1.0)
    assert np.allclose(np.transpose(q_t, (2, 1, 0)), q, rtol=1e-12, atol=1e-300)
