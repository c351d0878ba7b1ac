"""Seeded synthetic inputs for the FLD solver and its oracle.

This module only builds input fields (extinction sigma_t, albedo, emission j)
and light descriptions.  It holds none of the method's arithmetic: no flux
limiter, no stencil, no transmittance march.  Both the CUDA path and the FP64
oracle consume the FP32 arrays it returns, so neither side needs a twin of the
generator.

Array convention: numpy float32 of shape (nz, ny, nx), x fastest (C order),
voxel (i, j, k) centred at ((i + 1/2) h, (j + 1/2) h, (k + 1/2) h) on a grid of
spacing h.

The paper's datasets (Nebulae 200^3, MANIX CT, explosion) are not available;
its CPU testbed was a spherical cloud embedded in vacuum, driven by Perlin
noise (Sec. 5).  The fBm sphere cloud below stands in for
those workloads.  The paper does not define its noise, so the definition here
is this project's own:

  * lattice value noise: each integer lattice point (ix, iy, iz) of octave o
    gets a value in [0, 1) from a 64-bit SplitMix64-style finaliser of
    (seed, o, ix, iy, iz); values between lattice points are blended with the
    quintic fade t^3 (t (6 t - 15) + 10) along each axis (trilinear blend of
    the 8 corners);
  * fBm: 5 octaves, base frequency 4, lacunarity 2, gain 1/2, normalised by
    the sum of the octave amplitudes so the result lies in [0, 1];
  * evaluated in FP64 at voxel centres of the unit cube;
  * sigma_t = scale * max(0, fbm - threshold)^1.5 inside a sphere of radius
    0.45 about (1/2, 1/2, 1/2), and 0 (vacuum) outside; rounded to FP32.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "fbm_noise",
    "cloud_medium",
    "point_source_medium",
    "PointSource",
    "Light",
    "cloud_case",
    "batch_cases",
]

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _mix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014), uint64 -> uint64."""
    x = x.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        x ^= x >> np.uint64(30)
        x *= np.uint64(0xBF58476D1CE4E5B9)
        x ^= x >> np.uint64(27)
        x *= np.uint64(0x94D049BB133111EB)
        x ^= x >> np.uint64(31)
    return x


def _lattice(seed: int, octave: int, nx: int, ny: int, nz: int) -> np.ndarray:
    """Hash values in [0, 1) on the integer lattice [0, nx) x [0, ny) x [0, nz)."""
    ix = np.arange(nx, dtype=np.uint64)[None, None, :]
    iy = np.arange(ny, dtype=np.uint64)[None, :, None]
    iz = np.arange(nz, dtype=np.uint64)[:, None, None]
    with np.errstate(over="ignore"):
        key = (_mix64(np.array([seed], dtype=np.uint64))[0] * np.uint64(0x9E3779B97F4A7C15)
               + np.uint64(octave) * np.uint64(0xD1B54A32D192ED03))
        h = (ix * np.uint64(0x8CB92BA72F3D8DD7)) ^ (iy * np.uint64(0xC2B2AE3D27D4EB4F)) \
            ^ (iz * np.uint64(0x165667B19E3779F9)) ^ key
    h = _mix64(h)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _fade(t: np.ndarray) -> np.ndarray:
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def _axis(n: int, h: float, freq: float):
    u = (np.arange(n, dtype=np.float64) + 0.5) * h * freq
    i0 = np.floor(u).astype(np.int64)
    w = _fade(u - i0)
    return i0, w


def fbm_noise(nx: int, ny: int, nz: int, h: float, seed: int, octaves: int = 5,
              base_freq: float = 4.0, lacunarity: float = 2.0, gain: float = 0.5) -> np.ndarray:
    """fBm value noise in [0, 1] at the voxel centres, FP64, shape (nz, ny, nx)."""
    out = np.zeros((nz, ny, nx), dtype=np.float64)
    amp, amp_sum, freq = 1.0, 0.0, base_freq
    for o in range(octaves):
        ix0, wx = _axis(nx, h, freq)
        iy0, wy = _axis(ny, h, freq)
        iz0, wz = _axis(nz, h, freq)
        lat = _lattice(seed, o, int(ix0.max()) + 2, int(iy0.max()) + 2, int(iz0.max()) + 2)
        acc = np.zeros_like(out)
        for cz in (0, 1):
            fz = (wz if cz else 1.0 - wz)[:, None, None]
            for cy in (0, 1):
                fy = (wy if cy else 1.0 - wy)[None, :, None]
                for cx in (0, 1):
                    fx = (wx if cx else 1.0 - wx)[None, None, :]
                    vals = lat[np.ix_(iz0 + cz, iy0 + cy, ix0 + cx)]
                    acc += fz * fy * fx * vals
        out += amp * acc
        amp_sum += amp
        amp *= gain
        freq *= lacunarity
    return out / amp_sum


def cloud_medium(n: int, seed: int, albedo: float, *, scale: float = 200.0,
                 threshold: float = 0.35, radius: float = 0.45, ny: int | None = None,
                 nz: int | None = None):
    """fBm sphere cloud on the unit cube (h = 1/max extent).

    Returns (sigma_t, albedo) as float32 arrays of shape (nz, ny, nx).
    """
    nx = n
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    h = 1.0 / max(nx, ny, nz)
    f = fbm_noise(nx, ny, nz, h, seed)
    sig = scale * np.maximum(0.0, f - threshold) ** 1.5
    x = (np.arange(nx) + 0.5) * h - 0.5
    y = (np.arange(ny) + 0.5) * h - 0.5
    z = (np.arange(nz) + 0.5) * h - 0.5
    r2 = z[:, None, None] ** 2 + y[None, :, None] ** 2 + x[None, None, :] ** 2
    sig[r2 > radius * radius] = 0.0
    alb = np.full((nz, ny, nx), albedo, dtype=np.float32)
    return sig.astype(np.float32), alb


@dataclasses.dataclass
class PointSource:
    """A unit-power point source modelled as one emitting voxel (Sec. 6.1)."""
    n: int
    h: float
    sigma_t: np.ndarray
    albedo: np.ndarray
    j: np.ndarray
    centre: tuple  # (i, j, k) of the emitting voxel
    power: float


def point_source_medium(n: int, sigma_t: float = 10.0, sigma_s: float = 9.0,
                        power: float = 1.0, centre=None) -> PointSource:
    """Homogeneous cube with one emitting voxel, j = power / h^3 there.

    The emitting voxel is (n // 2, n // 2, n // 2) unless given; on odd n it is
    the geometric centre of the unit cube.
    """
    h = 1.0 / n
    sig = np.full((n, n, n), sigma_t, dtype=np.float32)
    alb = np.full((n, n, n), sigma_s / sigma_t, dtype=np.float32)
    j = np.zeros((n, n, n), dtype=np.float32)
    c = (n // 2, n // 2, n // 2) if centre is None else tuple(centre)
    j[c[2], c[1], c[0]] = power / h ** 3
    return PointSource(n=n, h=h, sigma_t=sig, albedo=alb, j=j, centre=c, power=power)


@dataclasses.dataclass
class Light:
    """Directional light (propagation direction `dir`, radiance L) or point light."""
    kind: str                 # "directional" | "point"
    dir: tuple = (0.0, 0.0, -1.0)
    radiance: float = 1.0
    pos: tuple = (0.5, 0.5, 1.5)
    power: float = 1.0


@dataclasses.dataclass
class Case:
    name: str
    n: int
    h: float
    seed: int
    albedo: float
    sigma_t: np.ndarray
    alb: np.ndarray
    light: Light


def cloud_case(n: int, seed: int = 0, albedo: float = 0.95, light: Light | None = None,
               name: str | None = None) -> Case:
    """One heterogeneous cloud solve: fBm medium lit by a unit directional
    light travelling along -z (step h/2 for the transmittance march)."""
    sig, alb = cloud_medium(n, seed, albedo)
    if light is None:
        light = Light(kind="directional", dir=(0.0, 0.0, -1.0), radiance=1.0)
    return Case(name=name or f"cloud{n}_s{seed}", n=n, h=1.0 / n, seed=seed, albedo=albedo,
                sigma_t=sig, alb=alb, light=light)


def batch_cases(count: int = 64, seed: int = 1234,
                sizes=(32, 48, 64, 96, 128, 160)):
    """Independent solves of uneven size: edge drawn uniformly from `sizes`,
    per-solve fBm seed, albedo ~ U[0.8, 0.99], point or directional light
    chosen by seed.  Returns a list of Case (media are generated lazily by
    the caller through `materialise`)."""
    rng = np.random.default_rng(seed)
    specs = []
    for b in range(count):
        n = int(rng.choice(sizes))
        s = int(rng.integers(0, 2 ** 31 - 1))
        a = float(rng.uniform(0.8, 0.99))
        if rng.integers(0, 2) == 0:
            th = rng.uniform(0.0, 0.35 * np.pi)
            ph = rng.uniform(0.0, 2.0 * np.pi)
            d = (float(np.sin(th) * np.cos(ph)), float(np.sin(th) * np.sin(ph)), -float(np.cos(th)))
            light = Light(kind="directional", dir=d, radiance=1.0)
        else:
            p = (float(rng.uniform(0.1, 0.9)), float(rng.uniform(0.1, 0.9)), float(rng.uniform(1.05, 1.5)))
            light = Light(kind="point", pos=p, power=4.0 * np.pi * float(np.sum((np.array(p) - 0.5) ** 2)))
        specs.append(dict(n=n, seed=s, albedo=a, light=light))
    return specs


@dataclasses.dataclass
class Scene:
    """A synthetic stand-in for one of the paper's rendered datasets."""
    name: str
    sigma_t: np.ndarray           # (nz, ny, nx) float32
    albedos: list                 # one (nz, ny, nx) float32 albedo per colour channel
    emission: np.ndarray | None   # (nz, ny, nx) float32 self-emission j, or None
    h: float
    light_dir: tuple              # direction the light travels
    light_radiance: float


def paper_scene(name: str) -> Scene:
    """Stand-ins for the paper's three rendered datasets, with their grid
    shapes (Sec. 6.2): "nebulae" -- 200^3, albedo 0.9, one directional light;
    "manix" -- 256 x 329 x 256 (x, y, z), extinction and a per-channel (RGB)
    albedo from one density via a transfer function; "explosion" -- 201 x
    272 x 230, albedo 1, a black-body-like emission field from a second noise
    field ("temperature", j ~ T^4 where hot) plus the light.  The densities
    are fBm sphere clouds (cloud_medium); the light comes from above."""
    light = (0.25, -1.0, -0.35)
    if name == "nebulae":
        sig, alb = cloud_medium(200, seed=11, albedo=0.9)
        return Scene(name, sig, [alb], None, 1.0 / 200, light, 1.0)
    if name == "manix":
        nx, ny, nz = 256, 329, 256
        sig, _ = cloud_medium(nx, seed=12, albedo=1.0, ny=ny, nz=nz)
        d = sig / max(float(sig.max()), 1e-30)                 # density in [0, 1]
        # transfer function: dense "bone" scatters white, thin "tissue" reddish
        base = ((0.97, 0.25), (0.85, 0.45), (0.75, 0.6))         # (albedo at d = 0, drop to d = 1) per channel
        albs = [np.clip(a0 - drop * (1.0 - d) * (d > 0), 0.0, 1.0).astype(np.float32) for a0, drop in base]
        return Scene(name, sig, albs, None, 1.0 / ny, light, 1.0)
    if name == "explosion":
        nx, ny, nz = 201, 272, 230
        sig, alb = cloud_medium(nx, seed=13, albedo=1.0, ny=ny, nz=nz)
        temp = fbm_noise(nx, ny, nz, 1.0 / ny, seed=14)
        j = (40.0 * np.maximum(0.0, temp - 0.55) ** 4 / 0.45 ** 4) * (sig > 0)
        return Scene(name, sig, [alb], j.astype(np.float32), 1.0 / ny, light, 1.0)
    raise ValueError(f"unknown scene {name!r}")
