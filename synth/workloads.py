"""The paper's workloads as seeded synthetic stand-ins (input recipes only).

The paper's own images (the DIC Challenge 2.0 Star5 set, the 32000 x 32000
Cu SEM pair, its radial-stretch renders) are not available, so each workload
below is a synthetic speckle pair with the sizes, bit depths, subset settings
and kind of deformation of the paper's cases (Sec. 3, Sec. 4, Sec. 5).
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

from . import ImageSpec, Speckle, affine_field, sine_field, FIELD_AFFINE

SEED_BASE = 12941


@dataclass(frozen=True)
class Workload:
    name: str
    width: int
    height: int
    dtype: str            # "u8" | "u16" | "f32" | "f64"
    ref: ImageSpec
    deformed: ImageSpec
    subset_size: int
    subset_step: int
    shape: str            # "rigid" | "affine" | "quadratic"
    seeds: tuple          # ((x, y), ...) in pixels; snapped to the grid by the library
    search_radius: int
    precision: str = "mixed"   # "fp64" | "mixed"

    @property
    def field(self):
        return self.deformed.field


def _pair(seed, dtype, gray_max, speckle_kw, fld, noise_frac):
    sp = Speckle(seed=seed, **speckle_kw)
    noise = noise_frac * gray_max
    return (ImageSpec(sp, gray_max=gray_max, noise=noise, noise_tag=1),
            ImageSpec(sp, field=fld, gray_max=gray_max, noise=noise, noise_tag=2))


# 2000 dots on 256^2 px, sigma in [1.5, 3) px
OPTICAL = dict(density=2000.0 / (256.0 * 256.0), sigma=(1.5, 3.0), cell=16)
# SEM-like: 0.5-1.5 px dots at 0.15 dots/px^2 (the same coverage as OPTICAL)
SEM = dict(density=0.15, sigma=(0.5, 1.5), cell=8)


def affine_256_u8() -> Workload:
    """256x256 u8 pair, u = 2.35, v = -1.70 px, exx = 1e-3, eyy = -5e-4, exy = 2e-4
    (symmetric shear) about the image centre; subset 21, step 5, affine; one seed."""
    W = H = 256
    fld = affine_field(W, H, u0=2.35, v0=-1.70, exx=1e-3, exy=2e-4, eyx=2e-4, eyy=-5e-4)
    ref, dfm = _pair(SEED_BASE + 1, "u8", 255.0, OPTICAL, fld, 0.0)
    return Workload("affine_256_u8", W, H, "u8", ref, dfm, 21, 5, "affine", ((125, 125),), 8,
                    precision="fp64")


def sine_2048_u16(width=2048, height=2048) -> Workload:
    """12-bit u16 pair, v = 0.5 sin(2 pi y / T(x)), T from 10 to 300 px across x,
    1% noise; subset 31, step 2, quadratic; seed at the centre."""
    W, H = width, height
    fld = sine_field(W, 0.5, 10.0, 300.0)
    ref, dfm = _pair(SEED_BASE + 2, "u16", 4095.0, OPTICAL, fld, 0.01)
    r = 15
    cx = r + 2 * ((W // 2 - 1 - r) // 2)
    cy = r + 2 * ((H // 2 - 1 - r) // 2)
    return Workload("sine_%d_u16" % W, W, H, "u16", ref, dfm, 31, 2, "quadratic", ((cx, cy),), 4)


def gigapixel_u8(size=32768) -> Workload:
    """size^2 u8 SEM-like pair (32768^2 is 1.07 Gpx): affine field plus a 0.8 px
    slip along the diagonal; subset 41, step 10, affine; 16 seeds at the centres
    of a 4x4 block grid; search radius 32."""
    W = H = size
    fld = affine_field(W, H, u0=3.3, v0=-1.2, exx=5e-4, exy=1e-4, eyx=1e-4, eyy=-2e-4, jump=0.8)
    ref, dfm = _pair(SEED_BASE + 3, "u8", 255.0, SEM, fld, 0.01)
    b = size // 4
    seeds = tuple((b // 2 + i * b, b // 2 + j * b) for j in range(4) for i in range(4))
    return Workload("gigapixel_%d_u8" % size, W, H, "u8", ref, dfm, 41, 10, "affine", seeds, 32)


def sequence_frame(k, n_frames=200, width=4096, height=3000, subset_size=21, shape="affine",
                   max_strain=2e-2, nu=0.3) -> Workload:
    """Frame k of an incremental uniaxial sequence: u = e_k X', v = -nu e_k Y' with
    e_k ramping linearly to max_strain at the last frame; 1% noise; step 10."""
    e = max_strain * k / (n_frames - 1)
    fld = affine_field(width, height, exx=e, eyy=-nu * e)
    sp = Speckle(seed=SEED_BASE + 4, **OPTICAL)
    G = 65535.0
    ref = ImageSpec(sp, gray_max=G, noise=0.01 * G, noise_tag=1000)
    dfm = ImageSpec(sp, field=fld, gray_max=G, noise=0.01 * G, noise_tag=1000 + k)
    return Workload("sequence_%dx%d_u16_f%d" % (width, height, k), width, height, "u16", ref, dfm,
                    subset_size, 10, shape, ((width // 2, height // 2),), 8)


@dataclass(frozen=True)
class ServingJob:
    """One request of a serving stream: a pair of a pooled reference and its own
    deformed image, with the job's own subset settings."""
    index: int
    arrival_s: float
    ref_index: int
    workload: Workload


def serving_stream(n_jobs=500, rate=20.0, pool=8, side=(512, 16384), seed=SEED_BASE + 5):
    """Poisson arrivals at ``rate`` jobs/s. References come from a pool of ``pool``
    square speckle images (side log-uniform in ``side``, u8 or u16 with p = 1/2,
    1% noise); each job draws one with repeats, an odd subset size in [15, 61], a
    step in 1..10, the affine or quadratic shape (p = 1/2), and a random affine
    field about the centre with |u| <= 5 px and strains up to 1e-2 in magnitude;
    one seed at the centre, search radius 8."""
    rng = np.random.default_rng(seed)
    refs = []
    for i in range(pool):
        s = int(round(float(np.exp(rng.uniform(np.log(side[0]), np.log(side[1]))))))
        dtype = "u8" if rng.random() < 0.5 else "u16"
        refs.append((s, dtype, 255.0 if dtype == "u8" else 65535.0, Speckle(seed=seed * 100 + i, **OPTICAL)))
    t = 0.0
    jobs = []
    for j in range(n_jobs):
        t += float(rng.exponential(1.0 / rate))
        i = int(rng.integers(pool))
        s, dtype, G, sp = refs[i]
        S = 2 * int(rng.integers(7, 31)) + 1
        step = int(rng.integers(1, 11))
        shape = "affine" if rng.random() < 0.5 else "quadratic"
        u0, v0 = (float(a) for a in rng.uniform(-3.5, 3.5, size=2))
        exx, exy, eyx, eyy = (float(a) for a in rng.uniform(-1e-2, 1e-2, size=4))
        fld = affine_field(s, s, u0=u0, v0=v0, exx=exx, exy=exy, eyx=eyx, eyy=eyy)
        ref = ImageSpec(sp, gray_max=G, noise=0.01 * G, noise_tag=1)
        dfm = ImageSpec(sp, field=fld, gray_max=G, noise=0.01 * G, noise_tag=100 + j)
        w = Workload("serve_%d_ref%d_%d_%s" % (j, i, s, dtype), s, s, dtype, ref, dfm, S, step, shape,
                     ((s // 2, s // 2),), 8)
        jobs.append(ServingJob(j, t, i, w))
    return jobs


def scaled(w: Workload, **kw) -> Workload:
    return replace(w, **kw)
