"""Named synthetic workloads (sizes, parameters and seeds) for tests and the bench.

Each workload is an adaptive-optics loop of the kind the paper simulates in
Section 5 (Shack-Hartmann sensor in Fried geometry, von Karman turbulence, AR(1)
phase model with a = 0.99, noise sigma = 0.1 rad), scaled from an 8x8 toy to an
80x80 ELT-sized sensor. Only inputs live here; the estimator's arithmetic does not.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    nsub: int                 # subapertures per side
    pitch: float              # subaperture size (m)
    obscuration: float        # central obscuration ratio of the circular pupil
    square: bool              # square pupil: every subaperture valid
    m: int                    # ensemble size
    window: int               # localization window, subapertures per side
    taper: int                # 0 = box, 1 = Gaspari-Cohn on R^-1
    loc_len: float            # Gaspari-Cohn half-support c in pitches (0 = window/4)
    rho: float                # multiplicative inflation
    sigma: float              # slope noise std (rad)
    a_ar1: float              # AR(1) coefficient of the forecast model
    r0: float                 # Fried parameter (m)
    L0: float                 # outer scale (m)
    frames: int
    truth: str                # "ar1" (fresh screens) or "frozen" (frozen flow)
    precision: int            # 0 = FP32 analysis, 1 = FP64 analysis
    seeds: tuple              # (truth, slope noise, forecast-noise bank)
    px_per_pitch: int = 25    # frozen-flow screen pixels per pitch (1 px shift/frame)
    bank_count: int = 16

    @property
    def sigma2(self) -> float:
        return self.sigma * self.sigma

    @property
    def noise_std(self) -> float:
        """Scale of the forecast-noise screens, sqrt(1 - a^2) (stationary AR(1))."""
        return math.sqrt(1.0 - self.a_ar1 * self.a_ar1)


# 8x8 square pupil, m = 10, 3x3 box window, FP64 analysis, AR(1) truth.
TOY_8X8 = Workload("toy-8x8-m10-w3-fp64", nsub=8, pitch=0.5, obscuration=0.0, square=True,
                   m=10, window=3, taper=0, loc_len=0.0, rho=1.05, sigma=0.1, a_ar1=0.99,
                   r0=0.15, L0=25.0, frames=100, truth="ar1", precision=1, seeds=(11, 12, 13))

# 16 m telescope: 32x32, obscuration 0.14, m = 24, 5x5 Gaspari-Cohn window, frozen flow 10 m/s.
TEL_16M = Workload("16m-32x32-m24-w5gc-fp32", nsub=32, pitch=0.5, obscuration=0.14,
                   square=False, m=24, window=5, taper=1, loc_len=0.0, rho=1.03, sigma=0.1,
                   a_ar1=0.99, r0=0.15, L0=25.0, frames=1000, truth="frozen", precision=0,
                   seeds=(21, 22, 23), px_per_pitch=25)

# ELT scale: 80x80 over 39 m, obscuration 0.14, m = 32, 7x7 box window, r0 = 0.12, L0 = 30.
# Screen spacing pitch/24 = 0.0203 m, one pixel per frame at 500 Hz (10.16 m/s).
ELT_80X80 = Workload("elt-80x80-m32-w7-fp32", nsub=80, pitch=39.0 / 80.0, obscuration=0.14,
                     square=False, m=32, window=7, taper=0, loc_len=0.0, rho=1.02, sigma=0.1,
                     a_ar1=0.99, r0=0.12, L0=30.0, frames=1000, truth="frozen", precision=0,
                     seeds=(31, 32, 33), px_per_pitch=24)

# Adjoint workload: the 16 m loop over 200 frames.
ADJ_16M = replace(TEL_16M, name="adjoint-16m-32x32-m24-200f", frames=200, seeds=(41, 42, 43))

# Brute-force case: 4x4 square sensor (5x5 nodes).
TINY_4X4 = Workload("tiny-4x4-m8-w3", nsub=4, pitch=0.5, obscuration=0.0, square=True, m=8,
                    window=3, taper=1, loc_len=1.0, rho=1.05, sigma=0.1, a_ar1=0.99, r0=0.15,
                    L0=25.0, frames=20, truth="ar1", precision=1, seeds=(1, 2, 3))

ALL = {w.name: w for w in (TOY_8X8, TEL_16M, ELT_80X80, ADJ_16M, TINY_4X4)}


def batched_instances(count: int = 48, seed: int = 50, frames: int = 500) -> list:
    """Many independent AO systems of different sizes: nsub ~ U{16..96},
    m ~ U{16, 24, 32, 48}, r0 ~ U(0.08, 0.2) m, pitch 0.5 m, obscuration 0.14,
    7x7 box window. Instance i uses seeds (5000+i, 6000+i, 7000+i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nsub = int(rng.integers(16, 97))
        m = int(rng.choice([16, 24, 32, 48]))
        r0 = float(rng.uniform(0.08, 0.2))
        out.append(Workload(f"inst{i}-{nsub}x{nsub}-m{m}", nsub=nsub, pitch=0.5,
                            obscuration=0.14, square=False, m=m, window=7, taper=0,
                            loc_len=0.0, rho=1.02, sigma=0.1, a_ar1=0.99, r0=r0, L0=25.0,
                            frames=frames, truth="frozen", precision=0,
                            seeds=(5000 + i, 6000 + i, 7000 + i), px_per_pitch=25))
    return out
