"""Named synthetic workloads (sizes, parameters and seeds) for tests and the bench.

Each workload is an adaptive-optics loop of the kind the paper simulates in
Section 5 (Shack-Hartmann sensor in Fried geometry, von Karman turbulence, AR(1)
phase model, slope noise sigma = 0.1 rad), scaled from an 8x8 toy to an
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
    q_model: float            # forecast-noise scale q; the AR(1) coefficient is sqrt(1 - q^2)
    r0: float                 # Fried parameter (m)
    L0: float                 # outer scale (m)
    frames: int
    truth: str                # "ar1" (fresh screens) or "frozen" (frozen flow)
    precision: int            # 0 = FP32 analysis, 1 = FP64 analysis
    seeds: tuple              # (truth, slope noise, forecast-noise bank)
    shift: float = 0.003      # frozen-flow displacement per frame, in pitches
    bank_count: int = 16
    partition: int = 0        # 0: per-node analysis; P: local domains of a P x P node partition
    piston: int = 0           # with a partition: differential-piston least squares
    row_split: int = 1        # FP32 per-node analysis: 2 = each column's rows on two lanes

    @property
    def sigma2(self) -> float:
        return self.sigma * self.sigma

    @property
    def noise_std(self) -> float:
        """Scale of the forecast-noise screens (the AR(1) model noise is
        q times a von Karman screen)."""
        return self.q_model

    @property
    def a_ar1(self) -> float:
        """AR(1) coefficient making the model stationary: a^2 + q^2 = 1."""
        return math.sqrt(1.0 - self.q_model * self.q_model)

    @property
    def wind_mps(self) -> float:
        """Frozen-flow speed at a 500 Hz frame rate."""
        return self.shift * self.pitch * 500.0


# The loop's turbulence is slow enough (about 0.3 sigma of slope change per frame)
# for the delayed-state LETKF to stay stable with 10-32 members, and every window
# is Gaspari-Cohn tapered; the model noise q is matched to the truth's change.

# 8x8 square pupil, m = 10, 3x3 window, FP64 analysis, AR(1) truth (twin experiment).
TOY_8X8 = Workload("toy-8x8-m10-w3-fp64", nsub=8, pitch=0.5, obscuration=0.0, square=True,
                   m=10, window=3, taper=1, loc_len=0.0, rho=1.05, sigma=0.1, q_model=0.003,
                   r0=0.15, L0=25.0, frames=100, truth="ar1", precision=1, seeds=(11, 12, 13))

# 16 m telescope: 32x32, obscuration 0.14, m = 24, 5x5 Gaspari-Cohn window, frozen flow.
TEL_16M = Workload("16m-32x32-m24-w5gc-fp32", nsub=32, pitch=0.5, obscuration=0.14,
                   square=False, m=24, window=5, taper=1, loc_len=0.0, rho=1.03, sigma=0.1,
                   q_model=0.006, r0=0.15, L0=25.0, frames=1000, truth="frozen", precision=0,
                   seeds=(21, 22, 23), shift=0.003)

# ELT scale: 80x80 over 39 m, obscuration 0.14, m = 32, 7x7 Gaspari-Cohn window,
# r0 = 0.12 m, L0 = 30 m, frozen flow.
ELT_80X80 = Workload("elt-80x80-m32-w7gc-fp32", nsub=80, pitch=39.0 / 80.0, obscuration=0.14,
                     square=False, m=32, window=7, taper=1, loc_len=0.0, rho=1.02, sigma=0.1,
                     q_model=0.005, r0=0.12, L0=30.0, frames=1000, truth="frozen", precision=0,
                     seeds=(31, 32, 33), shift=0.003)

# Adjoint workload: the 16 m loop over 200 frames.
ADJ_16M = replace(TEL_16M, name="adjoint-16m-32x32-m24-200f", frames=200, seeds=(41, 42, 43))

# Brute-force case: 4x4 square sensor (5x5 nodes).
TINY_4X4 = Workload("tiny-4x4-m8-w3", nsub=4, pitch=0.5, obscuration=0.0, square=True, m=8,
                    window=3, taper=1, loc_len=1.0, rho=1.05, sigma=0.1, q_model=0.003,
                    r0=0.15, L0=25.0, frames=20, truth="ar1", precision=1, seeds=(1, 2, 3))

# Multi-actuator local domains (Section 4) at the paper's own sizes (Section 5.3,
# Tables 1-2): m = 101, 5 x 5 windows, so that 4 x 4-node domains observe at most
# 8 x 8 subapertures (n_max = 32, p_max = 128), differential pistons removed.
# 16 m telescope without central obscuration (Section 5), 9 x 9 partition.
DOM_16M = Workload("dom-16m-32x32-m101-p9", nsub=32, pitch=0.5, obscuration=0.0, square=False,
                   m=101, window=5, taper=1, loc_len=0.0, rho=1.02, sigma=0.1, q_model=0.006,
                   r0=0.15, L0=25.0, frames=1000, truth="frozen", precision=0,
                   seeds=(81, 82, 83), shift=0.003, partition=9, piston=1)
# 40 m telescope, 80 x 80 sensor, 21 x 21 partition (373 domains, Section 5.3).
DOM_40M = Workload("dom-40m-80x80-m101-p21", nsub=80, pitch=0.5, obscuration=0.0, square=False,
                   m=101, window=5, taper=1, loc_len=0.0, rho=1.02, sigma=0.1, q_model=0.005,
                   r0=0.15, L0=25.0, frames=1000, truth="frozen", precision=0,
                   seeds=(91, 92, 93), shift=0.003, partition=21, piston=1)

ALL = {w.name: w for w in (TOY_8X8, TEL_16M, ELT_80X80, ADJ_16M, TINY_4X4, DOM_16M, DOM_40M)}


def batched_instances(count: int = 48, seed: int = 50, frames: int = 500) -> list:
    """Many independent AO systems of different sizes: nsub ~ U{16..96},
    m ~ U{16, 24, 32, 48}, r0 ~ U(0.08, 0.2) m, pitch 0.5 m, obscuration 0.14,
    7x7 Gaspari-Cohn window. Instance i uses seeds (5000+i, 6000+i, 7000+i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nsub = int(rng.integers(16, 97))
        m = int(rng.choice([16, 24, 32, 48]))
        r0 = float(rng.uniform(0.08, 0.2))
        out.append(Workload(f"inst{i}-{nsub}x{nsub}-m{m}", nsub=nsub, pitch=0.5,
                            obscuration=0.14, square=False, m=m, window=7, taper=1,
                            loc_len=0.0, rho=1.02, sigma=0.1, q_model=0.005, r0=r0, L0=25.0,
                            frames=frames, truth="frozen", precision=0,
                            seeds=(5000 + i, 6000 + i, 7000 + i), shift=0.003))
    return out
