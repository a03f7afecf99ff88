"""Pins of the oracle's forecast-noise draw (Section 3.1.2, Eq. Mem_pre).

The paper fixes only that the model noise v is zero-mean with covariance
Sigma_v. The reading here is Sigma_v = q^2 C_vK: q times a von Karman screen of
the turbulence, sampled at the actuator pitch, drawn by a SplitMix64 hash from a
bank of periodic screens (member i of forecast f: screen h % B at offset
((h >> 16) % G, (h >> 40) % G), h = SplitMix64(seed, f 2^16 + i)).

What pins ``oracle.bank_noise`` here, each against something other than itself:
* a draw worked by hand from SplitMix64's published output sequence
  (tests/golden/bank_noise_draw.txt): catches a wrong offset order, modulus,
  shift, axis or scale;
* the generator's definition (state = seed + (counter + 1) gamma): a frame's
  draws equal frame 0's draws of a shifted seed, which pins the frame counter;
* moments under uniformly random screens and offsets: the mean is zero and
  E[v(p) v(p')] is q^2 times the bank's own spatial covariance at lag p' - p,
  checked on an anisotropic bank so that transposed axes fail;
* the paper's covariance: the structure function of v divided by q^2 matches
  the von Karman structure function band-limited to the node grid, computed by
  numerical integration of the von Karman spectrum (independent of the FFT
  screens).
"""
import math
import os

import numpy as np
from scipy import integrate

import oracle
from paper_1408_7069_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GAMMA = 0x9E3779B97F4A7C15


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split(None, 1)
                out[k] = v
    return out


def test_splitmix64_published_sequence():
    g = _golden("bank_noise_draw.txt")
    for k in range(3):
        assert oracle.splitmix64(0, k) == int(g[f"h{k}"], 16)


def test_bank_noise_hand_worked_draw():
    g = _golden("bank_noise_draw.txt")
    B, G = int(g["bank_B"]), int(g["bank_G"])
    b, x, y = np.meshgrid(np.arange(B), np.arange(G), np.arange(G), indexing="ij")
    bank = (100 * b + 10 * x + y).astype(np.float32)
    nodes = np.array([[int(u) for u in t.split(",")] for t in g["nodes"].split()])
    v = oracle.bank_noise(bank, nodes, 3, seed=int(g["seed"]), frame=int(g["frame"]),
                          scale=float(g["scale"]))
    for i in range(3):
        expect = np.array([float(u) for u in g[f"member{i}"].split()])
        assert np.array_equal(v[:, i], expect), (i, v[:, i], expect)


def test_bank_noise_frame_counter_is_seed_shift():
    # SplitMix64's state after c + 1 steps is seed + (c + 1) gamma, so counter
    # f 2^16 + i from `seed` equals counter i from seed + f 2^16 gamma.
    bank = np.random.default_rng(0).standard_normal((5, 16, 16)).astype(np.float32)
    pts = np.array([[0, 0], [3, 9], [15, 2]])
    for f in (1, 7, 300):
        a = oracle.bank_noise(bank, pts, 6, seed=1234, frame=f, scale=1.0)
        shifted = (1234 + (f << 16) * GAMMA) % (1 << 64)
        b = oracle.bank_noise(bank, pts, 6, seed=shifted, frame=0, scale=1.0)
        assert np.array_equal(a, b)
    # and consecutive frames draw different members
    a0 = oracle.bank_noise(bank, pts, 6, seed=1234, frame=0, scale=1.0)
    a1 = oracle.bank_noise(bank, pts, 6, seed=1234, frame=1, scale=1.0)
    assert not np.array_equal(a0, a1)


def _draws(bank, pts, q, frames, m=8, seed=99):
    V = np.stack([oracle.bank_noise(bank, pts, m, seed, f, q) for f in range(frames)])
    return V.transpose(0, 2, 1).reshape(-1, len(pts))        # [draws, points]


def test_bank_noise_moments_follow_the_bank():
    # An anisotropic bank: white along axis 1, smoothed along axis 0, zero mean.
    rng = np.random.default_rng(3)
    raw = rng.standard_normal((8, 32, 32))
    bank = raw + np.roll(raw, 1, axis=1) + np.roll(raw, 2, axis=1)
    bank -= bank.mean(axis=(1, 2), keepdims=True)
    q = 0.37
    pts = np.array([[5, 5], [6, 5], [5, 6], [7, 5], [5, 8]])
    v = _draws(bank, pts, q, frames=1500)
    n = len(v)
    sd = q * bank.std()
    assert np.all(np.abs(v.mean(axis=0)) < 4.5 * sd / math.sqrt(n))

    def bank_cov(dx, dy):    # spatial covariance of the bank at lag (dx, dy)
        return float(np.mean(bank * np.roll(np.roll(bank, -dx, 1), -dy, 2)))

    for k, (dx, dy) in enumerate([(1, 0), (0, 1), (2, 0), (0, 3)], start=1):
        emp = float(np.mean(v[:, 0] * v[:, k]))
        exact = q * q * bank_cov(dx, dy)
        tol = 4.5 * q * q * bank.var() / math.sqrt(n)
        assert abs(emp - exact) < tol, ((dx, dy), emp, exact, tol)
    # the lags along axis 0 are strongly correlated, those along axis 1 are not
    assert bank_cov(1, 0) > 0.5 * bank.var() and abs(bank_cov(0, 1)) < 0.1 * bank.var()
    assert abs(float(np.mean(v[:, 0] ** 2)) / (q * q * bank.var()) - 1) < 0.1


def _vk_structure_band(r, r0, L0, pitch):
    """von Karman phase structure function at separation r (m) along an axis,
    band-limited to |fx|, |fy| <= 1 / (2 pitch): 2 * integral of the spectrum
    0.023 r0^-5/3 (f^2 + L0^-2)^-11/6 times (1 - cos 2 pi fx r)."""
    fN = 0.5 / pitch

    def psd(fx, fy):
        return 0.023 * r0 ** (-5.0 / 3.0) * (fx * fx + fy * fy + 1.0 / (L0 * L0)) ** (-11.0 / 6.0)

    val, _ = integrate.dblquad(lambda fy, fx: psd(fx, fy) * (1 - math.cos(2 * math.pi * fx * r)),
                               -fN, fN, -fN, fN, epsabs=1e-6, epsrel=1e-6)
    return 2.0 * val


def test_bank_noise_covariance_is_scaled_von_karman():
    q, r0, L0, pitch = 0.006, 0.15, 25.0, 0.5
    bank = synth.noise_bank(23, 16, 64, pitch, r0, L0).astype(np.float64)
    pts = np.array([[10, 10], [11, 10], [10, 12], [14, 10], [10, 14]])
    v = _draws(bank, pts, q, frames=1500)
    for k, lag in [(1, 1), (2, 2), (3, 4), (4, 4)]:
        d = float(np.mean((v[:, 0] - v[:, k]) ** 2)) / (q * q)
        ref = _vk_structure_band(lag * pitch, r0, L0, pitch)
        assert abs(d / ref - 1) < 0.08, (lag, d, ref)
    # the unbanded Kolmogorov law 6.88 (r / r0)^5/3 is approached only once the
    # sampled band is removed: at one pitch the grid holds about half of it
    d1 = float(np.mean((v[:, 0] - v[:, 1]) ** 2)) / (q * q)
    assert 0.4 < d1 / (6.88 * (pitch / r0) ** (5.0 / 3.0)) < 0.65
