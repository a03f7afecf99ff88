"""Seeded synthetic inputs for the LETKF adaptive-optics loop.

This module is the one piece shared by the CUDA path's harness (tests, bench) and
the CPU oracle's tests. It holds no arithmetic of the estimator itself: it draws
pupils, von Karman phase screens, turbulence sequences, noisy wavefront-sensor
slopes and the forecast-noise screen bank. Everything is deterministic in its
seeds.

The paper simulates a 16 m telescope with a 32x32 Shack-Hartmann sensor whose
valid subapertures are those more than 50 % illuminated (Section 5), von Karman
turbulence and frozen-flow layers (Section 5), and a two-frame-delay loop
(Section 2.1, Eq. Eq_Obs: the slopes of frame k see the phase of frame k-1).
The simulator here follows that set-up with one layer, phase sampled at the
Fried-geometry actuator nodes, and the Fried slope model of Appendix B
(two slopes per subaperture from the four corner phases).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# --------------------------------------------------------------------------
# Pupil geometry (Section 5: subapertures > 50 % illuminated are valid)
# --------------------------------------------------------------------------
def pupil_subap_mask(nsub: int, obscuration: float = 0.0, square: bool = False,
                     supersample: int = 16) -> np.ndarray:
    """uint8 [nsub, nsub] mask of valid subapertures, row-major (s, t).

    A subaperture is valid when more than half of a supersample x supersample
    grid of points inside it falls in the annulus obscuration*D/2 <= r <= D/2,
    D = nsub pitches, centred on the sensor. ``square`` marks every
    subaperture valid (a square pupil).
    """
    if square:
        return np.ones((nsub, nsub), np.uint8)
    u = (np.arange(supersample) + 0.5) / supersample
    c = nsub / 2.0
    s = np.arange(nsub)
    x = (s[:, None] + u[None, :]) - c          # [nsub, ss] coordinates along axis 0
    xx = x[:, None, :, None]
    yy = x[None, :, None, :]
    r = np.sqrt(xx * xx + yy * yy)              # [nsub, nsub, ss, ss]
    inside = (r <= c) & (r >= obscuration * c)
    frac = inside.mean(axis=(2, 3))
    return (frac > 0.5).astype(np.uint8)


# --------------------------------------------------------------------------
# Von Karman phase screens
# --------------------------------------------------------------------------
def von_karman_psd(f: np.ndarray, r0: float, L0: float) -> np.ndarray:
    """Phase power spectral density in rad^2 m^2 at spatial frequency f (cycles/m)."""
    return 0.023 * r0 ** (-5.0 / 3.0) * (f * f + 1.0 / (L0 * L0)) ** (-11.0 / 6.0)


def _fft_screen_pair(rng: np.random.Generator, nx: int, ny: int, dx: float,
                     r0: float, L0: float, subharmonics: bool) -> np.ndarray:
    """Complex screen whose real and imaginary parts are two independent
    von Karman screens on an nx x ny grid of spacing dx (metres)."""
    fx = np.fft.fftfreq(nx, dx)
    fy = np.fft.fftfreq(ny, dx)
    dfx, dfy = 1.0 / (nx * dx), 1.0 / (ny * dx)
    f = np.sqrt(fx[:, None] ** 2 + fy[None, :] ** 2)
    amp = np.sqrt(von_karman_psd(np.where(f == 0, 1.0, f), r0, L0) * dfx * dfy)
    amp[0, 0] = 0.0
    c = rng.standard_normal((nx, ny)) + 1j * rng.standard_normal((nx, ny))
    scr = np.fft.ifft2(c * amp) * (nx * ny)
    if subharmonics:
        # Low-order compensation (Lane, Glindemann & Dainty 1992): three levels of
        # 3x3 sub-frequencies below the FFT grid's first frequency.
        x = np.arange(nx) * dx
        y = np.arange(ny) * dx
        low = np.zeros((nx, ny), complex)
        for lev in range(1, 4):
            sx, sy = dfx / 3 ** lev, dfy / 3 ** lev
            for a in (-1, 0, 1):
                for b in (-1, 0, 1):
                    if a == 0 and b == 0:
                        continue
                    fxa, fyb = a * sx, b * sy
                    am = math.sqrt(von_karman_psd(np.array(math.hypot(fxa, fyb)), r0, L0) * sx * sy)
                    cc = rng.standard_normal() + 1j * rng.standard_normal()
                    low += cc * am * np.outer(np.exp(2j * np.pi * fxa * x), np.exp(2j * np.pi * fyb * y))
        low -= low.mean()
        scr = scr + low
    return scr


def von_karman_screens(seed: int, count: int, nx: int, ny: int, dx: float, r0: float,
                       L0: float, subharmonics: bool = True) -> np.ndarray:
    """``count`` independent float64 screens [count, nx, ny] in rad."""
    rng = np.random.default_rng(seed)
    out = np.empty((count, nx, ny))
    for k in range(0, count, 2):
        pair = _fft_screen_pair(rng, nx, ny, dx, r0, L0, subharmonics)
        out[k] = pair.real
        if k + 1 < count:
            out[k + 1] = pair.imag
    return out


def noise_bank(seed: int, count: int, size: int, pitch: float, r0: float, L0: float) -> np.ndarray:
    """Forecast-noise bank: ``count`` periodic von Karman screens [count, size, size]
    sampled at the actuator pitch, float32. Periodic (no subharmonics) so that a
    wrapped offset into a screen is still a valid screen."""
    return von_karman_screens(seed, count, size, size, pitch, r0, L0,
                              subharmonics=False).astype(np.float32)


def bank_size(nsub: int) -> int:
    """Side of the noise-bank screens for an nsub x nsub sensor."""
    g = 32
    while g < 2 * (nsub + 1):
        g *= 2
    return g


# --------------------------------------------------------------------------
# Turbulence sequences sampled at the actuator nodes (nsub+1)^2
# --------------------------------------------------------------------------
def ar1_truth(seed: int, frames: int, nsub: int, pitch: float, r0: float, L0: float,
              a: float) -> np.ndarray:
    """phi_{k+1} = a phi_k + sqrt(1-a^2) xi_k on the node grid, xi fresh screens.
    Returns float64 [frames, nsub+1, nsub+1]."""
    nn = nsub + 1
    size = 32
    while size < 4 * nn or size * pitch < 2 * L0:
        size *= 2
    scr = von_karman_screens(seed, frames, size, size, pitch, r0, L0)[:, :nn, :nn]
    out = np.empty((frames, nn, nn))
    out[0] = scr[0]
    q = math.sqrt(1.0 - a * a)
    for k in range(1, frames):
        out[k] = a * out[k - 1] + q * scr[k]
    return out


def frozen_flow_truth(seed: int, frames: int, nsub: int, pitch: float, r0: float, L0: float,
                      shift: float, px_per_pitch: int = 8) -> np.ndarray:
    """One frozen-flow layer moving ``shift`` pitches per frame along axis 0.

    The screen is drawn at spacing pitch/px_per_pitch; a sub-pixel position is
    read by linear interpolation along the flow axis (the nodes sit on screen
    columns). Returns float64 [frames, nsub+1, nsub+1]."""
    nn = nsub + 1
    dx = pitch / px_per_pitch
    span = (nn - 1) * px_per_pitch + 1
    nx = span + int(math.ceil(frames * shift * px_per_pitch)) + 2
    fx = 1
    while fx < nx:
        fx *= 2
    fy = 1
    while fy < span:
        fy *= 2
    scr = von_karman_screens(seed, 1, fx, fy, dx, r0, L0)[0]
    idx = np.arange(nn) * px_per_pitch
    out = np.empty((frames, nn, nn))
    for k in range(frames):
        pos = k * shift * px_per_pitch
        i0 = int(pos)
        f = pos - i0
        out[k] = (1 - f) * scr[np.ix_(idx + i0, idx)] + f * scr[np.ix_(idx + i0 + 1, idx)]
    return out


def prior_ensemble(seed: int, subap_mask: np.ndarray, m: int, a: float, q: float,
                   pitch: float, r0: float, L0: float) -> np.ndarray:
    """Initial forecast ensemble [n_pts, 2, m] drawn from the AR(1) model's
    stationary law: phi_{-1} a von Karman screen at the nodes, phi_0 =
    a phi_{-1} + q xi with xi an independent screen."""
    nodes = node_mask_of(subap_mask)
    pts = np.argwhere(nodes)
    g = bank_size(subap_mask.shape[0])
    scr = von_karman_screens(seed, 2 * m, g, g, pitch, r0, L0, subharmonics=False)
    X = np.empty((len(pts), 2, m))
    for i in range(m):
        prev = scr[2 * i][pts[:, 0], pts[:, 1]]
        nxt = scr[2 * i + 1][pts[:, 0], pts[:, 1]]
        X[:, 1, i] = prev
        X[:, 0, i] = a * prev + q * nxt
    return X


# --------------------------------------------------------------------------
# Wavefront sensor (Appendix B: Fried geometry, 2 slopes per subaperture)
# --------------------------------------------------------------------------
def wfs_slopes(phi_nodes: np.ndarray, subap_mask: np.ndarray) -> np.ndarray:
    """Noise-free Fried slopes of a node-grid phase [.., nsub+1, nsub+1].

    sx(s,t) = (phi[s+1,t] + phi[s+1,t+1] - phi[s,t] - phi[s,t+1]) / 2 and
    sy(s,t) = (phi[s,t+1] + phi[s+1,t+1] - phi[s,t] - phi[s+1,t]) / 2, in rad per
    subaperture. Output [.., p]: all sx of valid subapertures (row-major), then all sy.
    """
    p00 = phi_nodes[..., :-1, :-1]
    p10 = phi_nodes[..., 1:, :-1]
    p01 = phi_nodes[..., :-1, 1:]
    p11 = phi_nodes[..., 1:, 1:]
    sx = 0.5 * (p10 + p11 - p00 - p01)
    sy = 0.5 * (p01 + p11 - p00 - p10)
    sel = subap_mask.astype(bool)
    return np.concatenate([sx[..., sel], sy[..., sel]], axis=-1)


def node_mask_of(subap_mask: np.ndarray) -> np.ndarray:
    """Actuator nodes that are a corner of at least one valid subaperture."""
    m = subap_mask.astype(bool)
    n = np.zeros((m.shape[0] + 1, m.shape[1] + 1), bool)
    n[:-1, :-1] |= m
    n[1:, :-1] |= m
    n[:-1, 1:] |= m
    n[1:, 1:] |= m
    return n


@dataclass
class LoopInputs:
    """One synthetic closed-loop run.

    truth   [frames, n_pts]  phi^tur_k at the valid nodes (row-major order), float64
    slopes  [frames, p]      y_k = D phi^tur_{k-1} + w_k (y_0 sees a flat phase), float64
    bank    [B, G, G]        forecast-noise screens, float32
    X0      [n_pts, 2, m]    initial forecast ensemble (prior draw), float64
    """
    subap_mask: np.ndarray
    truth: np.ndarray
    slopes: np.ndarray
    bank: np.ndarray
    X0: np.ndarray


def make_loop_inputs(w, frames: int | None = None) -> LoopInputs:
    """Synthetic inputs for a workload description ``w`` (see ``workloads``)."""
    frames = w.frames if frames is None else frames
    seeds = w.seeds
    mask = pupil_subap_mask(w.nsub, w.obscuration, w.square)
    if w.truth == "ar1":
        phi = ar1_truth(seeds[0], frames, w.nsub, w.pitch, w.r0, w.L0, w.a_ar1)
    else:
        phi = frozen_flow_truth(seeds[0], frames, w.nsub, w.pitch, w.r0, w.L0, w.shift)
    nodes = node_mask_of(mask)
    truth = phi[:, nodes]
    clean = wfs_slopes(phi, mask)                      # slopes of frame k's phase
    rng = np.random.default_rng(seeds[1])
    noise = w.sigma * rng.standard_normal(clean.shape)
    slopes = np.empty_like(clean)
    slopes[0] = noise[0]                               # y_0 = D*0 + w_0
    slopes[1:] = clean[:-1] + noise[1:]                # y_k = D phi_{k-1} + w_k
    bank = noise_bank(seeds[2], w.bank_count, bank_size(w.nsub), w.pitch, w.r0, w.L0)
    X0 = prior_ensemble(seeds[0] + 1000, mask, w.m, w.a_ar1, w.noise_std, w.pitch, w.r0, w.L0)
    c = np.ascontiguousarray
    return LoopInputs(mask, c(truth), c(slopes), c(bank), c(X0))


def random_ensemble(seed: int, n_pts: int, m: int, scale: float = 1.0,
                    offset_scale: float = 5.0) -> np.ndarray:
    """A generic background ensemble [n_pts, 2, m] (float64): a smooth-ish mean plus
    member spread, for single-analysis parity cases."""
    rng = np.random.default_rng(seed)
    mean = offset_scale * rng.standard_normal((n_pts, 2, 1))
    return mean + scale * rng.standard_normal((n_pts, 2, m))


# --------------------------------------------------------------------------
# Deformable mirror calibration (the DM model the loop is simulated with)
# --------------------------------------------------------------------------
def dm_calibration(subap_mask: np.ndarray, coupling: float = 0.3, support: int = 2,
                   drop: float = 1e-6):
    """The simulated DM's calibration matrices over the valid nodes (row-major
    node order, actuators at the nodes): influence matrix N with
    N[b, a] = coupling^(di^2 + dj^2) for node offsets |di|, |dj| <= support, and
    the least-squares command matrix (N^T N)^-1 N^T with entries below `drop`
    times the largest magnitude dropped, as a controller would load them.
    Returns (N, P) as scipy CSR float64 matrices."""
    import scipy.sparse
    nodes = node_mask_of(subap_mask)
    pts = np.argwhere(nodes)
    index = -np.ones(nodes.shape, int)
    index[nodes] = np.arange(len(pts))
    rows, cols, vals = [], [], []
    for a, (i, j) in enumerate(pts):
        for di in range(-support, support + 1):
            for dj in range(-support, support + 1):
                ii, jj = i + di, j + dj
                if 0 <= ii < nodes.shape[0] and 0 <= jj < nodes.shape[1] and index[ii, jj] >= 0:
                    rows.append(index[ii, jj])
                    cols.append(a)
                    vals.append(coupling ** (di * di + dj * dj))
    n = len(pts)
    N = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(n, n))
    Nd = N.toarray()
    full = np.linalg.lstsq(Nd, np.eye(n), rcond=None)[0]
    P = scipy.sparse.csr_matrix(np.where(np.abs(full) >= drop * np.abs(full).max(), full, 0.0))
    return N, P
