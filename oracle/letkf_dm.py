"""Plain FP64 CPU oracle of the deformable-mirror side of the loop: influence
matrix, least-squares projection and the true closed loop.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module. It shares
no code with the CUDA library.

What it computes (Gray et al., arXiv:1408.7069):

* Correction (Section 2.1, Eq. Eq_Cor): phi^cor_k = N u_{k-1}, N the DM's
  influence matrix on the zonal basis (actuators at the valid nodes).
* Measurement (Section 2.1, Eq. Eq_Obs, with the observation matrix of
  Section 2.2): y_k = D1 (phi^tur_{k-1} - N u_{k-2}) + w_k, two frames of delay.
* Prediction of the slopes (Section 3.1.1; Appendix B Table 3): ybar =
  C1 xbar - D1 N u_{k-2}; the analysis therefore sees the pseudo-open-loop
  slopes y_k + D1 N u_{k-2}.
* Control (Section 2.2; Appendix B.3): u_k = P phihat_{k+1/k}, the predicted
  turbulent phase projected on the DM's space by least squares,
  P = (N^T N)^-1 N^T, stored sparse: entries below a relative 1e-6 of the
  largest are dropped (Appendix B.3 notes P's sparsity).
* Criterion (Section 2.1, Eq. Crit_Opt; Section 5): spatial variance of the
  residual phase phi^tur_k - phi^cor_k at the valid nodes, piston removed.

Readings of what the paper leaves open: N is separable and Gaussian,
N[b, a] = c^(di^2 + dj^2) for the node offset (di, dj) between actuator a and
node b with |di|, |dj| <= 2 (coupling c = 0.3 at one pitch, Section 5; the
5 x 5 support makes every row of D1 N hold 36 nonzeros, the Appendix B bound).
Appendix B.3 also mentions keeping only the actuators closer than 2 pitches;
with this influence matrix that truncation changes the command of a smooth
phase by about 75 % (the inverse's rows decay by only about 0.3 per pitch), so
it is not used; ``projection_matrix`` still offers it through ``radius``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse

from . import letkf_oracle as O


def influence_matrix(geom: O.Geometry, coupling: float = 0.3, support: int = 2):
    """N [n_pts, n_pts] (csr): N[b, a] = coupling^(di^2 + dj^2) for the offset
    (di, dj) from actuator a to node b, |di|, |dj| <= support."""
    pid = {tuple(p): k for k, p in enumerate(geom.points)}
    rows, cols, vals = [], [], []
    for a, (i, j) in enumerate(geom.points):
        for di in range(-support, support + 1):
            for dj in range(-support, support + 1):
                b = pid.get((i + di, j + dj))
                if b is not None:
                    rows.append(b)
                    cols.append(a)
                    vals.append(coupling ** (di * di + dj * dj))
    n = geom.n_pts
    return scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(n, n))


def projection_matrix(geom: O.Geometry, N, radius: float = np.inf, drop: float = 1e-6):
    """P [n_pts, n_pts] (csr): the least-squares projection (N^T N)^-1 N^T,
    entries below `drop` times the largest magnitude set to zero, and entries
    between actuators more than `radius` pitches apart too (by default none)."""
    Nd = N.toarray()
    Pf = np.linalg.solve(Nd.T @ Nd, Nd.T)
    Pf = np.where(np.abs(Pf) >= drop * np.abs(Pf).max(), Pf, 0.0)
    if np.isfinite(radius):
        d = geom.points[:, None, :] - geom.points[None, :, :]
        Pf = np.where(np.hypot(d[..., 0], d[..., 1]) <= radius + 1e-9, Pf, 0.0)
    return scipy.sparse.csr_matrix(Pf)


def closed_loop_dm(geom: O.Geometry, truth, wnoise, bank, m: int, sigma2: float, rho: float,
                   a: float, noise_scale: float, seed: int, frames: int, N, P, X0,
                   frame0: int = 0, analysis=None):
    """The true closed loop over `frames` frames from the forecast ensemble X0
    and zero commands (u_{-1} = u_{-2} = 0): at frame k the residual variance
    of phi^tur_k - N u_{k-1}, the measurement y_k = D1 (phi^tur_{k-1} - N u_{k-2})
    + w_k (phi^tur_{-1} = 0), the analysis of the pseudo-open-loop slopes
    y_k + D1 N u_{k-2}, the forecast with the bank noise of frame frame0 + k,
    and the command u_k = P phihat_{k+1/k}. truth [frames, n_pts] (phi^tur),
    wnoise [frames, p] (w_k). Returns (resvar [frames], final X, commands
    [frames, n_pts], measurements [frames, p])."""
    ana = O.analysis_batched if analysis is None else analysis
    X = np.array(X0, dtype=np.float64)
    n = geom.n_pts
    u1 = np.zeros(n)            # u_{k-1}
    u2 = np.zeros(n)            # u_{k-2}
    DN = geom.D1 @ N
    resvar = np.empty(frames)
    us, ys = [], []
    for k in range(frames):
        r = truth[k] - N @ u1
        r = r - r.mean()
        resvar[k] = float(np.mean(r * r))
        phi_prev = truth[k - 1] if k > 0 else np.zeros(n)
        y = geom.D1 @ (phi_prev - N @ u2) + wnoise[k]
        ys.append(y)
        Xa, _, _ = ana(geom, X, y + DN @ u2, sigma2, rho)
        X = O.forecast(Xa, O.bank_noise(bank, geom.points, m, seed, frame0 + k, noise_scale), a)
        u = P @ X[:, 0, :].mean(axis=-1)
        us.append(u)
        u2, u1 = u1, u
    return resvar, X, np.array(us), np.array(ys)
