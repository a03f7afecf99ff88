"""Plain FP64 CPU oracle of the local ensemble transform Kalman filter (LETKF).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module. It shares
no code, table or constant with the CUDA library; it reads the same seeded inputs.

What it computes (Gray et al., "Local ensemble transform Kalman filter, a fast
non-stationary control law for adaptive optics on ELTs", arXiv:1408.7069):

* State (Section 2.2): per actuator node g the two phase occurrences
  (phi_k(g), phi_{k-1}(g)); the ensemble is stored [n_pts, 2, m].
* Observation (Section 2.2, C1 = [0 D1]; Appendix B): Fried slopes of the
  phi_{k-1} row, sx then sy for the valid subapertures, row-major.
* Ensemble mean and anomalies (Section 3.1, Eq. Cov_emp).
* Local analysis (Section 4.2, Eqs. Sicz_majLoc .. X_{k/k}): for every node g,
  the window slopes S_g, R_l^-1 = diag(tau_j / sigma^2) (Section 4.1: the
  observation weight decreases with distance), A = (m-1)/rho I + C Yb_l with
  C = Yb_l^T R_l^-1, A = Q Lambda Q^T (Eq. Mat_T_QG), wbar = A^-1 C d,
  W = sqrt(m-1) A^{-1/2}, Xa = xbar + Xb' (wbar 1^T + W).
  With rho = 1, A = (m-1)(I + S_cz^T S_cz) of Section 4.2, and the mean and
  members coincide with Eq. Est_majLoc and the X_{k/k} equation.
* Forecast (Section 3.1.2, Eq. Mem_pre; Appendix B.2): phi_{k+1} = a phi_k + v,
  phi_k copied into the second row.
* Loop criterion (Section 2.1, Eq. Crit_Opt; Section 5): spatial variance of the
  piston-removed residual phi^tur_k - phihat_{k/k-1}.

Readings of points the paper leaves open are listed in the design notes:
inflation rho (Hunt et al. 2007 convention), odd windows anchored at the node
(subapertures s in [i - w//2, i - w//2 + w - 1]), Gaspari-Cohn taper on R^-1,
forecast noise drawn from a bank of periodic von Karman screens chosen by a
SplitMix64 hash (Steele, Lea & Flood 2014).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse

# ---------------------------------------------------------------------------
# Geometry
# ---------------------------------------------------------------------------


@dataclass
class Geometry:
    nsub: int
    subap_mask: np.ndarray        # bool [nsub, nsub]
    points: np.ndarray            # int [n_pts, 2] node (i, j), row-major
    subaps: np.ndarray            # int [n_sap, 2] valid subap (s, t), row-major
    D1: scipy.sparse.csr_matrix   # float64 [p, n_pts] Fried slope operator (4 nonzeros per row)
    win_idx: list                 # per point: int array of slope indices into y
    win_tau: list                 # per point: float64 taper of each slope
    win_dist: list = None         # per point: node-to-subaperture-centre distance (pitches)
    taper: int = 0
    loc_len: float = 0.0          # Gaspari-Cohn half-support actually used

    @property
    def n_pts(self) -> int:
        return len(self.points)

    @property
    def p(self) -> int:
        return 2 * len(self.subaps)


def gaspari_cohn(z):
    """Gaspari & Cohn (1999) compactly supported 5th-order piecewise rational
    correlation function of z = r / c: 1 at 0, 0 for z >= 2."""
    z = np.abs(np.asarray(z, dtype=np.float64))
    out = np.zeros_like(z)
    a = z <= 1.0
    b = (z > 1.0) & (z < 2.0)
    za = z[a]
    out[a] = -0.25 * za**5 + 0.5 * za**4 + 0.625 * za**3 - (5.0 / 3.0) * za**2 + 1.0
    zb = z[b]
    out[b] = (zb**5 / 12.0 - 0.5 * zb**4 + 0.625 * zb**3 + (5.0 / 3.0) * zb**2
              - 5.0 * zb + 4.0 - (2.0 / 3.0) / zb)
    return out


def gaspari_cohn_deriv(z):
    """d/dz of gaspari_cohn (differentiating its two polynomial pieces)."""
    z = np.abs(np.asarray(z, dtype=np.float64))
    out = np.zeros_like(z)
    a = z <= 1.0
    b = (z > 1.0) & (z < 2.0)
    za = z[a]
    out[a] = -1.25 * za**4 + 2.0 * za**3 + 1.875 * za**2 - (10.0 / 3.0) * za
    zb = z[b]
    out[b] = (5.0 / 12.0) * zb**4 - 2.0 * zb**3 + 1.875 * zb**2 + (10.0 / 3.0) * zb - 5.0 \
        + (2.0 / 3.0) / zb**2
    return out


def build_geometry(subap_mask, window: int, taper: int = 0, loc_len: float = 0.0) -> Geometry:
    """Valid nodes, Fried D1 and the per-node observation windows.

    * Valid nodes: corners of valid subapertures (Section 4.1: the phase is
      estimated at the actuators of the valid subapertures).
    * D1 (Appendix B): sx(s,t) = (phi[s+1,t] + phi[s+1,t+1] - phi[s,t] - phi[s,t+1]) / 2,
      sy(s,t) = (phi[s,t+1] + phi[s+1,t+1] - phi[s,t] - phi[s+1,t]) / 2.
    * Window of node (i, j) (Section 4.1, observation region): the valid
      subapertures (s, t) with i - w//2 <= s <= i - w//2 + w - 1, same for t.
      Both slopes of each such subaperture are observed.
    * Taper (Section 4.1, smooth localization): tau = 1 (box) or
      Gaspari-Cohn(dist / c), dist from the node to the subaperture centre in
      pitches, c = loc_len (default w / 4).
    """
    sm = np.asarray(subap_mask).astype(bool)
    nsub = sm.shape[0]
    nodes = np.zeros((nsub + 1, nsub + 1), bool)
    for s in range(nsub):
        for t in range(nsub):
            if sm[s, t]:
                nodes[s, t] = nodes[s + 1, t] = nodes[s, t + 1] = nodes[s + 1, t + 1] = True
    points = np.argwhere(nodes)                        # row-major
    subaps = np.argwhere(sm)
    pid = -np.ones((nsub + 1, nsub + 1), int)
    pid[nodes] = np.arange(len(points))
    sid = -np.ones((nsub, nsub), int)
    sid[sm] = np.arange(len(subaps))
    n_sap = len(subaps)
    D1 = scipy.sparse.lil_matrix((2 * n_sap, len(points)))
    for k, (s, t) in enumerate(subaps):
        D1[k, pid[s + 1, t]] += 0.5
        D1[k, pid[s + 1, t + 1]] += 0.5
        D1[k, pid[s, t]] -= 0.5
        D1[k, pid[s, t + 1]] -= 0.5
        D1[n_sap + k, pid[s, t + 1]] += 0.5
        D1[n_sap + k, pid[s + 1, t + 1]] += 0.5
        D1[n_sap + k, pid[s, t]] -= 0.5
        D1[n_sap + k, pid[s + 1, t]] -= 0.5
    D1 = D1.tocsr()
    h = window // 2
    c = loc_len if loc_len > 0 else window / 4.0
    win_idx, win_tau, win_dist = [], [], []
    for (i, j) in points:
        idx, tau, dist_l = [], [], []
        for s in range(i - h, i - h + window):
            for t in range(j - h, j - h + window):
                if 0 <= s < nsub and 0 <= t < nsub and sm[s, t]:
                    k = sid[s, t]
                    if taper == 1:
                        dist = math.hypot(s + 0.5 - i, t + 0.5 - j)
                        tk = float(gaspari_cohn(dist / c))
                    else:
                        tk = 1.0
                    idx += [k, n_sap + k]
                    tau += [tk, tk]
                    dd = math.hypot(s + 0.5 - i, t + 0.5 - j)
                    dist_l += [dd, dd]
        win_idx.append(np.array(idx, int))
        win_tau.append(np.array(tau, float))
        win_dist.append(np.array(dist_l, float))
    return Geometry(nsub, sm, points, subaps, D1, win_idx, win_tau, win_dist, taper, c)


# ---------------------------------------------------------------------------
# Analysis (Section 3.1 and 4.2)
# ---------------------------------------------------------------------------


def mean_anomalies(X):
    """Ensemble mean xbar [n_pts, 2] and unnormalised anomalies X - xbar
    (Section 3.1, Eq. Cov_emp: Z = anomalies / sqrt(m-1))."""
    xbar = X.mean(axis=-1)
    return xbar, X - xbar[..., None]


def local_transform(Yl, dl, wl, m: int, rho: float):
    """One local ensemble transform (Section 4.2, with Appendix A).

    Yl [p_l, m] window slope anomalies, dl [p_l] innovations, wl [p_l] diagonal
    of R_l^-1. Returns A, wbar, W with A = (m-1)/rho I + Yl^T R_l^-1 Yl,
    A = Q diag(lam) Q^T, wbar = Q diag(1/lam) Q^T (Yl^T R_l^-1 dl) and
    W = Q diag(sqrt((m-1)/lam)) Q^T.
    """
    C = Yl.T * wl[None, :]                       # Yb_l^T R_l^-1   [m, p_l]
    A = (m - 1) / rho * np.eye(m) + C @ Yl
    lam, Q = np.linalg.eigh(A)
    wbar = Q @ ((Q.T @ (C @ dl)) / lam)
    W = (Q * np.sqrt((m - 1) / lam)) @ Q.T
    return A, wbar, W


def observe(geom: Geometry, X):
    """Background mean, anomalies, slope anomalies Yb = D1 (phi_{k-1} anomalies)
    and predicted slopes ybar = D1 (phi_{k-1} mean) (Section 3.1.1, ybar = C1 xbar
    with a perfectly known correction, N = identity)."""
    xbar, Xp = mean_anomalies(X)
    Yb = geom.D1 @ Xp[:, 1, :]
    ybar = geom.D1 @ xbar[:, 1]
    return xbar, Xp, Yb, ybar


def analysis(geom: Geometry, Xb, y, sigma2: float, rho: float, return_local: bool = False):
    """Local analysis of every node, per-point loop (Section 4.2).

    Xb [n_pts, 2, m] background ensemble, y [p] slopes. Returns Xa, mean [n_pts, 2],
    spread [n_pts, 2] (sample std over members, m - 1), and optionally the
    per-point (A, wbar, W).
    """
    Xb = np.asarray(Xb, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m = Xb.shape[-1]
    xbar, Xp, Yb, ybar = observe(geom, Xb)
    d = y - ybar
    Xa = np.empty_like(Xb)
    local = []
    for g in range(geom.n_pts):
        idx = geom.win_idx[g]
        wl = geom.win_tau[g] / sigma2
        A, wbar, W = local_transform(Yb[idx], d[idx], wl, m, rho)
        Xa[g] = xbar[g][:, None] + Xp[g] @ (wbar[:, None] + W)
        if return_local:
            local.append((A, wbar, W))
    mean = Xa.mean(axis=-1)
    spread = Xa.std(axis=-1, ddof=1)
    if return_local:
        return Xa, mean, spread, local
    return Xa, mean, spread


def analysis_batched(geom: Geometry, Xb, y, sigma2: float, rho: float, nodes=None, obs=None):
    """The same analysis with every window padded to a common length with zero
    weight (exact: a zero weight adds nothing to A or C d) and one stacked
    numpy.linalg.eigh over the nodes. ``nodes`` (indices) restricts the work to
    a subset; the other nodes keep their background members. ``obs`` passes a
    precomputed observe(geom, Xb). Used to time the CPU baseline."""
    Xb = np.asarray(Xb, dtype=np.float64)
    m = Xb.shape[-1]
    xbar, Xp, Yb, ybar = observe(geom, Xb) if obs is None else obs
    d = np.asarray(y, dtype=np.float64) - ybar
    sel = np.arange(geom.n_pts) if nodes is None else np.asarray(nodes)
    L = max(len(geom.win_idx[g]) for g in sel)
    n = len(sel)
    idx = np.zeros((n, L), int)
    wts = np.zeros((n, L))
    for r, g in enumerate(sel):
        k = len(geom.win_idx[g])
        idx[r, :k] = geom.win_idx[g]
        wts[r, :k] = geom.win_tau[g] / sigma2
    Yl = Yb[idx]                                  # [n, L, m]
    dl = d[idx]                                   # [n, L]
    C = np.swapaxes(Yl, 1, 2) * wts[:, None, :]   # [n, m, L]
    A = C @ Yl + (m - 1) / rho * np.eye(m)[None]
    lam, Q = np.linalg.eigh(A)
    Cd = np.einsum("nml,nl->nm", C, dl)
    wbar = np.einsum("nij,nj->ni", Q, np.einsum("nji,nj->ni", Q, Cd) / lam)
    W = np.einsum("nij,nj,nkj->nik", Q, np.sqrt((m - 1) / lam), Q)
    T = wbar[:, :, None] + W
    Xa = Xb.copy()
    Xa[sel] = xbar[sel][..., None] + np.einsum("nrj,nji->nri", Xp[sel], T)
    return Xa, Xa.mean(axis=-1), Xa.std(axis=-1, ddof=1)


# ---------------------------------------------------------------------------
# Forecast (Section 3.1.2, Eq. Mem_pre) and its noise
# ---------------------------------------------------------------------------
_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed: int, counter: int) -> int:
    """Output of SplitMix64 (Steele, Lea & Flood 2014) whose state has been
    advanced counter + 1 times from ``seed``: z = seed + (counter+1) * gamma,
    then the two xor-shift-multiply rounds and a final xor-shift."""
    z = (seed + (counter + 1) * _GAMMA) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def bank_noise(bank, points, m: int, seed: int, frame: int, scale: float):
    """Forecast noise v [n_pts, m]: member i of forecast ``frame`` takes screen
    h % B of the bank at the offset ((h >> 16) % G, (h >> 40) % G), wrapped,
    with h = splitmix64(seed, frame * 2^16 + i), times ``scale``."""
    bank = np.asarray(bank)
    B, G, _ = bank.shape
    v = np.empty((len(points), m))
    for i in range(m):
        h = splitmix64(seed, (frame << 16) | i)
        b = h % B
        ox = (h >> 16) % G
        oy = (h >> 40) % G
        v[:, i] = bank[b, (points[:, 0] + ox) % G, (points[:, 1] + oy) % G]
    return scale * v


def forecast(Xa, v, a: float):
    """x_{k+1}^i = A1 x_{k/k}^i + v^i with A1 = [[a I, 0], [I, 0]] (Section 2.2, AR(1))."""
    Xb = np.empty_like(Xa)
    Xb[:, 0, :] = a * Xa[:, 0, :] + v
    Xb[:, 1, :] = Xa[:, 0, :]
    return Xb


def residual_variance(truth_k, X):
    """Spatial variance over valid nodes of phi^tur_k - phihat_{k/k-1}, piston
    removed (Section 2.1, Eq. Crit_Opt; Section 5)."""
    r = truth_k - X[:, 0, :].mean(axis=-1)
    r = r - r.mean()
    return float(np.mean(r * r))


def closed_loop(geom: Geometry, truth, slopes, bank, m: int, sigma2: float, rho: float,
                a: float, noise_scale: float, seed: int, frames: int, X0=None,
                batched: bool = False, frame0: int = 0):
    """Run the loop: at frame k record the residual of the prediction X_{k/k-1},
    analyse y_k, forecast with the bank noise of frame frame0 + k. Without X0
    the first prediction ensemble is all zeros (Section 3.1). ``batched`` uses
    the stacked form of the analysis. Returns (resvar [frames], final X,
    per-frame analysis means)."""
    X = np.zeros((geom.n_pts, 2, m)) if X0 is None else np.array(X0, dtype=np.float64)
    resvar = np.empty(frames)
    means = []
    ana = analysis_batched if batched else analysis
    for k in range(frames):
        resvar[k] = residual_variance(truth[k], X)
        Xa, mean, _ = ana(geom, X, slopes[k], sigma2, rho)
        means.append(mean)
        v = bank_noise(bank, geom.points, m, seed, frame0 + k, noise_scale)
        X = forecast(Xa, v, a)
    return resvar, X, np.array(means)


# ---------------------------------------------------------------------------
# Reverse mode of the closed loop (gradient of the mean residual variance)
# ---------------------------------------------------------------------------


def analysis_adjoint(geom: Geometry, Xb, y, sigma2: float, rho: float, Xa_bar):
    """Adjoint of one analysis (Section 4.2) at background Xb and slopes y.

    Xa_bar [n_pts, 2, m]: gradient of a scalar with respect to the analysis
    ensemble. Returns (Xb_bar [n_pts, 2, m], d/drho, d/dsigma2, d/dL) of that
    scalar, L the Gaspari-Cohn half-support. Per node, with c_j = tau_j/sigma2,
    A = (m-1)/rho I + sum_j c_j y_j y_j^T, b = sum_j c_j d_j y_j,
    wbar = A^-1 b, W = sqrt(m-1) A^-1/2 and Xa_r = xbar_r + X'_r (wbar 1^T + W):
      Xa_r -> xbar_r, X'_r, wbar, W;
      wbar -> b_bar = A^-1 wbar_bar, A_bar -= b_bar wbar^T;
      W -> A_bar += sqrt(m-1) Q (F o (Q^T W_bar Q)) Q^T, F_pq the divided
           difference of lambda^-1/2, -1/(sqrt(l_p) sqrt(l_q) (sqrt(l_p) + sqrt(l_q)));
      A, b -> y_j, d_j, c_j, (m-1)/rho; then the slopes back to the nodes
      through D1 and the anomaly / mean split (Section 3.1).
    """
    Xb = np.asarray(Xb, dtype=np.float64)
    n_pts, _, m = Xb.shape
    xbar, Xp, Yb, ybar = observe(geom, Xb)
    d = np.asarray(y, dtype=np.float64) - ybar
    Xp_bar = np.zeros_like(Xb)                 # adjoint of the anomalies X'
    xbar_bar = np.zeros((n_pts, 2))
    Yb_bar = np.zeros_like(Yb)
    d_bar = np.zeros_like(d)
    alpha = (m - 1) / rho
    g_alpha = g_s2 = g_L = 0.0
    one = np.ones(m)
    for g in range(n_pts):
        idx = geom.win_idx[g]
        tau = geom.win_tau[g]
        cw = tau / sigma2
        Yl = Yb[idx]
        dl = d[idx]
        A = alpha * np.eye(m) + (Yl.T * cw) @ Yl
        bvec = Yl.T @ (cw * dl)
        lam, Q = np.linalg.eigh(A)
        wbar = Q @ ((Q.T @ bvec) / lam)
        W = np.sqrt(m - 1) * (Q / np.sqrt(lam)) @ Q.T
        G = Xa_bar[g]                           # [2, m]
        ssum = G @ one                          # [2]
        xbar_bar[g] += ssum
        Xp_bar[g] += np.outer(ssum, wbar) + G @ W.T
        wbar_bar = Xp[g].T @ ssum
        W_bar = Xp[g].T @ G
        b_bar = Q @ ((Q.T @ wbar_bar) / lam)
        A_bar = -np.outer(b_bar, wbar)
        rl = np.sqrt(lam)
        F = -1.0 / (np.outer(rl, rl) * (rl[:, None] + rl[None, :]))
        A_bar += np.sqrt(m - 1) * Q @ (F * (Q.T @ W_bar @ Q)) @ Q.T
        As = 0.5 * (A_bar + A_bar.T)
        g_alpha += np.trace(As)
        Yb_bar[idx] += 2.0 * cw[:, None] * (Yl @ As) + np.outer(cw * dl, b_bar)
        yb = Yl @ b_bar
        d_bar[idx] += cw * yb
        c_bar = np.einsum("jm,mn,jn->j", Yl, As, Yl) + dl * yb
        g_s2 += np.sum(c_bar * (-cw / sigma2))
        if geom.taper == 1:
            z = geom.win_dist[g] / geom.loc_len
            dtau = gaspari_cohn_deriv(z) * (-z / geom.loc_len)
            g_L += np.sum(c_bar * dtau / sigma2)
    # slopes -> anomalies / means of the phi_{k-1} row (Yb = D1 X'_1, ybar = D1 xbar_1)
    Xp_bar[:, 1, :] += geom.D1.T @ Yb_bar
    xbar_bar[:, 1] += -(geom.D1.T @ d_bar)
    # X' = X - xbar 1^T, xbar = mean
    Xb_bar = Xp_bar - Xp_bar.mean(axis=-1, keepdims=True) + xbar_bar[..., None] / m
    g_rho = g_alpha * (-(m - 1) / rho**2)
    return Xb_bar, g_rho, g_s2, g_L


def residual_variance_grad(truth_k, X):
    """d/dX of residual_variance(truth_k, X)."""
    n_pts, _, m = X.shape
    r = truth_k - X[:, 0, :].mean(axis=-1)
    r = r - r.mean()
    G = np.zeros_like(X)
    G[:, 0, :] = (-2.0 / (n_pts * m)) * r[:, None]
    return G


def closed_loop_grad(geom: Geometry, truth, slopes, bank, m: int, sigma2: float, rho: float,
                     a: float, noise_scale: float, seed: int, frames: int, X0,
                     frame0: int = 0):
    """J = mean over the frames of the residual variance of the prediction
    (Section 2.1, Eq. Crit_Opt) and its gradient with respect to (rho, sigma2,
    L), by reverse mode through the analyses and AR(1) forecasts, from X0; the
    forecast after frame k draws the bank noise of frame frame0 + k."""
    X = np.array(X0, dtype=np.float64)
    Xs, J = [], 0.0
    for k in range(frames):
        Xs.append(X)
        J += residual_variance(truth[k], X)
        Xa, _, _ = analysis(geom, X, slopes[k], sigma2, rho)
        X = forecast(Xa, bank_noise(bank, geom.points, m, seed, frame0 + k, noise_scale), a)
    J /= frames
    grad = np.zeros(3)
    lam_next = np.zeros_like(X)                 # adjoint of X_{k+1}
    for k in range(frames - 1, -1, -1):
        Xa_bar = np.zeros_like(X)
        Xa_bar[:, 0, :] = a * lam_next[:, 0, :] + lam_next[:, 1, :]
        Xb_bar, gr, gs, gl = analysis_adjoint(geom, Xs[k], slopes[k], sigma2, rho, Xa_bar)
        grad += (gr, gs, gl)
        lam_next = Xb_bar + residual_variance_grad(truth[k], Xs[k]) / frames
    return J, grad, lam_next
