"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a number the
paper prints, a closed form, an independent formula of the same quantity
(global ETKF in the paper's S_cz / S_inov form, the exact Kalman filter, the
primal observation-space gain) or an invariant.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1408_7069_gb300 import opcount, synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_kv(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split(None, 1)
                out[k] = v
    return out


# --------------------------------------------------------------------- geometry
def test_geometry_16m_matches_section5():
    g = _golden_kv("geometry_16m.txt")
    mask = synth.pupil_subap_mask(int(g["nsub"]), float(g["obscuration"]))
    geom = oracle.build_geometry(mask, window=3)
    assert len(geom.subaps) == int(g["valid_subapertures"])
    assert geom.n_pts == int(g["valid_actuators"])
    assert geom.p == 2 * 812


def test_fried_operator_closed_forms():
    mask = synth.pupil_subap_mask(12, 0.3)
    geom = oracle.build_geometry(mask, window=3)
    i, j = geom.points[:, 0].astype(float), geom.points[:, 1].astype(float)
    ns = len(geom.subaps)
    # piston is unseen by a slope sensor
    assert np.abs(geom.D1 @ np.full(geom.n_pts, 3.7)).max() < 1e-14
    # a tilt alpha*i + beta*j gives sx = alpha, sy = beta (rad per subaperture)
    s = geom.D1 @ (0.3 * i - 1.1 * j)
    assert np.allclose(s[:ns], 0.3, atol=1e-14) and np.allclose(s[ns:], -1.1, atol=1e-14)
    # waffle (-1)^(i+j) is the Fried blind mode
    assert np.abs(geom.D1 @ (-1.0) ** (i + j)).max() < 1e-14
    # one subaperture by hand: corners p00=1, p10=2, p01=4, p11=8
    one = oracle.build_geometry(np.ones((1, 1)), window=1)
    phi = np.zeros(4)
    order = {tuple(p): k for k, p in enumerate(one.points)}
    phi[order[(0, 0)]], phi[order[(1, 0)]], phi[order[(0, 1)]], phi[order[(1, 1)]] = 1, 2, 4, 8
    assert np.allclose(one.D1 @ phi, [(2 + 8 - 1 - 4) / 2, (4 + 8 - 1 - 2) / 2])


def test_windows_anchor_and_truncation():
    geom = oracle.build_geometry(np.ones((6, 6)), window=3)
    pid = {tuple(p): k for k, p in enumerate(geom.points)}
    # interior node (3,3): subaps s,t in [2,4] -> 9 subaps, 18 slopes
    assert len(geom.win_idx[pid[(3, 3)]]) == 18
    # corner node (0,0): s,t in [-1,1] truncated to [0,1] -> 4 subaps
    assert len(geom.win_idx[pid[(0, 0)]]) == 8
    # far corner node (6,6): s,t in [5,7] truncated to [5] -> 1 subap
    assert len(geom.win_idx[pid[(6, 6)]]) == 2


def test_gaspari_cohn_shape():
    gc = oracle.gaspari_cohn
    assert gc(0.0) == pytest.approx(1.0)
    assert gc(2.0) == pytest.approx(0.0, abs=1e-15)
    assert gc(3.0) == 0.0
    h = 1e-6
    for z0 in (1.0, 2.0):        # value, slope and curvature continuous at the knots
        left = gc(np.array([z0 - 2 * h, z0 - h, z0 - 1e-12]))
        right = gc(np.array([z0 + 1e-12, z0 + h, z0 + 2 * h]))
        assert abs(left[2] - right[0]) < 1e-9
        dl = (left[2] - left[0]) / (2 * h)
        dr = (right[2] - right[0]) / (2 * h)
        assert abs(dl - dr) < 1e-5
    z = np.linspace(0, 2, 401)
    assert np.all(np.diff(gc(z)) <= 1e-15)
    # second derivative continuous at z = 1 and zero at z = 2 (C2, compact support)
    d2 = lambda f, z0, hh=1e-4: (f(z0 + hh) - 2 * f(z0) + f(z0 - hh)) / hh**2
    assert abs(d2(gc, 1.0 - 1e-3) - d2(gc, 1.0 + 1e-3)) < 1e-2
    assert abs(d2(gc, 2.0 - 1e-3)) < 1e-2


# ------------------------------------------------------------------ analysis pins
def _global_etkf(geom, Xb, y, sigma2, rho):
    """Global ETKF written in the paper's form (Section 3.1.1, Appendix A):
    Z = anomalies / sqrt(m-1) (pre-inflated by sqrt(rho)), S_cz = Sigma_w^-1/2 C1 Z,
    S_inov = Sigma_w^-1/2 (y - C1 xbar), T = (I + S_cz^T S_cz)^-1/2 via sqrtm,
    xhat from Eq. Est_majA3, X = sqrt(m-1) Z T + xhat."""
    n_pts, _, m = Xb.shape
    xbar = Xb.mean(-1)
    Z = np.sqrt(rho) * (Xb - xbar[..., None]) / np.sqrt(m - 1)
    Zf = Z.reshape(2 * n_pts, m)
    C1 = np.zeros((geom.p, 2 * n_pts))
    C1[:, 1::2] = geom.D1.toarray()
    s = 1 / np.sqrt(sigma2)
    Scz = s * (C1 @ Zf)
    Sinov = s * (y - C1 @ xbar.reshape(-1))
    M = np.eye(m) + Scz.T @ Scz
    T = np.linalg.inv(scipy.linalg.sqrtm(M).real)
    xhat = xbar.reshape(-1) + Zf @ Scz.T @ (Sinov - Scz @ np.linalg.solve(M, Scz.T @ Sinov))
    Xa = np.sqrt(m - 1) * Zf @ T + xhat[:, None]
    return Xa.reshape(n_pts, 2, m)


@pytest.mark.parametrize("rho", [1.0, 1.07])
def test_T1_full_window_is_global_etkf(rho):
    mask = np.ones((3, 3))
    geom = oracle.build_geometry(mask, window=8)      # covers the whole pupil from every node
    m, sigma2 = 12, 0.02
    Xb = synth.random_ensemble(5, geom.n_pts, m)
    y = np.random.default_rng(6).standard_normal(geom.p)
    Xa, mean, spread, local = oracle.analysis(geom, Xb, y, sigma2, rho, return_local=True)
    ref = _global_etkf(geom, Xb, y, sigma2, rho)
    assert np.allclose(Xa, ref, atol=1e-11, rtol=1e-11)
    # every node computed the same transform
    for A, wbar, W in local[1:]:
        assert np.allclose(W, local[0][2], atol=1e-12)
        assert np.allclose(wbar, local[0][1], atol=1e-12)


def test_T2_exact_kalman_filter():
    """Ensemble spanning the state with exact mean mu and covariance P: the
    analysis equals the Kalman filter (Section 2.2, Eqs. Est_maj, Cov_maj, K_Gain)
    with forecast covariance rho P."""
    geom = oracle.build_geometry(np.ones((2, 2)), window=8)
    n_pts = geom.n_pts
    n, m, sigma2, rho = 2 * n_pts, 20, 0.05, 1.1
    rng = np.random.default_rng(3)
    mu = rng.standard_normal(n)
    L = rng.standard_normal((n, n)) / np.sqrt(n) + np.eye(n)
    P = L @ L.T
    O = np.linalg.qr(np.column_stack([np.ones(m), rng.standard_normal((m, m - 1))]))[0]
    E = O[:, 1:n + 1].T                                   # n x m, E E^T = I, E 1 = 0
    Xp = np.linalg.cholesky(P) @ E * np.sqrt(m - 1)
    Xb = (mu[:, None] + Xp).reshape(n_pts, 2, m)
    y = rng.standard_normal(geom.p)
    Xa, mean, spread = oracle.analysis(geom, Xb, y, sigma2, rho)
    H = np.zeros((geom.p, n))
    H[:, 1::2] = geom.D1.toarray()
    Pf = rho * P
    K = Pf @ H.T @ np.linalg.inv(H @ Pf @ H.T + sigma2 * np.eye(geom.p))
    xa = mu + K @ (y - H @ mu)
    Pa = (np.eye(n) - K @ H) @ Pf
    Xaf = Xa.reshape(n, m)
    assert np.allclose(Xaf.mean(1), xa, atol=1e-11)
    Ca = np.cov(Xaf)
    assert np.allclose(Ca, Pa, atol=1e-11)


def test_T3_bruteforce_primal_gain_4x4():
    """Per node, the primal observation-space update (Eq. K_Gain with the sample
    covariance, restricted to the window, R_l = sigma^2 / tau) reproduces the
    ensemble-space result for the node's two rows (Appendix A, Section 4.2)."""
    from paper_1408_7069_gb300.workloads import TINY_4X4 as w
    mask = synth.pupil_subap_mask(w.nsub, square=True)
    geom = oracle.build_geometry(mask, w.window, w.taper, w.loc_len)
    Xb = synth.random_ensemble(9, geom.n_pts, w.m)
    y = np.random.default_rng(10).standard_normal(geom.p)
    Xa, mean, spread = oracle.analysis(geom, Xb, y, w.sigma2, w.rho)
    n = 2 * geom.n_pts
    Xf = Xb.reshape(n, w.m)
    xbar = Xf.mean(1)
    Xp = Xf - xbar[:, None]
    Pb = w.rho * Xp @ Xp.T / (w.m - 1)
    H = np.zeros((geom.p, n))
    H[:, 1::2] = geom.D1.toarray()
    for g in range(geom.n_pts):
        keep = geom.win_tau[g] > 0
        idx = geom.win_idx[g][keep]
        Hl = H[idx]
        Rl = np.diag(w.sigma2 / geom.win_tau[g][keep])
        K = Pb @ Hl.T @ np.linalg.inv(Hl @ Pb @ Hl.T + Rl)
        xa = xbar + K @ (y[idx] - Hl @ xbar)
        Pa = Pb - K @ Hl @ Pb
        rows = [2 * g, 2 * g + 1]
        assert np.allclose(mean[g], xa[rows], atol=1e-10)
        assert np.allclose(np.cov(Xa[g]), Pa[np.ix_(rows, rows)], atol=1e-10)


def test_T4_invariants_with_degenerate_edges():
    mask = synth.pupil_subap_mask(12, 0.25)
    geom = oracle.build_geometry(mask, window=5, taper=1)
    m, rho, sigma2 = 16, 1.03, 0.01
    Xb = synth.random_ensemble(11, geom.n_pts, m, scale=0.5)
    y = np.random.default_rng(12).standard_normal(geom.p)
    Xa, mean, spread, local = oracle.analysis(geom, Xb, y, sigma2, rho, return_local=True)
    xbar, Xp, Yb, ybar = oracle.observe(geom, Xb)
    assert np.linalg.matrix_rank(Yb) <= m - 1
    one = np.ones(m)
    n_degenerate = 0
    for g, (A, wbar, W) in enumerate(local):
        alpha = (m - 1) / rho
        assert np.allclose(W, W.T, atol=1e-12)
        assert np.allclose(W @ one, np.sqrt(rho) * one, atol=1e-10)       # W 1 = sqrt(rho) 1
        assert np.linalg.eigvalsh(A - alpha * np.eye(m)).min() > -1e-9    # A >= (m-1)/rho I
        assert np.allclose(W @ W @ A, (m - 1) * np.eye(m), atol=1e-8)    # W = sqrt(m-1) A^-1/2
        idx = geom.win_idx[g]
        Cd = (Yb[idx].T * (geom.win_tau[g] / sigma2)) @ (y - ybar)[idx]
        assert np.allclose(A @ wbar, Cd, atol=1e-9)                       # wbar = A^-1 C d
        if np.count_nonzero(geom.win_tau[g]) < m - 1:
            n_degenerate += 1
            Wref = np.sqrt(m - 1) * np.linalg.inv(scipy.linalg.sqrtm(A).real)
            assert np.allclose(W, Wref, atol=1e-9)
    assert n_degenerate > 0
    # analysis perturbations stay zero-mean: member mean = xbar + Xb' wbar
    for g, (A, wbar, W) in enumerate(local):
        assert np.allclose(mean[g], xbar[g] + Xp[g] @ wbar, atol=1e-10)


def test_zero_spread_background_is_unchanged():
    geom = oracle.build_geometry(synth.pupil_subap_mask(6, square=True), window=3)
    Xb = np.repeat(np.random.default_rng(1).standard_normal((geom.n_pts, 2, 1)), 8, axis=2)
    y = np.random.default_rng(2).standard_normal(geom.p)
    Xa, mean, spread = oracle.analysis(geom, Xb, y, 0.01, 1.05)
    assert np.allclose(Xa, Xb, atol=1e-13) and np.abs(spread).max() < 1e-13


def test_batched_form_matches_loop():
    geom = oracle.build_geometry(synth.pupil_subap_mask(10, 0.2), window=5, taper=1)
    Xb = synth.random_ensemble(4, geom.n_pts, 12)
    y = np.random.default_rng(5).standard_normal(geom.p)
    a = oracle.analysis(geom, Xb, y, 0.01, 1.02)
    b = oracle.analysis_batched(geom, Xb, y, 0.01, 1.02)
    for u, v in zip(a, b):
        assert np.allclose(u, v, atol=1e-10)


# ------------------------------------------------------------------ forecast pins
def test_forecast_is_ar1_shift():
    Xa = np.random.default_rng(0).standard_normal((7, 2, 5))
    v = np.random.default_rng(1).standard_normal((7, 5))
    Xb = oracle.forecast(Xa, v, 0.97)
    assert np.array_equal(Xb[:, 1], Xa[:, 0])
    assert np.allclose(Xb[:, 0], 0.97 * Xa[:, 0] + v, rtol=0, atol=0)


def test_splitmix64_published_vector():
    g = _golden_kv("splitmix64.txt")
    assert oracle.splitmix64(int(g["seed"]), 0) == int(g["first"], 16)


def test_residual_variance_removes_piston():
    X = np.zeros((5, 2, 3))
    X[:, 0, :] = np.arange(5)[:, None]
    truth = np.arange(5) + 4.0                     # prediction + piston
    assert oracle.residual_variance(truth, X) == pytest.approx(0.0, abs=1e-15)
    truth2 = np.arange(5) + np.array([1, -1, 1, -1, 0.0])
    assert oracle.residual_variance(truth2, X) == pytest.approx(4 / 5)


# ------------------------------------------------------------------ op counts
def test_table1_operation_counts():
    with open(os.path.join(GOLDEN, "table1_opcounts.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for kind, m, n, p, val in rows:
        m, n, p, val = int(m), int(n), int(p), float(val)
        got = opcount.update_ops(m, n, p) if kind == "update" else opcount.prediction_ops(m, n)
        assert abs(got - val) / val < 0.005, (kind, got, val)


def test_taper_support_matches_the_oracle_windows():
    """The kernels skip window cells outside the Gaspari-Cohn support; the
    executed-flops count takes their number from opcount. For an interior
    node of a full square pupil the oracle's window has exactly two slopes
    with a nonzero taper per such cell."""
    mask = np.ones((12, 12), bool)
    for window, loc_len in ((3, 0.0), (5, 0.0), (7, 0.0), (7, 1.2), (5, 3.0)):
        g = oracle.build_geometry(mask, window, taper=1, loc_len=loc_len)
        q = 6 * 13 + 6                                  # node (6, 6), row-major over 13 x 13
        nz = int(np.count_nonzero(np.asarray(g.win_tau[q]) > 0))
        assert nz == 2 * opcount.taper_support_cells(window, 1, loc_len), (window, loc_len, nz)
        assert opcount.taper_support_cells(window, 0) == window * window


# ------------------------------------------------------------------ synthetic turbulence
def test_T6_structure_function_kolmogorov():
    r0, dx = 0.15, 0.04
    scr = synth.von_karman_screens(7, 8, 256, 256, dx, r0, L0=1e4)
    for lag in (3, 6, 12):
        d = np.mean((scr[:, lag:, :] - scr[:, :-lag, :]) ** 2)
        expected = 6.88 * (lag * dx / r0) ** (5.0 / 3.0)
        assert abs(d / expected - 1) < 0.15, (lag, d, expected)


def test_synth_is_seed_deterministic():
    a = synth.von_karman_screens(3, 2, 32, 32, 0.5, 0.15, 25.0)
    b = synth.von_karman_screens(3, 2, 32, 32, 0.5, 0.15, 25.0)
    c = synth.von_karman_screens(4, 2, 32, 32, 0.5, 0.15, 25.0)
    assert np.array_equal(a, b) and not np.allclose(a, c)


def test_synth_slopes_delay():
    from paper_1408_7069_gb300.workloads import TOY_8X8
    inp = synth.make_loop_inputs(TOY_8X8, frames=5)
    mask = inp.subap_mask
    geom = oracle.build_geometry(mask, 3)
    # y_k - D phi_{k-1} is pure noise of std sigma
    phi_prev = inp.truth[1:4]
    resid = inp.slopes[2:5] - phi_prev @ geom.D1.T
    assert abs(resid.std() / TOY_8X8.sigma - 1) < 0.15
