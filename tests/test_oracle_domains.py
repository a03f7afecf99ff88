"""Pins of the domain oracle (multi-actuator local domains, Section 4, and the
differential-piston least squares, Section 4.4) to what the paper and the
mathematics fix:

* the domain counts and the largest local problem the paper prints
  (Section 5.1: 25 domains; Section 5.3: 373 domains, n_max = 32, p_max = 128,
  n = 10370 for the 40 m case);
* one-node domains are the per-node LETKF (the other, separately pinned oracle);
* one domain covering the pupil is the global ETKF in the paper's S_cz / S_inov
  form (Section 3.1.1), written here independently;
* every domain's mean update is the observation-space Kalman update with the
  ensemble covariance restricted to its rows and region (Section 2.2 Eq.
  K_Gain, via the identity of Appendix A);
* the piston least squares: piecewise-constant offsets are removed exactly,
  a brute-force constrained minimisation agrees, and the result is optimal.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

import oracle
from oracle import letkf_domains as LD
from paper_1408_7069_gb300 import synth


def test_domain_counts_of_section_5():
    # 40 m telescope, 80 x 80 sensor, 21 x 21 partition: 373 domains of at most
    # 16 actuators (n_max = 32) observing at most 128 slopes; n = 10370
    dg = LD.build_domains(synth.pupil_subap_mask(80, 0.0), 21, window=5)
    assert dg.n_dom == 373
    assert 2 * dg.geom.n_pts == 10370
    assert max(2 * len(n) for n in dg.dom_nodes) == 32
    assert max(len(o) for o in dg.dom_obs) == 128
    # 16 m telescope, 32 x 32 sensor, 5 x 5 partition: 25 domains
    dg = LD.build_domains(synth.pupil_subap_mask(32, 0.0), 5, window=5)
    assert dg.n_dom == 25
    # every node belongs to exactly one domain
    allnodes = np.sort(np.concatenate(dg.dom_nodes))
    assert np.array_equal(allnodes, np.arange(dg.geom.n_pts))


def test_one_node_domains_are_the_node_analysis():
    mask = synth.pupil_subap_mask(10, 0.2)
    w, c = 5, 1.3
    dg = LD.build_domains(mask, 11, window=w, taper=1, loc_len=c)
    geom = oracle.build_geometry(mask, w, taper=1, loc_len=c)
    assert dg.n_dom == geom.n_pts
    Xb = synth.random_ensemble(7, geom.n_pts, 12)
    y = np.random.default_rng(8).standard_normal(geom.p)
    a = LD.analysis_domains(dg, Xb, y, 0.02, 1.04, piston=False)
    b = oracle.analysis(geom, Xb, y, 0.02, 1.04)
    for u, v in zip(a, b):
        assert np.allclose(u, v, atol=1e-12, rtol=1e-12)


def _global_etkf(geom, Xb, y, sigma2, rho):
    """Global ETKF in the paper's form (Section 3.1.1, Appendix A) with the
    inflation applied to the anomalies: Z = sqrt(rho) X' / sqrt(m - 1),
    S_cz = Sigma_w^-1/2 C1 Z, S_inov = Sigma_w^-1/2 (y - C1 xbar),
    T = (I + S_cz^T S_cz)^-1/2, xhat by Eq. Est_majA4, X = sqrt(m-1) Z T + xhat."""
    n_pts, _, m = Xb.shape
    xbar = Xb.mean(-1).reshape(-1)
    Zf = np.sqrt(rho) * (Xb - Xb.mean(-1, keepdims=True)).reshape(2 * n_pts, m) / np.sqrt(m - 1)
    C1 = np.zeros((geom.p, 2 * n_pts))
    C1[:, 1::2] = geom.D1.toarray()
    Scz = (C1 @ Zf) / np.sqrt(sigma2)
    Sinov = (y - C1 @ xbar) / np.sqrt(sigma2)
    M = np.eye(m) + Scz.T @ Scz
    T = np.linalg.inv(scipy.linalg.sqrtm(M).real)
    xhat = xbar + Zf @ Scz.T @ (Sinov - Scz @ np.linalg.solve(M, Scz.T @ Sinov))
    return (np.sqrt(m - 1) * Zf @ T + xhat[:, None]).reshape(n_pts, 2, m)


@pytest.mark.parametrize("rho", [1.0, 1.06])
def test_single_domain_is_the_global_etkf(rho):
    mask = synth.pupil_subap_mask(6, 0.0)
    dg = LD.build_domains(mask, 1, window=16)       # one block, region = the pupil
    assert dg.n_dom == 1 and len(dg.dom_obs[0]) == dg.geom.p and len(dg.edges) == 0
    m = 14
    Xb = synth.random_ensemble(9, dg.geom.n_pts, m)
    y = np.random.default_rng(10).standard_normal(dg.geom.p)
    Xa, mean, spread = LD.analysis_domains(dg, Xb, y, 0.03, rho)
    assert np.allclose(Xa, _global_etkf(dg.geom, Xb, y, 0.03, rho), atol=1e-10, rtol=1e-10)


def test_domain_mean_is_the_primal_kalman_update():
    """x_d = xbar_d + P_dH^T (H P H^T + R_l / tau)^-1 (y_l - H xbar) per domain,
    P = rho X' X'^T / (m - 1) (rows of the domain against all phi_{k-1} rows)."""
    mask = synth.pupil_subap_mask(6, 0.0)
    dg = LD.build_domains(mask, 3, window=3, taper=1, loc_len=2.0)
    geom = dg.geom
    m, sigma2, rho = 9, 0.05, 1.08
    Xb = synth.random_ensemble(11, geom.n_pts, m)
    y = np.random.default_rng(12).standard_normal(geom.p)
    Xa, mean, _ = LD.analysis_domains(dg, Xb, y, sigma2, rho, piston=False)
    Xp = (Xb - Xb.mean(-1, keepdims=True)).reshape(2 * geom.n_pts, m)
    xbar = Xb.mean(-1).reshape(-1)
    H = np.zeros((geom.p, 2 * geom.n_pts))
    H[:, 1::2] = geom.D1.toarray()
    P = rho * Xp @ Xp.T / (m - 1)
    for nodes, idx, tau in zip(dg.dom_nodes, dg.dom_obs, dg.dom_tau):
        keep = tau > 0
        idx, tau = idx[keep], tau[keep]
        Hl = H[idx]
        rows = np.concatenate([[2 * g, 2 * g + 1] for g in nodes])
        S = Hl @ P @ Hl.T + np.diag(sigma2 / tau)
        xd = xbar[rows] + P[rows] @ Hl.T @ np.linalg.solve(S, y[idx] - Hl @ xbar)
        assert np.allclose(mean.reshape(-1)[rows], xd, atol=1e-10)


def test_piston_removes_piecewise_constant_offsets():
    dg = LD.build_domains(synth.pupil_subap_mask(16, 0.14), 5, window=5)
    p = np.random.default_rng(13).standard_normal((dg.n_dom, 2))
    delta = p[dg.node_dom]                          # each domain shifted by its own piston
    c = LD.piston_offsets(dg, delta)
    fixed = delta + c[dg.node_dom]
    counts = np.array([len(n) for n in dg.dom_nodes], float)
    level = (counts[:, None] * p).sum(0) / counts.sum()
    assert np.allclose(fixed, level[None, :], atol=1e-12)
    # a global constant changes nothing; zero increments need no correction
    assert np.allclose(LD.piston_offsets(dg, delta + 3.7), c, atol=1e-12)
    assert np.allclose(LD.piston_offsets(dg, np.zeros_like(delta)), 0.0, atol=1e-14)


def test_piston_least_squares_by_brute_force():
    dg = LD.build_domains(synth.pupil_subap_mask(6, 0.0), 3, window=3)
    rng = np.random.default_rng(14)
    delta = rng.standard_normal((dg.geom.n_pts, 2))
    c = LD.piston_offsets(dg, delta)
    counts = np.array([len(n) for n in dg.dom_nodes], float)
    di, dj = dg.node_dom[dg.edges[:, 0]], dg.node_dom[dg.edges[:, 1]]
    for r in range(2):
        jump = delta[dg.edges[:, 0], r] - delta[dg.edges[:, 1], r]

        def cost(x):
            return float(np.sum((jump + x[di] - x[dj]) ** 2))

        res = scipy.optimize.minimize(cost, np.zeros(dg.n_dom), method="SLSQP",
                                      constraints=[{"type": "eq", "fun": lambda x: counts @ x}],
                                      options={"ftol": 1e-14, "maxiter": 500})
        assert np.allclose(res.x, c[:, r], atol=1e-6)
        assert abs(counts @ c[:, r]) < 1e-10
        # optimal: no feasible perturbation lowers the cost
        base = cost(c[:, r])
        for _ in range(20):
            u = rng.standard_normal(dg.n_dom)
            u -= counts * (counts @ u) / (counts @ counts)
            assert cost(c[:, r] + 1e-3 * u) >= base - 1e-12


def test_piston_corrected_analysis_is_continuous():
    """After the correction no further piston lowers the border jumps: the
    least squares applied to the corrected increments returns zero, and the
    jumps are no larger than without the correction."""
    mask = synth.pupil_subap_mask(16, 0.14)
    dg = LD.build_domains(mask, 4, window=5, taper=1)
    m = 16
    Xb = synth.random_ensemble(15, dg.geom.n_pts, m)
    y = np.random.default_rng(16).standard_normal(dg.geom.p)
    xbar = Xb.mean(-1)
    Xa0, mean0, _ = LD.analysis_domains(dg, Xb, y, 0.02, 1.03, piston=False)
    Xa1, mean1, spread1, _, c = LD.analysis_domains(dg, Xb, y, 0.02, 1.03, return_parts=True)
    assert np.abs(c).max() > 1e-3                      # there was something to correct
    assert np.allclose(LD.piston_offsets(dg, mean1 - xbar), 0.0, atol=1e-10)

    def jumps(mean):
        d = mean - xbar
        return np.sum((d[dg.edges[:, 0]] - d[dg.edges[:, 1]]) ** 2)

    assert jumps(mean1) < jumps(mean0)
    # the correction moves whole domains: anomalies and spread are unchanged
    assert np.allclose(Xa1 - mean1[..., None], Xa0 - mean0[..., None], atol=1e-12)


def test_taper_is_one_inside_the_domain_box():
    """The localization weight depends on the distance to the domain's node
    box: every subaperture whose centre lies inside the box has weight 1, and
    the weight falls off outside it."""
    mask = synth.pupil_subap_mask(20, 0.0)
    dg = LD.build_domains(mask, 5, window=5, taper=1, loc_len=1.25)
    geom = dg.geom
    n_sap = len(geom.subaps)
    inside = outside = 0
    for nodes, idx, tau in zip(dg.dom_nodes, dg.dom_obs, dg.dom_tau):
        pts = geom.points[nodes]
        i0, i1, j0, j1 = pts[:, 0].min(), pts[:, 0].max(), pts[:, 1].min(), pts[:, 1].max()
        for k, t in zip(idx, tau):
            s, u = geom.subaps[k % n_sap] + 0.5
            if i0 <= s <= i1 and j0 <= u <= j1:
                assert t == 1.0
                inside += 1
            elif max(i0 - s, s - i1, j0 - u, u - j1) >= 1.0:
                assert t < 1.0
                outside += 1
    assert inside > 0 and outside > 0
