"""Pins of the DM oracle (Sections 2.1-2.2, Appendix B.3): the influence matrix
against the paper's coupling and the Appendix B sparsity of D1 N, the
least-squares projection against its defining property (P N = I before the
truncation), the calibration inputs the GPU receives against the oracle's own
matrices, and the closed loop with N = P = I against the pseudo-open-loop
oracle (a separately pinned function)."""
import numpy as np
import scipy.sparse

import oracle
from oracle import letkf_dm as DM
from paper_1408_7069_gb300 import synth, workloads as W


def test_influence_matrix_coupling_and_support():
    geom = oracle.build_geometry(synth.pupil_subap_mask(12, 0.0), 3)
    N = DM.influence_matrix(geom).toarray()
    pid = {tuple(p): k for k, p in enumerate(geom.points)}
    a = pid[(6, 6)]
    assert N[a, a] == 1.0
    assert np.isclose(N[pid[(7, 6)], a], 0.3) and np.isclose(N[pid[(6, 5)], a], 0.3)  # Section 5
    assert np.isclose(N[pid[(7, 7)], a], 0.09)
    assert N[pid[(9, 6)], a] == 0.0                    # beyond two pitches
    # Appendix B: every row of D1 N has at most 36 nonzeros, 36 inside the pupil
    DN = (geom.D1 @ scipy.sparse.csr_matrix(N)).tocsr()
    nnz = np.diff(DN.indptr)
    assert nnz.max() == 36 and (nnz == 36).sum() > 0


def test_projection_is_the_least_squares_left_inverse():
    geom = oracle.build_geometry(synth.pupil_subap_mask(10, 0.2), 3)
    N = DM.influence_matrix(geom)
    Pf = DM.projection_matrix(geom, N, drop=0.0).toarray()
    assert np.allclose(Pf @ N.toarray(), np.eye(geom.n_pts), atol=1e-10)
    # the least-squares solution by an independent route (SVD pseudo-inverse)
    assert np.allclose(Pf, np.linalg.pinv(N.toarray()), atol=1e-10)
    # the stored sparse P drops only negligible entries
    Ps = DM.projection_matrix(geom, N).toarray()
    assert (Ps == 0).mean() > 0.1
    assert np.abs(Ps - Pf).max() <= 1e-6 * np.abs(Pf).max()
    # the radius-2 truncation of Appendix B.3 would change a smooth phase's
    # command by far more than the analysis tolerances (why it is not used)
    P2 = DM.projection_matrix(geom, N, radius=2.0, drop=0.0).toarray()
    d = np.hypot(*(geom.points[:, None, :] - geom.points[None, :, :]).transpose(2, 0, 1))
    assert np.all(P2[d > 2.0 + 1e-9] == 0.0) and np.allclose(P2[d <= 2.0], Pf[d <= 2.0])
    phi = np.sin(0.3 * geom.points[:, 0]) + np.cos(0.2 * geom.points[:, 1])
    assert np.linalg.norm(P2 @ phi - Pf @ phi) > 0.3 * np.linalg.norm(Pf @ phi)


def test_synthetic_calibration_is_the_oracles():
    mask = synth.pupil_subap_mask(16, 0.14)
    geom = oracle.build_geometry(mask, 3)
    Ns, Ps = synth.dm_calibration(mask)
    No = DM.influence_matrix(geom)
    Po = DM.projection_matrix(geom, No)
    assert np.allclose(Ns.toarray(), No.toarray(), atol=0, rtol=0)
    assert np.allclose(Ps.toarray(), Po.toarray(), atol=1e-10)


def test_identity_mirror_is_the_pseudo_open_loop():
    w = W.TOY_8X8
    inp = synth.make_loop_inputs(w, frames=8)
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.loc_len)
    # w_k = y_k - D1 phi_{k-1} of the open-loop slopes (phi_{-1} = 0)
    prev = np.vstack([np.zeros((1, geom.n_pts)), inp.truth[:-1]])
    wnoise = inp.slopes - prev @ geom.D1.T
    I = scipy.sparse.identity(geom.n_pts, format="csr")
    rv, X, us, ys = DM.closed_loop_dm(geom, inp.truth, wnoise, inp.bank, w.m, w.sigma2, w.rho,
                                      w.a_ar1, w.noise_std, w.seeds[2], 8, I, I, inp.X0)
    rv0, X0, _ = oracle.closed_loop(geom, inp.truth, inp.slopes, inp.bank, w.m, w.sigma2, w.rho,
                                    w.a_ar1, w.noise_std, w.seeds[2], 8, X0=inp.X0, batched=True)
    # frame 0 has no command yet (u_{-1} = 0): its residual is the turbulence
    t0 = inp.truth[0] - inp.truth[0].mean()
    assert np.isclose(rv[0], np.mean(t0 * t0), rtol=1e-12)
    assert np.allclose(rv[1:], rv0[1:], rtol=1e-10, atol=0)
    assert np.allclose(X, X0, rtol=1e-10, atol=1e-12)
    # the command is the predicted phase
    assert np.allclose(us[-1], X0[:, 0, :].mean(-1), atol=1e-12)


def test_square_mirror_corrects_the_predicted_phase():
    """Actuators at the valid nodes make N square and invertible, so N P is the
    identity up to the dropped entries of P: the correction N u_{k-1} is the
    predicted phase, and the closed loop follows the pseudo-open-loop one
    (frames after the first, which has no command yet)."""
    w = W.TEL_16M
    inp = synth.make_loop_inputs(w, frames=12)
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.loc_len)
    prev = np.vstack([np.zeros((1, geom.n_pts)), inp.truth[:-1]])
    wnoise = inp.slopes - prev @ geom.D1.T
    N = DM.influence_matrix(geom)
    P = DM.projection_matrix(geom, N)
    assert np.abs((N @ P).toarray() - np.eye(geom.n_pts)).max() < 1e-4
    rv, _, us, _ = DM.closed_loop_dm(geom, inp.truth, wnoise, inp.bank, w.m, w.sigma2, w.rho,
                                     w.a_ar1, w.noise_std, w.seeds[2], 12, N, P, inp.X0)
    rv0, _, _ = oracle.closed_loop(geom, inp.truth, inp.slopes, inp.bank, w.m, w.sigma2, w.rho,
                                   w.a_ar1, w.noise_std, w.seeds[2], 12, X0=inp.X0, batched=True)
    assert np.all(np.isfinite(rv)) and np.max(np.abs(rv[1:] / rv0[1:] - 1)) < 1e-4
    # the commands are not the phase itself: the mirror's coupling is undone
    assert np.linalg.norm(us[-1] - (N @ us[-1])) > 0.1 * np.linalg.norm(us[-1])
