"""GPU parity of the deformable-mirror side of the loop (Sections 2.1-2.2,
Appendix B.3) against the DM oracle: the true closed loop (measurement of the
residual phase, pseudo-open-loop analysis, command from the prediction), the
command itself, the identity mirror against the pseudo-open-loop form, and the
calls that refuse a mirror."""
from dataclasses import replace

import numpy as np
import pytest
import scipy.sparse

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import letkf_dm as DM  # noqa: E402
from paper_1408_7069_gb300 import synth, workloads as W  # noqa: E402
from paper_1408_7069_gb300.letkf import Letkf, LetkfError  # noqa: E402

pytestmark = pytest.mark.gpu


def f32(a):
    return np.asarray(a).astype(np.float32).astype(np.float64)


def loop_inputs(w, frames):
    inp = synth.make_loop_inputs(w, frames=frames)
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.loc_len)
    prev = np.vstack([np.zeros((1, geom.n_pts)), inp.truth[:-1]])
    wnoise = inp.slopes - prev @ geom.D1.T                  # w_k of the open-loop slopes
    return inp, geom, f32(inp.truth), f32(wnoise)


@pytest.mark.parametrize("w", [W.TEL_16M, W.TOY_8X8], ids=["16m-fp32", "8x8-fp64"])
def test_dm_closed_loop_matches_oracle(w):
    frames = 10
    inp, geom, truth, wnoise = loop_inputs(w, frames)
    Ns, Ps = synth.dm_calibration(inp.subap_mask)
    No = DM.influence_matrix(geom)
    Po = DM.projection_matrix(geom, No)
    rt = np.float32 if w.precision == 0 else np.float64
    f = Letkf.from_workload(w, bank=inp.bank)
    f.set_state(torch.from_numpy(inp.X0.astype(rt)).cuda())
    f.set_dm(Ns, Ps)
    rv = f.run_dm(frames, torch.from_numpy(truth.astype(rt)).cuda(),
                  torch.from_numpy(wnoise.astype(rt)).cuda()).cpu().numpy()
    u = f.command().cpu().numpy()
    X = f.get_state().cpu().numpy()
    f.sync()
    f.close()
    rv_ref, X_ref, us, _ = DM.closed_loop_dm(geom, truth, wnoise, inp.bank, w.m, w.sigma2, w.rho,
                                             w.a_ar1, w.noise_std, w.seeds[2], frames, No, Po,
                                             f32(inp.X0) if w.precision == 0 else inp.X0)
    tol = 1e-3 if w.precision == 0 else 1e-8
    assert np.max(np.abs(rv - rv_ref) / rv_ref) <= tol, (rv, rv_ref)
    assert np.linalg.norm(u - us[-1]) <= tol * np.linalg.norm(us[-1])


def test_identity_mirror_equals_the_pseudo_open_loop_on_the_gpu():
    w = W.TEL_16M
    frames = 8
    inp, geom, truth, wnoise = loop_inputs(w, frames)
    X0 = torch.from_numpy(inp.X0.astype(np.float32)).cuda()
    I = scipy.sparse.identity(geom.n_pts, format="csr")
    f = Letkf.from_workload(w, bank=inp.bank)
    f.set_state(X0)
    rv0 = f.run(frames, torch.from_numpy(inp.slopes.astype(np.float32)).cuda(),
                torch.from_numpy(inp.truth.astype(np.float32)).cuda(), use_graph=False)
    f.sync()
    f.set_state(X0)
    f.set_frame(0)
    f.set_dm(I, I)
    rv1 = f.run_dm(frames, torch.from_numpy(truth.astype(np.float32)).cuda(),
                   torch.from_numpy(wnoise.astype(np.float32)).cuda(), use_graph=False)
    f.sync()
    f.close()
    a, b = rv0.cpu().numpy(), rv1.cpu().numpy()
    assert np.max(np.abs(a[1:] - b[1:]) / a[1:]) <= 1e-4


def test_command_is_the_projected_prediction():
    w = W.TEL_16M
    inp, geom, truth, wnoise = loop_inputs(w, 4)
    Ns, Ps = synth.dm_calibration(inp.subap_mask)
    f = Letkf.from_workload(w, bank=inp.bank)
    f.set_state(torch.from_numpy(inp.X0.astype(np.float32)).cuda())
    f.set_dm(Ns, Ps)
    f.forecast()
    u = f.command().cpu().numpy().astype(np.float64)
    X = f.get_state().cpu().numpy().astype(np.float64)
    f.sync()
    f.close()
    Po = DM.projection_matrix(geom, DM.influence_matrix(geom))
    ref = Po @ X[:, 0, :].mean(-1)
    assert np.linalg.norm(u - ref) <= 1e-5 * np.linalg.norm(ref)


def test_mirror_is_refused_where_it_does_not_apply():
    w = W.TEL_16M
    inp = synth.make_loop_inputs(w, frames=3)
    Ns, Ps = synth.dm_calibration(inp.subap_mask)
    f = Letkf.from_workload(w, bank=inp.bank)
    with pytest.raises(LetkfError, match="LETKF_ERR_STATE"):
        f.run_dm(1, torch.zeros(1, f.n_pts, device="cuda"), torch.zeros(1, f.p, device="cuda"))
    with pytest.raises(LetkfError, match="LETKF_ERR_STATE"):
        f.command()
    bad = Ns.copy()
    bad.indices = bad.indices.copy()
    bad.indices[0] = f.n_pts + 5
    with pytest.raises(LetkfError, match="LETKF_ERR_ARG"):
        f.set_dm(bad, Ps)
    f.set_dm(Ns, Ps)
    y = torch.from_numpy(inp.slopes.astype(np.float32)).cuda()
    t = torch.from_numpy(inp.truth.astype(np.float32)).cuda()
    with pytest.raises(LetkfError, match="LETKF_ERR_STATE"):
        f.grad(2, y, t)
    f.close()
    g = Letkf.batch([w, replace(w, seeds=(1, 2, 3))], [inp.bank, inp.bank])
    with pytest.raises(LetkfError, match="LETKF_ERR_ARG"):
        g.set_dm(Ns, Ps)
    g.close()
