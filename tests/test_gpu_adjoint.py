"""Reverse mode of the closed loop on the GPU (letkf_grad): the gradient of the
mean residual variance (Section 2.1, Eq. Crit_Opt) with respect to rho, sigma2
and the localization length L, against the oracle's reverse mode and against
finite differences of the GPU loop itself."""
import functools
from dataclasses import replace

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1408_7069_gb300 import synth, workloads as W  # noqa: E402
from paper_1408_7069_gb300 import letkf as L  # noqa: E402

pytestmark = pytest.mark.gpu


def loc_len(w):
    return w.loc_len if w.loc_len > 0 else w.window / 4.0


@functools.lru_cache(maxsize=None)
def loop_inputs(w, frames):
    return synth.make_loop_inputs(w, frames=frames)


def oracle_grad(w, inp, frames, rt):
    """Oracle J and gradient on the inputs as the GPU sees them (rounded to rt)."""
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, loc_len(w))
    c = lambda a: np.asarray(a).astype(rt).astype(np.float64)  # noqa: E731
    J, g, _ = oracle.closed_loop_grad(geom, c(inp.truth), c(inp.slopes), inp.bank, w.m, w.sigma2,
                                      w.rho, w.a_ar1, w.noise_std, w.seeds[2], frames, c(inp.X0))
    return J, g


def gpu_grad(w, inp, frames, ckpt=0, f=None):
    rt = np.float32 if w.precision == 0 else np.float64
    own = f is None
    if own:
        f = L.Letkf.from_workload(w, bank=inp.bank)
    f.set_state(torch.from_numpy(inp.X0.astype(rt)).cuda())
    f.set_frame(0)
    y = torch.from_numpy(inp.slopes[:frames].astype(rt)).cuda()
    t = torch.from_numpy(inp.truth[:frames].astype(rt)).cuda()
    J, g = f.grad(frames, y, t, ckpt)
    f.sync()
    if own:
        f.close()
    return J, g


FP32_CASES = [
    (replace(W.ADJ_16M, name="adj-20x20", nsub=20, seeds=(61, 62, 63)), 10),
    (W.ADJ_16M, 6),
    (replace(W.ADJ_16M, name="adj-m16-w7", nsub=16, m=16, window=7, seeds=(71, 72, 73)), 8),
]


@pytest.mark.parametrize("w,frames", FP32_CASES, ids=[c[0].name for c in FP32_CASES])
def test_fp32_gradient_matches_oracle(w, frames):
    inp = loop_inputs(w, frames)
    J, g = gpu_grad(w, inp, frames, ckpt=4)
    Jr, gr = oracle_grad(w, inp, frames, np.float32)
    assert J == pytest.approx(Jr, rel=1e-4)
    for k in range(3):
        assert abs(g[k] - gr[k]) <= 1e-3 * abs(gr[k]), (k, g, gr)


FP64_CASES = [W.TINY_4X4,
              replace(W.TINY_4X4, name="tiny-degenerate", m=16, seeds=(4, 5, 6)),
              replace(W.TOY_8X8, name="toy-gc", m=10, loc_len=1.2),
              replace(W.TOY_8X8, name="toy-notaper", m=12, taper=0, window=5, seeds=(14, 15, 16))]


@pytest.mark.parametrize("w", FP64_CASES, ids=[w.name for w in FP64_CASES])
def test_fp64_gradient_matches_oracle(w):
    """FP64 handles: the same arithmetic as the oracle up to rounding order (the
    degenerate case has windows with fewer slopes than m - 1, so exactly equal
    eigenvalues; without the taper dJ/dL is exactly zero)."""
    frames = 8
    inp = loop_inputs(w, frames)
    J, g = gpu_grad(w, inp, frames, ckpt=3)
    Jr, gr = oracle_grad(w, inp, frames, np.float64)
    assert J == pytest.approx(Jr, rel=1e-10)
    scale = np.max(np.abs(gr))
    for k in range(3):
        assert abs(g[k] - gr[k]) <= 1e-8 * max(abs(gr[k]), 1e-6 * scale), (k, g, gr)
    if w.taper == 0:
        assert g[2] == 0.0


def test_fp64_gradient_matches_gpu_finite_differences():
    """Central differences of the GPU loop itself (letkf_set_params + letkf_run),
    Richardson-extrapolated, against letkf_grad. The FP64 eigensolve starts
    from the identity here: started from the FP32 basis pass, the last bits of
    each analysis follow that basis, whose rotations change discontinuously with
    the parameters, and J(theta) carries noise of about 1e-10 relative, which
    the differences of step 1e-4 turn into about 2e-6 of the derivative. The
    gradient of the default (warm) start is compared with this one beside it."""
    w = replace(W.TOY_8X8, name="toy-gc", m=10, loc_len=1.2)
    frames = 8
    inp = loop_inputs(w, frames)
    f = L.Letkf.from_workload(w, bank=inp.bank)
    f.set_fp64_start(False)
    y = torch.from_numpy(inp.slopes[:frames]).cuda()
    t = torch.from_numpy(inp.truth[:frames]).cuda()
    X0 = torch.from_numpy(inp.X0).cuda()

    def J_at(rho, s2, Ll):
        f.set_params(rho, s2, Ll)
        f.set_state(X0)
        f.set_frame(0)
        rv = f.run(frames, y, t, use_graph=False)
        f.sync()
        return float(rv.cpu().numpy().mean())

    theta = np.array([w.rho, w.sigma2, loc_len(w)])

    def fd(k, h):
        def at(s):
            th = theta.copy()
            th[k] *= 1 + s
            return J_at(*th)
        d1 = (at(h) - at(-h)) / (2 * h * theta[k])
        d2 = (at(h / 2) - at(-h / 2)) / (h * theta[k])
        return (4 * d2 - d1) / 3

    num = [fd(k, 1e-4) for k in range(3)]
    f.set_params(*theta)
    J, g = gpu_grad(w, inp, frames, f=f)
    f.set_fp64_start(True)
    Jw, gw = gpu_grad(w, inp, frames, f=f)
    f.close()
    for k in range(3):
        assert abs(g[k] - num[k]) <= 1e-6 * max(abs(num[k]), 1e-9 * J), (g, num)
    # the two starts differ by rounding, which the 8-frame loop amplifies
    # (measured 7e-12 in J)
    assert Jw == pytest.approx(J, rel=1e-10)
    assert np.allclose(gw, g, rtol=1e-7, atol=0), (gw, g)


def test_checkpoint_spacing_and_replay_are_bitwise_invariant():
    w, frames = FP32_CASES[0][0], 12
    inp = loop_inputs(w, frames)
    f = L.Letkf.from_workload(w, bank=inp.bank)
    ref = gpu_grad(w, inp, frames, ckpt=0, f=f)
    again = gpu_grad(w, inp, frames, ckpt=0, f=f)     # graph replay
    assert again[0] == ref[0] and np.array_equal(again[1], ref[1])
    for ck in (1, 5, 12):
        out = gpu_grad(w, inp, frames, ckpt=ck, f=f)
        assert out[0] == ref[0] and np.array_equal(out[1], ref[1]), ck
    f.close()


def test_state_after_grad_equals_letkf_run():
    w, frames = FP32_CASES[0][0], 9
    inp = loop_inputs(w, frames)
    y = torch.from_numpy(inp.slopes[:frames].astype(np.float32)).cuda()
    t = torch.from_numpy(inp.truth[:frames].astype(np.float32)).cuda()
    X0 = torch.from_numpy(inp.X0.astype(np.float32)).cuda()
    a = L.Letkf.from_workload(w, bank=inp.bank)
    a.set_state(X0)
    J, _ = a.grad(frames, y, t, 4)
    a.forecast()                       # the frame counter moved on with the state
    Xa = a.get_state().cpu().numpy()
    b = L.Letkf.from_workload(w, bank=inp.bank)
    b.set_state(X0)
    rv = b.run(frames, y, t, use_graph=True)
    b.forecast()
    Xb = b.get_state().cpu().numpy()
    assert np.array_equal(Xa, Xb)
    assert J == pytest.approx(float(rv.cpu().numpy().mean()), rel=1e-14)
    a.close()
    b.close()


def test_autograd_function_returns_the_library_gradient():
    w, frames = FP32_CASES[0][0], 6
    inp = loop_inputs(w, frames)
    f = L.Letkf.from_workload(w, bank=inp.bank)
    y = torch.from_numpy(inp.slopes[:frames].astype(np.float32)).cuda()
    t = torch.from_numpy(inp.truth[:frames].astype(np.float32)).cuda()
    X0 = torch.from_numpy(inp.X0.astype(np.float32)).cuda()
    theta = [torch.tensor(v, dtype=torch.float64, requires_grad=True)
             for v in (w.rho, w.sigma2, loc_len(w))]
    J = L.letkf_loss(*theta, f, X0, y, t, frames, ckpt_every=2)
    (3.0 * J).backward()
    J2, g = gpu_grad(w, inp, frames, f=f)
    assert float(J.detach()) == J2
    for th, gk in zip(theta, g):
        assert float(th.grad) == pytest.approx(3.0 * gk, rel=1e-12)
    f.close()


def test_grad_rejects_unsupported_handles():
    inp = loop_inputs(W.TINY_4X4, 3)
    y = torch.zeros(3, 2 * int(inp.subap_mask.sum()), dtype=torch.float64).cuda()
    f = L.Letkf.from_workload(W.TINY_4X4, bank=None)
    t = torch.zeros(3, f.n_pts, dtype=torch.float64).cuda()
    with pytest.raises(L.LetkfError, match="LETKF_ERR_STATE"):
        f.grad(3, y, t)
    f.close()
    wide = replace(W.TINY_4X4, m=40, precision=0)
    g = L.Letkf.from_workload(wide, bank=inp.bank)
    with pytest.raises(L.LetkfError, match="LETKF_ERR_ARG"):
        g.grad(3, y.float(), t.float())
    g.close()
    b = L.Letkf.batch([W.TINY_4X4, W.TINY_4X4], [inp.bank, inp.bank])
    with pytest.raises(ValueError):
        b.grad(3, y, t)
    b.close()


def _golden(name):
    import os
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split(None, 1)
                out[k] = float(v)
    return out


def test_fp64_gradient_over_200_frames_matches_oracle_golden():
    """The 16 m system over 200 frames from the prior draw (checkpoint every 20
    frames) on an FP64 handle against the oracle's reverse mode, stored by
    tests/golden/make_adjoint_golden.py. Over this horizon J is rough in the
    parameters, so FP32 trajectories give gradients that differ by percents;
    the FP64 path must agree to rounding."""
    g0 = _golden("adjoint_16m_200f.txt")
    w = replace(W.ADJ_16M, precision=1)
    frames = W.ADJ_16M.frames
    inp = synth.make_loop_inputs(w, frames=frames)
    c = lambda a: np.asarray(a).astype(np.float32).astype(np.float64)  # noqa: E731
    f = L.Letkf.from_workload(w, bank=inp.bank)
    f.set_state(torch.from_numpy(c(inp.X0)).cuda())
    J, g = f.grad(frames, torch.from_numpy(c(inp.slopes[:frames])).cuda(),
                  torch.from_numpy(c(inp.truth[:frames])).cuda(), 20)
    f.sync()
    f.close()
    assert J == pytest.approx(g0["J"], rel=1e-9)
    for k, name in enumerate(("dJ_drho", "dJ_dsigma2", "dJ_dL")):
        assert g[k] == pytest.approx(g0[name], rel=1e-7), name
