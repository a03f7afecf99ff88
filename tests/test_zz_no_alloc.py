"""The allocation-free entry point (letkf_analyze_noalloc) for callers that
cannot allocate device memory at run time: it must give the same analysis as
the handle-based letkf_analyze and as the FP64 oracle, call after call,
although its scratch is one static array shared by every call; its status
query must report the faults and the nodes beyond the FP32 accuracy bound,
and a capturing stream must be refused. This file is collected last on
purpose."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1408_7069_gb300 import synth, workloads as W  # noqa: E402
from paper_1408_7069_gb300 import letkf as L  # noqa: E402

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _config(w, mask):
    c = L.letkf_config()
    c.nsub = mask.shape[0]
    c.subap_mask = mask.ctypes.data
    c.m, c.window, c.taper, c.loc_len = w.m, w.window, w.taper, w.loc_len
    c.rho, c.sigma2, c.a_ar1, c.noise_std = w.rho, w.sigma2, w.a_ar1, w.noise_std
    c.precision, c.fp64_kappa, c.seed, c.max_sweeps = 0, 0.0, w.seeds[2], 0
    return c


def _background(w, frames):
    """A loop background: the handle's own closed loop run for a few frames."""
    inp = synth.make_loop_inputs(w, frames=frames + 3)
    f = L.Letkf.from_workload(w, bank=inp.bank, precision=0)
    f.set_state(torch.from_numpy(inp.X0.astype(np.float32)).cuda())
    f.run(frames, torch.from_numpy(inp.slopes.astype(np.float32)).cuda(), use_graph=False)
    f.sync()
    X = f.get_state()
    f.close()
    return inp, X, torch.from_numpy(inp.slopes[frames].astype(np.float32)).cuda()


def _handle_analysis(w, X, y):
    f = L.Letkf.from_workload(w, precision=0)
    f.set_state(X.clone())
    mean, spread = f.analyze(y)
    f.sync()
    Xa = f.get_state()
    f.close()
    return Xa.cpu().numpy(), mean.cpu().numpy(), spread.cpu().numpy()


@pytest.mark.parametrize("w", [W.TEL_16M, W.TOY_8X8], ids=["16m-m24", "8x8-m10"])
def test_noalloc_matches_letkf_analyze_on_two_calls_in_a_row(w):
    inp, X, y = _background(w, 5)
    mask = np.ascontiguousarray(inp.subap_mask, dtype=np.uint8)
    cfg = _config(w, mask)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        Xref, mref, sref = _handle_analysis(w, X, y)
        Xn = X.clone()
        mean = torch.zeros_like(X[:, :, 0])
        spread = torch.zeros_like(X[:, :, 0])
        L.letkf_analyze_noalloc(cfg, Xn, y, mean, spread, stream)
        torch.cuda.synchronize()
        assert rel(mean.cpu().numpy(), mref) <= 1e-4
        assert rel(spread.cpu().numpy(), sref) <= 1e-3
        an = Xn.cpu().numpy()
        an = an - an.mean(-1, keepdims=True)
        ar = Xref - Xref.mean(-1, keepdims=True)
        assert rel(an, ar) <= 1e-3
        # the second call analyses the result of the first with the next slopes
        X, y = Xn, torch.from_numpy(inp.slopes[5 + call].astype(np.float32)).cuda()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    w = W.TEL_16M
    mask = np.ones((200, 200), np.uint8)
    cfg = _config(w, mask)
    X = torch.zeros(8, device="cuda")
    with pytest.raises(L.LetkfError) as e:
        L.letkf_analyze_noalloc(cfg, X, X)
    assert e.value.status == 1 and "128" in str(e.value)


def _anoms(X):
    return X - X.mean(-1, keepdims=True)


@pytest.mark.parametrize("w", [W.TEL_16M, W.TOY_8X8], ids=["16m-m24", "8x8-m10"])
def test_noalloc_matches_the_oracle(w):
    inp, X, y = _background(w, 5)
    mask = np.ascontiguousarray(inp.subap_mask, dtype=np.uint8)
    cfg = _config(w, mask)
    cfg.fp64_kappa = 300.0
    stream = torch.cuda.current_stream().cuda_stream
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.loc_len)
    for call in range(2):
        Xb = X.cpu().numpy().astype(np.float64)
        yb = y.cpu().numpy().astype(np.float64)
        Xr, mr, sr = oracle.analysis_batched(geom, Xb, yb, w.sigma2, w.rho)
        Xn = X.clone()
        mean = torch.zeros_like(X[:, :, 0])
        spread = torch.zeros_like(X[:, :, 0])
        L.letkf_analyze_noalloc(cfg, Xn, y, mean, spread, stream)
        st, nk = L.letkf_noalloc_status(stream)
        assert st == L.LETKF_OK and nk == 0      # no node above the accuracy bound
        assert rel(mean.cpu().numpy(), mr) <= 1e-4
        assert rel(spread.cpu().numpy(), sr) <= 1e-3
        assert rel(_anoms(Xn.cpu().numpy()), _anoms(Xr)) <= 1e-3
        X, y = Xn, torch.from_numpy(inp.slopes[5 + call].astype(np.float32)).cuda()


def test_noalloc_status_flags_kappa_and_sweep_limit():
    w = W.TEL_16M
    inp = synth.make_loop_inputs(w, frames=2)
    mask = np.ascontiguousarray(inp.subap_mask, dtype=np.uint8)
    X0 = torch.from_numpy(inp.X0.astype(np.float32)).cuda()
    y = torch.from_numpy(inp.slopes[1].astype(np.float32)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    cfg = _config(w, mask)
    # the prior draw: the node problems are ill-conditioned, beyond what the
    # FP32 mean solve resolves; they are counted
    cfg.fp64_kappa = 300.0
    L.letkf_analyze_noalloc(cfg, X0.clone(), y, None, None, stream)
    st, nk = L.letkf_noalloc_status(stream)
    assert st == L.LETKF_OK and nk > 100
    cfg.fp64_kappa = 0.0                          # no threshold: nothing counted
    L.letkf_analyze_noalloc(cfg, X0.clone(), y, None, None, stream)
    assert L.letkf_noalloc_status(stream) == (L.LETKF_OK, 0)
    cfg.max_sweeps = 1                            # one sweep cannot converge
    L.letkf_analyze_noalloc(cfg, X0.clone(), y, None, None, stream)
    assert L.letkf_noalloc_status(stream)[0] == 3  # LETKF_ERR_NOCONVERGE
    cfg.max_sweeps = 0                            # the next call starts clean
    L.letkf_analyze_noalloc(cfg, X0.clone(), y, None, None, stream)
    assert L.letkf_noalloc_status(stream)[0] == L.LETKF_OK


def test_noalloc_refuses_stream_capture():
    w = W.TOY_8X8
    inp = synth.make_loop_inputs(w, frames=2)
    mask = np.ascontiguousarray(inp.subap_mask, dtype=np.uint8)
    cfg = _config(w, mask)
    X = torch.from_numpy(inp.X0.astype(np.float32)).cuda()
    y = torch.from_numpy(inp.slopes[1].astype(np.float32)).cuda()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.stream(side):
        g.capture_begin()
        try:
            L.letkf_analyze_noalloc(cfg, X, y, None, None, side.cuda_stream)
        except L.LetkfError as e:
            err = e
        torch.zeros(1, device="cuda").add_(1.0)   # keep the captured graph non-empty
        g.capture_end()
    assert err is not None and err.status == 1 and "captured" in str(err)
    # the stream works normally afterwards
    L.letkf_analyze_noalloc(cfg, X, y, None, None, torch.cuda.current_stream().cuda_stream)
    assert L.letkf_noalloc_status(torch.cuda.current_stream().cuda_stream)[0] == L.LETKF_OK
