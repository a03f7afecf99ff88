"""GPU parity of the row-split form of the FP32 per-node analysis (each
column's rows on two lanes, letkf_set_row_split) against the FP64 oracle: the
Section 4.2 analysis teacher-forced in both split width classes (m <= 16 and
m <= 32), with and without the FP64 fallback (whose queued nodes start from
the basis the split kernel stores), the closed loop, the reverse mode (whose
forward pass stores every basis), batched instances, tile shapes, and the
calls that refuse the split."""
import functools
from dataclasses import replace

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1408_7069_gb300 import synth, workloads as W  # noqa: E402
from paper_1408_7069_gb300 import letkf as L  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = dict(mean=1e-4, spread=1e-3, anom=1e-3)

TOY12 = replace(W.TOY_8X8, name="toy-fp32-m12", precision=0, m=12, seeds=(17, 18, 19))
SMALL16 = replace(W.TEL_16M, name="16m-m16-w7", m=16, window=7, seeds=(24, 25, 26))


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@functools.lru_cache(maxsize=None)
def inputs(w, frames):
    inp = synth.make_loop_inputs(w, frames=frames)
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.loc_len)
    return inp, geom


def oracle_background(w, inp, geom, frames):
    X = inp.X0.copy()
    for k in range(frames):
        Xa, _, _ = oracle.analysis_batched(geom, X, inp.slopes[k], w.sigma2, w.rho)
        v = oracle.bank_noise(inp.bank, geom.points, w.m, w.seeds[2], k, w.noise_std)
        X = oracle.forecast(Xa, v, w.a_ar1)
    return X


def width_class(m):
    return 0 if m <= 16 else 1


def check(Xa, mean, spread, ref):
    rXa, rmean, rspread = ref
    assert rel(mean, rmean) <= TOL["mean"], rel(mean, rmean)
    assert rel(spread, rspread) <= TOL["spread"], rel(spread, rspread)
    anom = Xa - Xa.mean(-1, keepdims=True)
    ranom = rXa - rXa.mean(-1, keepdims=True)
    assert rel(anom, ranom) <= TOL["anom"], rel(anom, ranom)
    assert np.abs(mean - rmean).max() <= 10 * TOL["mean"] * np.sqrt(np.mean(rmean**2))
    assert np.abs(spread - rspread).max() <= 10 * TOL["spread"] * np.sqrt(np.mean(rspread**2))


CASES = [(W.TEL_16M, 0, 300.0), (W.TEL_16M, 6, 300.0), (W.TEL_16M, 3, 0.0),
         (TOY12, 0, 1.0000001), (TOY12, 4, 300.0), (SMALL16, 0, 300.0), (SMALL16, 5, 0.0),
         (W.ELT_80X80, 3, 300.0)]


@pytest.mark.parametrize("w,k,kappa", CASES, ids=[f"{w.name}-f{k}-k{c:g}" for w, k, c in CASES])
def test_split_analysis_teacher_forced(w, k, kappa):
    inp, geom = inputs(w, 8)
    Xb = (oracle_background(w, inp, geom, k) if k else inp.X0).astype(np.float32)
    y = inp.slopes[k].astype(np.float32)
    ref = oracle.analysis(geom, Xb.astype(np.float64), y.astype(np.float64), w.sigma2, w.rho)
    f = L.Letkf.from_workload(w, bank=inp.bank, fp64_kappa=kappa)
    f.set_row_split(width_class(w.m), 2)
    f.set_state(torch.from_numpy(Xb).cuda())
    mean, spread = f.analyze(torch.from_numpy(y).cuda())
    f.sync()
    nfp64, sweeps, _ = f.stats()
    if kappa == 0.0:
        assert nfp64 == 0
    if kappa == 1.0000001:
        assert nfp64 == f.n_pts                  # every node queued: all from the split basis
    assert 1 <= sweeps <= 20
    Xa = f.get_state().cpu().numpy().astype(np.float64)
    check(Xa, mean.cpu().numpy(), spread.cpu().numpy(), ref)
    f.close()


def test_split_and_whole_columns_agree_to_rounding():
    """The two forms compute the same analysis in another summation order: the
    frame's outputs agree to FP32 rounding, and each form is bitwise stable."""
    w = W.TEL_16M
    inp, geom = inputs(w, 8)
    Xb = oracle_background(w, inp, geom, 4).astype(np.float32)
    y = torch.from_numpy(inp.slopes[4].astype(np.float32)).cuda()
    out = {}
    for split in (1, 2, 2):
        f = L.Letkf.from_workload(w, bank=inp.bank)
        f.set_row_split(1, split)
        f.set_state(torch.from_numpy(Xb).cuda())
        mean, _ = f.analyze(y)
        f.sync()
        X = f.get_state().cpu().numpy()
        if split in out:
            assert np.array_equal(X, out[split])
        out[split] = X
        f.close()
    assert rel(out[2], out[1]) <= 1e-5, rel(out[2], out[1])


def test_split_closed_loop_matches_oracle():
    w, frames = W.TEL_16M, 60
    inp, geom = inputs(w, frames)
    rv_ref, X_ref, _ = oracle.closed_loop(
        geom, inp.truth.astype(np.float32).astype(np.float64),
        inp.slopes.astype(np.float32).astype(np.float64), inp.bank, w.m, w.sigma2, w.rho,
        w.a_ar1, w.noise_std, w.seeds[2], frames,
        X0=inp.X0.astype(np.float32).astype(np.float64), batched=True)
    f = L.Letkf.from_workload(w, bank=inp.bank)
    f.set_row_split(1, 2)
    f.set_jacobi(4e-6, 0.0)
    f.set_state(torch.from_numpy(inp.X0.astype(np.float32)).cuda())
    rv = f.run(frames, torch.from_numpy(inp.slopes.astype(np.float32)).cuda(),
               torch.from_numpy(inp.truth.astype(np.float32)).cuda(), use_graph=True)
    f.sync()
    f.close()
    dev = np.abs(rv.cpu().numpy() - rv_ref) / rv_ref
    # the thresholds of the whole-column form's strict closed-loop test
    assert dev[:20].max() <= 1e-3 and dev.max() <= 1e-2, dev.max()


def test_split_reverse_mode_matches_oracle():
    """letkf_grad's forward pass stores every node's basis from the split kernel."""
    w, frames = replace(W.ADJ_16M, name="adj-20x20", nsub=20, seeds=(61, 62, 63)), 10
    inp = synth.make_loop_inputs(w, frames=frames)
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.window / 4.0)
    c = lambda a: np.asarray(a).astype(np.float32).astype(np.float64)  # noqa: E731
    Jr, gr, _ = oracle.closed_loop_grad(geom, c(inp.truth), c(inp.slopes), inp.bank, w.m,
                                        w.sigma2, w.rho, w.a_ar1, w.noise_std, w.seeds[2],
                                        frames, c(inp.X0))
    f = L.Letkf.from_workload(w, bank=inp.bank)
    f.set_row_split(1, 2)
    f.set_state(torch.from_numpy(inp.X0.astype(np.float32)).cuda())
    J, g = f.grad(frames, torch.from_numpy(inp.slopes.astype(np.float32)).cuda(),
                  torch.from_numpy(inp.truth.astype(np.float32)).cuda(), 4)
    f.sync()
    f.close()
    assert J == pytest.approx(Jr, rel=1e-4)
    for k in range(3):
        assert abs(g[k] - gr[k]) <= 1e-3 * abs(gr[k]), (k, g, gr)


def test_row_split_workload_setting():
    w = replace(W.TEL_16M, row_split=2)
    inp, geom = inputs(W.TEL_16M, 8)
    y = torch.from_numpy(inp.slopes[0].astype(np.float32)).cuda()
    X0 = torch.from_numpy(inp.X0.astype(np.float32)).cuda()
    out = []
    for make in (lambda: L.Letkf.from_workload(w, bank=inp.bank),
                 lambda: L.Letkf.from_workload(W.TEL_16M, bank=inp.bank)):
        f = make()
        if len(out) == 1:
            f.set_row_split(1, 2)
        f.set_state(X0)
        f.analyze(y)
        f.sync()
        out.append(f.get_state().cpu().numpy())
        f.close()
    assert np.array_equal(out[0], out[1])


BATCH = [replace(W.TEL_16M, name="b16-m16", nsub=16, m=16, window=5, seeds=(101, 102, 103)),
         replace(W.TEL_16M, name="b20-m24", nsub=20, m=24, window=7, seeds=(104, 105, 106)),
         replace(W.TEL_16M, name="b12-m10", nsub=12, m=10, window=3, seeds=(107, 108, 109)),
         replace(W.TEL_16M, name="b24-m32", nsub=24, m=32, window=5, seeds=(110, 111, 112))]


def _batch(frames, shape=None):
    ins = [synth.make_loop_inputs(w, frames=frames) for w in BATCH]
    f = L.Letkf.batch(BATCH, [i.bank for i in ins])
    f.set_row_split(0, 2)
    f.set_row_split(1, 2)
    if shape is not None:
        ti, tj = L.tile_shapes()[shape]
        if ti * tj % 2:                       # class 0 takes two nodes per warp in the split form
            with pytest.raises(L.LetkfError, match="LETKF_ERR_ARG"):
                f.set_tile_shape(0, shape)
        else:
            f.set_tile_shape(0, shape)
        f.set_tile_shape(1, shape)            # one node per warp: every shape
    X0 = np.concatenate([i.X0.astype(np.float32).ravel() for i in ins])
    y = torch.from_numpy(np.concatenate([i.slopes.astype(np.float32) for i in ins], 1)).cuda()
    t = torch.from_numpy(np.concatenate([i.truth.astype(np.float32) for i in ins], 1)).cuda()
    f.set_state(torch.from_numpy(X0).cuda())
    rv = f.run(frames, y, t, use_graph=True)
    f.sync()
    X = f.get_state().cpu().numpy()
    f.close()
    return ins, X, rv.cpu().numpy()


def test_split_batch_matches_oracle_and_tile_shapes_leave_bits():
    frames = 8
    ins, ref, rv = _batch(frames)
    for k, (inp, w) in enumerate(zip(ins, BATCH)):
        geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.loc_len)
        rv_ref, _, _ = oracle.closed_loop(
            geom, inp.truth.astype(np.float32).astype(np.float64),
            inp.slopes.astype(np.float32).astype(np.float64), inp.bank, w.m, w.sigma2, w.rho,
            w.a_ar1, w.noise_std, w.seeds[2], frames,
            X0=inp.X0.astype(np.float32).astype(np.float64), batched=True)
        assert np.max(np.abs(rv[:, k] - rv_ref) / rv_ref) <= 1e-3, w.name
    _, X4, _ = _batch(4)
    for s in range(len(L.tile_shapes())):
        _, X, _ = _batch(4, shape=s)
        assert np.array_equal(X, X4), s


def test_row_split_is_refused_where_it_does_not_apply():
    inp, _ = inputs(W.TEL_16M, 8)
    f = L.Letkf.from_workload(W.TEL_16M, bank=inp.bank)
    for cls, split in ((2, 2), (1, 3), (1, 0), (3, 1)):
        with pytest.raises(L.LetkfError, match="LETKF_ERR_ARG"):
            f.set_row_split(cls, split)
    # a one-node tile holds whole warps only in the split form of class 1
    f.set_row_split(1, 2)
    one = [s for s, (a, b) in enumerate(L.tile_shapes()) if a * b == 1][0]
    f.set_tile_shape(1, one)
    with pytest.raises(L.LetkfError, match="LETKF_ERR_ARG"):
        f.set_row_split(1, 1)
    f.close()
    t8, _ = inputs(W.TOY_8X8, 8)
    g = L.Letkf.from_workload(W.TOY_8X8, bank=t8.bank)      # FP64 handle
    with pytest.raises(L.LetkfError, match="LETKF_ERR_ARG"):
        g.set_row_split(0, 2)
    g.set_row_split(0, 1)
    g.close()
    d = L.Letkf.from_workload(W.DOM_16M, bank=synth.make_loop_inputs(W.DOM_16M, 2).bank)
    with pytest.raises(L.LetkfError, match="LETKF_ERR_ARG"):
        d.set_row_split(1, 2)
    d.close()
