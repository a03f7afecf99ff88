"""Many AO instances of different sizes in one handle: per-instance parity with
the oracle, equality with the same instances run one handle each, and tile
shapes (autotuned or forced) leaving the arithmetic unchanged."""
import functools
from dataclasses import replace

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1408_7069_gb300 import synth, workloads as W  # noqa: E402
from paper_1408_7069_gb300 import letkf as L  # noqa: E402

pytestmark = pytest.mark.gpu

BATCH = [
    replace(W.TEL_16M, name="b0", nsub=20, m=24, window=5, seeds=(101, 102, 103)),
    replace(W.TEL_16M, name="b1", nsub=12, m=10, window=3, rho=1.05, seeds=(111, 112, 113)),
    replace(W.ELT_80X80, name="b2", nsub=28, m=32, window=7, seeds=(121, 122, 123)),
    replace(W.TEL_16M, name="b3", nsub=16, m=16, window=7, obscuration=0.0, seeds=(131, 132, 133)),
]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@functools.lru_cache(maxsize=None)
def inputs(frames):
    out = []
    for w in BATCH:
        inp = synth.make_loop_inputs(w, frames=frames)
        geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.loc_len)
        out.append((inp, geom))
    return out


def test_batch_teacher_forced_parity_per_instance():
    ins = inputs(4)
    f = L.Letkf.batch(BATCH, [i.bank for i, _ in ins])
    assert f.n_inst == len(BATCH)
    X0 = np.concatenate([i.X0.astype(np.float32).ravel() for i, _ in ins])
    y = np.concatenate([i.slopes[2].astype(np.float32) for i, _ in ins])
    f.set_state(torch.from_numpy(X0).cuda())
    mean, spread = f.analyze(torch.from_numpy(y).cuda())
    f.sync()
    Xs = [x.cpu().numpy() for x in f.split_state(f.get_state())]
    row = 0
    for (inp, geom), w, Xa in zip(ins, BATCH, Xs):
        Xb = inp.X0.astype(np.float32).astype(np.float64)
        rXa, rmean, rspread = oracle.analysis(geom, Xb, inp.slopes[2].astype(np.float32)
                                              .astype(np.float64), w.sigma2, w.rho)
        n = geom.n_pts
        assert rel(mean[row:row + n].cpu().numpy(), rmean) <= 1e-4, w.name
        assert rel(spread[row:row + n].cpu().numpy(), rspread) <= 1e-3, w.name
        row += n
    f.close()


def _run_batch(frames, tile=None, autotune=False):
    ins = inputs(frames)
    f = L.Letkf.batch(BATCH, [i.bank for i, _ in ins])
    X0 = np.concatenate([i.X0.astype(np.float32).ravel() for i, _ in ins])
    y = torch.from_numpy(np.concatenate([i.slopes.astype(np.float32) for i, _ in ins], 1)).cuda()
    t = torch.from_numpy(np.concatenate([i.truth.astype(np.float32) for i, _ in ins], 1)).cuda()
    f.set_state(torch.from_numpy(X0).cuda())
    if tile is not None:
        ti, tj = L.tile_shapes()[tile]
        for cls, per_warp in ((0, 4), (1, 2)):       # nodes per warp of the FP32 kernel
            if (ti * tj) % per_warp == 0:
                f.set_tile_shape(cls, tile)
            else:                                     # a tile must fill whole warps
                with pytest.raises(L.LetkfError, match="LETKF_ERR_ARG"):
                    f.set_tile_shape(cls, tile)
    if autotune:
        shapes, us = f.autotune(y[0].contiguous(), reps=2)
        assert all(0 <= s < len(L.tile_shapes()) for s in shapes)
    rv = f.run(frames, y, t, use_graph=True)
    f.sync()
    X = f.get_state().cpu().numpy()
    f.close()
    return X, rv.cpu().numpy()


def test_batch_equals_separate_handles_bitwise():
    frames = 6
    Xb, rvb = _run_batch(frames)
    ins = inputs(frames)
    parts, rvs = [], []
    for (inp, _), w in zip(ins, BATCH):
        f = L.Letkf.from_workload(w, bank=inp.bank)
        f.set_state(torch.from_numpy(inp.X0.astype(np.float32)).cuda())
        rv = f.run(frames, torch.from_numpy(inp.slopes.astype(np.float32)).cuda(),
                   torch.from_numpy(inp.truth.astype(np.float32)).cuda(), use_graph=True)
        f.sync()
        parts.append(f.get_state().cpu().numpy().ravel())
        rvs.append(rv.cpu().numpy())
        f.close()
    assert np.array_equal(Xb, np.concatenate(parts))
    assert np.array_equal(rvb, np.stack(rvs, 1))


def test_tile_shapes_and_autotune_leave_results_unchanged():
    frames = 4
    ref, _ = _run_batch(frames)
    for s in range(len(L.tile_shapes())):
        X, _ = _run_batch(frames, tile=s)
        assert np.array_equal(X, ref), s
    X, _ = _run_batch(frames, autotune=True)
    assert np.array_equal(X, ref)


def test_batch_closed_loop_matches_oracle_per_instance():
    frames = 10
    ins = inputs(frames)
    _, rv = _run_batch(frames)
    for k, ((inp, geom), w) in enumerate(zip(ins, BATCH)):
        rv_ref, _, _ = oracle.closed_loop(
            geom, inp.truth.astype(np.float32).astype(np.float64),
            inp.slopes.astype(np.float32).astype(np.float64), inp.bank, w.m, w.sigma2, w.rho,
            w.a_ar1, w.noise_std, w.seeds[2], frames,
            X0=inp.X0.astype(np.float32).astype(np.float64), batched=True)
        assert np.max(np.abs(rv[:, k] - rv_ref) / rv_ref) <= 1e-3, w.name


WIDE = [replace(W.ELT_80X80, name="w48", nsub=16, m=48, window=7, seeds=(141, 142, 143)),
        replace(W.TEL_16M, name="w40", nsub=12, m=40, window=5, seeds=(151, 152, 153)),
        replace(W.TEL_16M, name="w60", nsub=10, m=60, window=5, seeds=(161, 162, 163))]


@pytest.mark.parametrize("w", WIDE, ids=[w.name for w in WIDE])
def test_wide_ensemble_matches_oracle(w):
    """33..64 members (one node per warp, padded to 48 or 64 columns) on a
    steady-state loop background."""
    inp = synth.make_loop_inputs(w, frames=10)
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.loc_len)
    X = inp.X0.copy()
    for k in range(8):
        Xa, _, _ = oracle.analysis_batched(geom, X, inp.slopes[k], w.sigma2, w.rho)
        X = oracle.forecast(Xa, oracle.bank_noise(inp.bank, geom.points, w.m, w.seeds[2], k,
                                                  w.noise_std), w.a_ar1)
    Xb = X.astype(np.float32)
    y = inp.slopes[8].astype(np.float32)
    rXa, rmean, rspread = oracle.analysis(geom, Xb.astype(np.float64), y.astype(np.float64),
                                          w.sigma2, w.rho)
    f = L.Letkf.from_workload(w, bank=inp.bank)
    f.set_state(torch.from_numpy(Xb).cuda())
    mean, spread = f.analyze(torch.from_numpy(y).cuda())
    f.sync()
    Xa = f.get_state().cpu().numpy().astype(np.float64)
    assert rel(mean.cpu().numpy(), rmean) <= 1e-4
    assert rel(spread.cpu().numpy(), rspread) <= 1e-3
    an = Xa - Xa.mean(-1, keepdims=True)
    ar = rXa - rXa.mean(-1, keepdims=True)
    assert rel(an, ar) <= 1e-3
    f.close()


def test_mixed_batch_with_wide_ensembles_equals_separate_handles():
    ws = [BATCH[0], WIDE[0], BATCH[1], WIDE[1]]
    ins = [synth.make_loop_inputs(w, frames=5) for w in ws]
    f = L.Letkf.batch(ws, [i.bank for i in ins])
    X0 = np.concatenate([i.X0.astype(np.float32).ravel() for i in ins])
    y = torch.from_numpy(np.concatenate([i.slopes.astype(np.float32) for i in ins], 1)).cuda()
    f.set_state(torch.from_numpy(X0).cuda())
    f.run(5, y, use_graph=True)
    f.sync()
    Xb = f.get_state().cpu().numpy()
    f.close()
    parts = []
    for w, inp in zip(ws, ins):
        g = L.Letkf.from_workload(w, bank=inp.bank)
        g.set_state(torch.from_numpy(inp.X0.astype(np.float32)).cuda())
        g.run(5, torch.from_numpy(inp.slopes.astype(np.float32)).cuda(), use_graph=False)
        g.sync()
        parts.append(g.get_state().cpu().numpy().ravel())
        g.close()
    assert np.array_equal(Xb, np.concatenate(parts))


def test_wide_tile_shapes_leave_results_unchanged():
    """Instances padded to 48 and to 64 columns in one handle (two launches of
    the wide class): every allowed tile shape gives the same bits, and tiles
    of more than 8 nodes are refused for this class."""
    ws = [WIDE[0], WIDE[2], WIDE[1]]
    ins = [synth.make_loop_inputs(w, frames=4) for w in ws]
    X0 = np.concatenate([i.X0.astype(np.float32).ravel() for i in ins])
    y = torch.from_numpy(np.concatenate([i.slopes.astype(np.float32) for i in ins], 1)).cuda()
    ref = None
    for shape in range(len(L.tile_shapes())):
        f = L.Letkf.batch(ws, [i.bank for i in ins])
        ti, tj = L.tile_shapes()[shape]
        if ti * tj > 8:
            with pytest.raises(L.LetkfError, match="LETKF_ERR_ARG"):
                f.set_tile_shape(2, shape)
            f.close()
            continue
        f.set_tile_shape(2, shape)
        f.set_state(torch.from_numpy(X0).cuda())
        f.run(4, y, use_graph=False)
        f.sync()
        X = f.get_state().cpu().numpy()
        f.close()
        if ref is None:
            ref = X
        assert np.array_equal(X, ref), shape


@pytest.mark.parametrize("w", WIDE, ids=[w.name for w in WIDE])
def test_wide_ensemble_fp64_fallback_from_the_prior_draw(w):
    """The prior draw and the frames after it: ill-conditioned node problems
    (kappa_hat above the threshold) of the wide class are redone in FP64 and
    every frame matches the oracle, teacher-forced (the same FP32 background
    into both)."""
    inp = synth.make_loop_inputs(w, frames=5)
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.loc_len)
    f = L.Letkf.from_workload(w, bank=inp.bank)
    f.set_state(torch.from_numpy(inp.X0.astype(np.float32)).cuda())
    fp64 = []
    for k in range(4):
        Xb = f.get_state().cpu().numpy().astype(np.float64)
        y = inp.slopes[k].astype(np.float32)
        rXa, rmean, rspread = oracle.analysis_batched(geom, Xb, y.astype(np.float64), w.sigma2,
                                                      w.rho)
        mean, spread = f.analyze(torch.from_numpy(y).cuda())
        f.sync()
        fp64.append(f.stats()[0])
        Xa = f.get_state().cpu().numpy().astype(np.float64)
        assert rel(mean.cpu().numpy(), rmean) <= 1e-4, (k, rel(mean.cpu().numpy(), rmean))
        assert rel(spread.cpu().numpy(), rspread) <= 1e-3, k
        assert rel(Xa - Xa.mean(-1, keepdims=True), rXa - rXa.mean(-1, keepdims=True)) <= 1e-3, k
        f.forecast()
    assert fp64[0] > geom.n_pts // 2          # the prior draw sends most nodes to FP64
    f.close()


def _mix_inputs(ws, frames):
    import multiprocessing as mp
    import os
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.starmap(synth.make_loop_inputs, [(w, frames) for w in ws])


def test_config5_mix_teacher_forced_at_sampled_nodes():
    """The bench's 48-instance mix (nsub 16..96, m in {16, 24, 32, 48}) in one
    handle from the prior draw: at frames 0..3 the analysis of 48 sampled nodes
    of every instance matches the oracle's analysis of those nodes from the
    same FP32 background (norm-wise over the sample, 1e-4 mean, 1e-3 spread)."""
    ws = W.batched_instances(48, seed=50, frames=5)
    assert any(w.m == 48 for w in ws)
    ins = _mix_inputs(ws, 5)
    geoms = [oracle.build_geometry(i.subap_mask, w.window, w.taper, w.loc_len)
             for w, i in zip(ws, ins)]
    f = L.Letkf.batch(ws, [i.bank for i in ins])
    X0 = np.concatenate([i.X0.astype(np.float32).ravel() for i in ins])
    f.set_state(torch.from_numpy(X0).cuda())
    for k in range(4):
        Xs = [x.cpu().numpy().astype(np.float64) for x in f.split_state(f.get_state())]
        y = np.concatenate([i.slopes[k].astype(np.float32) for i in ins])
        mean, spread = f.analyze(torch.from_numpy(y).cuda())
        f.sync()
        nfp64 = f.stats()[0]
        if k == 0:
            assert nfp64 > 0
        mean, spread = mean.cpu().numpy(), spread.cpu().numpy()
        row = 0
        for w, inp, Xb, geom in zip(ws, ins, Xs, geoms):
            n = geom.n_pts
            sample = np.linspace(0, n - 1, 48).astype(int)
            _, rmean, rspread = oracle.analysis_batched(
                geom, Xb, inp.slopes[k].astype(np.float32).astype(np.float64), w.sigma2, w.rho,
                nodes=sample)
            gm, gs = mean[row:row + n][sample], spread[row:row + n][sample]
            assert rel(gm, rmean[sample]) <= 1e-4, (k, w.name, rel(gm, rmean[sample]))
            assert rel(gs, rspread[sample]) <= 1e-3, (k, w.name)
            row += n
        f.forecast()
    f.close()


def test_config5_reduced_mix_closed_loop():
    """The mix's wide (m = 48) instances plus three others, grids capped at
    24 x 24 so that the oracle runs every node: 10 closed-loop frames from the
    prior draw, the criterion of every instance within 1e-3 of the oracle's."""
    full = W.batched_instances(48, seed=50, frames=10)
    wide = [w for w in full if w.m == 48][:4]
    other = [w for w in full if w.m != 48][:3]
    ws = [replace(w, nsub=min(w.nsub, 24)) for w in wide + other]
    ins = _mix_inputs(ws, 10)
    f = L.Letkf.batch(ws, [i.bank for i in ins])
    X0 = np.concatenate([i.X0.astype(np.float32).ravel() for i in ins])
    y = torch.from_numpy(np.concatenate([i.slopes.astype(np.float32) for i in ins], 1)).cuda()
    t = torch.from_numpy(np.concatenate([i.truth.astype(np.float32) for i in ins], 1)).cuda()
    f.set_state(torch.from_numpy(X0).cuda())
    rv = f.run(10, y, t, use_graph=True).cpu().numpy()
    f.sync()
    f.close()
    for k, (w, inp) in enumerate(zip(ws, ins)):
        geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.loc_len)
        rv_ref, _, _ = oracle.closed_loop(
            geom, inp.truth.astype(np.float32).astype(np.float64),
            inp.slopes.astype(np.float32).astype(np.float64), inp.bank, w.m, w.sigma2, w.rho,
            w.a_ar1, w.noise_std, w.seeds[2], 10,
            X0=inp.X0.astype(np.float32).astype(np.float64), batched=True)
        assert np.max(np.abs(rv[:, k] - rv_ref) / rv_ref) <= 1e-3, (w.name, rv[:, k], rv_ref)


FP64_BATCH = [replace(W.TOY_8X8, name="f64-a", seeds=(151, 152, 153)),
              replace(W.TOY_8X8, name="f64-b", nsub=6, m=16, window=5, seeds=(154, 155, 156)),
              replace(W.TOY_8X8, name="f64-c", nsub=10, m=24, window=3, seeds=(157, 158, 159))]


def test_fp64_batch_matches_oracle_and_separate_handles():
    """FP64 instances of both FP64 width classes (m = 10, 16: 16 columns; m = 24:
    32 columns) in one handle: the FP32 basis pass runs over every instance's
    tiles before the warm FP64 sweeps. Per instance the closed loop matches the
    oracle at FP64 rounding and the batch equals the instances' own handles
    bitwise."""
    frames = 6
    ins = [synth.make_loop_inputs(w, frames=frames) for w in FP64_BATCH]
    f = L.Letkf.batch(FP64_BATCH, [i.bank for i in ins])
    X0 = np.concatenate([i.X0.ravel() for i in ins])
    y = torch.from_numpy(np.concatenate([i.slopes for i in ins], 1)).cuda()
    t = torch.from_numpy(np.concatenate([i.truth for i in ins], 1)).cuda()
    f.set_state(torch.from_numpy(X0).cuda())
    rv = f.run(frames, y, t, use_graph=True).cpu().numpy()
    f.sync()
    Xb = f.get_state().cpu().numpy()
    f.close()
    parts = []
    for k, (inp, w) in enumerate(zip(ins, FP64_BATCH)):
        geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.loc_len)
        rv_ref, _, _ = oracle.closed_loop(geom, inp.truth, inp.slopes, inp.bank, w.m, w.sigma2,
                                          w.rho, w.a_ar1, w.noise_std, w.seeds[2], frames,
                                          X0=inp.X0, batched=True)
        assert np.max(np.abs(rv[:, k] - rv_ref) / rv_ref) <= 1e-8, w.name
        g = L.Letkf.from_workload(w, bank=inp.bank)
        g.set_state(torch.from_numpy(inp.X0).cuda())
        g.run(frames, torch.from_numpy(inp.slopes).cuda(), torch.from_numpy(inp.truth).cuda(),
              use_graph=True)
        g.sync()
        parts.append(g.get_state().cpu().numpy().ravel())
        g.close()
    assert np.array_equal(Xb, np.concatenate(parts))
