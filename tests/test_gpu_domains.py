"""GPU parity of the multi-actuator local domains (Section 4) and the
differential-piston least squares (Section 4.4) against the domain oracle:
the partition itself, teacher-forced analyses at the paper's sizes (m = 101,
n_d <= 32, p_d <= 128), the piston constants, the degenerate partitions
(one node per domain, one domain for the pupil) and a closed loop."""
import functools
from dataclasses import replace

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import letkf_domains as LD  # noqa: E402
from paper_1408_7069_gb300 import synth, workloads as W  # noqa: E402
from paper_1408_7069_gb300.letkf import Letkf, LetkfError  # noqa: E402

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def anoms(X):
    return X - X.mean(-1, keepdims=True)


@functools.lru_cache(maxsize=None)
def loop_state(w, frames):
    """Inputs, domain geometry and the oracle's loop background after
    `frames` frames from the prior draw (FP32-rounded)."""
    inp = synth.make_loop_inputs(w, frames=frames + 12)
    dg = LD.build_domains(inp.subap_mask, w.partition, w.window, w.taper, w.loc_len)
    X = inp.X0.copy()
    for k in range(frames):
        Xa, _, _ = LD.analysis_domains(dg, X, inp.slopes[k], w.sigma2, w.rho, piston=bool(w.piston))
        X = oracle.forecast(Xa, oracle.bank_noise(inp.bank, dg.geom.points, w.m, w.seeds[2], k,
                                                  w.noise_std), w.a_ar1)
    return inp, dg, X.astype(np.float32)


def gpu_analysis(w, inp, X, y):
    f = Letkf.from_workload(w, bank=inp.bank)
    f.set_state(torch.from_numpy(X).cuda())
    mean, spread = f.analyze(torch.from_numpy(y).cuda())
    f.sync()
    out = f.get_state().cpu().numpy().astype(np.float64), mean.cpu().numpy(), spread.cpu().numpy()
    nfl = f.stats()[0]
    f.close()
    return out, nfl


def test_partition_matches_the_oracle():
    for w in (W.DOM_16M, W.DOM_40M):
        mask = synth.pupil_subap_mask(w.nsub, w.obscuration, w.square)
        dg = LD.build_domains(mask, w.partition, w.window, w.taper, w.loc_len)
        f = Letkf.from_workload(w)
        n, nd = f.domains()
        f.close()
        assert n == dg.n_dom
        assert np.array_equal(nd, dg.node_dom)
    assert LD.build_domains(synth.pupil_subap_mask(80, 0.0), 21, 5).n_dom == 373


@pytest.mark.parametrize("w,k", [(W.DOM_16M, 10), (W.DOM_16M, 14), (W.DOM_40M, 8)],
                         ids=["16m-f10", "16m-f14", "40m-f8"])
def test_domain_analysis_teacher_forced(w, k):
    inp, dg, Xb = loop_state(w, k)
    y = inp.slopes[k].astype(np.float32)
    (Xa, mean, spread), _ = gpu_analysis(w, inp, Xb, y)
    rXa, rmean, rspread = LD.analysis_domains(dg, Xb.astype(np.float64), y.astype(np.float64),
                                              w.sigma2, w.rho, piston=True)
    assert rel(mean, rmean) <= 1e-4, rel(mean, rmean)
    assert rel(spread, rspread) <= 1e-3, rel(spread, rspread)
    assert rel(anoms(Xa), anoms(rXa)) <= 1e-3, rel(anoms(Xa), anoms(rXa))
    # the analysis increment (what the update adds to the background mean)
    xbar = Xb.astype(np.float64).mean(-1)
    assert rel(mean - xbar, rmean - xbar) <= 2e-3, rel(mean - xbar, rmean - xbar)


def test_piston_constants_match_the_oracle():
    w = W.DOM_16M
    inp, dg, Xb = loop_state(w, 10)
    y = inp.slopes[10].astype(np.float32)
    (_, m_on, _), _ = gpu_analysis(w, inp, Xb, y)
    (_, m_off, _), _ = gpu_analysis(replace(w, piston=0), inp, Xb, y)
    *_, c = LD.analysis_domains(dg, Xb.astype(np.float64), y.astype(np.float64), w.sigma2, w.rho,
                                return_parts=True)
    shift = (m_on - m_off).astype(np.float64)           # per node: its domain's constant
    ref = c[dg.node_dom]
    assert np.abs(ref).max() > 1e-3
    assert np.max(np.abs(shift - ref)) <= 1e-3 * np.abs(ref).max()


def test_one_node_domains_are_the_node_analysis():
    w = replace(W.TEL_16M, name="dom-1node", nsub=12, m=40, window=5, partition=13, piston=0,
                seeds=(171, 172, 173))
    inp = synth.make_loop_inputs(w, frames=8)
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.loc_len)
    X = inp.X0.copy()
    for k in range(6):
        Xa, _, _ = oracle.analysis_batched(geom, X, inp.slopes[k], w.sigma2, w.rho)
        X = oracle.forecast(Xa, oracle.bank_noise(inp.bank, geom.points, w.m, w.seeds[2], k,
                                                  w.noise_std), w.a_ar1)
    Xb = X.astype(np.float32)
    y = inp.slopes[6].astype(np.float32)
    (Xa, mean, spread), _ = gpu_analysis(w, inp, Xb, y)
    rXa, rmean, rspread = oracle.analysis(geom, Xb.astype(np.float64), y.astype(np.float64),
                                          w.sigma2, w.rho)
    assert rel(mean, rmean) <= 1e-4 and rel(spread, rspread) <= 1e-3
    assert rel(anoms(Xa), anoms(rXa)) <= 1e-3


def test_single_domain_is_the_global_etkf():
    w = replace(W.TOY_8X8, name="dom-global", precision=0, m=24, window=18, taper=0,
                partition=1, piston=1, seeds=(181, 182, 183))
    inp = synth.make_loop_inputs(w, frames=4)
    dg = LD.build_domains(inp.subap_mask, 1, w.window, 0)
    assert dg.n_dom == 1 and len(dg.dom_obs[0]) == dg.geom.p
    Xb = inp.X0.astype(np.float32)
    y = inp.slopes[2].astype(np.float32)
    (Xa, mean, spread), _ = gpu_analysis(w, inp, Xb, y)
    rXa, rmean, rspread = LD.analysis_domains(dg, Xb.astype(np.float64), y.astype(np.float64),
                                              w.sigma2, w.rho)
    assert rel(mean, rmean) <= 1e-4 and rel(spread, rspread) <= 1e-3
    assert rel(anoms(Xa), anoms(rXa)) <= 1e-3


def test_domain_closed_loop_matches_oracle():
    w = W.DOM_16M
    frames, k0 = 10, 10
    inp, dg, Xb = loop_state(w, k0)
    f = Letkf.from_workload(w, bank=inp.bank)
    f.set_state(torch.from_numpy(Xb).cuda())
    f.set_frame(k0)
    y = torch.from_numpy(inp.slopes[k0:].astype(np.float32)).cuda()
    t = torch.from_numpy(inp.truth[k0:].astype(np.float32)).cuda()
    rv = f.run(frames, y, t, use_graph=True).cpu().numpy()
    f.sync()
    f.close()
    X = Xb.astype(np.float64)
    ref = []
    for k in range(k0, k0 + frames):
        ref.append(oracle.residual_variance(inp.truth[k].astype(np.float32).astype(np.float64), X))
        Xa, _, _ = LD.analysis_domains(dg, X, inp.slopes[k].astype(np.float32).astype(np.float64),
                                       w.sigma2, w.rho)
        X = oracle.forecast(Xa, oracle.bank_noise(inp.bank, dg.geom.points, w.m, w.seeds[2], k,
                                                  w.noise_std), w.a_ar1)
    ref = np.array(ref)
    assert np.max(np.abs(rv - ref) / ref) <= 1e-3, (rv, ref)


def test_domain_handles_refuse_what_they_do_not_support():
    w = W.DOM_16M
    with pytest.raises(LetkfError, match="LETKF_ERR_ARG"):
        Letkf.from_workload(replace(w, precision=1))
    with pytest.raises(LetkfError, match="LETKF_ERR_ARG"):
        Letkf.from_workload(replace(w, m=129))          # a partition of more than one domain
    with pytest.raises(LetkfError, match="LETKF_ERR_ARG"):
        Letkf.from_workload(replace(w, partition=1, m=1025))
    with pytest.raises(LetkfError, match="LETKF_ERR_ARG"):
        Letkf.batch([w, w], [None, None])
    inp = synth.make_loop_inputs(w, frames=3)
    f = Letkf.from_workload(w, bank=inp.bank)
    y = torch.from_numpy(inp.slopes[:3].astype(np.float32)).cuda()
    t = torch.from_numpy(inp.truth[:3].astype(np.float32)).cuda()
    with pytest.raises(LetkfError, match="LETKF_ERR_STATE"):
        f.grad(3, y, t)
    f.close()


@pytest.mark.parametrize("frames", [0, 3], ids=["prior-draw", "f3"])
def test_global_etkf_at_paper_size(frames):
    """One domain over the 16 m pupil (partition 1: every slope observed by
    every node, the global ETKF of Section 3.1.1) with m = 101: p = 1624
    slopes, n = 1754 state rows, kappa_hat of 1e4-1e5; the mean solve is
    refined in FP64 and every frame matches the oracle."""
    w = replace(W.DOM_16M, name="global-16m-m101", partition=1, piston=0, taper=0)
    inp = synth.make_loop_inputs(w, frames=frames + 2)
    dg = LD.build_domains(inp.subap_mask, 1, w.window, 0)
    assert dg.n_dom == 1 and len(dg.dom_obs[0]) == dg.geom.p == 1624
    X = inp.X0.copy()
    for k in range(frames):
        Xa, _, _ = LD.analysis_domains(dg, X, inp.slopes[k], w.sigma2, w.rho)
        X = oracle.forecast(Xa, oracle.bank_noise(inp.bank, dg.geom.points, w.m, w.seeds[2], k,
                                                  w.noise_std), w.a_ar1)
    Xb = X.astype(np.float32)
    y = inp.slopes[frames].astype(np.float32)
    (Xa, mean, spread), _ = gpu_analysis(w, inp, Xb, y)
    rXa, rmean, rspread = LD.analysis_domains(dg, Xb.astype(np.float64), y.astype(np.float64),
                                              w.sigma2, w.rho)
    assert rel(mean, rmean) <= 1e-4, rel(mean, rmean)
    assert rel(spread, rspread) <= 1e-3, rel(spread, rspread)
    assert rel(anoms(Xa), anoms(rXa)) <= 1e-3, rel(anoms(Xa), anoms(rXa))
    xbar = Xb.astype(np.float64).mean(-1)
    assert rel(mean - xbar, rmean - xbar) <= 1e-3, rel(mean - xbar, rmean - xbar)


@pytest.mark.parametrize("m,frames", [(200, 0), (200, 2), (626, 0)],
                         ids=["m200-prior", "m200-f2", "m626-prior"])
def test_global_etkf_wide_ensembles(m, frames):
    """The global ETKF beyond the one-CTA eigensolver's 128 columns (up to the
    paper's 626 members): Newton-Schulz root and FP64-refined mean solve
    against the oracle's eigendecomposition, 16 m pupil, all 1624 slopes."""
    w = replace(W.DOM_16M, name=f"global-16m-m{m}", m=m, partition=1, piston=0, taper=0)
    inp = synth.make_loop_inputs(w, frames=frames + 2)
    dg = LD.build_domains(inp.subap_mask, 1, w.window, 0)
    X = inp.X0.copy()
    for k in range(frames):
        Xa, _, _ = LD.analysis_domains(dg, X, inp.slopes[k], w.sigma2, w.rho)
        X = oracle.forecast(Xa, oracle.bank_noise(inp.bank, dg.geom.points, w.m, w.seeds[2], k,
                                                  w.noise_std), w.a_ar1)
    Xb = X.astype(np.float32)
    y = inp.slopes[frames].astype(np.float32)
    (Xa, mean, spread), _ = gpu_analysis(w, inp, Xb, y)
    rXa, rmean, rspread = LD.analysis_domains(dg, Xb.astype(np.float64), y.astype(np.float64),
                                              w.sigma2, w.rho)
    assert rel(mean, rmean) <= 1e-4, rel(mean, rmean)
    assert rel(spread, rspread) <= 1e-3, rel(spread, rspread)
    assert rel(anoms(Xa), anoms(rXa)) <= 1e-3, rel(anoms(Xa), anoms(rXa))
    xbar = Xb.astype(np.float64).mean(-1)
    assert rel(mean - xbar, rmean - xbar) <= 1e-3, rel(mean - xbar, rmean - xbar)
