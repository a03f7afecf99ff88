"""Pins of the oracle's reverse mode (gradient of the mean residual variance
with respect to inflation rho, noise variance sigma^2 and localization length
L) to central finite differences of the FP64 forward loop, including exactly
degenerate eigenvalue clusters (windows with fewer slopes than m - 1)."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from paper_1408_7069_gb300 import synth, workloads as W


def test_gaspari_cohn_derivative():
    z = np.linspace(0.01, 2.2, 300)
    h = 1e-6
    fd = (oracle.gaspari_cohn(z + h) - oracle.gaspari_cohn(z - h)) / (2 * h)
    assert np.allclose(oracle.gaspari_cohn_deriv(z), fd, atol=1e-7)


def _loop_inputs(w, frames):
    inp = synth.make_loop_inputs(w, frames=frames)
    return inp


def _J(w, inp, frames, rho, sigma2, L, X0):
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, L)
    rv, _, _ = oracle.closed_loop(geom, inp.truth, inp.slopes, inp.bank, w.m, sigma2, rho,
                                  w.a_ar1, w.noise_std, w.seeds[2], frames, X0=X0)
    return rv.mean()


def _fd(fun, x, h):
    """Central difference with relative step h, Richardson-extrapolated (h, h/2)."""
    d1 = (fun(x * (1 + h)) - fun(x * (1 - h))) / (2 * h * x)
    d2 = (fun(x * (1 + h / 2)) - fun(x * (1 - h / 2))) / (h * x)
    return (4 * d2 - d1) / 3


def test_analysis_adjoint_dot_product():
    """<Xa_bar, dXa> = <Xb_bar, dXb> for a random direction dXb."""
    w = W.TINY_4X4
    inp = _loop_inputs(w, 3)
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, w.loc_len)
    rng = np.random.default_rng(0)
    Xb = inp.X0 + 0.3 * rng.standard_normal(inp.X0.shape)
    G = rng.standard_normal(Xb.shape)
    dX = rng.standard_normal(Xb.shape)
    Xb_bar, _, _, _ = oracle.analysis_adjoint(geom, Xb, inp.slopes[1], w.sigma2, w.rho, G)
    h = 1e-6
    Xp, _, _ = oracle.analysis(geom, Xb + h * dX, inp.slopes[1], w.sigma2, w.rho)
    Xm, _, _ = oracle.analysis(geom, Xb - h * dX, inp.slopes[1], w.sigma2, w.rho)
    lhs = np.sum(G * (Xp - Xm)) / (2 * h)
    rhs = np.sum(Xb_bar * dX)
    assert abs(lhs - rhs) <= 1e-6 * abs(rhs)


CASES = [W.TINY_4X4,
         replace(W.TINY_4X4, name="tiny-degenerate", m=16, seeds=(4, 5, 6)),
         replace(W.TOY_8X8, name="toy-gc", m=10, loc_len=1.2)]


@pytest.mark.parametrize("w", CASES, ids=[w.name for w in CASES])
def test_closed_loop_gradient_matches_finite_differences(w):
    frames = 6
    inp = _loop_inputs(w, frames)
    X0 = inp.X0
    L0 = w.loc_len if w.loc_len > 0 else w.window / 4.0
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, L0)
    J, grad, _ = oracle.closed_loop_grad(geom, inp.truth, inp.slopes, inp.bank, w.m, w.sigma2,
                                         w.rho, w.a_ar1, w.noise_std, w.seeds[2], frames, X0)
    assert J == pytest.approx(_J(w, inp, frames, w.rho, w.sigma2, L0, X0), rel=1e-12)
    fd = [_fd(lambda r: _J(w, inp, frames, r, w.sigma2, L0, X0), w.rho, 1e-4),
          _fd(lambda s: _J(w, inp, frames, w.rho, s, L0, X0), w.sigma2, 1e-4),
          _fd(lambda L: _J(w, inp, frames, w.rho, w.sigma2, L, X0), L0, 1e-4)]
    for g, f in zip(grad, fd):
        assert abs(g - f) <= 1e-6 * max(abs(f), 1e-9 * abs(J)), (grad, fd)
