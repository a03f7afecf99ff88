"""Writes adjoint_16m_200f.txt: the oracle's mean residual variance J over 200
closed-loop frames of the 16 m system and its gradient (dJ/drho, dJ/dsigma2,
dJ/dL), by the oracle's reverse mode (Section 2.1 Eq. Crit_Opt through the
analyses of Section 4.2), on the seeded synthetic inputs rounded to FP32 as an
FP32 or FP64 handle receives them. Calls only the oracle and the input
generators. Run from the repository root:
    python tests/golden/make_adjoint_golden.py
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

import oracle  # noqa: E402
from paper_1408_7069_gb300 import synth, workloads as W  # noqa: E402


def main():
    w = W.ADJ_16M
    frames = w.frames
    inp = synth.make_loop_inputs(w, frames=frames)
    c = lambda a: np.asarray(a).astype(np.float32).astype(np.float64)  # noqa: E731
    L0 = w.loc_len if w.loc_len > 0 else w.window / 4.0
    geom = oracle.build_geometry(inp.subap_mask, w.window, w.taper, L0)
    J, g, _ = oracle.closed_loop_grad(geom, c(inp.truth), c(inp.slopes), inp.bank, w.m, w.sigma2,
                                      w.rho, w.a_ar1, w.noise_std, w.seeds[2], frames, c(inp.X0))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_16m_200f.txt")
    with open(out, "w") as f:
        f.write("# Oracle reverse mode of the closed loop, written by make_adjoint_golden.py.\n"
                f"# Workload {w.name}: {frames} frames from the prior draw X0, inputs rounded\n"
                "# to FP32, noise frames 0.., L = window / 4.\n")
        f.write(f"J {float(J)!r}\ndJ_drho {float(g[0])!r}\ndJ_dsigma2 {float(g[1])!r}\n"
                f"dJ_dL {float(g[2])!r}\n")
    print(out, J, g)


if __name__ == "__main__":
    main()
