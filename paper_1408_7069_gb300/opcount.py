"""Algorithmic operation counts of the paper (Appendix B), used as the numerator
of the roofline fraction.

Appendix B.1 counts the multiplications of one ETKF update on a zonal basis,
(m^2 + m) n + (m^2 + 7m + 41) p + 2 m^3 + 3 m^2 + (3 + gamma) m, and states that
the additions are of the same order; Table 1 quotes twice that number (7.65e6
for m = 101, n = 32, p = 128). Appendix B.2 counts the prediction step,
(3/2 m + 1) n multiplications plus (5/2 m - 1) n additions.
"""
from __future__ import annotations


def update_mults(m: int, n: int, p: int, gamma: int = 1) -> int:
    """Multiplications of one (local) update with state size n and p observations."""
    return (m * m + m) * n + (m * m + 7 * m + 41) * p + 2 * m ** 3 + 3 * m * m + (3 + gamma) * m


def update_ops(m: int, n: int, p: int, gamma: int = 1) -> int:
    """Multiplications plus as many additions (the Table 1 convention)."""
    return 2 * update_mults(m, n, p, gamma)


def prediction_ops(m: int, n: int) -> float:
    """(3/2 m + 1) n multiplications + (5/2 m - 1) n additions."""
    return (1.5 * m + 1) * n + (2.5 * m - 1) * n


def frame_analysis_ops(m: int, window_slopes) -> int:
    """Per-frame analysis ops of the per-node LETKF: every node is one local
    domain with n_d = 2 state rows and p_l = its window's slope count."""
    return sum(update_ops(m, 2, int(p)) for p in window_slopes)


def taper_support_cells(window: int, taper: int, loc_len: float = 0.0) -> int:
    """Window cells the analysis kernels visit: those whose subaperture centre,
    at (ds - w//2 + 0.5, dt - w//2 + 0.5) pitches from the node, lies inside
    the Gaspari-Cohn support (distance < 2 c, c = loc_len or w / 4); every
    cell for the box taper."""
    if taper != 1:
        return window * window
    hw = window // 2
    c = loc_len if loc_len > 0 else window / 4.0
    return sum(1 for ds in range(window) for dt in range(window)
               if ((ds - hw + 0.5) ** 2 + (dt - hw + 0.5) ** 2) ** 0.5 / c < 2.0)


def frame_executed_flops(mp: int, n_nodes: int, support_cells: int, mean_sweeps: float) -> float:
    """Flops the FP32 analysis kernel executes per frame (an FMA counts as two),
    from its loop structure, beside the paper's count. Per node: the Gram over
    the window cells inside the taper's support (two slopes each, 2 mp^2 flops
    per slope, both triangles of the mp x mp matrix, pupil or not); per Jacobi
    sweep mp rounds of mp/2 column pairs, each a dot product (2 mp) and a
    rotation of both columns, 4 mp in the even rounds (one FMA per element)
    and 6 mp in the odd ones (a multiply and an FMA), 3.5 mp^3 in all; the
    eigenvector normalisation, transform and apply (about 10 mp^2).
    mean_sweeps: the measured mean sweep count per node."""
    per_sweep = 3.5 * mp ** 3
    per_node = 2.0 * mp * mp * 2 * support_cells + mean_sweeps * per_sweep + 10.0 * mp * mp
    return float(n_nodes * per_node)
