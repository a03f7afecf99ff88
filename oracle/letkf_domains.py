"""Plain FP64 CPU oracle of the LETKF with multi-actuator local domains and the
differential-piston least squares.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module. It shares
no code, table or constant with the CUDA library.

What it computes (Gray et al., arXiv:1408.7069):

* Local domains (Section 4.1): the actuator nodes are split by a P x P
  partition of the node grid; the valid nodes of one block form a local domain
  of n_d = 2 x (its nodes) state rows (phi_k and phi_{k-1} of every node).
* Observation region (Section 4.1: the subapertures including and surrounding
  the domain): the union of the w x w windows of the domain's nodes (the
  per-node window of ``letkf_oracle.build_geometry``), both slopes of each
  valid subaperture; with w = 5 and 4 x 4-node domains it holds at most
  8 x 8 subapertures, the p_max = 128 slopes of Section 5.3.
* Smooth localization (Section 4.1): R^-1 = diag(tau / sigma^2) with tau the
  Gaspari-Cohn function of the distance from the subaperture centre to the
  domain's node box (zero inside it), in pitches, half-support c.
* Local update (Section 4.2, Eqs. Sicz_majLoc .. X_{k/k}, with the inflation
  reading of the per-node oracle): one ensemble transform per domain,
  applied to all n_d rows of the domain.
* Differential pistons (Section 4.4): the local updates leave each domain with
  its own unmeasured piston. A least-squares fit of one constant per domain
  and state row removes the discontinuities of the analysis increment
  (x_a - x_b mean) across every pair of 4-neighbour nodes that lie in different
  domains; the constants of each connected group of domains have zero
  node-weighted mean. They are added to every member of the domain's rows.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse.csgraph

from .letkf_oracle import Geometry, build_geometry, gaspari_cohn, local_transform, observe


@dataclass
class DomainGeometry:
    geom: Geometry                # per-node geometry (nodes, subapertures, D1)
    partition: int                # P: blocks per side of the node grid
    dom_nodes: list               # per domain: point ids, row-major
    dom_obs: list                 # per domain: slope indices into y (sx block, then sy)
    dom_tau: list                 # per domain: taper of each observed slope
    node_dom: np.ndarray          # [n_pts] domain of every node
    edges: np.ndarray             # [E, 2] point ids of 4-neighbours in different domains

    @property
    def n_dom(self) -> int:
        return len(self.dom_nodes)


def block_bounds(n: int, parts: int) -> list:
    """Start of each of `parts` blocks splitting range(n) as evenly as possible:
    block b covers [floor(b n / parts), floor((b + 1) n / parts))."""
    return [(b * n) // parts for b in range(parts + 1)]


def build_domains(subap_mask, partition: int, window: int, taper: int = 0,
                  loc_len: float = 0.0) -> DomainGeometry:
    """Local domains of a P x P partition of the (nsub + 1)^2 node grid and
    their observation regions (see the module docstring)."""
    geom = build_geometry(subap_mask, window)
    sm = geom.subap_mask
    nsub = geom.nsub
    nn = nsub + 1
    n_sap = len(geom.subaps)
    sid = -np.ones((nsub, nsub), int)
    sid[sm] = np.arange(n_sap)
    pid = -np.ones((nn, nn), int)
    pid[geom.points[:, 0], geom.points[:, 1]] = np.arange(geom.n_pts)
    bb = block_bounds(nn, partition)
    h = window // 2
    c = loc_len if loc_len > 0 else window / 4.0
    dom_nodes, dom_obs, dom_tau = [], [], []
    node_dom = -np.ones(geom.n_pts, int)
    for bi in range(partition):
        for bj in range(partition):
            ids = [pid[i, j] for i in range(bb[bi], bb[bi + 1]) for j in range(bb[bj], bb[bj + 1])
                   if pid[i, j] >= 0]
            if not ids:
                continue
            ids = np.array(ids, int)
            pts = geom.points[ids]
            i0, i1 = pts[:, 0].min(), pts[:, 0].max()
            j0, j1 = pts[:, 1].min(), pts[:, 1].max()
            region = set()
            for (i, j) in pts:            # union of the nodes' windows
                for s in range(i - h, i - h + window):
                    for t in range(j - h, j - h + window):
                        if 0 <= s < nsub and 0 <= t < nsub and sm[s, t]:
                            region.add((s, t))
            obs, tau = [], []
            for (s, t) in sorted(region):
                k = sid[s, t]
                if taper == 1:
                    dx = max(i0 - (s + 0.5), 0.0, (s + 0.5) - i1)
                    dy = max(j0 - (t + 0.5), 0.0, (t + 0.5) - j1)
                    tk = float(gaspari_cohn(math.hypot(dx, dy) / c))
                else:
                    tk = 1.0
                obs += [k, n_sap + k]
                tau += [tk, tk]
            node_dom[ids] = len(dom_nodes)
            dom_nodes.append(ids)
            dom_obs.append(np.array(obs, int))
            dom_tau.append(np.array(tau, float))
    edges = []
    for g, (i, j) in enumerate(geom.points):
        for (a, b) in ((i + 1, j), (i, j + 1)):
            if a < nn and b < nn and pid[a, b] >= 0 and node_dom[pid[a, b]] != node_dom[g]:
                edges.append((g, pid[a, b]))
    return DomainGeometry(geom, partition, dom_nodes, dom_obs, dom_tau, node_dom,
                          np.array(edges, int).reshape(-1, 2))


def piston_offsets(dg: DomainGeometry, delta):
    """Differential pistons (Section 4.4): per domain and state row the constant
    c minimising the sum over border edges (i, j) of
    ((delta_i + c_dom(i)) - (delta_j + c_dom(j)))^2, with zero node-weighted
    mean over every connected group of domains; delta [n_pts, 2] is the
    analysis increment. Solved as an equality-constrained least-squares
    problem (KKT system). Returns c [n_dom, 2]."""
    D = dg.n_dom
    delta = np.asarray(delta, dtype=np.float64)
    if len(dg.edges) == 0:
        return np.zeros((D, 2))
    di, dj = dg.node_dom[dg.edges[:, 0]], dg.node_dom[dg.edges[:, 1]]
    E = np.zeros((len(dg.edges), D))
    E[np.arange(len(dg.edges)), di] += 1.0
    E[np.arange(len(dg.edges)), dj] -= 1.0
    adj = scipy.sparse.coo_matrix((np.ones(len(di)), (di, dj)), shape=(D, D))
    ncomp, comp = scipy.sparse.csgraph.connected_components(adj, directed=False)
    counts = np.array([len(n) for n in dg.dom_nodes], float)
    C = np.zeros((ncomp, D))
    C[comp, np.arange(D)] = counts
    K = np.block([[E.T @ E, C.T], [C, np.zeros((ncomp, ncomp))]])
    out = np.zeros((D, 2))
    for r in range(2):
        jump = delta[dg.edges[:, 0], r] - delta[dg.edges[:, 1], r]
        rhs = np.concatenate([-E.T @ jump, np.zeros(ncomp)])
        out[:, r] = np.linalg.solve(K, rhs)[:D]
    return out


def analysis_domains(dg: DomainGeometry, Xb, y, sigma2: float, rho: float,
                     piston: bool = True, return_parts: bool = False):
    """Local analysis per domain (Section 4.2) and, with ``piston``, the
    differential-piston correction (Section 4.4). Xb [n_pts, 2, m], y [p].
    Returns Xa, mean [n_pts, 2], spread [n_pts, 2] (members' sample std, m - 1),
    and with ``return_parts`` also the per-domain (A, wbar, W) and the piston
    constants [n_dom, 2]."""
    Xb = np.asarray(Xb, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m = Xb.shape[-1]
    xbar, Xp, Yb, ybar = observe(dg.geom, Xb)
    d = y - ybar
    Xa = np.empty_like(Xb)
    parts = []
    for nodes, idx, tau in zip(dg.dom_nodes, dg.dom_obs, dg.dom_tau):
        A, wbar, W = local_transform(Yb[idx], d[idx], tau / sigma2, m, rho)
        T = wbar[:, None] + W
        for g in nodes:
            Xa[g] = xbar[g][:, None] + Xp[g] @ T
        parts.append((A, wbar, W))
    cpist = np.zeros((dg.n_dom, 2))
    if piston:
        cpist = piston_offsets(dg, Xa.mean(axis=-1) - xbar)
        Xa += cpist[dg.node_dom][:, :, None]
    mean = Xa.mean(axis=-1)
    spread = Xa.std(axis=-1, ddof=1)
    if return_parts:
        return Xa, mean, spread, parts, cpist
    return Xa, mean, spread
