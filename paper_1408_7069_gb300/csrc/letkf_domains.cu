// Local analysis on multi-actuator domains (Section 4.1-4.2) and the
// differential-piston least squares (Section 4.4).
//
// The node grid is split by a P x P partition (block b of a side covers nodes
// [floor(b N / P), floor((b + 1) N / P)), N = nsub + 1); the valid nodes of a
// block form a local domain of n_d = 2 x nodes state rows. Its observation
// region is the union of its nodes' w x w windows, both slopes of every valid
// subaperture, weighted by R^-1 = diag(tau / sigma2), tau = Gaspari-Cohn of the
// distance from the subaperture centre to the domain's node box (0 inside).
//
// One CTA per domain, 4 MPD threads, MPD = m padded to a multiple of 8
// (identity on the padding):
//   gather  S = diag(sqrt(tau/sigma2)) Yb_region (p_d x MPD), s = sqrt(tau/sigma2) d,
//           the domain's anomaly rows X' (n_d x MPD), into shared memory
//   Gram    A = (m-1)/rho I + S^T S, c = S^T s
//   EVD     one-sided Jacobi on the columns of B = A: MPD/2 groups of 8 lanes,
//           group g holds columns 2g and 2g+1, lane l of it rows l, l+8, ...;
//           the MPD rounds of a sweep follow the odd-even transposition order
//           (even round: own pair; odd round: the pair straddling two groups,
//           the last group swapping), columns moving between groups through
//           shared memory after every round. Converged columns are lambda q.
//   apply   G = X' Q, z = Lambda^-1 Q^T c, Xa_r = xbar_r + sum_c G_rc (z_c +
//           sqrt((m-1)/lambda_c) Q_jc) for every row r of the domain
// A partition of 1 (one domain over the whole grid, the global ETKF of
// Section 3.1.1 when the window covers the pupil) runs as the multi-kernel
// pipeline below instead, for any number of slopes and nodes.
// Then the piston kernels: per domain and state row the constant that
// minimises the squared jumps of the mean increment across border edges
// (4-neighbour nodes in different domains), c = K b with b the per-domain
// edge sums and K the Laplacian's constrained pseudo-inverse (zero
// node-weighted mean per connected group of domains), precomputed on the host
// in FP64; every member of the domain's rows moves by c.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "letkf_device.cuh"

struct LkDom {
  int n_dom = 0, max_nodes = 0, max_obs = 0, rpl = 0, piston = 0;
  int *node_off = nullptr, *node_ids = nullptr;   // CSR: domain -> point ids
  int *obs_off = nullptr, *obs_slot = nullptr;    // CSR: domain -> grid slot (cell * 2 + slope)
  float *obs_w = nullptr;                         // tau / sigma2 of each observed slope
  int *node_dom = nullptr;                        // [n_pts]
  int2 *edges = nullptr;                          // [E] (i, j) point ids, dom(i) != dom(j)
  int *dedge_off = nullptr, *dedge = nullptr;     // per domain: incident edges, +(e+1) / -(e+1)
  float *KT = nullptr;                            // [D][D] K transposed
  float *delta = nullptr;                         // [n_pts][2] mean increments
  float *cpist = nullptr;                         // [D][2] piston constants
  std::vector<double> tau;                        // host: tau of each observed slope
  // one domain covering the grid (partition 1): the global ETKF pipeline
  int global = 0, kchunks = 0, mpt = 0;
  void *ns_ws = nullptr;                          // Newton-Schulz workspace (global, m > 64)
  double *gpart = nullptr;                        // [kchunks][MPD][MPD] Gram partial sums
  double *cpart = nullptr;                        // [kchunks][MPD]
  float *T = nullptr;                             // [m][m] transform wbar 1^T + W
};

namespace {

constexpr int DM_GROUP = 8;      // lanes per column pair

__device__ __forceinline__ float group8_sum(float v) {
  v += __shfl_xor_sync(FULL, v, 4);
  v += __shfl_xor_sync(FULL, v, 2);
  v += __shfl_xor_sync(FULL, v, 1);
  return v;
}

struct DomArgs {
  const int *node_off, *node_ids, *obs_off, *obs_slot;
  const float *obs_w;
  float *mean, *spread, *delta;
  int *counters;
  float tol, stop, kappa_thr;
  int max_sweeps, max_obs, max_rows;
};

// Shared-memory layout (floats): S / Q region, s, c, z, sroot, the column
// exchange [2][G][MPD] and its norms [2][G] (G = X'Q reuses the exchange after
// the sweeps when it fits, so that two CTAs share an SM), X' [rows][MPD],
// xbar [rows], 4 reduction slots.
struct DomLayout {
  int ld, sq, sv, cv, zv, sr, xb, xn, xd, gm, xm, red, total;
};
__host__ __device__ inline DomLayout dom_layout(int mpd, int max_obs, int max_rows) {
  DomLayout L;
  L.ld = mpd + 1;
  const int srows = max_obs > mpd ? max_obs : mpd;
  L.sq = 0;
  L.sv = L.sq + srows * L.ld;
  L.cv = L.sv + max_obs;
  L.zv = L.cv + mpd;
  L.sr = L.zv + mpd;
  L.xb = L.sr + mpd;
  L.xn = L.xb + 2 * (mpd / 2) * mpd;
  L.xd = L.xn + 2 * (mpd / 2);
  L.xm = L.xd + max_rows * mpd;
  L.red = L.xm + max_rows;
  L.total = L.red + 4;
  if (max_rows <= mpd) {
    L.gm = L.xb;                       // [rows][MPD] <= [2][MPD/2][MPD]
  } else {
    L.gm = L.total;
    L.total += max_rows * mpd;
  }
  return L;
}

// One round on the group's pair (P, Q): rotate (or, for the idle slot of an
// odd round, swap) with the rotation that makes the two columns orthogonal,
// from the tracked squared norms and the group-reduced dot product. Returns
// bit 0: rotated, bit 1: rotated with a cosine above the stop cosine.
template <int RPL>
__device__ __forceinline__ int dom_round(float (&P)[RPL], float (&Q)[RPL], float &nP, float &nQ,
                                         float tol2, float stop2, bool idle) {
  float part = 0.f;
#pragma unroll
  for (int i = 0; i < RPL; ++i) part = fmaf(P[i], Q[i], part);
  const float dot = group8_sum(part);
  const float x = nQ - nP, y = 2.f * dot;
  const float rh = rsqrtf(fmaxf(fmaf(x, x, y * y), 1e-37f));
  const float c2 = fmaf(0.5f * fabsf(x), rh, 0.5f);
  const float rc = rsqrtf(c2);
  const float cr = c2 * rc;
  const float sr = (x >= 0.f ? y : -y) * (0.5f * rh) * rc;
  const float t = sr * rc;
  const float dd = dot * dot, nn = nP * nQ;
  const bool rot = !idle && dd > tol2 * nn;
  const float c = rot ? cr : (idle ? 0.f : 1.f);
  const float s = rot ? sr : (idle ? 1.f : 0.f);
  const float nP2 = rot ? fmaf(-t, dot, nP) : (idle ? nQ : nP);
  const float nQ2 = rot ? fmaf(t, dot, nQ) : (idle ? nP : nQ);
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    const float p = P[i], q = Q[i];
    P[i] = fmaf(c, p, -s * q);
    Q[i] = fmaf(c, q, s * p);
  }
  nP = nP2;
  nQ = nQ2;
  return (rot ? 1 : 0) | ((rot && dd > stop2 * nn) ? 2 : 0);
}

// Column transfer between groups: every group publishes V (its rows) and n,
// then takes those of group `src`. Double-buffered, one barrier.
template <int RPL>
__device__ __forceinline__ void dom_xfer(float (&V)[RPL], float &n, float *xb, float *xn, int &buf,
                                         int g, int l, int src) {
  constexpr int MPD = 8 * RPL;
  float *b = xb + (size_t)buf * (MPD / 2) * MPD;
  float *bn = xn + buf * (MPD / 2);
#pragma unroll
  for (int i = 0; i < RPL; ++i) b[g * MPD + l + 8 * i] = V[i];
  if (l == 0) bn[g] = n;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < RPL; ++i) V[i] = b[src * MPD + l + 8 * i];
  n = bn[src];
  buf ^= 1;
}

template <int RPL>
__global__ void __launch_bounds__(32 * RPL)
    domain_kernel(const LkInst *__restrict__ insts, DomArgs a) {
  constexpr int MPD = 8 * RPL, G = MPD / 2, NT = 4 * MPD;
  extern __shared__ __align__(16) float dsm[];
  lk_pdl_wait();
  const LkInst &I = insts[0];
  const int m = I.m, tid = threadIdx.x;
  const int dom = blockIdx.x;
  const int o0 = a.obs_off[dom], np = a.obs_off[dom + 1] - o0;
  const int n0 = a.node_off[dom], nd = 2 * (a.node_off[dom + 1] - n0);
  const DomLayout Ly = dom_layout(MPD, a.max_obs, a.max_rows);
  const int LD = Ly.ld;
  float *Sq = dsm + Ly.sq, *sv = dsm + Ly.sv, *cv = dsm + Ly.cv, *zv = dsm + Ly.zv;
  float *srt = dsm + Ly.sr, *xb = dsm + Ly.xb, *xn = dsm + Ly.xn, *Xd = dsm + Ly.xd;
  float *Gm = dsm + Ly.gm, *xm = dsm + Ly.xm, *red = dsm + Ly.red;
  const float *Ybp = static_cast<const float *>(I.Ybp);
  const float *dp = static_cast<const float *>(I.dp);
  float *X = static_cast<float *>(I.X);

  // ---- gather: S, s, the anomaly rows; tr(S^T S) for kappa_hat ----
  if (tid == 0) red[0] = 0.f;
  __syncthreads();
  float tr = 0.f;
  for (int e = tid; e < np * MPD; e += NT) {
    const int k = e / MPD, i = e - k * MPD;
    const int slot = a.obs_slot[o0 + k];
    const float sw = sqrtf(a.obs_w[o0 + k]);
    const float v = i < m ? sw * Ybp[(size_t)slot * m + i] : 0.f;
    Sq[k * LD + i] = v;
    tr = fmaf(v, v, tr);
  }
  for (int k = tid; k < np; k += NT) sv[k] = sqrtf(a.obs_w[o0 + k]) * dp[a.obs_slot[o0 + k]];
  for (int e = tid; e < nd * MPD; e += NT) {
    const int r = e / MPD, j = e - r * MPD;
    const int pid = a.node_ids[n0 + (r >> 1)];
    Xd[r * MPD + j] = j < m ? X[((size_t)pid * 2 + (r & 1)) * m + j] : 0.f;
  }
  tr = lk_warp_sum(tr);
  if ((tid & 31) == 0) atomicAdd(&red[0], tr);
  __syncthreads();
  const float inv_m = 1.f / float(m);
  for (int r = tid >> 5; r < nd; r += NT / 32) {   // warp per row: mean, anomalies
    float s = 0.f;
    for (int j = tid & 31; j < m; j += 32) s += Xd[r * MPD + j];
    s = lk_warp_sum(s) * inv_m;
    for (int j = tid & 31; j < m; j += 32) Xd[r * MPD + j] -= s;
    if ((tid & 31) == 0) xm[r] = s;
  }
  const float alpha = float(I.alpha);
  if (tid == 0 && a.kappa_thr > 0.f && 1.f + red[0] / alpha > a.kappa_thr)
    atomicAdd(&a.counters[1], 1);
  __syncthreads();

  // ---- Gram in the Jacobi layout, and c = S^T s ----
  const int g = tid >> 3, l = tid & 7;
  const int cP = 2 * g, cQ = 2 * g + 1;
  float P[RPL], Q[RPL];
#pragma unroll
  for (int i = 0; i < RPL; ++i) P[i] = Q[i] = 0.f;
  for (int k = 0; k < np; ++k) {
    const float *row = Sq + k * LD;
    const float sp = row[cP], sq = row[cQ];
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      const float sr = row[l + 8 * i];
      P[i] = fmaf(sr, sp, P[i]);
      Q[i] = fmaf(sr, sq, Q[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    const int r = l + 8 * i;
    if (r == cP) P[i] += cP < m ? alpha : 1.f;
    if (r == cQ) Q[i] += cQ < m ? alpha : 1.f;
  }
  if (tid < MPD) {
    float s = 0.f;
    for (int k = 0; k < np; ++k) s = fmaf(Sq[k * LD + tid], sv[k], s);
    cv[tid] = s;
  }

  // ---- Jacobi sweeps ----
  const float tol2 = a.tol * a.tol, stop2 = a.stop * a.stop;
  int buf = 0, sweeps = 0;
  bool conv = false;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    float pp = 0.f, qq = 0.f;
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      pp = fmaf(P[i], P[i], pp);
      qq = fmaf(Q[i], Q[i], qq);
    }
    float nP = group8_sum(pp), nQ = group8_sum(qq);
    int flags = 0;
    for (int r = 0; r < G; ++r) {
      flags |= dom_round<RPL>(P, Q, nP, nQ, tol2, stop2, false);
      dom_xfer<RPL>(Q, nQ, xb, xn, buf, g, l, g + 1 < G ? g + 1 : 0);
      flags |= dom_round<RPL>(P, Q, nP, nQ, tol2, stop2, g == G - 1);
      dom_xfer<RPL>(P, nP, xb, xn, buf, g, l, g > 0 ? g - 1 : G - 1);
    }
    sweeps = sweep + 1;
    if (!__syncthreads_or(flags & 2)) {
      conv = true;
      break;
    }
  }
  if (tid == 0) {
    atomicMax(&a.counters[2], sweeps);
    atomicAdd(&a.counters[3], sweeps);
    if (!conv) atomicOr(&a.counters[0], LK_BIT_NOCONVERGE);
  }

  // ---- eigenpairs: lambda = |b|, q = b / lambda, into Q (aliases S) ----
  float pp = 0.f, qq = 0.f;
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    pp = fmaf(P[i], P[i], pp);
    qq = fmaf(Q[i], Q[i], qq);
  }
  const float lP = sqrtf(group8_sum(pp)), lQ = sqrtf(group8_sum(qq));
  __syncthreads();                                  // every read of S is done
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    Sq[(l + 8 * i) * LD + cP] = P[i] / lP;
    Sq[(l + 8 * i) * LD + cQ] = Q[i] / lQ;
  }
  if (l == 0) {
    zv[cP] = lP;
    zv[cQ] = lQ;
  }
  __syncthreads();
  if (tid < MPD) {                                  // z = Lambda^-1 Q^T c, sqrt((m-1)/lambda)
    const float lam = zv[tid];
    float u = 0.f;
    for (int r = 0; r < MPD; ++r) u = fmaf(Sq[r * LD + tid], cv[r], u);
    srt[tid] = sqrtf(float(m - 1) / lam);
    zv[tid] = u / lam;
  }
  for (int e = tid; e < nd * MPD; e += NT) {        // G = X' Q
    const int r = e / MPD, c = e - r * MPD;
    float s = 0.f;
    for (int j = 0; j < MPD; ++j) s = fmaf(Xd[r * MPD + j], Sq[j * LD + c], s);
    Gm[r * MPD + c] = s;
  }
  __syncthreads();

  // ---- apply: a warp per row ----
  const int lane = tid & 31;
  for (int r = tid >> 5; r < nd; r += NT / 32) {
    const int pid = a.node_ids[n0 + (r >> 1)], comp = r & 1;
    float wb = 0.f;                                 // X'_r wbar: the mean increment
    for (int c = lane; c < MPD; c += 32) wb = fmaf(Gm[r * MPD + c], zv[c], wb);
    wb = lk_warp_sum(wb);
    float sum = 0.f, sq = 0.f;
    float *xrow = X + ((size_t)pid * 2 + comp) * m;
    for (int j = lane; j < m; j += 32) {
      float q = 0.f;
      for (int c = 0; c < MPD; ++c) q = fmaf(Gm[r * MPD + c] * srt[c], Sq[j * LD + c], q);
      const float xa = xm[r] + wb + q;
      xrow[j] = xa;
      sum += xa;
    }
    const float mu = lk_warp_sum(sum) * inv_m;
    for (int j = lane; j < m; j += 32) {
      const float dv = xrow[j] - mu;
      sq = fmaf(dv, dv, sq);
    }
    const float sp = sqrtf(lk_warp_sum(sq) / float(m - 1));
    if (lane == 0) {
      if (a.mean) a.mean[(size_t)pid * 2 + comp] = mu;
      if (a.spread) a.spread[(size_t)pid * 2 + comp] = sp;
      a.delta[(size_t)pid * 2 + comp] = mu - xm[r];
      if (!isfinite(mu) || !isfinite(sp)) atomicOr(&a.counters[0], LK_BIT_NONFINITE);
    }
  }
}

// b_d = sum over the border edges of domain d of (delta_other - delta_own) for
// both state rows (a fixed order: the domain's incident edge list), then
// c = K b with one thread per domain. One CTA.
__global__ void __launch_bounds__(1024)
    piston_solve_kernel(int n_dom, const int2 *__restrict__ edges, const int *__restrict__ dedge_off,
                        const int *__restrict__ dedge, const float *__restrict__ delta,
                        const float *__restrict__ KT, float *__restrict__ cpist) {
  extern __shared__ __align__(16) float bsm[];   // [2][n_dom]
  lk_pdl_wait();
  for (int d = threadIdx.x; d < n_dom; d += blockDim.x) {
    float b0 = 0.f, b1 = 0.f;
    for (int q = dedge_off[d]; q < dedge_off[d + 1]; ++q) {
      const int se = dedge[q];
      const int2 ed = edges[(se > 0 ? se : -se) - 1];
      const int own = se > 0 ? ed.x : ed.y, oth = se > 0 ? ed.y : ed.x;
      b0 += delta[2 * oth] - delta[2 * own];
      b1 += delta[2 * oth + 1] - delta[2 * own + 1];
    }
    bsm[d] = b0;
    bsm[n_dom + d] = b1;
  }
  __syncthreads();
  for (int d = threadIdx.x; d < n_dom; d += blockDim.x) {
    float c0 = 0.f, c1 = 0.f;
    for (int e = 0; e < n_dom; ++e) {
      const float k = KT[(size_t)e * n_dom + d];
      c0 = fmaf(k, bsm[e], c0);
      c1 = fmaf(k, bsm[n_dom + e], c1);
    }
    cpist[2 * d] = c0;
    cpist[2 * d + 1] = c1;
  }
}

// Every member of every node row moves by its domain's constant (and so does
// the analysis mean). A warp per node.
__global__ void __launch_bounds__(LK_WARP_CTA)
    piston_apply_kernel(const LkInst *__restrict__ insts, const int *__restrict__ node_dom,
                        const float *__restrict__ cpist, float *__restrict__ mean) {
  lk_pdl_wait();
  const LkInst &I = insts[0];
  const int node = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (node >= I.n_pts) return;
  const int d = node_dom[node];
  const float c0 = cpist[2 * d], c1 = cpist[2 * d + 1];
  float *x = static_cast<float *>(I.X) + (size_t)node * 2 * I.m;
  for (int j = lane; j < I.m; j += 32) {
    x[j] += c0;
    x[I.m + j] += c1;
  }
  if (lane == 0 && mean) {
    mean[2 * node] += c0;
    mean[2 * node + 1] += c1;
  }
}

// ---------------------------------------------------------------------------
// One domain covering the grid (partition 1): the global ETKF (Section 3.1.1)
// for any number of slopes and nodes, as three kernels:
//   gram    partial sums of A = S^T S and c = S^T s over chunks of slopes, one
//           CTA per (upper-triangle 32 x 32 tile of A, chunk): every term
//           w_k y_ka y_kb (w = tau / sigma2, y the grid's FP32 values) formed
//           exactly as two floats (FMA two-products) and accumulated as an
//           unevaluated float pair (two-sum, the error carried in the low
//           part): about 1e-11 relative to the sum of |terms| over a chunk, on
//           the FP32 pipe, against FP64 FMAs at 1/75 of its rate
//   solve   one CTA: A = (m-1)/rho I + the partials (FP64), its FP32 rounding
//           diagonalised by the domain kernel's Jacobi (A = Q Lambda Q^T), then
//           wbar = A^-1 c by mixed-precision iterative refinement (residual
//           c - A wbar in FP64, correction Q Lambda^-1 Q^T r in FP32: the error
//           contracts by about kappa eps32 per step, so a few steps reach the
//           FP64 solution although kappa_hat reaches 1e4-1e5 for the whole
//           pupil), and T = wbar 1^T + Q ((m-1) Lambda^-1)^(1/2) Q^T
//   apply   a CTA per 16 state rows: Xa_r = xbar_r + X'_r T, mean, spread
// ---------------------------------------------------------------------------
constexpr int GL_TILE = 32, GL_KC = 64, GL_REFINE = 4;

// hi + lo += w a b: the product a b as two floats (FMA two-product), each times w
// (again two-product for the high part), added to the pair by Knuth's two-sum.
// The _rn intrinsics keep the compiler from contracting the steps.
__device__ __forceinline__ void gl_add_wab(float &hi, float &lo, float w, float a, float b) {
  const float ph = __fmul_rn(a, b);
  const float pl = fmaf(a, b, -ph);
  const float qh = __fmul_rn(w, ph);
  const float ql = fmaf(w, ph, -qh);
  const float t = fmaf(w, pl, ql);
  const float s = __fadd_rn(hi, qh);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(qh, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, t));
}

__global__ void __launch_bounds__(256)
    global_gram_kernel(const LkInst *__restrict__ insts, const int *__restrict__ obs_slot,
                       const float *__restrict__ obs_w, int np, int mpt,
                       double *__restrict__ gpart, double *__restrict__ cpart) {
  __shared__ float si[GL_KC][GL_TILE + 1], sj[GL_KC][GL_TILE + 1], sw[GL_KC], sd[GL_KC];
  lk_pdl_wait();
  const LkInst &I = insts[0];
  const int m = I.m;
  const float *Ybp = static_cast<const float *>(I.Ybp);
  const float *dp = static_cast<const float *>(I.dp);
  // upper-triangle tile (ti <= tj) from blockIdx.x
  const int nt = mpt / GL_TILE;
  int ti = 0, tj = blockIdx.x;
  while (tj >= nt - ti) {
    tj -= nt - ti;
    ++ti;
  }
  tj += ti;
  const int kc = blockIdx.y, k0 = kc * GL_KC;
  const int kn = np - k0 < GL_KC ? np - k0 : GL_KC;
  for (int e = threadIdx.x; e < GL_KC * GL_TILE; e += blockDim.x) {
    const int k = e / GL_TILE, i = e - k * GL_TILE;
    float a = 0.f, b = 0.f;
    if (k < kn) {
      const int slot = obs_slot[k0 + k];
      const int ri = ti * GL_TILE + i, rj = tj * GL_TILE + i;
      if (ri < m) a = Ybp[(size_t)slot * m + ri];
      if (rj < m) b = Ybp[(size_t)slot * m + rj];
    }
    si[k][i] = a;
    sj[k][i] = b;
  }
  for (int k = threadIdx.x; k < GL_KC; k += blockDim.x) {
    sw[k] = k < kn ? obs_w[k0 + k] : 0.f;
    sd[k] = k < kn ? dp[obs_slot[k0 + k]] : 0.f;
  }
  __syncthreads();
  const int a0 = (threadIdx.x / 16) * 2, b0 = (threadIdx.x % 16) * 2;
  float hi[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, lo[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k = 0; k < GL_KC; ++k) {
    const float w = sw[k];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) gl_add_wab(hi[x][y], lo[x][y], w, si[k][a0 + x], sj[k][b0 + y]);
  }
  double *out = gpart + (size_t)kc * mpt * mpt;
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y)
      out[(size_t)(ti * GL_TILE + a0 + x) * mpt + tj * GL_TILE + b0 + y] =
          (double)hi[x][y] + (double)lo[x][y];
  if (ti == tj && threadIdx.x < GL_TILE) {
    float ch = 0.f, cl = 0.f;
    for (int k = 0; k < GL_KC; ++k) gl_add_wab(ch, cl, sw[k], si[k][threadIdx.x], sd[k]);
    cpart[(size_t)kc * mpt + ti * GL_TILE + threadIdx.x] = (double)ch + (double)cl;
  }
}

// Shared memory of the solve kernel: A (FP64, [MPD][MPD+1]), c, wbar, r (FP64),
// then one float region used first as the Jacobi's column exchange and then
// for Q ([MPD][MPD+1]), and lambda, t, sroot.
template <int RPL>
__host__ __device__ constexpr size_t gsolve_qfloats() {
  constexpr size_t MPD = 8 * RPL, q = MPD * (MPD + 1), x = 2 * (MPD / 2) * MPD + 2 * (MPD / 2);
  return q > x ? q : x;
}
template <int RPL>
size_t global_solve_smem() {
  constexpr int MPD = 8 * RPL;
  return sizeof(double) * ((size_t)MPD * (MPD + 1) + 3 * MPD) +
         sizeof(float) * (gsolve_qfloats<RPL>() + 3 * MPD);
}

template <int RPL>
__global__ void __launch_bounds__(32 * RPL)
    global_solve_kernel(const LkInst *__restrict__ insts, const double *__restrict__ gpart,
                        const double *__restrict__ cpart, int kchunks, int mpt,
                        float *__restrict__ T, float tol, float stop, int max_sweeps,
                        int *__restrict__ counters) {
  constexpr int MPD = 8 * RPL, G = MPD / 2, NT = 4 * MPD, LD = MPD + 1;
  extern __shared__ __align__(16) double gsm[];
  lk_pdl_wait();
  const LkInst &I = insts[0];
  const int m = I.m, tid = threadIdx.x;
  double *A = gsm;                              // [MPD][LD] FP64
  double *c64 = A + MPD * LD, *w64 = c64 + MPD, *r64 = w64 + MPD;
  float *Qs = reinterpret_cast<float *>(r64 + MPD);   // [MPD][LD], after the sweeps
  float *xb = Qs, *xn = xb + 2 * G * MPD;             // exchange, during the sweeps
  float *lam = Qs + gsolve_qfloats<RPL>(), *tv = lam + MPD, *sr = tv + MPD;
  const double alpha = I.alpha;
  // ---- A and c from the partial sums: element (i, j) of the upper triangle
  // was summed in tile (min / 32, max / 32) at (min, max) ----
  for (int e = tid; e < MPD * MPD; e += NT) {
    const int i = e / MPD, j = e - i * MPD;
    const int a = i <= j ? i : j, b = i <= j ? j : i;
    double s = 0.0;
    for (int k = 0; k < kchunks; ++k) s += gpart[((size_t)k * mpt + a) * mpt + b];
    if (i == j) s += i < m ? alpha : 1.0;
    A[i * LD + j] = s;
  }
  if (tid < MPD) {
    double s = 0.0;
    for (int k = 0; k < kchunks; ++k) s += cpart[(size_t)k * mpt + tid];
    c64[tid] = s;
    w64[tid] = 0.0;
  }
  __syncthreads();
  // ---- FP32 Jacobi on the rounded A (the domain kernel's layout and rounds) ----
  const int g = tid >> 3, l = tid & 7;
  float P[RPL], Q[RPL];
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    P[i] = (float)A[(l + 8 * i) * LD + 2 * g];
    Q[i] = (float)A[(l + 8 * i) * LD + 2 * g + 1];
  }
  const float tol2 = tol * tol, stop2 = stop * stop;
  int buf = 0, sweeps = 0;
  bool conv = false;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    float pp = 0.f, qq = 0.f;
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      pp = fmaf(P[i], P[i], pp);
      qq = fmaf(Q[i], Q[i], qq);
    }
    float nP = group8_sum(pp), nQ = group8_sum(qq);
    int flags = 0;
    for (int r = 0; r < G; ++r) {
      flags |= dom_round<RPL>(P, Q, nP, nQ, tol2, stop2, false);
      dom_xfer<RPL>(Q, nQ, xb, xn, buf, g, l, g + 1 < G ? g + 1 : 0);
      flags |= dom_round<RPL>(P, Q, nP, nQ, tol2, stop2, g == G - 1);
      dom_xfer<RPL>(P, nP, xb, xn, buf, g, l, g > 0 ? g - 1 : G - 1);
    }
    sweeps = sweep + 1;
    if (!__syncthreads_or(flags & 2)) {
      conv = true;
      break;
    }
  }
  if (tid == 0) {
    atomicMax(&counters[2], sweeps);
    atomicAdd(&counters[3], sweeps);
    if (!conv) atomicOr(&counters[0], LK_BIT_NOCONVERGE);
  }
  float pp = 0.f, qq = 0.f;
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    pp = fmaf(P[i], P[i], pp);
    qq = fmaf(Q[i], Q[i], qq);
  }
  const float lP = sqrtf(group8_sum(pp)), lQ = sqrtf(group8_sum(qq));
  __syncthreads();                              // the exchange region becomes Q
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    Qs[(l + 8 * i) * LD + 2 * g] = P[i] / lP;
    Qs[(l + 8 * i) * LD + 2 * g + 1] = Q[i] / lQ;
  }
  if (l == 0) {
    lam[2 * g] = lP;
    lam[2 * g + 1] = lQ;
  }
  __syncthreads();
  if (tid < MPD) sr[tid] = sqrtf(float(m - 1) / lam[tid]);
  // ---- wbar = A^-1 c by iterative refinement ----
  for (int it = 0; it < GL_REFINE; ++it) {
    if (tid < MPD) {                              // r = c - A w (FP64)
      double s = c64[tid];
      for (int j = 0; j < MPD; ++j) s = fma(-A[tid * LD + j], w64[j], s);
      r64[tid] = s;
    }
    __syncthreads();
    if (tid < MPD) {                              // t = Lambda^-1 Q^T r
      float s = 0.f;
      for (int j = 0; j < MPD; ++j) s = fmaf(Qs[j * LD + tid], (float)r64[j], s);
      tv[tid] = s / lam[tid];
    }
    __syncthreads();
    if (tid < MPD) {                              // w += Q t
      float s = 0.f;
      for (int c = 0; c < MPD; ++c) s = fmaf(Qs[tid * LD + c], tv[c], s);
      w64[tid] += (double)s;
    }
    __syncthreads();
  }
  // ---- T = wbar 1^T + Q diag(sroot) Q^T ----
  for (int e = tid; e < m * m; e += NT) {
    const int i = e / m, j = e - i * m;
    float s = 0.f;
    for (int c = 0; c < MPD; ++c) s = fmaf(Qs[i * LD + c] * sr[c], Qs[j * LD + c], s);
    T[e] = (float)w64[i] + s;
  }
}

// Xa_r = xbar_r + X'_r T for 16 state rows per CTA (rows = node-major, 2 per node).
__global__ void __launch_bounds__(256)
    global_apply_kernel(const LkInst *__restrict__ insts, const float *__restrict__ T,
                        float *__restrict__ mean, float *__restrict__ spread,
                        int *__restrict__ counters) {
  extern __shared__ __align__(16) float asm_[];
  lk_pdl_wait();
  const LkInst &I = insts[0];
  const int m = I.m, tid = threadIdx.x;
  float *Ts = asm_;                               // [m][m]
  float *xr = Ts + m * m;                         // [16][m]
  for (int e = tid; e < m * m; e += blockDim.x) Ts[e] = T[e];
  const long long r0 = (long long)blockIdx.x * 16, nrows = 2LL * I.n_pts;
  float *X = static_cast<float *>(I.X);
  for (int e = tid; e < 16 * m; e += blockDim.x) {
    const long long r = r0 + e / m;
    xr[e] = r < nrows ? X[r * m + e % m] : 0.f;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  const float inv_m = 1.f / float(m);
  for (int q = warp; q < 16; q += 8) {
    const long long r = r0 + q;
    if (r >= nrows) break;
    float s = 0.f;
    for (int j = lane; j < m; j += 32) s += xr[q * m + j];
    const float xbar = lk_warp_sum(s) * inv_m;
    float sum = 0.f;
    for (int j = lane; j < m; j += 32) {
      float acc = 0.f;
      for (int i = 0; i < m; ++i) acc = fmaf(xr[q * m + i] - xbar, Ts[i * m + j], acc);
      const float xa = xbar + acc;
      X[r * m + j] = xa;
      sum += xa;
    }
    const float mu = lk_warp_sum(sum) * inv_m;
    float sq = 0.f;
    for (int j = lane; j < m; j += 32) {
      const float dv = X[r * m + j] - mu;
      sq = fmaf(dv, dv, sq);
    }
    const float sp = sqrtf(lk_warp_sum(sq) / float(m - 1));
    if (lane == 0) {
      if (mean) mean[r] = mu;
      if (spread) spread[r] = sp;
      if (!isfinite(mu) || !isfinite(sp)) atomicOr(&counters[0], LK_BIT_NONFINITE);
    }
  }
}

constexpr int gl_mpt(int mpd) { return ((mpd + GL_TILE - 1) / GL_TILE) * GL_TILE; }

template <int RPL>
cudaError_t launch_global_rpl(letkf_ctx *h, void *mean, void *spread) {
  const LkDom &D = *h->dom;
  const LkInst &I = h->inst[0];
  constexpr int MPT = gl_mpt(8 * RPL), NT = MPT / GL_TILE;
  cudaError_t e = lk_launch_pdl(global_gram_kernel, dim3(NT * (NT + 1) / 2, D.kchunks), 256, 0,
                                h->stream, h->d_inst, (const int *)D.obs_slot,
                                (const float *)D.obs_w, D.max_obs, MPT, D.gpart, D.cpart);
  if (e != cudaSuccess) return e;
  e = lk_launch_pdl(global_solve_kernel<RPL>, 1, 32 * RPL, global_solve_smem<RPL>(), h->stream,
                    h->d_inst, (const double *)D.gpart, (const double *)D.cpart, D.kchunks, MPT,
                    D.T, (float)h->tol32, (float)(h->stop32 > h->tol32 ? h->stop32 : h->tol32),
                    h->max_sweeps, h->counters);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((2LL * I.n_pts + 15) / 16);
  return lk_launch_pdl(global_apply_kernel, blocks, 256,
                       sizeof(float) * ((size_t)I.m * I.m + 16 * (size_t)I.m), h->stream,
                       h->d_inst, (const float *)D.T, static_cast<float *>(mean),
                       static_cast<float *>(spread), h->counters);
}

template <int RPL>
cudaError_t setup_global_rpl(const LkDom &D, int m) {
  cudaError_t e = cudaFuncSetAttribute(global_solve_kernel<RPL>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)global_solve_smem<RPL>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(global_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(float) * ((size_t)m * m + 16 * (size_t)m)));
  (void)D;
  return e;
}

template <int RPL>
cudaError_t launch_rpl(letkf_ctx *h, const DomArgs &a) {
  const LkDom &D = *h->dom;
  const size_t smem = (size_t)dom_layout(8 * RPL, D.max_obs, 2 * D.max_nodes).total * sizeof(float);
  return lk_launch_pdl(domain_kernel<RPL>, (unsigned)D.n_dom, 32 * RPL, smem, h->stream,
                       h->d_inst, a);
}

template <int RPL>
cudaError_t setup_rpl(const LkDom &D) {
  const size_t smem = (size_t)dom_layout(8 * RPL, D.max_obs, 2 * D.max_nodes).total * sizeof(float);
  return cudaFuncSetAttribute(domain_kernel<RPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

// Rows per lane of the Jacobi layout (MPD = 8 RPL columns); 0: wider than the
// one-CTA layout takes (the global ETKF's Newton-Schulz path, letkf_global.cu).
int rpl_of(int m) {
  return m <= 16 ? 2 : m <= 32 ? 4 : m <= 64 ? 8 : m <= 104 ? 13 : m <= 128 ? 16 : 0;
}

constexpr int NS_ITERS = 40;      // Newton-Schulz iterations of the wide global path (at most 64;
                                  // converged iterations are skipped on the device)

template <typename T>
cudaError_t dup(T **dst, const std::vector<T> &src) {
  *dst = nullptr;
  if (src.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void **)dst, src.size() * sizeof(T));
  if (e == cudaSuccess) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

// Cholesky solve of the SPD system M X = B in place (n x n, B n x k), FP64.
bool chol_solve(std::vector<double> &M, int n, std::vector<double> &B, int k) {
  for (int j = 0; j < n; ++j) {
    double s = M[(size_t)j * n + j];
    for (int q = 0; q < j; ++q) s -= M[(size_t)j * n + q] * M[(size_t)j * n + q];
    if (!(s > 0)) return false;
    const double d = sqrt(s);
    M[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = M[(size_t)i * n + j];
      for (int q = 0; q < j; ++q) t -= M[(size_t)i * n + q] * M[(size_t)j * n + q];
      M[(size_t)i * n + j] = t / d;
    }
  }
  for (int c = 0; c < k; ++c) {
    for (int i = 0; i < n; ++i) {                 // L y = b
      double t = B[(size_t)i * k + c];
      for (int q = 0; q < i; ++q) t -= M[(size_t)i * n + q] * B[(size_t)q * k + c];
      B[(size_t)i * k + c] = t / M[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {            // L^T x = y
      double t = B[(size_t)i * k + c];
      for (int q = i + 1; q < n; ++q) t -= M[(size_t)q * n + i] * B[(size_t)q * k + c];
      B[(size_t)i * k + c] = t / M[(size_t)i * n + i];
    }
  }
  return true;
}

}  // namespace

// Domain tables of a single-instance handle (cfg.partition > 0); the per-node
// geometry (nodes, subapertures, grid) is already in h->inst[0].
letkf_status lk_domains_build(letkf_ctx *h, const letkf_config &c, const std::vector<int> &pid,
                              const std::vector<int2> &pts, const std::vector<int2> &saps,
                              std::string &err) {
  const LkInst &I = h->inst[0];
  const int nsub = c.nsub, nn = nsub + 1, P = c.partition, w = c.window, hw = w / 2;
  LkDom *D = new (std::nothrow) LkDom();
  if (!D) return LETKF_ERR_NOMEM;
  h->dom = D;
  D->piston = c.piston != 0;
  std::vector<int> sid((size_t)nsub * nsub, -1);
  for (size_t k = 0; k < saps.size(); ++k) sid[(size_t)saps[k].x * nsub + saps[k].y] = (int)k;
  std::vector<int> bb(P + 1);
  for (int b = 0; b <= P; ++b) bb[b] = (int)(((long long)b * nn) / P);
  const double cl = c.loc_len > 0 ? c.loc_len : w / 4.0;
  std::vector<int> node_off{0}, node_ids, obs_off{0}, obs_slot, node_dom(pts.size(), -1);
  std::vector<char> mark((size_t)nsub * nsub, 0);
  for (int bi = 0; bi < P; ++bi)
    for (int bj = 0; bj < P; ++bj) {
      std::vector<int> ids;
      for (int i = bb[bi]; i < bb[bi + 1]; ++i)
        for (int j = bb[bj]; j < bb[bj + 1]; ++j)
          if (pid[(size_t)i * nn + j] >= 0) ids.push_back(pid[(size_t)i * nn + j]);
      if (ids.empty()) continue;
      int i0 = nn, i1 = -1, j0 = nn, j1 = -1;
      for (int q : ids) {
        i0 = std::min(i0, pts[q].x);
        i1 = std::max(i1, pts[q].x);
        j0 = std::min(j0, pts[q].y);
        j1 = std::max(j1, pts[q].y);
        node_dom[q] = (int)node_off.size() - 1;
        node_ids.push_back(q);
      }
      node_off.push_back((int)node_ids.size());
      // union of the nodes' windows, row-major over the subaperture grid
      std::vector<int> region;
      for (int q : ids)
        for (int s = pts[q].x - hw; s < pts[q].x - hw + w; ++s)
          for (int t = pts[q].y - hw; t < pts[q].y - hw + w; ++t)
            if (s >= 0 && s < nsub && t >= 0 && t < nsub && sid[(size_t)s * nsub + t] >= 0 &&
                !mark[(size_t)s * nsub + t]) {
              mark[(size_t)s * nsub + t] = 1;
              region.push_back(s * nsub + t);
            }
      std::sort(region.begin(), region.end());
      for (int st : region) {
        const int s = st / nsub, t = st % nsub;
        mark[(size_t)st] = 0;
        double tau = 1.0;
        if (c.taper == 1) {
          const double dx = std::max({i0 - (s + 0.5), 0.0, (s + 0.5) - i1});
          const double dy = std::max({j0 - (t + 0.5), 0.0, (t + 0.5) - j1});
          tau = lk_gaspari_cohn(hypot(dx, dy) / cl);
        }
        const long long cell = (long long)(s + I.h) * I.gs_cols + (t + I.h);
        obs_slot.push_back((int)(cell * 2));
        obs_slot.push_back((int)(cell * 2 + 1));
        D->tau.push_back(tau);
        D->tau.push_back(tau);
      }
      obs_off.push_back((int)obs_slot.size());
      D->max_obs = std::max(D->max_obs, (int)region.size() * 2);
      D->max_nodes = std::max(D->max_nodes, (int)ids.size());
    }
  D->n_dom = (int)node_off.size() - 1;
  // the global ETKF of more than 64 members takes the Newton-Schulz path
  // (m = 101: 0.59 ms against 0.72 ms for the one-CTA Jacobi, measured)
  D->rpl = (P == 1 && c.m > 64) ? 0 : rpl_of(c.m);
  D->global = P == 1;
  if (D->rpl == 0 && !D->global) {
    err = "local domains of more than one take m <= 128";
    return LETKF_ERR_ARG;
  }
  const int mpd = D->rpl ? 8 * D->rpl : ((c.m + 63) / 64) * 64;
  const size_t smem = (size_t)dom_layout(mpd, D->max_obs, 2 * D->max_nodes).total * sizeof(float);
  int dev_smem = 0;
  cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (!D->global && smem > (size_t)dev_smem) {
    err = "local domains too large for one CTA's shared memory (fewer nodes per domain, a "
          "smaller window or fewer members)";
    return LETKF_ERR_ARG;
  }
  // border edges and their incidence per domain
  std::vector<int2> edges;
  for (size_t q = 0; q < pts.size(); ++q) {
    const int i = pts[q].x, j = pts[q].y;
    const int nb[2] = {i + 1 < nn ? pid[(size_t)(i + 1) * nn + j] : -1,
                       j + 1 < nn ? pid[(size_t)i * nn + j + 1] : -1};
    for (int o : nb)
      if (o >= 0 && node_dom[o] != node_dom[q]) edges.push_back(make_int2((int)q, o));
  }
  const int Dn = D->n_dom;
  std::vector<std::vector<int>> inc(Dn);
  for (size_t e = 0; e < edges.size(); ++e) {
    inc[node_dom[edges[e].x]].push_back((int)e + 1);
    inc[node_dom[edges[e].y]].push_back(-((int)e + 1));
  }
  std::vector<int> dedge_off{0}, dedge;
  for (auto &v : inc) {
    dedge.insert(dedge.end(), v.begin(), v.end());
    dedge_off.push_back((int)dedge.size());
  }
  // K = (I - sum_comp 1_c w_c^T) L^+, L^+ = M^-1 - sum_comp u_c u_c^T with
  // M = L + sum_comp u_c u_c^T (u_c: normalised indicator of a connected group)
  std::vector<double> Lm((size_t)Dn * Dn, 0.0);
  for (const int2 &ed : edges) {
    const int a = node_dom[ed.x], b = node_dom[ed.y];
    Lm[(size_t)a * Dn + a] += 1;
    Lm[(size_t)b * Dn + b] += 1;
    Lm[(size_t)a * Dn + b] -= 1;
    Lm[(size_t)b * Dn + a] -= 1;
  }
  std::vector<int> comp(Dn, -1);
  int ncomp = 0;
  for (int s = 0; s < Dn; ++s) {
    if (comp[s] >= 0) continue;
    std::vector<int> stack{s};
    comp[s] = ncomp;
    while (!stack.empty()) {
      const int u = stack.back();
      stack.pop_back();
      for (int v = 0; v < Dn; ++v)
        if (comp[v] < 0 && Lm[(size_t)u * Dn + v] != 0.0) {
          comp[v] = ncomp;
          stack.push_back(v);
        }
    }
    ++ncomp;
  }
  std::vector<double> csize(ncomp, 0.0), cnodes(ncomp, 0.0);
  for (int d = 0; d < Dn; ++d) {
    csize[comp[d]] += 1;
    cnodes[comp[d]] += node_off[d + 1] - node_off[d];
  }
  std::vector<double> M = Lm;
  for (int a = 0; a < Dn; ++a)
    for (int b = 0; b < Dn; ++b)
      if (comp[a] == comp[b]) M[(size_t)a * Dn + b] += 1.0 / csize[comp[a]];
  std::vector<double> Lp((size_t)Dn * Dn, 0.0);
  for (int d = 0; d < Dn; ++d) Lp[(size_t)d * Dn + d] = 1.0;
  if (!chol_solve(M, Dn, Lp, Dn)) {
    err = "piston system is not positive definite";
    return LETKF_ERR_ARG;
  }
  for (int a = 0; a < Dn; ++a)
    for (int b = 0; b < Dn; ++b)
      if (comp[a] == comp[b]) Lp[(size_t)a * Dn + b] -= 1.0 / csize[comp[a]];
  // weighted centring per group: K = Lp - 1_c (w_c^T Lp)
  std::vector<double> wrow((size_t)ncomp * Dn, 0.0);
  for (int d = 0; d < Dn; ++d) {
    const double wd = (node_off[d + 1] - node_off[d]) / cnodes[comp[d]];
    for (int b = 0; b < Dn; ++b) wrow[(size_t)comp[d] * Dn + b] += wd * Lp[(size_t)d * Dn + b];
  }
  std::vector<float> KT((size_t)Dn * Dn);
  for (int a = 0; a < Dn; ++a)
    for (int b = 0; b < Dn; ++b)
      KT[(size_t)b * Dn + a] = (float)(Lp[(size_t)a * Dn + b] - wrow[(size_t)comp[a] * Dn + b]);
  std::vector<float> wv(D->tau.size());
  for (size_t q = 0; q < wv.size(); ++q) wv[q] = (float)(D->tau[q] / c.sigma2);
  cudaError_t e = dup(&D->node_off, node_off);
  if (e == cudaSuccess) e = dup(&D->node_ids, node_ids);
  if (e == cudaSuccess) e = dup(&D->obs_off, obs_off);
  if (e == cudaSuccess) e = dup(&D->obs_slot, obs_slot);
  if (e == cudaSuccess) e = dup(&D->obs_w, wv);
  if (e == cudaSuccess) e = dup(&D->node_dom, node_dom);
  if (e == cudaSuccess && !edges.empty()) e = dup(&D->edges, edges);
  if (e == cudaSuccess) e = dup(&D->dedge_off, dedge_off);
  if (e == cudaSuccess && !dedge.empty()) e = dup(&D->dedge, dedge);
  if (e == cudaSuccess) e = dup(&D->KT, KT);
  if (e == cudaSuccess) e = cudaMalloc((void **)&D->delta, pts.size() * 2 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void **)&D->cpist, (size_t)Dn * 2 * sizeof(float));
  if (e == cudaSuccess && D->global) {
    const int mpt = D->rpl ? gl_mpt(mpd) : mpd;
    D->mpt = mpt;
    D->kchunks = (D->max_obs + GL_KC - 1) / GL_KC;
    if (D->kchunks < 1) D->kchunks = 1;
    e = cudaMalloc((void **)&D->gpart, (size_t)D->kchunks * mpt * mpt * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(D->gpart, 0, (size_t)D->kchunks * mpt * mpt * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&D->cpart, (size_t)D->kchunks * mpt * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(D->cpart, 0, (size_t)D->kchunks * mpt * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&D->T, (size_t)c.m * c.m * sizeof(float));
    if (e == cudaSuccess && D->rpl == 0) {
      const long long n_pad = ((2LL * (long long)pts.size() + lk_ns_tile() - 1) / lk_ns_tile()) *
                              lk_ns_tile();
      e = cudaMalloc(&D->ns_ws, lk_ns_workspace_bytes(mpt, n_pad));
    } else if (e == cudaSuccess) {
      switch (D->rpl) {
        case 2: e = setup_global_rpl<2>(*D, c.m); break;
        case 4: e = setup_global_rpl<4>(*D, c.m); break;
        case 8: e = setup_global_rpl<8>(*D, c.m); break;
        case 13: e = setup_global_rpl<13>(*D, c.m); break;
        default: e = setup_global_rpl<16>(*D, c.m); break;
      }
    }
  } else if (e == cudaSuccess) {
    switch (D->rpl) {
      case 2: e = setup_rpl<2>(*D); break;
      case 4: e = setup_rpl<4>(*D); break;
      case 8: e = setup_rpl<8>(*D); break;
      case 13: e = setup_rpl<13>(*D); break;
      default: e = setup_rpl<16>(*D); break;
    }
  }
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return LETKF_ERR_CUDA;
  }
  return LETKF_OK;
}

// New sigma2 / taper half-support: the domain weights tau / sigma2 again.
letkf_status lk_domains_set_params(letkf_ctx *h, const letkf_config &c, const std::vector<int> &pid,
                                   const std::vector<int2> &pts, const std::vector<int2> &saps,
                                   std::string &err) {
  lk_domains_release(h);
  return lk_domains_build(h, c, pid, pts, saps, err);
}

void lk_domains_release(letkf_ctx *h) {
  LkDom *D = h->dom;
  if (!D) return;
  void *bufs[] = {D->node_off, D->node_ids, D->obs_off, D->obs_slot, D->obs_w, D->node_dom,
                  D->edges,    D->dedge_off, D->dedge,   D->KT,       D->delta, D->cpist,
                  D->gpart,    D->cpart,     D->T,       D->ns_ws};
  for (void *p : bufs)
    if (p) cudaFree(p);
  delete D;
  h->dom = nullptr;
}

int lk_domain_count(const letkf_ctx *h) { return h->dom ? h->dom->n_dom : 0; }

int lk_domain_of_nodes(const letkf_ctx *h, int *node_dom_host) {
  if (!h->dom) return 0;
  return cudaMemcpy(node_dom_host, h->dom->node_dom, h->inst[0].n_pts * sizeof(int),
                    cudaMemcpyDeviceToHost) == cudaSuccess;
}

int lk_domain_obs_counts(const letkf_ctx *h, int *obs_host) {
  if (!h->dom) return 0;
  std::vector<int> off(h->dom->n_dom + 1);
  if (cudaMemcpy(off.data(), h->dom->obs_off, off.size() * sizeof(int), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return 0;
  for (int d = 0; d < h->dom->n_dom; ++d) obs_host[d] = off[d + 1] - off[d];
  return 1;
}

// Analysis of every domain, then (with the piston correction) the piston
// constants and their application.
cudaError_t lk_launch_domains(letkf_ctx *h, void *mean, void *spread) {
  const LkDom &D = *h->dom;
  if (D.global && D.rpl == 0) {
    const int nt = D.mpt / GL_TILE;
    cudaError_t e = lk_launch_pdl(global_gram_kernel, dim3(nt * (nt + 1) / 2, D.kchunks), 256, 0,
                                  h->stream, h->d_inst, (const int *)D.obs_slot,
                                  (const float *)D.obs_w, D.max_obs, D.mpt, D.gpart, D.cpart);
    if (e != cudaSuccess) return e;
    return lk_launch_ns_global(h, D.gpart, D.cpart, D.kchunks, D.mpt, NS_ITERS, D.ns_ws, mean,
                               spread);
  }
  if (D.global) {
    switch (D.rpl) {
      case 2: return launch_global_rpl<2>(h, mean, spread);
      case 4: return launch_global_rpl<4>(h, mean, spread);
      case 8: return launch_global_rpl<8>(h, mean, spread);
      case 13: return launch_global_rpl<13>(h, mean, spread);
      default: return launch_global_rpl<16>(h, mean, spread);
    }
  }
  DomArgs a;
  a.node_off = D.node_off;
  a.node_ids = D.node_ids;
  a.obs_off = D.obs_off;
  a.obs_slot = D.obs_slot;
  a.obs_w = D.obs_w;
  a.mean = static_cast<float *>(mean);
  a.spread = static_cast<float *>(spread);
  a.delta = D.delta;
  a.counters = h->counters;
  a.tol = (float)h->tol32;
  a.stop = (float)(h->stop32 > h->tol32 ? h->stop32 : h->tol32);
  a.kappa_thr = h->fp64_kappa > 0 ? (float)h->fp64_kappa : 0.f;
  a.max_sweeps = h->max_sweeps;
  a.max_obs = D.max_obs;
  a.max_rows = 2 * D.max_nodes;
  cudaError_t e;
  switch (D.rpl) {
    case 2: e = launch_rpl<2>(h, a); break;
    case 4: e = launch_rpl<4>(h, a); break;
    case 8: e = launch_rpl<8>(h, a); break;
    case 13: e = launch_rpl<13>(h, a); break;
    default: e = launch_rpl<16>(h, a); break;
  }
  if (e != cudaSuccess || !D.piston || D.n_dom < 2) return e;
  e = lk_launch_pdl(piston_solve_kernel, 1, 1024, (size_t)2 * D.n_dom * sizeof(float), h->stream,
                    D.n_dom, (const int2 *)D.edges, (const int *)D.dedge_off,
                    (const int *)D.dedge, (const float *)D.delta, (const float *)D.KT, D.cpist);
  if (e != cudaSuccess) return e;
  const LkInst &I = h->inst[0];
  const unsigned blocks = (unsigned)(((long long)I.n_pts * 32 + LK_WARP_CTA - 1) / LK_WARP_CTA);
  return lk_launch_pdl(piston_apply_kernel, blocks, LK_WARP_CTA, 0, h->stream, h->d_inst,
                       (const int *)D.node_dom, (const float *)D.cpist, static_cast<float *>(mean));
}
