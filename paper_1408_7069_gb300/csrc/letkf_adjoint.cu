// Reverse mode of the closed loop: gradient of the mean residual variance over
// a window of frames (Section 2.1, Eq. Crit_Opt) with respect to the inflation
// rho, the slope noise variance sigma2 and the Gaspari-Cohn localization
// length L, through the analyses of Section 4.2 and the AR(1) forecasts of
// Section 3.1.2.
//
// Per node and frame (one warp, lane = member / eigen-column), with
// c_j = tau_j / sigma2, the analysis is recomputed from the stored background
// and differentiated:
//   Xa_r = xbar_r + X'_r (wbar 1^T + W)      -> xbar_r, X'_r, wbar, W
//   wbar = A^-1 b                             -> b_bar = A^-1 wbar_bar, A_bar -= b_bar wbar^T
//   W = sqrt(m-1) A^-1/2                      -> A_bar += sqrt(m-1) V (F o (V^T W_bar V)) V^T
//        with F_pq = -1 / (sqrt(l_p) sqrt(l_q) (sqrt(l_p) + sqrt(l_q))), the divided
//        difference of l^-1/2 written so that it is exact at l_p = l_q: degenerate
//        clusters (windows with fewer slopes than m - 1) need no gap test.
//        W_bar = sum_r X'_r^T G_r has rank 2, so V^T W_bar V = sum_r (V^T X'_r)(V^T G_r)^T.
//   A = (m-1)/rho I + sum_j c_j y_j y_j^T, b = sum_j c_j d_j y_j
//                                             -> y_j, d_j, c_j, rho
// The eigenbasis comes from the forward analysis of the same frame: FP32 nodes
// refine the stored basis with a B-only Jacobi (one sweep at most in practice);
// nodes whose kappa_hat bound sends them to FP64 in the forward analysis are
// queued and redone in FP64 with accumulated eigenvectors, starting from the
// FP32 basis U0 that the forward pair kernel stored for the node (FP64 handles
// start from the FP32-rounded FP64 basis their forward node kernel stored).
//
// Every node writes the adjoints of its window's slopes to its own slots; a
// subaperture kernel sums them over the nodes whose window holds the slope (in
// a fixed order), and a node kernel takes them back through the Fried operator,
// undoes the anomaly / mean split (Section 3.1), adds the criterion's gradient
// and applies the adjoint of the forecast. The result is bitwise reproducible.
//
// letkf_grad: forward over the frames storing the background and the analysis
// eigenbases of the last segment and a checkpoint (ensemble, warm-start bases,
// frame counters) at the start of every segment of ckpt_every frames; backward
// segment by segment, recomputing the segment's forward from its checkpoint.
#include <math.h>
#include <string.h>

#include <string>
#include <type_traits>
#include <vector>

#include "letkf_device.cuh"

struct LkAdjWork {
  int frames = 0, ckpt = 0, n_seg = 0;
  void *x_seg = nullptr;            // [ckpt][state] backgrounds of one segment
  void *basis_seg = nullptr;        // [ckpt][n_pts][mp][mp] analysis eigenbases of one segment
                                    // (FP32; FP64 on FP64 handles)
  void *ckpt_x = nullptr;           // [n_seg][state]
  float *ckpt_basis = nullptr;      // [n_seg][n_pts][mp][mp] warm-start bases at segment start
  long long *ckpt_frame = nullptr;  // [n_seg][2] frame counters at segment start
  void *fin_x = nullptr;            // state after the forward pass
  float *fin_basis = nullptr;
  long long *fin_frame = nullptr;
  double *resvar = nullptr;         // [frames]
  double *lam[2] = {nullptr, nullptr};  // [n_pts][2][m] adjoint of the analysis ensemble
  double *xp_bar = nullptr;         // [n_pts][2][m]
  double *xbar_bar = nullptr;       // [n_pts][2]
  double *ybw = nullptr;            // [n_pts][w*w][2][m] per-node window slope adjoints
  double *dbw = nullptr;            // [n_pts][w*w][2] per-node window innovation adjoints
  double *ybar = nullptr;           // [gs_rows*gs_cols][2][m] slope adjoints (padded grid)
  double *dbar = nullptr;           // [gs_rows*gs_cols][2]
  double *theta = nullptr;          // [n_pts][3] per-node (rho, sigma2, L) partials
  double *acc = nullptr;            // [5]: [0..2] accumulated gradient, [3] the frame's residual piston, [4] scratch
  double *dtap = nullptr;           // [w*w] d(tau/sigma2)/dL
  int2 *queue = nullptr;            // [n_pts] nodes redone in FP64
  int *queue_len = nullptr;
  cudaGraphExec_t graph = nullptr;
  const void *graph_y = nullptr, *graph_truth = nullptr;
};

// Phase clocks (a library built with -DLK_PHASE_CLOCKS only): lane 0 of every
// node adds the SM cycles of each phase of adjoint_node_kernel, [0..5] for the
// FP32 form and [6..11] for the FP64 one: window staging, Gram and the start
// of the eigensolve, Jacobi sweeps, adjoint of the transform up to A_bar,
// window slopes, nodes.
#ifdef LK_PHASE_CLOCKS
__device__ unsigned long long g_lk_adj_clocks[12];
#define LK_ADJ_STAMP(t) const long long t = clock64()
#else
#define LK_ADJ_STAMP(t)
#endif

namespace {

// One warp per CTA: the node kernels are bound by their SM's FP64 and dependency
// latency, so the nodes are spread over as many SMs as possible.
constexpr int ADJ_WARPS = 1;

// Per-warp vector slots in shared memory (MP elements each).
enum { S_LAM, S_B, S_XP0, S_XP1, S_G0, S_G1, S_Z, S_WB, S_GX0, S_GX1, S_H0, S_H1, S_WBB, S_Q, S_BB,
       S_N };

template <int MP, typename S, typename T>
__host__ __device__ size_t adj_warp_bytes(int w) {
  const size_t wc = (size_t)w * w;
  return align16(wc * 2 * MP * sizeof(S)) + align16(wc * 2 * sizeof(S)) +
         align16(wc * sizeof(T)) + align16(wc * sizeof(double)) +
         2 * align16((size_t)MP * (MP + 1) * sizeof(T)) + (size_t)S_N * MP * sizeof(T);
}

struct AdjArgs {
  const double *lam_a;   // adjoint of this frame's analysis ensemble
  double *xp_bar, *xbar_bar, *ybw, *dbw, *theta;
  const double *dtap;
  double rho, sigma2;
  int max_sweeps;
  int *counters;
};

// hi + lo += a * b with the product's and the sum's rounding errors kept in lo
// (FMA two-product and Knuth's two-sum): a compensated FP32 accumulation. The
// _rn intrinsics keep the compiler from contracting the steps into FMAs.
__device__ __forceinline__ void df_add_prod(float &hi, float &lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = fmaf(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(se, pe));
}

// Adjoint of one node's analysis. T = float: FP32 handle, warm start from the
// frame's stored eigenbasis U0 and B-only Jacobi, nodes above kappa_thr queued.
// T = double: accumulated eigenvectors, started from the FP32-rounded basis U0
// that the frame's forward analysis stored: the FP64 node kernel's for FP64
// handles, or, with `list` (the FP64 queue of an FP32 handle), the forward pair
// kernel's for the queued node.
template <int MP, typename S, typename T>
__global__ void __launch_bounds__(ADJ_WARPS * 32)
    adjoint_node_kernel(const LkInst *__restrict__ insts, const int2 *__restrict__ list,
                        const int *__restrict__ list_len, const float *__restrict__ U0,
                        const double *__restrict__ U64, float kappa_thr,
                        int2 *__restrict__ queue, int *__restrict__ queue_len, T tol, AdjArgs a) {
  constexpr bool kWarm = std::is_same<T, float>::value;
  LK_ADJ_STAMP(ph0);
  extern __shared__ __align__(16) unsigned char smem[];
  const LkInst &I = insts[0];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int pid = blockIdx.x * ADJ_WARPS + warp;
  if (list) {
    if (pid >= *list_len) return;
    pid = list[pid].y;
  } else if (pid >= I.n_pts) {
    return;
  }
  const int w = I.w, wc = w * w, m = I.m;
  const bool col = lane < MP, mem = lane < m;
  unsigned char *base = smem + (size_t)warp * adj_warp_bytes<MP, S, T>(w);
  S *win = reinterpret_cast<S *>(base);
  size_t off = align16((size_t)wc * 2 * MP * sizeof(S));
  S *dwin = reinterpret_cast<S *>(base + off);
  off += align16((size_t)wc * 2 * sizeof(S));
  T *tap = reinterpret_cast<T *>(base + off);
  off += align16((size_t)wc * sizeof(T));
  double *dtap = reinterpret_cast<double *>(base + off);
  off += align16((size_t)wc * sizeof(double));
  T *Vs = reinterpret_cast<T *>(base + off);   // Vs[i*(MP+1)+j] = V[i][j]
  off += align16((size_t)MP * (MP + 1) * sizeof(T));
  T *Ms = reinterpret_cast<T *>(base + off);
  off += align16((size_t)MP * (MP + 1) * sizeof(T));
  T *vec = reinterpret_cast<T *>(base + off);
  auto V = [&](int slot) { return vec + slot * MP; };

  // ---- the node's window ----
  const int2 ij = I.pts[pid];
  const S *Ybp = static_cast<const S *>(I.Ybp);
  const S *dp = static_cast<const S *>(I.dp);
  const S *taper = static_cast<const S *>(I.taper);
  // eight loads in flight per lane before their stores (the window's cells are
  // independent; one at a time, each waited out its L2 latency)
  for (int e0 = lane; e0 < wc * 2 * MP; e0 += 8 * 32) {
    S v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + 32 * u;
      v[u] = S(0);
      if (e < wc * 2 * MP) {
        const int cell = e / (2 * MP);
        const int r = e - cell * 2 * MP;
        const int c = r / MP;
        const int mm = r - c * MP;
        const int ds = cell / w, dt = cell - (cell / w) * w;
        const size_t src = (size_t)(ij.x + ds) * I.gs_cols + (ij.y + dt);
        if (mm < m) v[u] = Ybp[(src * 2 + c) * m + mm];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (e0 + 32 * u < wc * 2 * MP) win[e0 + 32 * u] = v[u];
  }
  for (int e = lane; e < wc * 2; e += 32) {
    const int cell = e >> 1;
    const int ds = cell / w, dt = cell - (cell / w) * w;
    const size_t src = (size_t)(ij.x + ds) * I.gs_cols + (ij.y + dt);
    dwin[e] = dp[src * 2 + (e & 1)];
  }
  for (int e = lane; e < wc; e += 32) {
    tap[e] = T(taper[e]);
    dtap[e] = a.dtap[e];
  }
  __syncwarp();
  LK_ADJ_STAMP(ph1);

  // ---- A, b and the eigendecomposition A = V diag(lam) V^T ----
#ifdef LK_PHASE_CLOCKS
  long long ph2 = 0;
#endif
  T b[MP], diag, cd;
  gram<MP, S, T>(win, dwin, w, tap, w, m, T(I.alpha), b, diag, cd);
  T v[MP];
  if constexpr (kWarm) {
    if (kappa_thr > 0.f) {
      const float trg = lk_warp_sum(diag);
      if (1.f + trg / float(I.alpha) > kappa_thr) {
        if (lane == 0) queue[atomicAdd(queue_len, 1)] = make_int2(0, pid);
        return;
      }
    }
    // B = A U0 (rows of A staged in Ms, lane = basis column)
    if (col) {
#pragma unroll
      for (int k = 0; k < MP; ++k) Ms[lane * (MP + 1) + k] = b[k];
    }
    const float *u0 = U0 + (size_t)pid * MP * MP;
#pragma unroll
    for (int k = 0; k < MP; ++k) v[k] = col ? u0[k * MP + lane] : 0.f;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < MP; ++i) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < MP; ++k) s = fma(Ms[i * (MP + 1) + k], v[k], s);
      b[i] = s;
    }
    __syncwarp();
    LK_ADJ_STAMP(ph2w);
    // U0 is this frame's converged basis, so the first sweep's rotations are at
    // rounding level: stop after the first sweep whose cosines all stay below
    // 1e-3 (one sweep, leaving pairs within about 1e-6) instead of running a
    // second sweep only to find no rotation
    jacobi<MP, T, false>(b, v, tol, a.max_sweeps, a.counters, T(1e-3));
#ifdef LK_PHASE_CLOCKS
    ph2 = ph2w;
#endif
  } else if (U64) {
    // FP64 handles: the forward analysis's FP64 eigenvectors V (orthonormal and
    // converged to FP64 rounding) are taken as they are, B = A V, lambda = |A v|
    if (col) {
#pragma unroll
      for (int k = 0; k < MP; ++k) Ms[lane * (MP + 1) + k] = b[k];
    }
    const double *u = U64 + (size_t)pid * MP * MP;
#pragma unroll
    for (int k = 0; k < MP; ++k) v[k] = col ? T(u[k * MP + lane]) : T(0);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < MP; ++i) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < MP; ++k) s = fma(Ms[i * (MP + 1) + k], v[k], s);
      b[i] = s;
    }
    __syncwarp();
#ifdef LK_PHASE_CLOCKS
    ph2 = clock64();
#endif
  } else {
    if (U0) {
      warm_basis<MP, T>(b, v, U0 + (size_t)pid * MP * MP, Ms, Vs);
    } else {
#pragma unroll
      for (int k = 0; k < MP; ++k) v[k] = (k == lane) ? T(1) : T(0);
    }
#ifdef LK_PHASE_CLOCKS
    ph2 = clock64();
#endif
    jacobi<MP, T, true>(b, v, tol, a.max_sweeps, a.counters, U0 ? T(LK_WARM_STOP64) : T(0));
  }
  LK_ADJ_STAMP(ph3);
  const T nrm = dot4<MP, T>(b, b);
  const T lam = (col && nrm > T(0)) ? sqrt(nrm) : T(1);   // |A v_j| = lambda_j
  if constexpr (kWarm) {
    const T inv = T(1) / lam;
#pragma unroll
    for (int k = 0; k < MP; ++k) v[k] = b[k] * inv;         // B = V diag(lam)
  }

  // ---- anomalies and the incoming adjoint ----
  const S *X = static_cast<const S *>(I.X) + (size_t)pid * 2 * m;
  const T x0 = mem ? T(X[lane]) : T(0);
  const T x1 = mem ? T(X[m + lane]) : T(0);
  const T xb0 = lk_warp_sum(x0) / T(m), xb1 = lk_warp_sum(x1) / T(m);
  const T g0 = mem ? T(a.lam_a[((size_t)pid * 2 + 0) * m + lane]) : T(0);
  const T g1 = mem ? T(a.lam_a[((size_t)pid * 2 + 1) * m + lane]) : T(0);
  const T s0 = lk_warp_sum(g0), s1 = lk_warp_sum(g1);
  if (col) {
#pragma unroll
    for (int k = 0; k < MP; ++k) Vs[k * (MP + 1) + lane] = v[k];
    V(S_LAM)[lane] = lam;
    V(S_B)[lane] = cd;
    V(S_XP0)[lane] = mem ? x0 - xb0 : T(0);
    V(S_XP1)[lane] = mem ? x1 - xb1 : T(0);
    V(S_G0)[lane] = g0;
    V(S_G1)[lane] = g1;
  }
  __syncwarp();
  // lane j: projections on eigenvector j
  if (col) {
    T u = 0, gx0 = 0, gx1 = 0, h0 = 0, h1 = 0;
#pragma unroll
    for (int k = 0; k < MP; ++k) {
      u = fma(v[k], V(S_B)[k], u);
      gx0 = fma(v[k], V(S_XP0)[k], gx0);
      gx1 = fma(v[k], V(S_XP1)[k], gx1);
      h0 = fma(v[k], V(S_G0)[k], h0);
      h1 = fma(v[k], V(S_G1)[k], h1);
    }
    V(S_Z)[lane] = u / lam;
    V(S_GX0)[lane] = gx0;
    V(S_GX1)[lane] = gx1;
    V(S_H0)[lane] = h0;
    V(S_H1)[lane] = h1;
  }
  __syncwarp();
  // lane i: wbar, the direct adjoints of X' and xbar, wbar_bar = X'^T (G 1)
  const T sq = sqrt(T(m - 1));
  if (col) {
    const T *vr = Vs + lane * (MP + 1);
    T wb = 0, wg0 = 0, wg1 = 0;
#pragma unroll
    for (int j = 0; j < MP; ++j) {
      const T rs = T(1) / sqrt(V(S_LAM)[j]);
      wb = fma(vr[j], V(S_Z)[j], wb);
      wg0 = fma(vr[j], rs * V(S_H0)[j], wg0);
      wg1 = fma(vr[j], rs * V(S_H1)[j], wg1);
    }
    V(S_WB)[lane] = wb;
    V(S_WBB)[lane] = s0 * V(S_XP0)[lane] + s1 * V(S_XP1)[lane];
    if (mem) {
      a.xp_bar[((size_t)pid * 2 + 0) * m + lane] = double(s0 * wb + sq * wg0);
      a.xp_bar[((size_t)pid * 2 + 1) * m + lane] = double(s1 * wb + sq * wg1);
    }
  }
  if (lane == 0) {
    a.xbar_bar[(size_t)pid * 2 + 0] = double(s0);
    a.xbar_bar[(size_t)pid * 2 + 1] = double(s1);
  }
  __syncwarp();
  // b_bar = V diag(1/lam) V^T wbar_bar
  if (col) {
    T q = 0;
#pragma unroll
    for (int k = 0; k < MP; ++k) q = fma(v[k], V(S_WBB)[k], q);
    V(S_Q)[lane] = q / lam;
  }
  __syncwarp();
  if (col) {
    const T *vr = Vs + lane * (MP + 1);
    T bb = 0;
#pragma unroll
    for (int p = 0; p < MP; ++p) bb = fma(vr[p], V(S_Q)[p], bb);
    V(S_BB)[lane] = bb;
  }
  __syncwarp();
  // T1 = V (F o M), M = sum_r (V^T X'_r)(V^T G_r)^T; lane q forms column q
  if (col) {
    const T rq = sqrt(lam);
    const T hq0 = V(S_H0)[lane], hq1 = V(S_H1)[lane];
    T mcol[MP];
#pragma unroll
    for (int p = 0; p < MP; ++p) {
      const T rp = sqrt(V(S_LAM)[p]);
      const T F = T(-1) / (rp * rq * (rp + rq));
      mcol[p] = F * (V(S_GX0)[p] * hq0 + V(S_GX1)[p] * hq1);
    }
    for (int i = 0; i < MP; ++i) {
      const T *vr = Vs + i * (MP + 1);
      T t = 0;
#pragma unroll
      for (int p = 0; p < MP; ++p) t = fma(vr[p], mcol[p], t);
      Ms[i * (MP + 1) + lane] = t;
    }
  }
  __syncwarp();
  // A_bar = sqrt(m-1) T1 V^T - b_bar wbar^T, then its symmetric part; lane l holds column l
  T as[MP];
  if (col) {
    const T *vl = Vs + lane * (MP + 1);
    const T wl = V(S_WB)[lane];
#pragma unroll
    for (int i = 0; i < MP; ++i) {
      const T *ti = Ms + i * (MP + 1);
      T t = 0;
#pragma unroll
      for (int q = 0; q < MP; ++q) t = fma(ti[q], vl[q], t);
      as[i] = sq * t - V(S_BB)[i] * wl;
    }
  } else {
#pragma unroll
    for (int i = 0; i < MP; ++i) as[i] = T(0);
  }
  __syncwarp();
  if (col) {
#pragma unroll
    for (int i = 0; i < MP; ++i) Ms[i * (MP + 1) + lane] = as[i];
  }
  __syncwarp();
  T dg = 0;
  if (col) {
#pragma unroll
    for (int i = 0; i < MP; ++i) {
      as[i] = T(0.5) * (as[i] + Ms[lane * (MP + 1) + i]);
      if (i == lane) dg = as[i];
    }
  }
  const double alpha_bar = double(lk_warp_sum(dg));   // d/d((m-1)/rho) = tr(A_bar)
  LK_ADJ_STAMP(ph4);

  // ---- window slopes: y_bar_j = 2 c_j A_bar y_j + c_j d_j b_bar, d_bar_j, c_bar_j ----
  // sum_j c_bar_j c_j and sum_j c_bar_j dc_j/dL, whose terms cancel strongly
  // over the window: in FP64 for FP64 handles; for FP32 handles as compensated
  // FP32 sums (the products' and the additions' rounding errors carried in a
  // second float, about FP64 accuracy without the FP64 pipe); dc_j/dsigma2 =
  // -c_j / sigma2 is applied once per node
  const T bbl = col ? V(S_BB)[lane] : T(0);
  double gs2 = 0, gL = 0;
  float gs2h = 0.f, gs2l = 0.f, gLh = 0.f, gLl = 0.f;
  double *yb_out = a.ybw + (size_t)pid * wc * 2 * m;
  double *db_out = a.dbw + (size_t)pid * wc * 2;
  for (int cell = 0; cell < wc; ++cell) {
    const T cj = tap[cell];
    if (cj == T(0) && dtap[cell] == 0.0) {
      // outside the taper's support for every nearby L: no slope of the cell
      // reaches A, C d or J
      if (mem)
        for (int c = 0; c < 2; ++c) yb_out[((size_t)cell * 2 + c) * m + lane] = 0.0;
      if (lane == 0) db_out[cell * 2] = db_out[cell * 2 + 1] = 0.0;
      continue;
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const S *yv = win + (size_t)cell * 2 * MP + c * MP;
      const T yl = col ? T(yv[lane]) : T(0);
      // (A_bar y_j)_lane as four interleaved chains: a quarter of the latency
      T a4[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int i = 0; i < MP; ++i) a4[i & 3] = fma(as[i], T(yv[i]), a4[i & 3]);
      const T ay = (a4[0] + a4[1]) + (a4[2] + a4[3]);
      const T dj = T(dwin[cell * 2 + c]);
      const T yb = lk_warp_sum(yl * bbl);
      const T yay = lk_warp_sum(yl * ay);
      if (mem) yb_out[((size_t)cell * 2 + c) * m + lane] = double(T(2) * cj * ay + cj * dj * bbl);
      if (lane == 0) db_out[cell * 2 + c] = double(cj * yb);
      if constexpr (std::is_same<T, float>::value) {
        const float cb = fmaf(dj, yb, yay);
        df_add_prod(gs2h, gs2l, cb, cj);
        df_add_prod(gLh, gLl, cb, (float)dtap[cell]);
      } else {
        const double cbar = double(fma(dj, yb, yay));
        gs2 = fma(cbar, double(cj), gs2);
        gL = fma(cbar, dtap[cell], gL);
      }
    }
  }
  if constexpr (std::is_same<T, float>::value) {
    gs2 = (double)gs2h + (double)gs2l;
    gL = (double)gLh + (double)gLl;
  }
  if (lane == 0) {
    a.theta[(size_t)pid * 3 + 0] = alpha_bar * (-(m - 1) / (a.rho * a.rho));
    a.theta[(size_t)pid * 3 + 1] = -gs2 / a.sigma2;
    a.theta[(size_t)pid * 3 + 2] = gL;
  }
#ifdef LK_PHASE_CLOCKS
  __syncwarp();
  LK_ADJ_STAMP(ph5);
  if (lane == 0) {
    unsigned long long *pc = g_lk_adj_clocks + (kWarm ? 0 : 6);
    atomicAdd(&pc[0], (unsigned long long)(ph1 - ph0));
    atomicAdd(&pc[1], (unsigned long long)(ph2 - ph1));
    atomicAdd(&pc[2], (unsigned long long)(ph3 - ph2));
    atomicAdd(&pc[3], (unsigned long long)(ph4 - ph3));
    atomicAdd(&pc[4], (unsigned long long)(ph5 - ph4));
    atomicAdd(&pc[5], 1ull);
  }
#endif
}

// Warp per valid subaperture (s, t): sums the slope adjoints the nodes whose
// window holds (s, t) wrote, in a fixed order (node row, then column), into the
// padded grid. The candidate nodes are looked up 32 at a time, one per lane,
// so that the loads of their adjoints do not wait on one another.
__global__ void __launch_bounds__(LK_WARP_CTA)
    adjoint_subap_kernel(const LkInst *__restrict__ insts, const double *__restrict__ ybw,
                         const double *__restrict__ dbw, double *__restrict__ ybar,
                         double *__restrict__ dbar) {
  const LkInst &I = insts[0];
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= I.n_sap) return;
  const int2 st = I.saps[q];
  const int w = I.w, wc = w * w, m = I.m, nn = I.nsub + 1;
  const bool mem = lane < m;
  const int i0 = st.x + I.h - w + 1, j0 = st.y + I.h - w + 1;
  double y0 = 0, y1 = 0, d0 = 0, d1 = 0;
  for (int c0 = 0; c0 < wc; c0 += 32) {
    // lane: candidate node c0 + lane of the w x w block of nodes, row-major
    long long cell = -1;
    const int c = c0 + lane;
    if (c < wc) {
      const int i = i0 + c / w, j = j0 + c % w;
      if (i >= 0 && i < nn && j >= 0 && j < nn) {
        const int pid = I.pid_map[i * nn + j];
        if (pid >= 0) cell = (long long)pid * wc + (long long)(st.x - i + I.h) * w + (st.y - j + I.h);
      }
    }
    const int nc = wc - c0 < 32 ? wc - c0 : 32;
    // eight candidates at a time: their loads first (all in flight together),
    // then the sums in candidate order
    for (int u0 = 0; u0 < nc; u0 += 8) {
      double a0[8], a1[8], e0[8], e1[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const long long cu = __shfl_sync(FULL, cell, (u0 + u) & 31);
        const bool ok = u0 + u < nc && cu >= 0;
        a0[u] = ok && mem ? ybw[(cu * 2 + 0) * m + lane] : 0.0;
        a1[u] = ok && mem ? ybw[(cu * 2 + 1) * m + lane] : 0.0;
        e0[u] = ok ? dbw[cu * 2 + 0] : 0.0;
        e1[u] = ok ? dbw[cu * 2 + 1] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (u0 + u >= nc) break;
        y0 += a0[u];
        y1 += a1[u];
        d0 += e0[u];
        d1 += e1[u];
      }
    }
  }
  const size_t g = (size_t)(st.x + I.h) * I.gs_cols + (st.y + I.h);
  if (mem) {
    ybar[(g * 2 + 0) * m + lane] = y0;
    ybar[(g * 2 + 1) * m + lane] = y1;
  }
  if (lane == 0) {
    dbar[g * 2 + 0] = d0;
    dbar[g * 2 + 1] = d1;
  }
}

// Warp per node, lane = member: slope adjoints back to the phi_{k-1} row through
// the Fried operator (Yb = D1 X'_1, ybar = D1 xbar_1), the anomaly / mean split,
// the criterion's gradient, then the adjoint of the forecast
// x_{k+1} = A1 x_{k/k} + v (row 0 <- a row 0 + row 1, row 1 <- 0).
template <typename S>
__global__ void __launch_bounds__(LK_WARP_CTA)
    adjoint_gather_kernel(const LkInst *__restrict__ insts, const double *__restrict__ xp_bar,
                          const double *__restrict__ xbar_bar, const double *__restrict__ ybar,
                          const double *__restrict__ dbar, const S *__restrict__ truth,
                          const double *__restrict__ ebar, double crit_scale,
                          double *__restrict__ lam_out) {
  const LkInst &I = insts[0];
  const int pid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (pid >= I.n_pts) return;
  const int m = I.m;
  const int2 ij = I.pts[pid];
  const bool mem = lane < m;
  double r0 = mem ? xp_bar[((size_t)pid * 2 + 0) * m + lane] : 0.0;
  double r1 = mem ? xp_bar[((size_t)pid * 2 + 1) * m + lane] : 0.0;
  const double xb0 = xbar_bar[(size_t)pid * 2 + 0];
  double xb1 = xbar_bar[(size_t)pid * 2 + 1];
  for (int a = 0; a < 2; ++a)
    for (int bq = 0; bq < 2; ++bq) {
      const int s = ij.x - 1 + a, t = ij.y - 1 + bq;
      if (s < 0 || t < 0 || s >= I.nsub || t >= I.nsub) continue;
      const double cx = (ij.x == s + 1) ? 0.5 : -0.5;   // d sx(s,t) / d phi(i,j)
      const double cy = (ij.y == t + 1) ? 0.5 : -0.5;   // d sy(s,t) / d phi(i,j)
      const size_t cell = (size_t)(s + I.h) * I.gs_cols + (t + I.h);
      if (mem) r1 += cx * ybar[(cell * 2 + 0) * m + lane] + cy * ybar[(cell * 2 + 1) * m + lane];
      xb1 -= cx * dbar[cell * 2 + 0] + cy * dbar[cell * 2 + 1];
    }
  const double m0 = lk_warp_sum(r0) / m, m1 = lk_warp_sum(r1) / m;
  double l0 = mem ? r0 - m0 + xb0 / m : 0.0;
  const double l1 = mem ? r1 - m1 + xb1 / m : 0.0;
  // d/dX[g,0,i] of the piston-removed spatial variance of truth - mean(row 0)
  const S *X = static_cast<const S *>(I.X) + (size_t)pid * 2 * m;
  const double mu = lk_warp_sum(mem ? double(X[lane]) : 0.0) / m;
  const double e = double(truth[pid]) - mu - ebar[0];
  l0 += crit_scale * e;
  if (mem) {
    lam_out[((size_t)pid * 2 + 0) * m + lane] = I.a_ar1 * l0 + l1;
    lam_out[((size_t)pid * 2 + 1) * m + lane] = 0.0;
  }
}

// acc[c] += sum over nodes of part[n][c] (c < 3), in a fixed order.
__global__ void __launch_bounds__(256) theta_reduce_kernel(const double *__restrict__ part, int n,
                                                            double *__restrict__ acc) {
  __shared__ double sh[3][8];
  double s[3] = {0, 0, 0};
  for (int g = threadIdx.x; g < n; g += blockDim.x)
    for (int c = 0; c < 3; ++c) s[c] += part[(size_t)g * 3 + c];
  for (int c = 0; c < 3; ++c) {
    s[c] = lk_warp_sum(s[c]);
    if ((threadIdx.x & 31) == 0) sh[c][threadIdx.x >> 5] = s[c];
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) {
      double t = 0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[c][k];
      acc[c] += t;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

letkf_status gfail(letkf_ctx *h, letkf_status st, const std::string &msg) {
  h->err = msg;
  return st;
}

#define LK_ACUDA(h, call)                                                                     \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return gfail((h), LETKF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// d/dz of the Gaspari & Cohn (1999) function of z = r / c (their Eq. 4.10),
// differentiated term by term.
double gaspari_cohn_dz(double z) {
  if (z <= 1.0) return (((-1.25 * z + 2.0) * z + 1.875) * z - 10.0 / 3.0) * z;
  if (z < 2.0)
    return (((5.0 / 12.0 * z - 2.0) * z + 1.875) * z + 10.0 / 3.0) * z - 5.0 + (2.0 / 3.0) / (z * z);
  return 0.0;
}

template <int MP, typename S, typename T>
size_t node_smem(const LkInst &I) {
  return (size_t)ADJ_WARPS * adj_warp_bytes<MP, S, T>(I.w);
}

template <int MP, typename S, typename T>
cudaError_t set_node_smem(const LkInst &I) {
  return cudaFuncSetAttribute(adjoint_node_kernel<MP, S, T>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)node_smem<MP, S, T>(I));
}

cudaError_t setup_kernels(letkf_ctx *h) {
  const LkInst &I = h->inst[0];
  if (h->precision == 1)
    return I.mp == 16 ? set_node_smem<16, double, double>(I) : set_node_smem<32, double, double>(I);
  cudaError_t e = I.mp == 16 ? set_node_smem<16, float, float>(I) : set_node_smem<32, float, float>(I);
  if (e == cudaSuccess)
    e = I.mp == 16 ? set_node_smem<16, float, double>(I) : set_node_smem<32, float, double>(I);
  return e;
}

size_t max_node_smem(const letkf_ctx *h) {
  const LkInst &I = h->inst[0];
  size_t b = 0;
  auto upd = [&](size_t x) { b = x > b ? x : b; };
  if (h->precision == 1) {
    upd(I.mp == 16 ? node_smem<16, double, double>(I) : node_smem<32, double, double>(I));
  } else {
    upd(I.mp == 16 ? node_smem<16, float, float>(I) : node_smem<32, float, float>(I));
    upd(I.mp == 16 ? node_smem<16, float, double>(I) : node_smem<32, float, double>(I));
  }
  return b;
}

template <int MP>
cudaError_t launch_nodes(letkf_ctx *h, LkAdjWork *W, const void *bk, const AdjArgs &a) {
  const LkInst &I = h->inst[0];
  const int blocks = (I.n_pts + ADJ_WARPS - 1) / ADJ_WARPS;
  if (h->precision == 1) {
    // FP64 handles: the FP64 eigenbasis the forward node64 kernel stored
    adjoint_node_kernel<MP, double, double>
        <<<blocks, ADJ_WARPS * 32, node_smem<MP, double, double>(I), h->stream>>>(
            h->d_inst, nullptr, nullptr, nullptr, static_cast<const double *>(bk), 0.f, nullptr,
            nullptr, h->tol64, a);
    return cudaGetLastError();
  }
  const float *U0 = static_cast<const float *>(bk);
  const float kthr = h->fp64_kappa > 0 ? (float)h->fp64_kappa : 0.f;
  adjoint_node_kernel<MP, float, float>
      <<<blocks, ADJ_WARPS * 32, node_smem<MP, float, float>(I), h->stream>>>(
          h->d_inst, nullptr, nullptr, U0, nullptr, kthr, W->queue, W->queue_len,
          (float)h->tol32, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || kthr <= 0.f) return e;
  adjoint_node_kernel<MP, float, double>
      <<<blocks, ADJ_WARPS * 32, node_smem<MP, float, double>(I), h->stream>>>(
          h->d_inst, W->queue, W->queue_len, U0, nullptr, 0.f, nullptr, nullptr, h->tol64, a);
  return cudaGetLastError();
}

void free_work(LkAdjWork *W) {
  if (!W) return;
  if (W->graph) cudaGraphExecDestroy(W->graph);
  void *bufs[] = {W->x_seg,    W->basis_seg, W->ckpt_x,   W->ckpt_basis, W->ckpt_frame, W->fin_x,
                  W->fin_basis, W->fin_frame, W->resvar,   W->lam[0],     W->lam[1],     W->xp_bar,
                  W->xbar_bar,  W->ybw,       W->dbw,      W->ybar,       W->dbar,       W->theta,
                  W->acc,       W->dtap,      W->queue,    W->queue_len};
  for (void *p : bufs)
    if (p) cudaFree(p);
  delete W;
}

template <typename P>
cudaError_t walloc(P **p, size_t bytes) {
  return cudaMalloc((void **)p, bytes ? bytes : 16);
}

// (Re)allocates the workspace for `frames` frames in segments of `ckpt`.
letkf_status ensure_work(letkf_ctx *h, int frames, int ckpt) {
  LkAdjWork *W = h->adj;
  if (W && W->frames == frames && W->ckpt == ckpt) return LETKF_OK;
  free_work(W);
  h->adj = W = new LkAdjWork();
  W->frames = frames;
  W->ckpt = ckpt;
  W->n_seg = (frames + ckpt - 1) / ckpt;
  const LkInst &I = h->inst[0];
  const size_t st = (size_t)h->state_total * h->rsz;
  const size_t bas = (size_t)I.n_pts * I.mp * I.mp * sizeof(float);
  const size_t bas_seg = (size_t)I.n_pts * I.mp * I.mp * (h->precision == 1 ? 8 : 4);
  const size_t ns = (size_t)I.n_pts * 2 * I.m * sizeof(double);
  const size_t wc = (size_t)I.w * I.w;
  const size_t cells = (size_t)I.gs_rows * I.gs_cols;
  cudaError_t e = walloc(&W->x_seg, (size_t)ckpt * st);
  if (e == cudaSuccess) e = walloc(&W->basis_seg, (size_t)ckpt * bas_seg);
  if (e == cudaSuccess) e = walloc(&W->ckpt_x, (size_t)W->n_seg * st);
  if (e == cudaSuccess) e = walloc(&W->ckpt_basis, (size_t)W->n_seg * bas);
  if (e == cudaSuccess) e = walloc(&W->ckpt_frame, (size_t)W->n_seg * 2 * sizeof(long long));
  if (e == cudaSuccess) e = walloc(&W->fin_x, st);
  if (e == cudaSuccess) e = walloc(&W->fin_basis, bas);
  if (e == cudaSuccess) e = walloc(&W->fin_frame, 2 * sizeof(long long));
  if (e == cudaSuccess) e = walloc(&W->resvar, (size_t)frames * sizeof(double));
  if (e == cudaSuccess) e = walloc(&W->lam[0], ns);
  if (e == cudaSuccess) e = walloc(&W->lam[1], ns);
  if (e == cudaSuccess) e = walloc(&W->xp_bar, ns);
  if (e == cudaSuccess) e = walloc(&W->xbar_bar, (size_t)I.n_pts * 2 * sizeof(double));
  if (e == cudaSuccess) e = walloc(&W->ybw, (size_t)I.n_pts * wc * 2 * I.m * sizeof(double));
  if (e == cudaSuccess) e = walloc(&W->dbw, (size_t)I.n_pts * wc * 2 * sizeof(double));
  if (e == cudaSuccess) e = walloc(&W->ybar, cells * 2 * I.m * sizeof(double));
  if (e == cudaSuccess) e = walloc(&W->dbar, cells * 2 * sizeof(double));
  if (e == cudaSuccess) e = walloc(&W->theta, (size_t)I.n_pts * 3 * sizeof(double));
  if (e == cudaSuccess) e = walloc(&W->acc, 5 * sizeof(double));
  if (e == cudaSuccess) e = walloc(&W->dtap, wc * sizeof(double));
  if (e == cudaSuccess) e = walloc(&W->queue, (size_t)I.n_pts * sizeof(int2));
  if (e == cudaSuccess) e = walloc(&W->queue_len, sizeof(int));
  // slope adjoints of subapertures outside the pupil stay zero
  if (e == cudaSuccess) e = cudaMemset(W->ybar, 0, cells * 2 * I.m * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(W->dbar, 0, cells * 2 * sizeof(double));
  if (e != cudaSuccess) {
    free_work(W);
    h->adj = nullptr;
    return gfail(h, LETKF_ERR_NOMEM, std::string("adjoint workspace: ") + cudaGetErrorString(e));
  }
  return LETKF_OK;
}

// Copies between the handle's state (ensemble, warm-start bases, frame
// counters) and a saved copy.
cudaError_t save_state(letkf_ctx *h, void *x, float *basis, long long *frame) {
  const LkInst &I = h->inst[0];
  cudaError_t e = cudaMemcpyAsync(x, h->X, h->state_total * h->rsz, cudaMemcpyDeviceToDevice,
                                  h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(basis, h->basis, (size_t)I.n_pts * I.mp * I.mp * sizeof(float),
                        cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(frame, h->frame, 2 * sizeof(long long), cudaMemcpyDeviceToDevice,
                        h->stream);
  return e;
}

cudaError_t load_state(letkf_ctx *h, const void *x, const float *basis, const long long *frame) {
  const LkInst &I = h->inst[0];
  cudaError_t e = cudaMemcpyAsync(h->X, x, h->state_total * h->rsz, cudaMemcpyDeviceToDevice,
                                  h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->basis, basis, (size_t)I.n_pts * I.mp * I.mp * sizeof(float),
                        cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->frame, frame, 2 * sizeof(long long), cudaMemcpyDeviceToDevice,
                        h->stream);
  return e;
}

// One forward frame (prediction in h->X): optional residual, analysis (its
// background kept in xk, its eigenbases in bk: FP64 on FP64 handles),
// forecast with the bank noise.
cudaError_t forward_frame(letkf_ctx *h, const void *y_seq, const void *truth_seq, double *resvar,
                          void *xk, void *bk, bool forecast) {
  const LkInst &I = h->inst[0];
  const long long *ridx = h->frame + 1;
  cudaError_t e = cudaSuccess;
  if (resvar) e = lk_launch_residual(h, truth_seq, resvar, ridx);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(xk, h->X, h->state_total * h->rsz, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess) e = lk_launch_obs(h, y_seq, ridx);
  if (e == cudaSuccess) e = lk_launch_analysis(h, nullptr, nullptr);
  const size_t nb = (size_t)I.n_pts * I.mp * I.mp;
  if (e == cudaSuccess)
    e = h->basis64 ? cudaMemcpyAsync(bk, h->basis64, nb * sizeof(double), cudaMemcpyDeviceToDevice,
                                     h->stream)
                   : cudaMemcpyAsync(bk, h->basis, nb * sizeof(float), cudaMemcpyDeviceToDevice,
                                     h->stream);
  if (e == cudaSuccess && forecast) e = lk_launch_forecast(h, nullptr);
  return e;
}

// One backward frame: background xk, analysis eigenbases bk, adjoint of the
// analysis lam_in -> adjoint of the previous analysis lam_out.
cudaError_t backward_frame(letkf_ctx *h, LkAdjWork *W, const void *y_k, const void *truth_k,
                           const void *xk, const void *bk, const double *lam_in, double *lam_out,
                           double crit_scale) {
  const LkInst &I = h->inst[0];
  cudaError_t e = cudaMemcpyAsync(h->X, xk, h->state_total * h->rsz, cudaMemcpyDeviceToDevice,
                                  h->stream);
  if (e == cudaSuccess) e = lk_launch_obs(h, y_k, nullptr);
  if (e == cudaSuccess) e = cudaMemsetAsync(W->queue_len, 0, sizeof(int), h->stream);
  if (e != cudaSuccess) return e;
  AdjArgs a;
  a.lam_a = lam_in;
  a.xp_bar = W->xp_bar;
  a.xbar_bar = W->xbar_bar;
  a.ybw = W->ybw;
  a.dbw = W->dbw;
  a.theta = W->theta;
  a.dtap = W->dtap;
  a.rho = h->cfg.rho;
  a.sigma2 = h->cfg.sigma2;
  a.max_sweeps = h->max_sweeps;
  a.counters = h->counters;
  e = I.mp == 16 ? launch_nodes<16>(h, W, bk, a) : launch_nodes<32>(h, W, bk, a);
  if (e != cudaSuccess) return e;
  theta_reduce_kernel<<<1, 256, 0, h->stream>>>(W->theta, I.n_pts, W->acc);
  adjoint_subap_kernel<<<(I.n_sap * 32 + LK_WARP_CTA - 1) / LK_WARP_CTA, LK_WARP_CTA, 0,
                         h->stream>>>(h->d_inst, W->ybw, W->dbw, W->ybar, W->dbar);
  const int blocks = (int)(((long long)I.n_pts * 32 + LK_WARP_CTA - 1) / LK_WARP_CTA);
  // the piston of the frame's residual (acc[3]; its variance goes to acc[4])
  e = lk_launch_residual(h, truth_k, W->acc + 4, nullptr, W->acc + 3);
  if (e != cudaSuccess) return e;
  if (h->precision == 1) {
    adjoint_gather_kernel<double><<<blocks, LK_WARP_CTA, 0, h->stream>>>(
        h->d_inst, W->xp_bar, W->xbar_bar, W->ybar, W->dbar, (const double *)truth_k, W->acc + 3,
        crit_scale, lam_out);
  } else {
    adjoint_gather_kernel<float><<<blocks, LK_WARP_CTA, 0, h->stream>>>(
        h->d_inst, W->xp_bar, W->xbar_bar, W->ybar, W->dbar, (const float *)truth_k, W->acc + 3,
        crit_scale, lam_out);
  }
  return cudaGetLastError();
}

// The whole gradient computation, enqueued on h->stream.
letkf_status enqueue_grad(letkf_ctx *h, int frames, const void *y_seq, const void *truth_seq) {
  LkAdjWork *W = h->adj;
  const LkInst &I = h->inst[0];
  const int C = W->ckpt;
  const size_t st = (size_t)h->state_total * h->rsz;
  const size_t bas = (size_t)I.n_pts * I.mp * I.mp;   // floats
  const size_t bseg = bas * (h->precision == 1 ? 8 : 4);  // bytes per frame in basis_seg
  char *bs = static_cast<char *>(W->basis_seg);
  const char *ys = static_cast<const char *>(y_seq);
  const char *ts = static_cast<const char *>(truth_seq);
  char *xs = static_cast<char *>(W->x_seg);
  const double crit_scale = -2.0 / ((double)I.n_pts * I.m * frames);
  LK_ACUDA(h, cudaMemsetAsync(h->frame + 1, 0, sizeof(long long), h->stream));
  // ---- forward ----
  for (int k = 0; k < frames; ++k) {
    const int seg = k / C, slot = k % C;
    if (slot == 0)
      LK_ACUDA(h, save_state(h, static_cast<char *>(W->ckpt_x) + (size_t)seg * st,
                             W->ckpt_basis + (size_t)seg * bas, W->ckpt_frame + 2 * seg));
    LK_ACUDA(h, forward_frame(h, y_seq, truth_seq, W->resvar, xs + (size_t)slot * st,
                              bs + (size_t)slot * bseg, true));
  }
  LK_ACUDA(h, save_state(h, W->fin_x, W->fin_basis, W->fin_frame));
  // ---- backward ----
  LK_ACUDA(h, cudaMemsetAsync(W->lam[0], 0, (size_t)I.n_pts * 2 * I.m * sizeof(double),
                              h->stream));
  LK_ACUDA(h, cudaMemsetAsync(W->acc, 0, 5 * sizeof(double), h->stream));
  int cur = 0;
  for (int seg = W->n_seg - 1; seg >= 0; --seg) {
    const int s = seg * C, e = (s + C < frames) ? s + C : frames;
    if (seg != W->n_seg - 1) {   // the last segment is still in the segment buffers
      LK_ACUDA(h, load_state(h, static_cast<char *>(W->ckpt_x) + (size_t)seg * st,
                             W->ckpt_basis + (size_t)seg * bas, W->ckpt_frame + 2 * seg));
      for (int k = s; k < e; ++k)
        LK_ACUDA(h, forward_frame(h, y_seq, nullptr, nullptr, xs + (size_t)(k - s) * st,
                                  bs + (size_t)(k - s) * bseg, k + 1 < e));
    }
    for (int k = e - 1; k >= s; --k) {
      LK_ACUDA(h, backward_frame(h, W, ys + (size_t)k * h->p_total * h->rsz,
                                 ts + (size_t)k * h->n_pts_total * h->rsz,
                                 xs + (size_t)(k - s) * st, bs + (size_t)(k - s) * bseg,
                                 W->lam[cur], W->lam[cur ^ 1], crit_scale));
      cur ^= 1;
    }
  }
  LK_ACUDA(h, load_state(h, W->fin_x, W->fin_basis, W->fin_frame));
  return LETKF_OK;
}

}  // namespace

void lk_adjoint_release(letkf_ctx *h) {
  free_work(h->adj);
  h->adj = nullptr;
}

extern "C" letkf_status letkf_grad(letkf_t h, int32_t frames, const void *y_seq_dev,
                                   const void *truth_seq_dev, int32_t ckpt_every, double *J_out,
                                   double *grad_out) {
  if (!h) return LETKF_ERR_ARG;
  if (frames < 1) return gfail(h, LETKF_ERR_ARG, "frames must be >= 1");
  if (!y_seq_dev || !truth_seq_dev)
    return gfail(h, LETKF_ERR_ARG, "y_seq_dev and truth_seq_dev are required");
  if (h->n_inst != 1) return gfail(h, LETKF_ERR_ARG, "letkf_grad takes a single-instance handle");
  if (h->dom) return gfail(h, LETKF_ERR_STATE, "letkf_grad has no local-domain form");
  if (h->inst[0].dm)
    return gfail(h, LETKF_ERR_STATE, "letkf_grad differentiates the pseudo-open-loop form only");
  const LkInst &I = h->inst[0];
  if (I.mp > 32) return gfail(h, LETKF_ERR_ARG, "letkf_grad supports m <= 32");
  if (!I.bank) return gfail(h, LETKF_ERR_STATE, "letkf_grad needs the instance's noise bank");
  int dev_prev = -1;
  if (cudaGetDevice(&dev_prev) == cudaSuccess && dev_prev != h->device) cudaSetDevice(h->device);
  struct Restore {
    int d;
    ~Restore() {
      if (d >= 0) cudaSetDevice(d);
    }
  } restore{dev_prev != h->device ? dev_prev : -1};

  int dev_smem = 0;
  LK_ACUDA(h, cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                     h->device));
  if (max_node_smem(h) > (size_t)dev_smem)
    return gfail(h, LETKF_ERR_ARG, "localization window too wide for the adjoint kernels");
  const int C = (ckpt_every <= 0 || ckpt_every > frames) ? frames : ckpt_every;
  LK_ACUDA(h, cudaStreamSynchronize(h->stream));
  letkf_status st = ensure_work(h, frames, C);
  if (st != LETKF_OK) return st;
  LkAdjWork *W = h->adj;
  // d(tau/sigma2)/dL of every window offset (zero without the taper)
  {
    const int w = I.w, hw = w / 2;
    const double L = h->cfg.loc_len > 0 ? h->cfg.loc_len : w / 4.0;
    std::vector<double> dt((size_t)w * w, 0.0);
    if (h->cfg.taper == 1)
      for (int ds = 0; ds < w; ++ds)
        for (int dd = 0; dd < w; ++dd) {
          const double z = hypot(ds - hw + 0.5, dd - hw + 0.5) / L;
          dt[(size_t)ds * w + dd] = gaspari_cohn_dz(z) * (-z / L) / h->cfg.sigma2;
        }
    LK_ACUDA(h, cudaMemcpy(W->dtap, dt.data(), dt.size() * sizeof(double),
                           cudaMemcpyHostToDevice));
  }
  LK_ACUDA(h, setup_kernels(h));
  // the forward analyses keep every node's eigenbasis for the backward pass
  struct KeepBasis {
    letkf_ctx *h;
    ~KeepBasis() { h->keep_basis = 0; }
  } keep{h};
  h->keep_basis = 1;
  if (h->stream) {
    if (!W->graph || W->graph_y != y_seq_dev || W->graph_truth != truth_seq_dev) {
      if (W->graph) {
        cudaGraphExecDestroy(W->graph);
        W->graph = nullptr;
      }
      LK_ACUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      st = enqueue_grad(h, frames, y_seq_dev, truth_seq_dev);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
      if (st != LETKF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess)
        return gfail(h, LETKF_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&W->graph, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess)
        return gfail(h, LETKF_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
      W->graph_y = y_seq_dev;
      W->graph_truth = truth_seq_dev;
    }
    LK_ACUDA(h, cudaGraphLaunch(W->graph, h->stream));
  } else {
    st = enqueue_grad(h, frames, y_seq_dev, truth_seq_dev);
    if (st != LETKF_OK) return st;
  }
  std::vector<double> rv(frames);
  double acc[4];
  LK_ACUDA(h, cudaMemcpyAsync(rv.data(), W->resvar, frames * sizeof(double),
                              cudaMemcpyDeviceToHost, h->stream));
  LK_ACUDA(h, cudaMemcpyAsync(acc, W->acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LK_ACUDA(h, cudaStreamSynchronize(h->stream));
  h->frame_host += frames;
  double J = 0;
  for (int k = 0; k < frames; ++k) J += rv[k];
  if (J_out) *J_out = J / frames;
  if (grad_out)
    for (int c = 0; c < 3; ++c) grad_out[c] = acc[c];
  return LETKF_OK;
}

extern "C" letkf_status letkf_adjoint_phase_clocks(uint64_t *out) {
#ifdef LK_PHASE_CLOCKS
  if (!out) return LETKF_ERR_ARG;
  unsigned long long v[12] = {};
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(v, g_lk_adj_clocks, sizeof(v));
  const unsigned long long z[12] = {};
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_lk_adj_clocks, z, sizeof(z));
  if (e != cudaSuccess) return LETKF_ERR_CUDA;
  for (int i = 0; i < 12; ++i) out[i] = v[i];
  return LETKF_OK;
#else
  (void)out;
  return LETKF_ERR_STATE;
#endif
}
