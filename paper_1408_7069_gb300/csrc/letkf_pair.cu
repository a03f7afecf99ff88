// FP32 local analysis for ensembles of 17..32 members (Section 4.2 with
// Section 3.1 and Appendix A), two nodes per warp.
//
// Lanes 16h .. 16h+15 of a warp serve node h of the pair. Lane i of a node
// holds two columns of the node's 32-column problem (padded with identity
// columns above m): on entry rows 2i and 2i+1 of
//   A = (m-1)/rho I + sum_j tau_j/sigma2 Yb_j Yb_j^T     (symmetric, so also columns),
// as 16 float2 each, so that packed FP32 FMAs (two lanes of arithmetic per
// instruction) do the Gram, the rotations and the dot products.
//
// Eigensolve: one-sided (Hestenes) Jacobi on the columns of B = A, which
// converge to V diag(lambda) (|A v| = lambda for A > 0). A sweep visits all
// 496 column pairs in 32 rounds of the odd-even transposition network: in an
// even round lane i rotates its own pair (positions 2i, 2i+1); in an odd round
// it rotates positions (2i+1, 2i+2), where position 2i+2 came from lane i+1.
// After each rotation the two columns trade positions (the network's swap),
// so between rounds every lane passes exactly one column to a neighbour: the Q
// column down after an even round, the P column up after an odd round. One
// shuffle moves 32 values per pair visit, half of what a lane-per-column
// layout needs. The end slot of an odd round (positions 31 and 0, held by lane
// 15) does not rotate; it swaps its columns (an exact 90-degree rotation, the
// sign being irrelevant), which keeps the register roles of every lane the same.
// A rotation is applied as P' = c P - s Q, Q' = s P + c Q, exact for c = 1,
// s = 0 (no rotation) and for the swap. A node whose sweep made no rotation is
// converged and freezes (its lanes shuffle from themselves), so its result does
// not depend on the node that shares its warp.
//
// kappa_hat = 1 + rho tr(G)/(m-1) bounds the condition number before the
// eigensolve; nodes above the threshold are queued for the FP64 list kernel.
#include <math.h>
#include <stdint.h>

#include "letkf_device.cuh"

#define LK_PAIR_SHAPES(X) X(0, 2, 4) X(1, 4, 4) X(2, 2, 2) X(3, 1, 8)

namespace {

constexpr int PMP = 32;               // padded width of the node problem
constexpr int CELLF = 2 * PMP + 4;    // floats per halo cell: +4 shifts banks between neighbours
constexpr int NODE_SCR = 3 * PMP + 4;  // floats of scratch per node (C d, X'_0, X'_1)

// Shared-memory layout of one CTA (bytes).
struct PairLayout {
  size_t dh, tap, scr, total;
};
template <int TI, int TJ>
__host__ __device__ PairLayout pair_layout(int w) {
  PairLayout L;
  const size_t ncell = (size_t)(TI + w - 1) * (TJ + w - 1);
  L.dh = align16(ncell * CELLF * sizeof(float));
  L.tap = align16(L.dh + ncell * 2 * sizeof(float));
  L.scr = align16(L.tap + (size_t)w * w * sizeof(float));
  L.total = L.scr + (size_t)TI * TJ * NODE_SCR * sizeof(float);
  return L;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Sum over the 16 lanes of a node.
__device__ __forceinline__ float half_sum(float v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

__device__ __forceinline__ float dot16(const float2 (&a)[16], const float2 (&b)[16]) {
  float2 s0 = f2(0.f), s1 = f2(0.f), s2 = f2(0.f), s3 = f2(0.f);
#pragma unroll
  for (int k = 0; k < 16; k += 4) {
    s0 = fma2(a[k], b[k], s0);
    s1 = fma2(a[k + 1], b[k + 1], s1);
    s2 = fma2(a[k + 2], b[k + 2], s2);
    s3 = fma2(a[k + 3], b[k + 3], s3);
  }
  return ((s0.x + s0.y) + (s1.x + s1.y)) + ((s2.x + s2.y) + (s3.x + s3.y));
}

// One round on this lane's pair (P, Q) with tracked squared norms. `idle`:
// the end slot of an odd round, which swaps instead of rotating. Returns
// whether the pair was rotated.
__device__ __forceinline__ int pair_round(float2 (&P)[16], float2 (&Q)[16], float &nP, float &nQ,
                                          float tol2, bool idle, bool frozen) {
  const float dot = dot16(P, Q);
  // tan(theta) for the rotation that makes the pair orthogonal, with
  // x = |q|^2 - |p|^2, y = 2 p.q: t = sign(x) y / (|x| + sqrt(x^2 + y^2)), |theta| <= pi/4
  const float x = nQ - nP, y = 2.f * dot;
  const float h2 = fmaf(x, x, y * y);
  const float h = h2 * rsqrtf(fmaxf(h2, 1e-37f));
  const float t = (x >= 0.f ? y : -y) / (fabsf(x) + h);
  const float cr = rsqrtf(fmaf(t, t, 1.f));
  const bool rot = !frozen && !idle && dot * dot > tol2 * nP * nQ;
  const bool swp = idle && !frozen;
  // P' = c P - s Q, Q' = s P + c Q: exact for the swap (c = 0, s = 1) and for no
  // rotation (c = 1, s = 0). A three-shear form would save one packed FMA per
  // element pair but its swap leaks rounding of the larger column into the
  // smaller one, which stalls convergence when their norms differ by kappa.
  const float c = rot ? cr : (swp ? 0.f : 1.f);
  const float s = rot ? cr * t : (swp ? 1.f : 0.f);
  const float nP2 = rot ? fmaf(-t, dot, nP) : (swp ? nQ : nP);
  const float nQ2 = rot ? fmaf(t, dot, nQ) : (swp ? nP : nQ);
  const float2 cc = f2(c), ms = f2(-s), ps = f2(s);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float2 p = P[k], q = Q[k];
    P[k] = fma2(cc, p, mul2(ms, q));
    Q[k] = fma2(cc, q, mul2(ps, p));
  }
  nP = nP2;
  nQ = nQ2;
  return rot ? 1 : 0;
}

__device__ __forceinline__ void shfl_cols(float2 (&X)[16], int src) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    X[k].x = __shfl_sync(FULL, X[k].x, src);
    X[k].y = __shfl_sync(FULL, X[k].y, src);
  }
}

__device__ __forceinline__ float norm16(const float2 (&a)[16]) { return dot16(a, a); }

// Sum of v over the 16 lanes of a node, scattered: on return v[0] of lane i
// holds element i (members 2i, 2i+1) of the sum. Recursive halving: at offset
// o a lane keeps the half selected by bit o of its index and adds the partner's
// copy of that half.
__device__ __forceinline__ float2 reduce_scatter16(float2 (&v)[16], int li) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    const bool b = (li & o) != 0;
#pragma unroll
    for (int e = 0; e < o; ++e) {
      const float2 lo = v[e], hi = v[e + o];
      const float2 keep = b ? hi : lo;
      float2 send = b ? lo : hi;
      send.x = __shfl_xor_sync(FULL, send.x, o);
      send.y = __shfl_xor_sync(FULL, send.y, o);
      v[e] = make_float2(keep.x + send.x, keep.y + send.y);
    }
  }
  return v[0];
}

// Stages the tile's halo (slope anomalies and innovations) and the taper table.
template <int TI, int TJ>
__device__ __forceinline__ void stage_pair_tile(const LkInst &I, int i0, int j0, float *halo,
                                                float *dh, float *tap) {
  const int w = I.w, m = I.m;
  const int HJ = TJ + w - 1;
  const int ncell = (TI + w - 1) * HJ;
  const float *Ybp = static_cast<const float *>(I.Ybp);
  const float *dp = static_cast<const float *>(I.dp);
  const float *taper = static_cast<const float *>(I.taper);
  if (m == PMP && (reinterpret_cast<uintptr_t>(Ybp) & 15) == 0) {
    // a cell's two slope rows are 64 contiguous floats in the grid: float4 copies
    for (int e4 = threadIdx.x; e4 < ncell * 16; e4 += blockDim.x) {
      const int cell = e4 >> 4, q = e4 & 15;
      const int hi = cell / HJ, hj = cell - hi * HJ;
      const size_t src = (size_t)(i0 + hi) * I.gs_cols + (j0 + hj);
      reinterpret_cast<float4 *>(halo + (size_t)cell * CELLF)[q] =
          reinterpret_cast<const float4 *>(Ybp + src * 2 * PMP)[q];
    }
  } else {
    for (int e = threadIdx.x; e < ncell * CELLF; e += blockDim.x) {
    const int cell = e / CELLF;
    const int r = e - cell * CELLF;
    float v = 0.f;
    if (r < 2 * PMP) {
      const int c = r / PMP;
      const int mm = r - c * PMP;
      const int hi = cell / HJ, hj = cell - (cell / HJ) * HJ;
      const size_t src = (size_t)(i0 + hi) * I.gs_cols + (j0 + hj);
      if (mm < m) v = Ybp[(src * 2 + c) * m + mm];
    }
    halo[e] = v;
    }
  }
  for (int e = threadIdx.x; e < ncell * 2; e += blockDim.x) {
    const int cell = e >> 1;
    const int hi = cell / HJ, hj = cell - (cell / HJ) * HJ;
    const size_t src = (size_t)(i0 + hi) * I.gs_cols + (j0 + hj);
    dh[e] = dp[src * 2 + (e & 1)];
  }
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) tap[e] = taper[e];
}

// One CTA per tile of TI x TJ nodes of one instance; warp w serves nodes 2w
// and 2w+1 of the tile (row-major).
// Register cap: 128 per thread, so that 16 warps (32 nodes) fit on an SM.
template <int TI, int TJ>
__global__ void __launch_bounds__(TI *TJ * 16)
    analysis_pair_kernel(const LkInst *__restrict__ insts, const LkTile *__restrict__ tiles,
                         float *__restrict__ mean, float *__restrict__ spread, float tol,
                         int max_sweeps, float kappa_thr, int *__restrict__ counters,
                         int2 *__restrict__ worklist, int keep_basis) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LkTile tl = tiles[blockIdx.x];
  const LkInst &I = insts[tl.inst];
  const int w = I.w, m = I.m;
  const PairLayout Ly = pair_layout<TI, TJ>(w);
  const int HJ = TJ + w - 1;
  float *halo = reinterpret_cast<float *>(smem);
  float *dh = reinterpret_cast<float *>(smem + Ly.dh);
  float *tap = reinterpret_cast<float *>(smem + Ly.tap);
  stage_pair_tile<TI, TJ>(I, tl.i0, tl.j0, halo, dh, tap);
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int hh = lane >> 4, li = lane & 15;
  const int node = (threadIdx.x >> 5) * 2 + hh;            // node of the tile
  const int ti = node / TJ, tj = node - (node / TJ) * TJ;
  const int gi = tl.i0 + ti, gj = tl.j0 + tj;
  int pid = -1;
  if (gi <= I.nsub && gj <= I.nsub) pid = I.pid_map[gi * (I.nsub + 1) + gj];
  float *scr = reinterpret_cast<float *>(smem + Ly.scr) + (size_t)node * NODE_SCR;

  // ---- Gram: rows 2li and 2li+1 of A, C d, diagonal of G ----
  float2 P[16], Q[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    P[k] = f2(0.f);
    Q[k] = f2(0.f);
  }
  float diag = 0.f, cd0 = 0.f, cd1 = 0.f;
  const float *hwin = halo + (size_t)(ti * HJ + tj) * CELLF;
  const float *dwin = dh + (size_t)(ti * HJ + tj) * 2;
  for (int ds = 0; ds < w; ++ds) {
    for (int dt = 0; dt < w; ++dt) {
      const int cell = ds * HJ + dt;
      const float tw = tap[ds * w + dt];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float *yv = hwin + (size_t)cell * CELLF + c * PMP;
        const float2 yl = reinterpret_cast<const float2 *>(yv)[li];
        const float cy0 = tw * yl.x, cy1 = tw * yl.y;
        diag = fmaf(cy0, yl.x, fmaf(cy1, yl.y, diag));
        const float dj = dwin[cell * 2 + c];
        cd0 = fmaf(cy0, dj, cd0);
        cd1 = fmaf(cy1, dj, cd1);
        const float2 c0 = f2(cy0), c1 = f2(cy1);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float4 y4 = reinterpret_cast<const float4 *>(yv)[k];
          const float2 ya = make_float2(y4.x, y4.y), yb = make_float2(y4.z, y4.w);
          P[2 * k] = fma2(c0, ya, P[2 * k]);
          P[2 * k + 1] = fma2(c0, yb, P[2 * k + 1]);
          Q[2 * k] = fma2(c1, ya, Q[2 * k]);
          Q[2 * k + 1] = fma2(c1, yb, Q[2 * k + 1]);
        }
      }
    }
  }
  const float alpha = float(I.alpha);
  bool active = pid >= 0;
  if (kappa_thr > 0.f) {
    const float trg = half_sum(diag);
    if (active && 1.f + trg / alpha > kappa_thr) {
      if (li == 0) {
        worklist[atomicAdd(&counters[4 + 1], 1)] = make_int2(tl.inst, pid);
        atomicAdd(&counters[1], 1);
      }
      active = false;
    }
  }
  // (m-1)/rho on the diagonal, 1 on the padding; inactive nodes get the identity
  const float dP = (2 * li < m) ? alpha : 1.f, dQ = (2 * li + 1 < m) ? alpha : 1.f;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (!active) {
      P[k] = f2(0.f);
      Q[k] = f2(0.f);
    }
    if (k == li) {
      P[k].x = active ? P[k].x + dP : 1.f;
      Q[k].y = active ? Q[k].y + dQ : 1.f;
    }
  }

  // ---- Jacobi sweeps ----
  const float tol2 = tol * tol;
  const int up = (lane & 16) | ((li + 1) & 15), dn = (lane & 16) | ((li + 15) & 15);
  bool conv = !active;
  int sweeps = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (__all_sync(FULL, conv)) break;
    float nP = norm16(P), nQ = norm16(Q);
    int rotated = 0;
    const int su = conv ? lane : up, sd = conv ? lane : dn;
#pragma unroll 1
    for (int r = 0; r < 16; ++r) {
      rotated |= pair_round(P, Q, nP, nQ, tol2, false, conv);
      shfl_cols(Q, su);
      nQ = __shfl_sync(FULL, nQ, su);
      rotated |= pair_round(P, Q, nP, nQ, tol2, li == 15, conv);
      shfl_cols(P, sd);
      nP = __shfl_sync(FULL, nP, sd);
    }
    const unsigned any = __ballot_sync(FULL, rotated);
    if (!conv) {
      sweeps = sweep + 1;
      if (((any >> (16 * hh)) & 0xffffu) == 0u) conv = true;
    }
  }
  if (active && li == 0) {
    atomicMax(&counters[2], sweeps);
    atomicAdd(&counters[3], sweeps);
    if (!conv) atomicOr(&counters[0], LK_BIT_NOCONVERGE);
  }

  // ---- eigenpairs: lambda = |b|, v = b / lambda ----
  const float lP = sqrtf(norm16(P)), lQ = sqrtf(norm16(Q));
  {
    const float iP = 1.f / lP, iQ = 1.f / lQ;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      P[k] = mul2(f2(iP), P[k]);
      Q[k] = mul2(f2(iQ), Q[k]);
    }
  }

  // ---- eigenbasis for the reverse mode: U[k][2li], U[k][2li+1] ----
  if (keep_basis && active) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      ok = ok && isfinite(P[k].x) && isfinite(P[k].y) && isfinite(Q[k].x) && isfinite(Q[k].y);
    float *U = I.basis + (size_t)pid * PMP * PMP;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float2 r0 = ok ? make_float2(P[k].x, Q[k].x)
                           : make_float2(k == li ? 1.f : 0.f, 0.f);
      const float2 r1 = ok ? make_float2(P[k].y, Q[k].y)
                           : make_float2(0.f, k == li ? 1.f : 0.f);
      reinterpret_cast<float2 *>(U + (2 * k) * PMP)[li] = r0;
      reinterpret_cast<float2 *>(U + (2 * k + 1) * PMP)[li] = r1;
    }
  }
  // ---- transform and apply (Section 4.2): Xa_r = xbar_r + X'_r wbar + X'_r W ----
  float *vcd = scr;                     // C d
  float *vx0 = vcd + PMP;               // X'_0
  float *vx1 = vx0 + PMP;               // X'_1
  float *xrow = active ? static_cast<float *>(I.X) + (size_t)pid * 2 * m : nullptr;
  const int m0 = 2 * li, m1 = 2 * li + 1;
  const float x00 = (active && m0 < m) ? xrow[m0] : 0.f;
  const float x01 = (active && m1 < m) ? xrow[m1] : 0.f;
  const float x10 = (active && m0 < m) ? xrow[m + m0] : 0.f;
  const float x11 = (active && m1 < m) ? xrow[m + m1] : 0.f;
  const float inv_m = 1.f / float(m);
  const float xb0 = half_sum(x00 + x01) * inv_m;
  const float xb1 = half_sum(x10 + x11) * inv_m;
  reinterpret_cast<float2 *>(vcd)[li] = make_float2(cd0, cd1);
  reinterpret_cast<float2 *>(vx0)[li] =
      make_float2(m0 < m ? x00 - xb0 : 0.f, m1 < m ? x01 - xb0 : 0.f);
  reinterpret_cast<float2 *>(vx1)[li] =
      make_float2(m0 < m ? x10 - xb1 : 0.f, m1 < m ? x11 - xb1 : 0.f);
  __syncwarp();
  // projections of C d and of the two anomaly rows on this lane's eigenvectors
  float2 uP = f2(0.f), uQ = f2(0.f), a0P = f2(0.f), a0Q = f2(0.f), a1P = f2(0.f), a1Q = f2(0.f);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float2 cdv = reinterpret_cast<const float2 *>(vcd)[k];
    const float2 x0v = reinterpret_cast<const float2 *>(vx0)[k];
    const float2 x1v = reinterpret_cast<const float2 *>(vx1)[k];
    uP = fma2(P[k], cdv, uP);
    uQ = fma2(Q[k], cdv, uQ);
    a0P = fma2(P[k], x0v, a0P);
    a0Q = fma2(Q[k], x0v, a0Q);
    a1P = fma2(P[k], x1v, a1P);
    a1Q = fma2(Q[k], x1v, a1Q);
  }
  const float gP0 = a0P.x + a0P.y, gQ0 = a0Q.x + a0Q.y;
  const float gP1 = a1P.x + a1P.y, gQ1 = a1Q.x + a1Q.y;
  const float zP = (uP.x + uP.y) / lP, zQ = (uQ.x + uQ.y) / lQ;
  const float w0 = half_sum(gP0 * zP + gQ0 * zQ);          // X'_0 wbar
  const float w1 = half_sum(gP1 * zP + gQ1 * zQ);          // X'_1 wbar
  const float rP = sqrtf(float(m - 1) / lP), rQ = sqrtf(float(m - 1) / lQ);
  // X'_r W = sum_j h_r,j v_j^T with h_r,j = (X'_r v_j) sqrt((m-1)/lambda_j): this
  // lane's two terms, summed over the node's lanes and scattered by member
  float2 v0[16], v1[16];
  {
    const float2 hP0 = f2(gP0 * rP), hQ0 = f2(gQ0 * rQ), hP1 = f2(gP1 * rP), hQ1 = f2(gQ1 * rQ);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      v0[k] = fma2(hP0, P[k], mul2(hQ0, Q[k]));
      v1[k] = fma2(hP1, P[k], mul2(hQ1, Q[k]));
    }
  }
  const float2 q0 = reduce_scatter16(v0, li);
  const float2 q1 = reduce_scatter16(v1, li);
  const float q00 = q0.x, q01 = q0.y, q10 = q1.x, q11 = q1.y;
  const float xa00 = xb0 + w0 + q00, xa01 = xb0 + w0 + q01;
  const float xa10 = xb1 + w1 + q10, xa11 = xb1 + w1 + q11;
  if (active) {
    if (m0 < m) {
      xrow[m0] = xa00;
      xrow[m + m0] = xa10;
    }
    if (m1 < m) {
      xrow[m1] = xa01;
      xrow[m + m1] = xa11;
    }
  }
  const float e00 = m0 < m ? xa00 : 0.f, e01 = m1 < m ? xa01 : 0.f;
  const float e10 = m0 < m ? xa10 : 0.f, e11 = m1 < m ? xa11 : 0.f;
  const float mu0 = half_sum(e00 + e01) * inv_m;
  const float mu1 = half_sum(e10 + e11) * inv_m;
  const float d00 = m0 < m ? xa00 - mu0 : 0.f, d01 = m1 < m ? xa01 - mu0 : 0.f;
  const float d10 = m0 < m ? xa10 - mu1 : 0.f, d11 = m1 < m ? xa11 - mu1 : 0.f;
  const float sp0 = sqrtf(half_sum(d00 * d00 + d01 * d01) / float(m - 1));
  const float sp1 = sqrtf(half_sum(d10 * d10 + d11 * d11) / float(m - 1));
  if (active && li == 0) {
    const long long row = I.node_off + pid;
    if (mean) {
      mean[2 * row] = mu0;
      mean[2 * row + 1] = mu1;
    }
    if (spread) {
      spread[2 * row] = sp0;
      spread[2 * row + 1] = sp1;
    }
    if (!isfinite(mu0) || !isfinite(mu1) || !isfinite(sp0) || !isfinite(sp1))
      atomicOr(&counters[0], LK_BIT_NONFINITE);
  }
}

template <int TI, int TJ>
cudaError_t launch_shape(letkf_ctx *h, int cls, float *mean, float *spread, float tol, float kthr) {
  size_t need = 0;
  for (const LkInst &I : h->inst)
    if (I.mp == PMP) {
      const size_t b = pair_layout<TI, TJ>(I.w).total;
      need = b > need ? b : need;
    }
  analysis_pair_kernel<TI, TJ><<<h->n_tiles[cls], TI * TJ * 16, need, h->stream>>>(
      h->d_inst, h->tiles[cls], mean, spread, tol, h->max_sweeps, kthr, h->counters,
      h->worklist + (size_t)cls * h->n_pts_total, h->keep_basis);
  return cudaGetLastError();
}

template <int TI, int TJ>
cudaError_t set_shape_smem(int w) {
  return cudaFuncSetAttribute(analysis_pair_kernel<TI, TJ>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)pair_layout<TI, TJ>(w).total);
}

}  // namespace

cudaError_t lk_launch_pair(letkf_ctx *h, int cls, void *mean, void *spread, float tol, float kthr) {
  switch (h->tile_shape[cls]) {
#define LK_CASE(id, ti, tj) \
  case id:                  \
    return launch_shape<ti, tj>(h, cls, (float *)mean, (float *)spread, tol, kthr);
    LK_PAIR_SHAPES(LK_CASE)
#undef LK_CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t lk_setup_pair(letkf_ctx *h) {
  int wmax = 0;
  for (const LkInst &I : h->inst)
    if (I.mp == PMP) wmax = I.w > wmax ? I.w : wmax;
  if (wmax == 0 || h->precision != 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
#define LK_SET(id, ti, tj) \
  if (e == cudaSuccess) e = set_shape_smem<ti, tj>(wmax);
  LK_PAIR_SHAPES(LK_SET)
#undef LK_SET
  return e;
}
