// FP32 local analysis (Section 4.2 with Section 3.1 and Appendix A) with two
// columns of the node problem per lane.
//
// The node problem is padded to MP = 16, 32, 48 or 64 columns (identity on the
// padding). A node is served by LPN = MP/2 lanes: 4 nodes per warp for MP = 16,
// 2 for MP = 32, 1 for MP = 48 (lanes 24..31 idle) and 64. Lane i of a node
// holds two columns, on entry rows 2i and 2i+1 of
//   A = (m-1)/rho I + sum_j tau_j/sigma2 Yb_j Yb_j^T     (symmetric, so also columns),
// as MP/2 float2 each, so that packed FP32 FMAs (two lanes of arithmetic per
// instruction) do the Gram, the rotations and the dot products.
//
// Eigensolve: one-sided (Hestenes) Jacobi on the columns of B = A, which
// converge to V diag(lambda) (|A v| = lambda for A > 0). A sweep visits all
// MP (MP-1)/2 column pairs in MP rounds of the odd-even transposition network:
// in an even round lane i rotates its own pair (positions 2i, 2i+1); in an odd
// round it rotates positions (2i+1, 2i+2), where position 2i+2 came from lane
// i+1. After each rotation the two columns trade positions (the network's
// swap), so between rounds every lane passes exactly one column to a
// neighbour: the Q column down after an even round, the P column up after an
// odd round. One shuffle moves MP values per pair visit, half of what a
// lane-per-column layout needs. The end slot of an odd round (positions MP-1
// and 0, held by the node's last lane) does not rotate; it swaps its columns
// (a 90-degree rotation, the sign being irrelevant), which keeps the register
// roles of every lane the same. Even rounds have no end slot, so they apply
// their rotations without the cosine, P' = P - t Q, Q' = Q + t P (half the
// packed FMAs), and leave the cosine as the scale of both columns; the odd
// round folds the two scales into its rotation P' = c P - s Q, Q' = s P + c Q
// and writes both columns back at scale 1. No rotation of a frozen node
// changes a bit. A node is converged after a sweep whose rotations all had cosines
// at most the stop cosine (letkf_set_jacobi; with stop <= the rotation
// threshold, a sweep without rotations) and then freezes (its lanes shuffle
// from themselves), so its result does not depend on the nodes that share its
// warp.
//
// kappa_hat = 1 + rho tr(G)/(m-1) bounds the condition number before the
// eigensolve; nodes above the threshold still take this FP32 sweep, store
// their eigenbasis (the start of their FP64 sweep) and leave X alone: they are
// queued, per width class, for the FP64 list kernels of letkf_node64.cu
// (MP = 16 and 32: node64_list_kernel; MP = 48 and 64 share one queue:
// node64w_list_kernel), which write them.
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "letkf_device.cuh"

// Phase clocks (a library built with -DLK_PHASE_CLOCKS only): lane 0 of every
// warp adds the SM cycles it spent in each phase of the kernel, summed over
// warps: [0] halo staging, [1] Gram and kappa_hat, [2] Jacobi sweeps,
// [3] eigenpairs, transform and apply, [4] number of warps.
#ifdef LK_PHASE_CLOCKS
__device__ unsigned long long g_lk_phase_clocks[5];
#define LK_PHASE_STAMP(t) const long long t = clock64()
#else
#define LK_PHASE_STAMP(t)
#endif

namespace {

constexpr int pow2_ceil(int x) { return x <= 1 ? 1 : 2 * pow2_ceil((x + 1) / 2); }

// MP = 24 (ensembles of 17..24 members of the m <= 32 class) computes on 24
// columns but keeps the class's 32 x 32 basis layout (MPS): its nodes' bases
// are the 24 x 24 block of a 32 x 32 store whose padding stays the identity.
template <int MP>
struct PairCfg {
  static constexpr int LPN = MP / 2;                           // lanes per node
  static constexpr int GL = MP <= 32 ? pow2_ceil(LPN) : 32;    // lanes of a node's group (power of 2)
  static constexpr int NPW = 32 / GL;                          // nodes per warp
  static constexpr int K2 = MP / 2;                            // float2 per column
  static constexpr int CELLF = 2 * MP + 4;                     // floats per halo cell (+4: bank shift)
  static constexpr int NODE_SCR = 3 * MP + 4;                  // scratch floats per node
  static constexpr int MPS = MP == 24 ? 32 : MP;               // columns of the stored basis
};

// Shared-memory layout of one CTA (bytes).
struct PairLayout {
  size_t dh, tap, scr, total;
};
template <int MP, int TI, int TJ>
__host__ __device__ PairLayout pair_layout(int w) {
  using C = PairCfg<MP>;
  PairLayout L;
  const size_t ncell = (size_t)(TI + w - 1) * (TJ + w - 1);
  L.dh = align16(ncell * C::CELLF * sizeof(float));
  L.tap = align16(L.dh + ncell * 2 * sizeof(float));
  L.scr = align16(L.tap + (size_t)w * w * sizeof(float));
  L.total = L.scr + (size_t)TI * TJ * C::NODE_SCR * sizeof(float);
  return L;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Sum over the lanes of a node's group (idle lanes contribute zero).
template <int GL>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = GL / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Dot product of two MP-element columns with four independent packed chains.
template <int K2>
__device__ __forceinline__ float dotk(const float2 (&a)[K2], const float2 (&b)[K2]) {
  constexpr int NC = K2 >= 4 ? 4 : K2;
  float2 s[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) s[c] = mul2(a[c], b[c]);
#pragma unroll
  for (int k = NC; k < K2; ++k) s[k % NC] = fma2(a[k], b[k], s[k % NC]);
#pragma unroll
  for (int w = NC / 2; w > 0; w >>= 1)
#pragma unroll
    for (int c = 0; c < w; ++c) s[c] = __fadd2_rn(s[c], s[c + w]);
  return s[0].x + s[0].y;
}

// Adds the partner lane's partial sum (XO > 0: the columns' rows are split
// between lanes XO apart). Float addition commutes, so both lanes get the
// same bits.
template <int XO>
__device__ __forceinline__ float combine(float v) {
  if constexpr (XO > 0) v += __shfl_xor_sync(FULL, v, XO);
  return v;
}

// The rotation that makes a pair orthogonal, |theta| <= pi/4, from the true
// squared norms and dot product: x = |q|^2 - |p|^2, y = 2 p.q, h = sqrt(x^2 + y^2),
// cos 2theta = |x|/h, sin 2theta = sign(x) y / h, c = sqrt((1 + cos 2theta)/2)
// >= 1/sqrt(2), s = sin 2theta / (2c), t = s / c. Two reciprocal square roots,
// no divide. `rot`: the pair is rotated (not frozen, not the end slot, and
// cos(p, q) above the rotation threshold); `big`: above the stopping cosine.
struct Rot {
  float c, s, t;
  bool rot, big;
};

__device__ __forceinline__ Rot rotation(float nP, float nQ, float dot, float tol2, float stop2,
                                        bool skip) {
  const float x = nQ - nP, y = 2.f * dot;
  const float rh = lk_rsqrt_normal(fmaxf(fmaf(x, x, y * y), 1e-37f));
  const float c2 = fmaf(0.5f * fabsf(x), rh, 0.5f);
  const float rc = lk_rsqrt_normal(c2);
  Rot R;
  R.c = c2 * rc;
  R.s = (x >= 0.f ? y : -y) * (0.5f * rh) * rc;
  R.t = R.s * rc;
  const float dd = dot * dot, nn = nP * nQ;
  R.rot = !skip && dd > tol2 * nn;
  R.big = R.rot && dd > stop2 * nn;
  return R;
}

// Even round of the odd-even network on this lane's pair (P, Q), both stored
// at scale 1 (the odd round before normalised them), with tracked true
// squared norms. The rotation is applied without its cosine,
// P' = P - t Q, Q' = Q + t P (one packed FMA per element pair, exact for
// t = 0), and the cosine is returned in `cs` as the scale of both stored
// columns: the true columns are cs P' and cs Q'. XO > 0: the lane holds half
// of the pair's rows, the other half is on lane ^ XO, which computes the same
// rotation. Returns whether the pair was rotated with cos(p, q) above the
// stopping cosine.
template <int K2, int XO = 0>
__device__ __forceinline__ bool pair_round_even(float2 (&P)[K2], float2 (&Q)[K2], float &nP,
                                               float &nQ, float &cs, float tol2, float stop2,
                                               bool frozen) {
  const float dot = combine<XO>(dotk<K2>(P, Q));
  const Rot R = rotation(nP, nQ, dot, tol2, stop2, frozen);
  const float t = R.rot ? R.t : 0.f;
  cs = R.rot ? R.c : 1.f;
  nP = fmaf(-t, dot, nP);
  nQ = fmaf(t, dot, nQ);
  const float2 mt = f2(-t), pt = f2(t);
#pragma unroll
  for (int k = 0; k < K2; ++k) {
    const float2 p = P[k], q = Q[k];
    P[k] = fma2(mt, q, p);
    Q[k] = fma2(pt, p, q);
  }
  return R.big;
}

// Odd round on (P, Q) stored at scales a and b (the cosines of the even rounds
// that produced them; 1 for a frozen node). The true rotation
// p' = c p - s q, q' = s p + c q of the true columns p = a P, q = b Q is
// written back at scale 1: P' = (c a) P - (s b) Q, Q' = (s a) P + (c b) Q.
// `idle`: the end slot, which swaps instead of rotating (c = 0, s = 1, so
// P' = -b Q and Q' = a P: each column only rescaled, nothing of the other
// mixed in). No rotation at a = b = 1 is exact.
template <int K2, int XO = 0>
__device__ __forceinline__ bool pair_round_odd(float2 (&P)[K2], float2 (&Q)[K2], float &nP,
                                              float &nQ, float a, float b, float tol2,
                                              float stop2, bool idle, bool frozen) {
  const float dot = combine<XO>(dotk<K2>(P, Q)) * (a * b);
  const Rot R = rotation(nP, nQ, dot, tol2, stop2, frozen || idle);
  const bool swp = idle && !frozen;
  const float c = R.rot ? R.c : (swp ? 0.f : 1.f);
  const float s = R.rot ? R.s : (swp ? 1.f : 0.f);
  const float nP2 = R.rot ? fmaf(-R.t, dot, nP) : (swp ? nQ : nP);
  const float nQ2 = R.rot ? fmaf(R.t, dot, nQ) : (swp ? nP : nQ);
  const float2 ca = f2(c * a), msb = f2(-(s * b)), sa = f2(s * a), cb = f2(c * b);
#pragma unroll
  for (int k = 0; k < K2; ++k) {
    const float2 p = P[k], q = Q[k];
    P[k] = fma2(ca, p, mul2(msb, q));
    Q[k] = fma2(cb, q, mul2(sa, p));
  }
  nP = nP2;
  nQ = nQ2;
  return R.big;
}

template <int K2>
__device__ __forceinline__ void shfl_cols(float2 (&X)[K2], int src) {
#pragma unroll
  for (int k = 0; k < K2; ++k) {
    X[k].x = __shfl_sync(FULL, X[k].x, src);
    X[k].y = __shfl_sync(FULL, X[k].y, src);
  }
}

// Sum of v over the GL lanes of a group, scattered: on return v[0] of lane i
// (i < GL) holds element i of the sum. Recursive halving: at offset o a lane
// keeps the half selected by bit o of its index and adds the partner's copy.
template <int GL>
__device__ __forceinline__ float2 reduce_scatter(float2 (&v)[GL], int li) {
#pragma unroll
  for (int o = GL / 2; o > 0; o >>= 1) {
    const bool b = (li & o) != 0;
#pragma unroll
    for (int e = 0; e < o; ++e) {
      const float2 lo = v[e], hi = v[e + o];
      const float2 keep = b ? hi : lo;
      float2 send = b ? lo : hi;
      send.x = __shfl_xor_sync(FULL, send.x, o);
      send.y = __shfl_xor_sync(FULL, send.y, o);
      v[e] = __fadd2_rn(keep, send);
    }
  }
  return v[0];
}

// Stages the tile's halo (slope anomalies and innovations) and the taper table.
// S: the handle's storage type (double on FP64 handles, whose FP32 basis pass
// rounds the window to float here).
template <int MP, int TI, int TJ, typename S = float>
__device__ __forceinline__ void stage_pair_tile(const LkInst &I, int i0, int j0, float *halo,
                                                float *dh, float *tap) {
  using C = PairCfg<MP>;
  const int w = I.w, m = I.m;
  const int HJ = TJ + w - 1;
  const int ncell = (TI + w - 1) * HJ;
  const S *Ybp = static_cast<const S *>(I.Ybp);
  const S *dp = static_cast<const S *>(I.dp);
  const S *taper = static_cast<const S *>(I.taper);
  if (std::is_same<S, float>::value && m == MP && (reinterpret_cast<uintptr_t>(Ybp) & 15) == 0) {
    // a cell's two slope rows are 2 MP contiguous floats in the grid: float4 copies
    constexpr int Q4 = MP / 2;
    for (int e4 = threadIdx.x; e4 < ncell * Q4; e4 += blockDim.x) {
      const int cell = e4 / Q4, q = e4 - cell * Q4;
      const int hi = cell / HJ, hj = cell - hi * HJ;
      const size_t src = (size_t)(i0 + hi) * I.gs_cols + (j0 + hj);
      reinterpret_cast<float4 *>(halo + (size_t)cell * C::CELLF)[q] =
          reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(Ybp) + src * 2 * MP)[q];
    }
  } else {
    for (int e = threadIdx.x; e < ncell * C::CELLF; e += blockDim.x) {
      const int cell = e / C::CELLF;
      const int r = e - cell * C::CELLF;
      float v = 0.f;
      if (r < 2 * MP) {
        const int c = r / MP;
        const int mm = r - c * MP;
        const int hi = cell / HJ, hj = cell - hi * HJ;
        const size_t src = (size_t)(i0 + hi) * I.gs_cols + (j0 + hj);
        if (mm < m) v = (float)Ybp[(src * 2 + c) * m + mm];
      }
      halo[e] = v;
    }
  }
  for (int e = threadIdx.x; e < ncell * 2; e += blockDim.x) {
    const int cell = e >> 1;
    const int hi = cell / HJ, hj = cell - hi * HJ;
    const size_t src = (size_t)(i0 + hi) * I.gs_cols + (j0 + hj);
    dh[e] = (float)dp[src * 2 + (e & 1)];
  }
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) tap[e] = (float)taper[e];
}

// One CTA per tile of TI x TJ nodes of one instance; the nodes of the tile are
// taken in row-major order, NPW per warp. `queue`: FP64 worklist counter slot
// (MP <= 32), NULL for no fallback.
// Threads per CTA, and CTAs per SM to budget registers for: 128 per thread
// for MP <= 32 (16 warps per SM), whatever the wide problems need otherwise.
template <int MP, int TI, int TJ>
struct PairLaunch {
  static constexpr int threads = TI * TJ * 32 / PairCfg<MP>::NPW;
  static constexpr int regs = MP <= 32 ? 128 : (MP == 48 ? 168 : 0);   // budget per thread
  static constexpr int min_ctas =
      regs == 0 || 65536 / (threads * (regs ? regs : 1)) == 0 ? 1 : 65536 / (threads * regs);
};

// BASIS (FP64 handles, S = double): the FP32 eigensolve alone, storing every
// node's eigenbasis as the start of the FP64 sweep of node64_kernel; nothing
// is queued and X is not touched.
template <int MP, int TI, int TJ, typename S = float, bool BASIS = false>
__global__ void __launch_bounds__(PairLaunch<MP, TI, TJ>::threads, PairLaunch<MP, TI, TJ>::min_ctas)
    analysis_pair_kernel(const LkInst *__restrict__ insts, const LkTile *__restrict__ tiles,
                         float *__restrict__ mean, float *__restrict__ spread, float tol,
                         float stop, int max_sweeps, float kappa_thr, int *__restrict__ counters,
                         int *__restrict__ queue, int2 *__restrict__ worklist, int keep_basis) {
  lk_pdl_wait();   // no early trigger: the next kernel launches as this one's CTAs exit
  LK_PHASE_STAMP(ph0);
  using C = PairCfg<MP>;
  constexpr int K2 = C::K2, LPN = C::LPN, GL = C::GL;
  extern __shared__ __align__(16) unsigned char smem[];
  const LkTile tl = tiles[blockIdx.x];
  const LkInst &I = insts[tl.inst];
  const int w = I.w, m = I.m;
  const PairLayout Ly = pair_layout<MP, TI, TJ>(w);
  const int HJ = TJ + w - 1;
  float *halo = reinterpret_cast<float *>(smem);
  float *dh = reinterpret_cast<float *>(smem + Ly.dh);
  float *tap = reinterpret_cast<float *>(smem + Ly.tap);
  stage_pair_tile<MP, TI, TJ, S>(I, tl.i0, tl.j0, halo, dh, tap);
  __syncthreads();
  LK_PHASE_STAMP(ph1);

  const int lane = threadIdx.x & 31;
  const int grp = lane / GL, li = lane - grp * GL;    // node of the warp, lane within the node
  const bool live = li < LPN;                        // lanes 24..31 idle when MP = 48
  const int node = (threadIdx.x >> 5) * C::NPW + grp;  // node of the tile
  const int ti = node / TJ, tj = node - (node / TJ) * TJ;
  const int gi = tl.i0 + ti, gj = tl.j0 + tj;
  int pid = -1;
  if (gi <= I.nsub && gj <= I.nsub) pid = I.pid_map[gi * (I.nsub + 1) + gj];
  float *scr = reinterpret_cast<float *>(smem + Ly.scr) + (size_t)node * C::NODE_SCR;

  // ---- Gram: rows 2li and 2li+1 of A, C d, diagonal of G ----
  float2 P[K2], Q[K2];
#pragma unroll
  for (int k = 0; k < K2; ++k) {
    P[k] = f2(0.f);
    Q[k] = f2(0.f);
  }
  float diag = 0.f, cd0 = 0.f, cd1 = 0.f;
  const float *hwin = halo + (size_t)(ti * HJ + tj) * C::CELLF;
  const float *dwin = dh + (size_t)(ti * HJ + tj) * 2;
  const int lr = live ? li : 0;                      // idle lanes read row pair 0, then drop it
  for (int ds = 0; ds < w; ++ds) {
    for (int dt = 0; dt < w; ++dt) {
      const int cell = ds * HJ + dt;
      const float tw = tap[ds * w + dt];
      if (tw == 0.f) continue;                       // outside the taper's support
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float *yv = hwin + (size_t)cell * C::CELLF + c * MP;
        const float2 yl = reinterpret_cast<const float2 *>(yv)[lr];
        const float cy0 = tw * yl.x, cy1 = tw * yl.y;
        diag = fmaf(cy0, yl.x, fmaf(cy1, yl.y, diag));
        const float dj = dwin[cell * 2 + c];
        cd0 = fmaf(cy0, dj, cd0);
        cd1 = fmaf(cy1, dj, cd1);
        const float2 c0 = f2(cy0), c1 = f2(cy1);
#pragma unroll
        for (int k = 0; k < K2 / 2; ++k) {
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
  if (!live) diag = cd0 = cd1 = 0.f;
  const float alpha = float(I.alpha);
  const bool active = pid >= 0;
  // kappa_hat above the threshold: the node's mean solve needs the FP64 Gram.
  // It still takes this FP32 eigensolve, whose basis is stored as the start of
  // the FP64 list kernel's sweep; X is left alone and the node is queued.
  bool queued = false;
  if (queue) {
    const float trg = group_sum<GL>(diag);
    if (active && 1.f + trg / alpha > kappa_thr) {
      if (li == 0) {
        worklist[atomicAdd(queue, 1)] = make_int2(tl.inst, pid);
        atomicAdd(&counters[1], 1);
      }
      queued = true;
    }
  }
  // (m-1)/rho on the diagonal, 1 on the padding; inactive nodes and idle lanes
  // get identity columns
  const bool own = active && live;
  const float dP = (2 * li < m) ? alpha : 1.f, dQ = (2 * li + 1 < m) ? alpha : 1.f;
#pragma unroll
  for (int k = 0; k < K2; ++k) {
    if (!own) {
      P[k] = f2(0.f);
      Q[k] = f2(0.f);
    }
    if (k == li) {
      P[k].x = own ? P[k].x + dP : 1.f;
      Q[k].y = own ? Q[k].y + dQ : 1.f;
    }
  }
  if (!live) {                                       // unit columns, never touched again
    P[0].x = 1.f;
    Q[0].y = 1.f;
  }

  // ---- Jacobi sweeps ----
  LK_PHASE_STAMP(ph2);
  const float tol2 = tol * tol, stop2 = stop * stop;
  const int base = grp * GL;
  const int up = live ? base + (li + 1) % LPN : lane;
  const int dn = live ? base + (li + LPN - 1) % LPN : lane;
  bool conv = !active;
  int sweeps = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (__all_sync(FULL, conv)) break;
    float nP = dotk<K2>(P, P), nQ = dotk<K2>(Q, Q);
    bool rotated = false;
    const bool frz = conv || !live;
    const int su = frz ? lane : up, sd = frz ? lane : dn;
#pragma unroll 2
    for (int r = 0; r < MP / 2; ++r) {
      float cs;
      rotated |= pair_round_even<K2>(P, Q, nP, nQ, cs, tol2, stop2, frz);
      shfl_cols<K2>(Q, su);
      nQ = __shfl_sync(FULL, nQ, su);
      const float cq = __shfl_sync(FULL, cs, su);
      rotated |= pair_round_odd<K2>(P, Q, nP, nQ, cs, cq, tol2, stop2, li == LPN - 1, frz);
      shfl_cols<K2>(P, sd);
      nP = __shfl_sync(FULL, nP, sd);
    }
    // Converged after a sweep whose rotations all had cos(p, q) <= stop. With
    // stop <= tol that is a sweep without rotations (every pair orthogonal to
    // tol); a larger stop ends one or two sweeps earlier, leaving pairs within
    // about stop^2 except inside near-degenerate clusters, whose mixing does
    // not change W.
    const unsigned big = __ballot_sync(FULL, rotated);
    const unsigned gmask = (GL == 32) ? 0xffffffffu : (((1u << GL) - 1u) << base);
    if (!conv) {
      sweeps = sweep + 1;
      if ((big & gmask) == 0u) conv = true;
    }
  }
  if (active && li == 0) {
    atomicMax(&counters[2], sweeps);
    atomicAdd(&counters[3], sweeps);
    if (!conv) atomicOr(&counters[0], LK_BIT_NOCONVERGE);
  }

  // ---- eigenpairs: lambda = |b|, v = b / lambda ----
  LK_PHASE_STAMP(ph3);
  const float lP = sqrtf(dotk<K2>(P, P)), lQ = sqrtf(dotk<K2>(Q, Q));
  {
    const float iP = 1.f / lP, iQ = 1.f / lQ;
#pragma unroll
    for (int k = 0; k < K2; ++k) {
      P[k] = mul2(f2(iP), P[k]);
      Q[k] = mul2(f2(iQ), Q[k]);
    }
  }
  // ---- eigenbasis for the reverse mode and for queued nodes: U[k][2li], U[k][2li+1] ----
  if ((BASIS || keep_basis || queued) && active && live) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < K2; ++k)
      ok = ok && isfinite(P[k].x) && isfinite(P[k].y) && isfinite(Q[k].x) && isfinite(Q[k].y);
    constexpr int MPS = C::MPS;
    float *U = I.basis + (size_t)pid * MPS * MPS;
#pragma unroll
    for (int k = 0; k < K2; ++k) {
      const float2 r0 = ok ? make_float2(P[k].x, Q[k].x) : make_float2(k == li ? 1.f : 0.f, 0.f);
      const float2 r1 = ok ? make_float2(P[k].y, Q[k].y) : make_float2(0.f, k == li ? 1.f : 0.f);
      reinterpret_cast<float2 *>(U + (2 * k) * MPS)[li] = r0;
      reinterpret_cast<float2 *>(U + (2 * k + 1) * MPS)[li] = r1;
    }
  }
  if constexpr (BASIS) return;

  // ---- transform and apply (Section 4.2): Xa_r = xbar_r + X'_r wbar + X'_r W ----
  float *vcd = scr;                     // C d
  float *vx0 = vcd + MP;                // X'_0
  float *vx1 = vx0 + MP;                // X'_1
  const bool wr = active && !queued;
  float *xrow = wr ? static_cast<float *>(I.X) + (size_t)pid * 2 * m : nullptr;
  const int m0 = 2 * li, m1 = 2 * li + 1;
  const bool in0 = live && m0 < m, in1 = live && m1 < m;
  const float x00 = (wr && in0) ? xrow[m0] : 0.f;
  const float x01 = (wr && in1) ? xrow[m1] : 0.f;
  const float x10 = (wr && in0) ? xrow[m + m0] : 0.f;
  const float x11 = (wr && in1) ? xrow[m + m1] : 0.f;
  const float inv_m = 1.f / float(m);
  const float xb0 = group_sum<GL>(x00 + x01) * inv_m;
  const float xb1 = group_sum<GL>(x10 + x11) * inv_m;
  if (live) {
    reinterpret_cast<float2 *>(vcd)[li] = make_float2(cd0, cd1);
    reinterpret_cast<float2 *>(vx0)[li] = make_float2(in0 ? x00 - xb0 : 0.f, in1 ? x01 - xb0 : 0.f);
    reinterpret_cast<float2 *>(vx1)[li] = make_float2(in0 ? x10 - xb1 : 0.f, in1 ? x11 - xb1 : 0.f);
  }
  __syncwarp();
  // projections of C d and of the two anomaly rows on this lane's eigenvectors
  float2 uP = f2(0.f), uQ = f2(0.f), a0P = f2(0.f), a0Q = f2(0.f), a1P = f2(0.f), a1Q = f2(0.f);
#pragma unroll
  for (int k = 0; k < K2; ++k) {
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
  const float gP0 = live ? a0P.x + a0P.y : 0.f, gQ0 = live ? a0Q.x + a0Q.y : 0.f;
  const float gP1 = live ? a1P.x + a1P.y : 0.f, gQ1 = live ? a1Q.x + a1Q.y : 0.f;
  const float zP = (uP.x + uP.y) / lP, zQ = (uQ.x + uQ.y) / lQ;
  const float w0 = group_sum<GL>(gP0 * zP + gQ0 * zQ);    // X'_0 wbar
  const float w1 = group_sum<GL>(gP1 * zP + gQ1 * zQ);    // X'_1 wbar
  const float rP = sqrtf(float(m - 1) / lP), rQ = sqrtf(float(m - 1) / lQ);
  // X'_r W = sum_j h_r,j v_j^T with h_r,j = (X'_r v_j) sqrt((m-1)/lambda_j): this
  // lane's two terms, summed over the node's lanes and scattered by member
  float2 v0[GL], v1[GL];
  {
    const float2 hP0 = f2(gP0 * rP), hQ0 = f2(gQ0 * rQ), hP1 = f2(gP1 * rP), hQ1 = f2(gQ1 * rQ);
#pragma unroll
    for (int k = 0; k < GL; ++k) {
      if (k < K2) {
        v0[k] = fma2(hP0, P[k], mul2(hQ0, Q[k]));
        v1[k] = fma2(hP1, P[k], mul2(hQ1, Q[k]));
      } else {
        v0[k] = f2(0.f);
        v1[k] = f2(0.f);
      }
    }
  }
  const float2 q0 = reduce_scatter<GL>(v0, li);
  const float2 q1 = reduce_scatter<GL>(v1, li);
  const float xa00 = xb0 + w0 + q0.x, xa01 = xb0 + w0 + q0.y;
  const float xa10 = xb1 + w1 + q1.x, xa11 = xb1 + w1 + q1.y;
  if (wr) {
    if (in0) {
      xrow[m0] = xa00;
      xrow[m + m0] = xa10;
    }
    if (in1) {
      xrow[m1] = xa01;
      xrow[m + m1] = xa11;
    }
  }
  const float e00 = in0 ? xa00 : 0.f, e01 = in1 ? xa01 : 0.f;
  const float e10 = in0 ? xa10 : 0.f, e11 = in1 ? xa11 : 0.f;
  const float mu0 = group_sum<GL>(e00 + e01) * inv_m;
  const float mu1 = group_sum<GL>(e10 + e11) * inv_m;
  const float d00 = in0 ? xa00 - mu0 : 0.f, d01 = in1 ? xa01 - mu0 : 0.f;
  const float d10 = in0 ? xa10 - mu1 : 0.f, d11 = in1 ? xa11 - mu1 : 0.f;
  const float sp0 = sqrtf(group_sum<GL>(d00 * d00 + d01 * d01) / float(m - 1));
  const float sp1 = sqrtf(group_sum<GL>(d10 * d10 + d11 * d11) / float(m - 1));
  if (wr && li == 0) {
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
#ifdef LK_PHASE_CLOCKS
  __syncwarp();
  LK_PHASE_STAMP(ph4);
  if (lane == 0) {
    atomicAdd(&g_lk_phase_clocks[0], (unsigned long long)(ph1 - ph0));
    atomicAdd(&g_lk_phase_clocks[1], (unsigned long long)(ph2 - ph1));
    atomicAdd(&g_lk_phase_clocks[2], (unsigned long long)(ph3 - ph2));
    atomicAdd(&g_lk_phase_clocks[3], (unsigned long long)(ph4 - ph3));
    atomicAdd(&g_lk_phase_clocks[4], 1ull);
  }
#endif
}

// ---------------------------------------------------------------------------
// Row-split form (MP = 16 and 32): each column's rows are split between two
// lanes, so a node takes 2 MP/2 = MP lanes: lane (h, li) of the node, h = 0, 1
// the row half and li = 0 .. MP/2 - 1 the column pair, holds rows
// [MP h / 2, MP (h + 1) / 2) of columns 2li and 2li + 1. The odd-even network
// runs on each half as on the whole columns; every dot product adds the
// partner half's partial sum (lane ^ MP/2), so both halves compute the same
// rotation. A round's chain (dot product, rotation, column shuffle) is half as
// long and a system has twice as many warps: this pays where the nodes fill
// few warps per SM (latency-bound systems), not where the SMs are full.
template <int MP>
struct SplitCfg {
  static_assert(MP == 16 || MP == 32, "row split for MP = 16 and 32");
  static constexpr int LPN = MP / 2;      // column-pair lanes per half
  static constexpr int GL = MP;           // lanes of a node
  static constexpr int NPW = 32 / GL;     // nodes per warp
  static constexpr int KH = MP / 4;       // float2 per column and lane
};

template <int MP, int TI, int TJ>
struct SplitLaunch {
  static constexpr int threads = TI * TJ * SplitCfg<MP>::GL;
  static constexpr int min_ctas = 65536 / (threads * 128) > 0 ? 65536 / (threads * 128) : 1;
};

template <int MP, int TI, int TJ>
__global__ void __launch_bounds__(SplitLaunch<MP, TI, TJ>::threads, SplitLaunch<MP, TI, TJ>::min_ctas)
    analysis_split_kernel(const LkInst *__restrict__ insts, const LkTile *__restrict__ tiles,
                          float *__restrict__ mean, float *__restrict__ spread, float tol,
                          float stop, int max_sweeps, float kappa_thr, int *__restrict__ counters,
                          int *__restrict__ queue, int2 *__restrict__ worklist, int keep_basis) {
  lk_pdl_wait();
  LK_PHASE_STAMP(ph0);
  using C = PairCfg<MP>;
  using S = SplitCfg<MP>;
  constexpr int KH = S::KH, LPN = S::LPN, GL = S::GL;
  extern __shared__ __align__(16) unsigned char smem[];
  const LkTile tl = tiles[blockIdx.x];
  const LkInst &I = insts[tl.inst];
  const int w = I.w, m = I.m;
  const PairLayout Ly = pair_layout<MP, TI, TJ>(w);
  const int HJ = TJ + w - 1;
  float *halo = reinterpret_cast<float *>(smem);
  float *dh = reinterpret_cast<float *>(smem + Ly.dh);
  float *tap = reinterpret_cast<float *>(smem + Ly.tap);
  stage_pair_tile<MP, TI, TJ>(I, tl.i0, tl.j0, halo, dh, tap);
  __syncthreads();
  LK_PHASE_STAMP(ph1);

  const int lane = threadIdx.x & 31;
  const int grp = lane / GL, gl = lane - grp * GL;   // node of the warp, lane within the node
  const int hh = gl / LPN, li = gl - hh * LPN;       // row half, column pair
  const int node = (threadIdx.x >> 5) * S::NPW + grp;
  const int ti = node / TJ, tj = node - (node / TJ) * TJ;
  const int gi = tl.i0 + ti, gj = tl.j0 + tj;
  int pid = -1;
  if (gi <= I.nsub && gj <= I.nsub) pid = I.pid_map[gi * (I.nsub + 1) + gj];
  float *scr = reinterpret_cast<float *>(smem + Ly.scr) + (size_t)node * C::NODE_SCR;

  // ---- Gram: this half's rows of columns 2li and 2li+1 of A, C d, diagonal of G ----
  float2 P[KH], Q[KH];
#pragma unroll
  for (int k = 0; k < KH; ++k) {
    P[k] = f2(0.f);
    Q[k] = f2(0.f);
  }
  float diag = 0.f, cd0 = 0.f, cd1 = 0.f;
  const float *hwin = halo + (size_t)(ti * HJ + tj) * C::CELLF;
  const float *dwin = dh + (size_t)(ti * HJ + tj) * 2;
  for (int ds = 0; ds < w; ++ds) {
    for (int dt = 0; dt < w; ++dt) {
      const int cell = ds * HJ + dt;
      const float tw = tap[ds * w + dt];
      if (tw == 0.f) continue;                       // outside the taper's support
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float *yv = hwin + (size_t)cell * C::CELLF + c * MP;
        const float2 yl = reinterpret_cast<const float2 *>(yv)[li];
        const float cy0 = tw * yl.x, cy1 = tw * yl.y;
        diag = fmaf(cy0, yl.x, fmaf(cy1, yl.y, diag));
        const float dj = dwin[cell * 2 + c];
        cd0 = fmaf(cy0, dj, cd0);
        cd1 = fmaf(cy1, dj, cd1);
        const float2 c0 = f2(cy0), c1 = f2(cy1);
        const float4 *y4p = reinterpret_cast<const float4 *>(yv) + hh * (KH / 2);
#pragma unroll
        for (int k = 0; k < KH / 2; ++k) {
          const float4 y4 = y4p[k];
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
  const bool active = pid >= 0;
  bool queued = false;
  if (queue) {
    const float trg = group_sum<LPN>(diag);          // the same in both halves
    if (active && 1.f + trg / alpha > kappa_thr) {
      if (gl == 0) {
        worklist[atomicAdd(queue, 1)] = make_int2(tl.inst, pid);
        atomicAdd(&counters[1], 1);
      }
      queued = true;
    }
  }
  const float dP = (2 * li < m) ? alpha : 1.f, dQ = (2 * li + 1 < m) ? alpha : 1.f;
#pragma unroll
  for (int k = 0; k < KH; ++k) {
    if (!active) {
      P[k] = f2(0.f);
      Q[k] = f2(0.f);
    }
    if (hh * KH + k == li) {
      P[k].x = active ? P[k].x + dP : 1.f;
      Q[k].y = active ? Q[k].y + dQ : 1.f;
    }
  }

  // ---- Jacobi sweeps ----
  LK_PHASE_STAMP(ph2);
  const float tol2 = tol * tol, stop2 = stop * stop;
  const int base = grp * GL + hh * LPN;
  const int up = base + (li + 1) % LPN;
  const int dn = base + (li + LPN - 1) % LPN;
  bool conv = !active;
  int sweeps = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (__all_sync(FULL, conv)) break;
    float nP = combine<LPN>(dotk<KH>(P, P)), nQ = combine<LPN>(dotk<KH>(Q, Q));
    bool rotated = false;
    const int su = conv ? lane : up, sd = conv ? lane : dn;
#pragma unroll 2
    for (int r = 0; r < MP / 2; ++r) {
      float cs;
      rotated |= pair_round_even<KH, LPN>(P, Q, nP, nQ, cs, tol2, stop2, conv);
      shfl_cols<KH>(Q, su);
      nQ = __shfl_sync(FULL, nQ, su);
      const float cq = __shfl_sync(FULL, cs, su);
      rotated |= pair_round_odd<KH, LPN>(P, Q, nP, nQ, cs, cq, tol2, stop2, li == LPN - 1, conv);
      shfl_cols<KH>(P, sd);
      nP = __shfl_sync(FULL, nP, sd);
    }
    const unsigned big = __ballot_sync(FULL, rotated);
    const unsigned gmask = (GL == 32) ? 0xffffffffu : (((1u << GL) - 1u) << (grp * GL));
    if (!conv) {
      sweeps = sweep + 1;
      if ((big & gmask) == 0u) conv = true;
    }
  }
  if (active && gl == 0) {
    atomicMax(&counters[2], sweeps);
    atomicAdd(&counters[3], sweeps);
    if (!conv) atomicOr(&counters[0], LK_BIT_NOCONVERGE);
  }

  // ---- eigenpairs: lambda = |b|, v = b / lambda ----
  LK_PHASE_STAMP(ph3);
  const float lP = sqrtf(combine<LPN>(dotk<KH>(P, P)));
  const float lQ = sqrtf(combine<LPN>(dotk<KH>(Q, Q)));
  {
    const float iP = 1.f / lP, iQ = 1.f / lQ;
#pragma unroll
    for (int k = 0; k < KH; ++k) {
      P[k] = mul2(f2(iP), P[k]);
      Q[k] = mul2(f2(iQ), Q[k]);
    }
  }
  {
    // finite on both halves of the two columns: the shuffle runs on every lane
    // (two nodes share a warp when MP = 16, and only one of them may store)
    bool ok = true;
#pragma unroll
    for (int k = 0; k < KH; ++k)
      ok = ok && isfinite(P[k].x) && isfinite(P[k].y) && isfinite(Q[k].x) && isfinite(Q[k].y);
    ok = __shfl_xor_sync(FULL, (int)ok, LPN) && ok;
    if ((keep_basis || queued) && active) {
      float *U = I.basis + (size_t)pid * MP * MP;
#pragma unroll
      for (int k = 0; k < KH; ++k) {
        const int r = hh * KH + k;
        const float2 r0 = ok ? make_float2(P[k].x, Q[k].x) : make_float2(r == li ? 1.f : 0.f, 0.f);
        const float2 r1 = ok ? make_float2(P[k].y, Q[k].y) : make_float2(0.f, r == li ? 1.f : 0.f);
        reinterpret_cast<float2 *>(U + (2 * r) * MP)[li] = r0;
        reinterpret_cast<float2 *>(U + (2 * r + 1) * MP)[li] = r1;
      }
    }
  }

  // ---- transform and apply (Section 4.2): Xa_r = xbar_r + X'_r wbar + X'_r W ----
  float *vcd = scr;
  float *vx0 = vcd + MP;
  float *vx1 = vx0 + MP;
  const bool wr = active && !queued;
  float *xrow = wr ? static_cast<float *>(I.X) + (size_t)pid * 2 * m : nullptr;
  const bool in0 = 2 * li < m, in1 = 2 * li + 1 < m;
  const float x00 = (wr && in0) ? xrow[2 * li] : 0.f;
  const float x01 = (wr && in1) ? xrow[2 * li + 1] : 0.f;
  const float x10 = (wr && in0) ? xrow[m + 2 * li] : 0.f;
  const float x11 = (wr && in1) ? xrow[m + 2 * li + 1] : 0.f;
  const float inv_m = 1.f / float(m);
  const float xb0 = group_sum<LPN>(x00 + x01) * inv_m;
  const float xb1 = group_sum<LPN>(x10 + x11) * inv_m;
  if (hh == 0) {
    reinterpret_cast<float2 *>(vcd)[li] = make_float2(cd0, cd1);
    reinterpret_cast<float2 *>(vx0)[li] = make_float2(in0 ? x00 - xb0 : 0.f, in1 ? x01 - xb0 : 0.f);
    reinterpret_cast<float2 *>(vx1)[li] = make_float2(in0 ? x10 - xb1 : 0.f, in1 ? x11 - xb1 : 0.f);
  }
  __syncwarp();
  float2 uP = f2(0.f), uQ = f2(0.f), a0P = f2(0.f), a0Q = f2(0.f), a1P = f2(0.f), a1Q = f2(0.f);
#pragma unroll
  for (int k = 0; k < KH; ++k) {
    const int r = hh * KH + k;
    const float2 cdv = reinterpret_cast<const float2 *>(vcd)[r];
    const float2 x0v = reinterpret_cast<const float2 *>(vx0)[r];
    const float2 x1v = reinterpret_cast<const float2 *>(vx1)[r];
    uP = fma2(P[k], cdv, uP);
    uQ = fma2(Q[k], cdv, uQ);
    a0P = fma2(P[k], x0v, a0P);
    a0Q = fma2(Q[k], x0v, a0Q);
    a1P = fma2(P[k], x1v, a1P);
    a1Q = fma2(Q[k], x1v, a1Q);
  }
  const float gP0 = combine<LPN>(a0P.x + a0P.y), gQ0 = combine<LPN>(a0Q.x + a0Q.y);
  const float gP1 = combine<LPN>(a1P.x + a1P.y), gQ1 = combine<LPN>(a1Q.x + a1Q.y);
  const float zP = combine<LPN>(uP.x + uP.y) / lP, zQ = combine<LPN>(uQ.x + uQ.y) / lQ;
  const float w0 = group_sum<LPN>(gP0 * zP + gQ0 * zQ);    // X'_0 wbar
  const float w1 = group_sum<LPN>(gP1 * zP + gQ1 * zQ);    // X'_1 wbar
  const float rP = sqrtf(float(m - 1) / lP), rQ = sqrtf(float(m - 1) / lQ);
  // X'_r W: this lane's terms on its half's rows, summed over the half's LPN
  // lanes; lane li < KH of half h ends with row pair h KH + li
  float2 v0[KH], v1[KH];
  {
    const float2 hP0 = f2(gP0 * rP), hQ0 = f2(gQ0 * rQ), hP1 = f2(gP1 * rP), hQ1 = f2(gQ1 * rQ);
#pragma unroll
    for (int k = 0; k < KH; ++k) {
      v0[k] = fma2(hP0, P[k], mul2(hQ0, Q[k]));
      v1[k] = fma2(hP1, P[k], mul2(hQ1, Q[k]));
    }
  }
  float2 q0 = reduce_scatter<KH>(v0, li), q1 = reduce_scatter<KH>(v1, li);
  q0.x += __shfl_xor_sync(FULL, q0.x, KH);
  q0.y += __shfl_xor_sync(FULL, q0.y, KH);
  q1.x += __shfl_xor_sync(FULL, q1.x, KH);
  q1.y += __shfl_xor_sync(FULL, q1.y, KH);
  const int r0 = hh * KH + (li & (KH - 1));
  const bool own = li < KH;
  const bool o0 = own && 2 * r0 < m, o1 = own && 2 * r0 + 1 < m;
  const float xa00 = xb0 + w0 + q0.x, xa01 = xb0 + w0 + q0.y;
  const float xa10 = xb1 + w1 + q1.x, xa11 = xb1 + w1 + q1.y;
  if (wr) {
    if (o0) {
      xrow[2 * r0] = xa00;
      xrow[m + 2 * r0] = xa10;
    }
    if (o1) {
      xrow[2 * r0 + 1] = xa01;
      xrow[m + 2 * r0 + 1] = xa11;
    }
  }
  const float e00 = o0 ? xa00 : 0.f, e01 = o1 ? xa01 : 0.f;
  const float e10 = o0 ? xa10 : 0.f, e11 = o1 ? xa11 : 0.f;
  const float mu0 = group_sum<GL>(e00 + e01) * inv_m;
  const float mu1 = group_sum<GL>(e10 + e11) * inv_m;
  const float d00 = o0 ? xa00 - mu0 : 0.f, d01 = o1 ? xa01 - mu0 : 0.f;
  const float d10 = o0 ? xa10 - mu1 : 0.f, d11 = o1 ? xa11 - mu1 : 0.f;
  const float sp0 = sqrtf(group_sum<GL>(d00 * d00 + d01 * d01) / float(m - 1));
  const float sp1 = sqrtf(group_sum<GL>(d10 * d10 + d11 * d11) / float(m - 1));
  if (wr && gl == 0) {
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
#ifdef LK_PHASE_CLOCKS
  __syncwarp();
  LK_PHASE_STAMP(ph4);
  if (lane == 0) {
    atomicAdd(&g_lk_phase_clocks[0], (unsigned long long)(ph1 - ph0));
    atomicAdd(&g_lk_phase_clocks[1], (unsigned long long)(ph2 - ph1));
    atomicAdd(&g_lk_phase_clocks[2], (unsigned long long)(ph3 - ph2));
    atomicAdd(&g_lk_phase_clocks[3], (unsigned long long)(ph4 - ph3));
    atomicAdd(&g_lk_phase_clocks[4], 1ull);
  }
#endif
}

// A tile fills whole warps (its node count is a multiple of the nodes per
// warp), and wide problems (one node per warp) take tiles of at most 8 nodes:
// a 16-warp CTA would leave fewer registers per thread than the two columns need.
template <int MP, int TI, int TJ>
constexpr bool shape_ok() {
  return (TI * TJ) % PairCfg<MP>::NPW == 0 && (PairCfg<MP>::NPW > 1 || TI * TJ <= 8);
}
// The row-split form: whole warps of nodes (two per warp for MP = 16).
template <int MP, int TI, int TJ>
constexpr bool split_shape_ok() {
  if constexpr (MP != 16 && MP != 32) return false;
  else return (TI * TJ) % SplitCfg<MP>::NPW == 0;
}

// The instances a kernel of width MP serves: MP = 24 those of the m <= 32
// class with at most 24 members, MP = 32 that class (its tile list decides
// which), otherwise the instances padded to MP.
template <int MP>
bool serves(const LkInst &I) {
  if constexpr (MP == 24) return I.mp == 32 && I.m <= 24;
  else return I.mp == MP;
}

template <int MP, int TI, int TJ, bool SPLIT>
cudaError_t launch_shape(letkf_ctx *h, const LkTile *tiles, int n_tiles, float *mean,
                         float *spread, float kthr, int *queue, int2 *worklist) {
  if (n_tiles == 0) return cudaSuccess;
  if constexpr (SPLIT ? !split_shape_ok<MP, TI, TJ>() : !shape_ok<MP, TI, TJ>()) {
    return cudaErrorInvalidConfiguration;
  } else {
  size_t need = 0;
  for (const LkInst &I : h->inst)
    if (serves<MP>(I)) {
      const size_t b = pair_layout<MP, TI, TJ>(I.w).total;
      need = b > need ? b : need;
    }
  if constexpr (SPLIT)
    return lk_launch_pdl(analysis_split_kernel<MP, TI, TJ>, n_tiles,
                         SplitLaunch<MP, TI, TJ>::threads, need, h->stream, h->d_inst, tiles, mean,
                         spread, (float)h->tol32, (float)h->stop32, h->max_sweeps, kthr,
                         h->counters, queue, worklist, h->keep_basis);
  else
    return lk_launch_pdl(analysis_pair_kernel<MP, TI, TJ>, n_tiles,
                         TI * TJ * 32 / PairCfg<MP>::NPW, need, h->stream, h->d_inst, tiles, mean,
                         spread, (float)h->tol32, (float)h->stop32, h->max_sweeps, kthr,
                         h->counters, queue, worklist, h->keep_basis);
  }
}

template <int MP>
cudaError_t launch_mp(letkf_ctx *h, int cls, const LkTile *tiles, int n_tiles, float *mean,
                      float *spread) {
  const float kthr = h->fp64_kappa > 0 ? (float)h->fp64_kappa : 0.f;
  int *queue = kthr > 0.f ? h->counters + 4 + cls : nullptr;
  int2 *wl = h->worklist + (size_t)cls * h->n_pts_total;
  const bool split = (MP == 16 || MP == 32) && h->row_split[cls] == 2;
  switch (h->tile_shape[cls]) {
#define LK_CASE(id, ti, tj)                                                                   \
  case id:                                                                                    \
    return split ? launch_shape<MP, ti, tj, true>(h, tiles, n_tiles, mean, spread, kthr, queue, \
                                                  wl)                                         \
                 : launch_shape<MP, ti, tj, false>(h, tiles, n_tiles, mean, spread, kthr, queue, \
                                                   wl);
    LK_FOR_SHAPES(LK_CASE)
#undef LK_CASE
  }
  return cudaErrorInvalidValue;
}

// FP64 handles: the FP32 basis pass over one width class (MP = 16 or 32).
template <int MP, int TI, int TJ>
cudaError_t launch_basis_shape(letkf_ctx *h, int cls) {
  if (h->n_tiles[cls] == 0) return cudaSuccess;
  if constexpr (!shape_ok<MP, TI, TJ>()) {
    return cudaErrorInvalidConfiguration;
  } else {
    size_t need = 0;
    for (const LkInst &I : h->inst)
      if (I.mp == MP) {
        const size_t b = pair_layout<MP, TI, TJ>(I.w).total;
        need = b > need ? b : need;
      }
    return lk_launch_pdl(analysis_pair_kernel<MP, TI, TJ, double, true>, h->n_tiles[cls],
                         TI * TJ * 32 / PairCfg<MP>::NPW, need, h->stream, h->d_inst,
                         h->tiles[cls], (float *)nullptr, (float *)nullptr, (float)h->tol32,
                         (float)h->stop32, h->max_sweeps, 0.f, h->counters, (int *)nullptr,
                         (int2 *)nullptr, 1);
  }
}

template <int MP>
cudaError_t launch_basis(letkf_ctx *h, int cls) {
  switch (h->tile_shape[cls]) {
#define LK_CASE(id, ti, tj) \
  case id:                  \
    return launch_basis_shape<MP, ti, tj>(h, cls);
    LK_FOR_SHAPES(LK_CASE)
#undef LK_CASE
  }
  return cudaErrorInvalidValue;
}

template <int MP, int TI, int TJ>
cudaError_t set_shape_smem(int w, bool fp64) {
  const int bytes = (int)pair_layout<MP, TI, TJ>(w).total;
  cudaError_t e = cudaSuccess;
  if constexpr (shape_ok<MP, TI, TJ>()) {
    if (fp64) {
      if constexpr (MP == 16 || MP == 32)
        e = cudaFuncSetAttribute(analysis_pair_kernel<MP, TI, TJ, double, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      return e;
    }
    e = cudaFuncSetAttribute(analysis_pair_kernel<MP, TI, TJ>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  }
  if constexpr (split_shape_ok<MP, TI, TJ>())
    if (e == cudaSuccess && !fp64)
      e = cudaFuncSetAttribute(analysis_split_kernel<MP, TI, TJ>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

template <int MP>
cudaError_t setup_mp(letkf_ctx *h) {
  int wmax = 0;
  for (const LkInst &I : h->inst)
    if (serves<MP>(I)) wmax = I.w > wmax ? I.w : wmax;
  if (wmax == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
#define LK_SET(id, ti, tj) \
  if (e == cudaSuccess) e = set_shape_smem<MP, ti, tj>(wmax, h->precision == 1);
  LK_FOR_SHAPES(LK_SET)
#undef LK_SET
  return e;
}

}  // namespace

// Class 0: MP = 16; class 1: tiles of instances with m <= 24 first (tile_split
// of them, none in the row-split form) on MP = 24, then MP = 32; class 2: tiles
// of MP = 64 instances first, then MP = 48.
cudaError_t lk_launch_pair(letkf_ctx *h, int cls, void *mean, void *spread) {
  float *mo = static_cast<float *>(mean), *so = static_cast<float *>(spread);
  if (cls == 0) return launch_mp<16>(h, 0, h->tiles[0], h->n_tiles[0], mo, so);
  if (cls == 1) {
    const int n24 = h->tile_split[1];
    cudaError_t e = launch_mp<24>(h, 1, h->tiles[1], n24, mo, so);
    if (e == cudaSuccess)
      e = launch_mp<32>(h, 1, h->tiles[1] + n24, h->n_tiles[1] - n24, mo, so);
    return e;
  }
  const int split = h->tile_split[2];
  cudaError_t e = launch_mp<64>(h, 2, h->tiles[2], split, mo, so);
  if (e == cudaSuccess)
    e = launch_mp<48>(h, 2, h->tiles[2] + split, h->n_tiles[2] - split, mo, so);
  return e;
}

bool lk_shape_ok(const letkf_ctx *h, int cls, int shape) {
  return lk_shape_split_ok(h, cls, shape, h->row_split[cls]);
}

bool lk_shape_split_ok(const letkf_ctx *h, int cls, int shape, int split) {
  int ti, tj;
  lk_tile_shape(shape, &ti, &tj);
  // FP64 handles analyse one node per CTA; their FP32 basis pass takes the
  // tiles of the whole-column form
  if (h->precision == 1 && split != 1) return false;
  if (split == 2) {
    switch (cls) {
      case 0: return (ti * tj) % SplitCfg<16>::NPW == 0;
      case 1: return (ti * tj) % SplitCfg<32>::NPW == 0;
      default: return false;
    }
  }
  switch (cls) {
    case 0: return (ti * tj) % PairCfg<16>::NPW == 0;
    case 1: return (ti * tj) % PairCfg<32>::NPW == 0;
    default: return ti * tj <= 8;
  }
}

cudaError_t lk_launch_pair_basis(letkf_ctx *h, int cls) {
  if (cls == 0) return launch_basis<16>(h, 0);
  if (cls == 1) return launch_basis<32>(h, 1);
  return cudaErrorInvalidValue;              // FP64 handles hold m <= 32
}

cudaError_t lk_setup_pair(letkf_ctx *h) {
  cudaError_t e = setup_mp<16>(h);
  if (e == cudaSuccess && h->precision == 0) e = setup_mp<24>(h);
  if (e == cudaSuccess) e = setup_mp<32>(h);
  if (e == cudaSuccess) e = setup_mp<48>(h);
  if (e == cudaSuccess) e = setup_mp<64>(h);
  return e;
}

extern "C" letkf_status letkf_phase_clocks(uint64_t *out) {
#ifdef LK_PHASE_CLOCKS
  if (!out) return LETKF_ERR_ARG;
  unsigned long long v[5] = {0, 0, 0, 0, 0};
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(v, g_lk_phase_clocks, sizeof(v));
  const unsigned long long z[5] = {0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_lk_phase_clocks, z, sizeof(z));
  if (e != cudaSuccess) return LETKF_ERR_CUDA;
  for (int i = 0; i < 5; ++i) out[i] = v[i];
  return LETKF_OK;
#else
  (void)out;
  return LETKF_ERR_STATE;
#endif
}
