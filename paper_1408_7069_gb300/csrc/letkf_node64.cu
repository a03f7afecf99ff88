// FP64 local analysis of one node per CTA (Section 4.2 with Section 3.1 and
// Appendix A), for FP64 handles and for the nodes of FP32 handles whose
// kappa_hat sent them to FP64.
//
// GB300's FP64 rate is 0.5 FMA per clock per SMSP, so a warp-wide FP64
// instruction holds its SMSP for about 64 clocks: one warp per node leaves
// three of an SM's four FP64 units idle and puts every row of the node on one
// instruction stream. Here a CTA of four warps holds one node, with the rows
// of every column split over them:
//   thread t: column c = t % MP, row block rb = t / MP (MP = 32: four blocks of
//   8 rows, one per warp; MP = 16: eight blocks of 2 rows, two per warp).
// A column's partner in a Jacobi step (c ^ step) sits in the same warp and row
// block, so the rotation exchanges rows by shuffles; only the per-column sums
// (dot products, norms, projections) cross row blocks, through shared memory,
// in a fixed order and with one barrier each. Every thread of a column
// computes the same rotation from the same sums, so the result does not depend
// on which block holds which rows.
//
//   Gram   A = (m-1)/rho I + sum_j tau_j/sigma2 Yb_j Yb_j^T, C d   (FP64, from the grid)
//   EVD    one-sided Jacobi on the columns of B = A V, V accumulated: from the
//          identity, or from a stored FP32 eigenbasis made orthonormal by
//          Newton-Schulz steps (one for the queued nodes of FP32 handles, two
//          for FP64 handles, whose FP32 basis pass precedes this kernel)
//   apply  wbar = V Lambda^-1 V^T C d, W = V ((m-1) Lambda^-1)^(1/2) V^T,
//          Xa_r = xbar_r + X'_r wbar + X'_r W for the node's two rows
#include <math.h>

#include <atomic>

#include "letkf_device.cuh"

namespace {

constexpr int N64_THREADS = 128;

template <int MP>
struct N64 {
  static constexpr int NB = N64_THREADS / MP;   // row blocks
  static constexpr int RB = MP / NB;            // rows per thread
  static constexpr int LD = MP + 1;             // shared-memory row stride of the matrices
};

// Shared memory of one CTA, in doubles: three [MP][LD] matrices (A, V, and the
// Newton-Schulz product or the output staging), the double-buffered column
// sums [2][NB][MP] and eight vectors of MP.
template <int MP>
__host__ __device__ constexpr size_t n64_smem_doubles() {
  // A, V, G; the column sums; 8 vectors; FP32 copies of V and of I - G (one
  // [MP][LD] double array holds both)
  return 4 * (size_t)MP * N64<MP>::LD + 2 * (size_t)N64<MP>::NB * MP + 8 * (size_t)MP;
}

template <int MP>
struct N64Smem {
  double *As, *Vs, *Gs, *red, *vec;
  float *Vf, *Ef;
  __device__ explicit N64Smem(double *base) {
    constexpr int LD = N64<MP>::LD;
    As = base;
    Vs = As + MP * LD;
    Gs = Vs + MP * LD;
    red = Gs + MP * LD;
    vec = red + 2 * N64<MP>::NB * MP;
    Vf = reinterpret_cast<float *>(vec + 8 * MP);
    Ef = Vf + MP * LD;
  }
};

// Sum over the row blocks of column c of the per-thread partial x, in block
// order; every thread of the column gets the same value. One barrier; the two
// buffers alternate, so a fast warp cannot overwrite sums a slow one still reads.
template <int MP>
__device__ __forceinline__ double colsum(double x, double *red, int &buf) {
  constexpr int NB = N64<MP>::NB;
  const int c = threadIdx.x % MP, rb = threadIdx.x / MP;
  double *r = red + (size_t)buf * NB * MP;
  r[rb * MP + c] = x;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < NB; ++q) s += r[q * MP + c];
  buf ^= 1;
  return s;
}

// The node's analysis. S: storage type of the grid, ensemble and outputs;
// WARM: start the sweep from the FP32 basis U (row-major MP x MP) instead of
// the identity; stop: see jacobi().
// WARM: ns_steps Newton-Schulz steps make the stored FP32 basis orthonormal
// before the sweep. Each squares the orthogonality error: the FP32 eigensolve
// leaves about 1e-6 (its last sweep rotated by cosines up to 1e-3), so one step
// gives about 1e-12, enough for FP32 outputs, and two reach FP64 rounding,
// which the FP64 outputs need (the Jacobi rotations keep whatever error V
// starts with, and W = V Lambda^-1/2 V^T inherits it). A step is
// V <- V + V E / 2 with E = I - V^T V: V^T V in FP64, since E is what is left of
// it, but the product V E in FP32, since it is a correction of size |E| that
// FP32 carries to |E| eps32 (1e-13 after the first step, 1e-19 after the second).
// The FP64 FMAs of a step halve.
template <int MP, typename S, bool WARM>
__device__ void node64(const LkInst &I, int pid, S *__restrict__ mean_out,
                       S *__restrict__ spread_out, double tol, double stop, int max_sweeps,
                       int *__restrict__ counters, double *smem, bool keep_basis = false,
                       int ns_steps = 1) {
  constexpr int NB = N64<MP>::NB, RB = N64<MP>::RB, LD = N64<MP>::LD;
  const int tid = threadIdx.x, c = tid % MP, rb = tid / MP, r0 = rb * RB;
  const int m = I.m, w = I.w;
  N64Smem<MP> sm(smem);
  int buf = 0;

  // ---- Gram: rows r0 .. r0+RB-1 of column c of A, and (C d)_c ----
  const int2 ij = I.pts[pid];
  const S *Ybp = static_cast<const S *>(I.Ybp);
  const S *dp = static_cast<const S *>(I.dp);
  const S *taper = static_cast<const S *>(I.taper);
  double b[RB], v[RB];
#pragma unroll
  for (int i = 0; i < RB; ++i) b[i] = 0.0;
  double cd = 0.0;
  for (int ds = 0; ds < w; ++ds) {
    for (int dt = 0; dt < w; ++dt) {
      const size_t src = (size_t)(ij.x + ds) * I.gs_cols + (ij.y + dt);
      const double tw = (double)taper[ds * w + dt];
      if (tw == 0.0) continue;                       // outside the taper's support
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const S *yv = Ybp + (src * 2 + cc) * m;
        const double yc = c < m ? (double)yv[c] : 0.0;
        const double cy = tw * yc;
        cd = fma(cy, (double)dp[src * 2 + cc], cd);
#pragma unroll
        for (int i = 0; i < RB; ++i) {
          const int r = r0 + i;
          b[i] = fma(cy, r < m ? (double)yv[r] : 0.0, b[i]);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < RB; ++i)
    if (r0 + i == c) b[i] += c < m ? I.alpha : 1.0;   // (m-1)/rho I, identity on the padding

  // ---- starting basis ----
  if constexpr (WARM) {
    // V from the FP32 basis; ns_steps x (V <- V (3I - V^T V)/2); B = A V
    const float *U = I.basis + (size_t)pid * MP * MP;
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      v[i] = (double)U[(r0 + i) * MP + c];
      sm.As[(r0 + i) * LD + c] = b[i];
      sm.Vs[(r0 + i) * LD + c] = v[i];
    }
    __syncthreads();
    for (int step = 0; step < ns_steps; ++step) {
#pragma unroll
      for (int i = 0; i < RB; ++i) {                 // G[j][c] = (V^T V)[j][c], j in my rows
        const int j = r0 + i;
        double g = 0.0;
#pragma unroll 8
        for (int k = 0; k < MP; ++k) g = fma(sm.Vs[k * LD + j], sm.Vs[k * LD + c], g);
        sm.Gs[j * LD + c] = g;
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < RB; ++i) {                 // FP32 copies of E = I - G and of V
        const int j = r0 + i;
        sm.Ef[j * LD + c] = (float)((j == c ? 1.0 : 0.0) - sm.Gs[j * LD + c]);
        sm.Vf[j * LD + c] = (float)v[i];
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < RB; ++i) {                 // V'[r][c] = V[r][c] + 0.5 (V E)[r][c]
        const int r = r0 + i;
        float t = 0.f;
#pragma unroll 8
        for (int j = 0; j < MP; ++j) t = fmaf(sm.Vf[r * LD + j], sm.Ef[j * LD + c], t);
        v[i] = fma(0.5, (double)t, v[i]);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < RB; ++i) sm.Vs[(r0 + i) * LD + c] = v[i];
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RB; ++i) {                   // B[r][c] = (A V')[r][c]
      const int r = r0 + i;
      double t = 0.0;
#pragma unroll 8
      for (int k = 0; k < MP; ++k) t = fma(sm.As[r * LD + k], sm.Vs[k * LD + c], t);
      b[i] = t;
    }
  } else {
#pragma unroll
    for (int i = 0; i < RB; ++i) v[i] = (r0 + i == c) ? 1.0 : 0.0;
  }

  // ---- sweeps (the rotation of jacobi_step, rows split over the blocks) ----
  // Per step: every thread shuffles in its partner's rows and forms its part of
  // the pair's dot product; warp 0 alone (lane = column) adds the parts, keeps
  // the column norms and computes the rotations, which every thread then reads
  // back and applies to its rows. The rotation's FP64 chain thus runs once per
  // node instead of once per warp. Two barriers per step (parts written, then
  // rotations written); between them a single buffer each for the parts (red)
  // and the rotations (rot) is race-free.
  if (stop < tol) stop = tol;
  double *rot = sm.vec;                      // [2][MP]: c, signed s of each column's rotation
  const bool w0 = tid < 32;
  const int cw = tid % MP;                   // warp 0: its lane's column
  int sweep = 0;
  bool converged = false;
  for (; sweep < max_sweeps; ++sweep) {
    double part = 0.0;
#pragma unroll
    for (int i = 0; i < RB; ++i) part = fma(b[i], b[i], part);
    sm.red[rb * MP + c] = part;
    __syncthreads();
    double nrm = 0.0;
    if (w0)
      for (int q = 0; q < NB; ++q) nrm += sm.red[q * MP + cw];
    int flags = 0;
    for (int t = 1; t < MP; ++t) {
      double pb[RB];
#pragma unroll
      for (int i = 0; i < RB; ++i) pb[i] = __shfl_xor_sync(FULL, b[i], t);
      double pd = 0.0;
#pragma unroll
      for (int i = 0; i < RB; ++i) pd = fma(b[i], pb[i], pd);
      if (t == 1) __syncthreads();           // warp 0 has read the sweep's norms
      sm.red[rb * MP + c] = pd;
      __syncthreads();
      if (w0) {
        double dot = 0.0;
        for (int q = 0; q < NB; ++q) dot += sm.red[q * MP + cw];
        const double pn = __shfl_xor_sync(FULL, nrm, t);
        const bool isp = cw < (cw ^ t);      // column p of the pair (p < q)
        const double app = isp ? nrm : pn, aqq = isp ? pn : nrm;
        const double scale = sqrt(app * aqq);
        double cs = 1.0, sn = 0.0, tr = 0.0;
        if (fabs(dot) > tol * scale) {
          // the tangent t of the rotation angle (|theta| <= pi/4) in FP32, from
          // x = aqq - app and y = 2 dot formed in FP64: cos 2theta = |x|/h,
          // c^2 = (1 + cos 2theta)/2, t = sin 2theta / (2 c^2), h = sqrt(x^2 + y^2).
          // Then c = (1 + t^2)^-1/2 and s = c t in FP64, so the rotation is
          // orthogonal to FP64 rounding; an FP32-accurate angle leaves the pair's
          // cosine at ~1e-7 of its value, which the next sweep removes.
          const float x = (float)(aqq - app), y = (float)(2.0 * dot);
          const float rh = lk_rsqrt_normal(fmaxf(fmaf(x, x, y * y), 1e-37f));
          const float c2 = fmaf(0.5f * fabsf(x), rh, 0.5f);
          const float t = (x >= 0.f ? y : -y) * (0.5f * rh) / c2;
          tr = (double)t;
          cs = rsqrt(fma(tr, tr, 1.0));
          sn = cs * tr;
          flags |= fabs(dot) > stop * scale ? 3 : 1;
        }
        nrm = isp ? (app - tr * dot) : (aqq + tr * dot);
        if (tid < MP) {
          rot[cw] = cs;
          rot[MP + cw] = isp ? -sn : sn;     // p' = c p - s q ; q' = s p + c q
        }
      }
      __syncthreads();
      const double cs = rot[c], sg = rot[MP + c];
#pragma unroll
      for (int i = 0; i < RB; ++i) b[i] = fma(sg, pb[i], cs * b[i]);
      double pv[RB];
#pragma unroll
      for (int i = 0; i < RB; ++i) pv[i] = __shfl_xor_sync(FULL, v[i], t);
#pragma unroll
      for (int i = 0; i < RB; ++i) v[i] = fma(sg, pv[i], cs * v[i]);
    }
    if (!__syncthreads_or(flags & 2)) {
      converged = true;
      break;
    }
  }
  if (tid == 0) {
    atomicMax(&counters[2], converged ? sweep + 1 : sweep);
    atomicAdd(&counters[3], converged ? sweep + 1 : sweep);
    if (!converged) atomicOr(&counters[0], LK_BIT_NOCONVERGE);
  }
  if (keep_basis) {
    // the eigenvectors for the reverse mode: in FP64 on FP64 handles (it takes
    // them as they are), else rounded to FP32 (it refines them in FP64 instead
    // of sweeping from the identity again)
    if (I.basis64) {
      double *U = I.basis64 + (size_t)pid * MP * MP;
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        const int r = r0 + i;
        U[r * MP + c] = isfinite(v[i]) ? v[i] : (r == c ? 1.0 : 0.0);
      }
    } else {
      float *U = I.basis + (size_t)pid * MP * MP;
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        const int r = r0 + i;
        U[r * MP + c] = isfinite(v[i]) ? (float)v[i] : (r == c ? 1.f : 0.f);
      }
    }
  }
  __syncthreads();                           // rot (in vec) is reused below

  // ---- weights and update: lambda_c = |B e_c|, column c of V is v ----
  double part = 0.0;
#pragma unroll
  for (int i = 0; i < RB; ++i) part = fma(b[i], b[i], part);
  const double nb = colsum<MP>(part, sm.red, buf);
  const double lam = nb > 0.0 ? sqrt(nb) : 1.0;
  S *xrow = static_cast<S *>(I.X) + (size_t)pid * 2 * m;
  double *cdv = sm.vec, *xs0 = cdv + MP, *xs1 = xs0 + MP;
  double *gz0 = xs1 + MP, *gz1 = gz0 + MP, *gs0 = gz1 + MP, *gs1 = gs0 + MP;
  if (rb == 0) {
    cdv[c] = cd;
    xs0[c] = c < m ? (double)xrow[c] : 0.0;
    xs1[c] = c < m ? (double)xrow[m + c] : 0.0;
  }
  __syncthreads();
  double xb0 = 0.0, xb1 = 0.0;
  for (int j = 0; j < MP; ++j) {
    xb0 += xs0[j];
    xb1 += xs1[j];
  }
  const double inv_m = 1.0 / m;
  xb0 *= inv_m;
  xb1 *= inv_m;
  double pu = 0.0, p0 = 0.0, p1 = 0.0;
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    const int r = r0 + i;
    pu = fma(v[i], cdv[r], pu);                           // (V^T C d)_c
    p0 = fma(v[i], r < m ? xs0[r] - xb0 : 0.0, p0);       // (X'_0 V)_c
    p1 = fma(v[i], r < m ? xs1[r] - xb1 : 0.0, p1);
  }
  const double u = colsum<MP>(pu, sm.red, buf);
  const double g0 = colsum<MP>(p0, sm.red, buf);
  const double g1 = colsum<MP>(p1, sm.red, buf);
  // every eigenvector gets its root: a warm start leaves the padding's unit
  // eigenvectors (lambda = 1) in arbitrary columns, and their g0, g1 are zero
  const double z = u / lam, sroot = sqrt((m - 1) / lam);
  if (rb == 0) {
    gz0[c] = g0 * z;
    gz1[c] = g1 * z;
    gs0[c] = g0 * sroot;
    gs1[c] = g1 * sroot;
  }
  __syncthreads();
  // (X'_r W)_j = sum_c V[j][c] g_r,c sroot_c: the terms, then a row sum per member
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    const int r = r0 + i;
    sm.Gs[r * LD + c] = v[i] * gs0[c];
    sm.As[r * LD + c] = v[i] * gs1[c];
  }
  __syncthreads();
  if (tid < 32) {
    const int j = tid;
    const bool mem = j < m;
    double q0 = 0.0, q1 = 0.0, P0 = 0.0, P1 = 0.0;
    if (j < MP) {
      for (int k = 0; k < MP; ++k) {
        q0 += sm.Gs[j * LD + k];
        q1 += sm.As[j * LD + k];
      }
    }
    for (int k = 0; k < MP; ++k) {                        // X'_r wbar
      P0 += gz0[k];
      P1 += gz1[k];
    }
    const double xa0 = xb0 + P0 + q0, xa1 = xb1 + P1 + q1;
    if (mem) {
      xrow[j] = S(xa0);
      xrow[m + j] = S(xa1);
    }
    const double mu0 = lk_warp_sum(mem ? xa0 : 0.0) * inv_m;
    const double mu1 = lk_warp_sum(mem ? xa1 : 0.0) * inv_m;
    const double e0 = mem ? xa0 - mu0 : 0.0, e1 = mem ? xa1 - mu1 : 0.0;
    const double sp0 = sqrt(lk_warp_sum(e0 * e0) / (m - 1));
    const double sp1 = sqrt(lk_warp_sum(e1 * e1) / (m - 1));
    if (j == 0) {
      if (mean_out) {
        mean_out[0] = S(mu0);
        mean_out[1] = S(mu1);
      }
      if (spread_out) {
        spread_out[0] = S(sp0);
        spread_out[1] = S(sp1);
      }
      if (!isfinite(mu0) || !isfinite(mu1) || !isfinite(sp0) || !isfinite(sp1))
        atomicOr(&counters[0], LK_BIT_NONFINITE);
    }
  }
}

// FP64 handles: one CTA per node of width class MP (items: every node of the
// handle; nodes of the other class leave at once). WARM: the sweep starts from
// the FP32 eigenbasis the basis pass of the pair kernel stored (made
// orthonormal to FP64 rounding by two Newton-Schulz steps) and stops after a
// sweep whose cosines all stay below LK_WARM_STOP64; otherwise from the
// identity, with a last sweep without rotations.
template <int MP, typename S, bool WARM>
__global__ void __launch_bounds__(N64_THREADS)
    node64_kernel(const LkInst *__restrict__ insts, const int2 *__restrict__ items,
                  S *__restrict__ mean, S *__restrict__ spread, double tol, int max_sweeps,
                  int *__restrict__ counters, int keep_basis) {
  extern __shared__ __align__(16) double n64_smem[];
  lk_pdl_wait();   // no early trigger (long kernel): dependents launch as its CTAs exit
  const int2 it = items[blockIdx.x];
  const LkInst &I = insts[it.x];
  if (I.mp != MP) return;
  const long long row = I.node_off + it.y;
  node64<MP, S, WARM>(I, it.y, mean ? mean + 2 * row : nullptr, spread ? spread + 2 * row : nullptr,
                      tol, WARM ? LK_WARM_STOP64 : 0.0, max_sweeps, counters, n64_smem,
                      keep_basis != 0, 2);
}

// FP32 handles: the nodes the pair kernel queued, a fixed grid of CTAs walking
// the queue, each sweep started from the node's stored FP32 basis.
template <int MP>
__global__ void __launch_bounds__(N64_THREADS)
    node64_list_kernel(const LkInst *__restrict__ insts, const int2 *__restrict__ worklist,
                       const int *__restrict__ queue_len, float *__restrict__ mean,
                       float *__restrict__ spread, double tol, int max_sweeps,
                       int *__restrict__ counters) {
  extern __shared__ __align__(16) double n64_smem[];
  lk_pdl_wait();   // no early trigger (long kernel): dependents launch as its CTAs exit
  const int qn = *queue_len;
  for (int idx = blockIdx.x; idx < qn; idx += gridDim.x) {
    const int2 it = worklist[idx];
    const LkInst &I = insts[it.x];
    const long long row = I.node_off + it.y;
    node64<MP, float, true>(I, it.y, mean ? mean + 2 * row : nullptr,
                            spread ? spread + 2 * row : nullptr, tol, LK_WARM_STOP64, max_sweeps,
                            counters, n64_smem);
    __syncthreads();                       // shared memory is reused by the next node
  }
}

// ---------------------------------------------------------------------------
// FP64 fallback of the wide class (m = 33..64): the nodes the pair kernel
// queued for MP = 48 and MP = 64, both padded to 64 columns here (identity on
// the padding). One CTA of eight warps per node: thread t holds column
// c = t % 64 of a row block rb = t / 64 of 16 rows (two warps per block).
// The partner column c ^ t of a Jacobi step lies in the other warp of the
// block for t >= 32, so columns are exchanged through shared memory, not by
// shuffles. The eigensolve is one-sided Jacobi on B = A V0 alone, V0 the
// node's stored FP32 eigenbasis made orthonormal by one Newton-Schulz step:
// for A > 0 the converged columns are lambda_c q_c, so q_c = b_c / |b_c|
// needs no accumulated V (the lost relative accuracy of the small eigenpairs,
// about eps64 kappa_hat, stays far below the FP32 outputs).
// ---------------------------------------------------------------------------
constexpr int N64W_MP = 64;
constexpr int N64W_THREADS = 256;
constexpr int N64W_NB = N64W_THREADS / N64W_MP;   // 4 row blocks
constexpr int N64W_RB = N64W_MP / N64W_NB;        // 16 rows per thread
constexpr int N64W_LD = N64W_MP + 1;

// Shared memory in doubles: three [64][65] matrices (A, V and G during the
// Newton-Schulz step; B exchange and output terms later), column sums [2][4][64],
// 12 vectors of 64.
__host__ __device__ constexpr size_t n64w_smem_doubles() {
  return 3 * (size_t)N64W_MP * N64W_LD + 2 * (size_t)N64W_NB * N64W_MP + 12 * (size_t)N64W_MP;
}

// Sum over the row blocks of column c (every thread of the column gets it).
__device__ __forceinline__ double colsum_w(double x, double *red, int &buf) {
  const int c = threadIdx.x % N64W_MP, rb = threadIdx.x / N64W_MP;
  double *r = red + (size_t)buf * N64W_NB * N64W_MP;
  r[rb * N64W_MP + c] = x;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < N64W_NB; ++q) s += r[q * N64W_MP + c];
  buf ^= 1;
  return s;
}

__device__ void node64w(const LkInst &I, int pid, float *__restrict__ mean_out,
                        float *__restrict__ spread_out, double tol, double stop, int max_sweeps,
                        int *__restrict__ counters, double *smem) {
  constexpr int MP = N64W_MP, NB = N64W_NB, RB = N64W_RB, LD = N64W_LD;
  const int tid = threadIdx.x, c = tid % MP, rb = tid / MP, r0 = rb * RB;
  const int m = I.m, w = I.w, ms = I.mp;        // ms: width of the stored basis (48 or 64)
  double *M0 = smem, *M1 = M0 + MP * LD, *M2 = M1 + MP * LD;
  double *red = M2 + MP * LD, *vec = red + 2 * NB * MP;
  int buf = 0;

  // ---- Gram (FP64): rows r0 .. r0+RB-1 of column c of A, and (C d)_c ----
  const int2 ij = I.pts[pid];
  const float *Ybp = static_cast<const float *>(I.Ybp);
  const float *dp = static_cast<const float *>(I.dp);
  const float *taper = static_cast<const float *>(I.taper);
  double b[RB];
#pragma unroll
  for (int i = 0; i < RB; ++i) b[i] = 0.0;
  double cd = 0.0;
  for (int ds = 0; ds < w; ++ds) {
    for (int dt = 0; dt < w; ++dt) {
      const size_t src = (size_t)(ij.x + ds) * I.gs_cols + (ij.y + dt);
      const double tw = (double)taper[ds * w + dt];
      if (tw == 0.0) continue;                       // outside the taper's support
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const float *yv = Ybp + (src * 2 + cc) * m;
        const double cy = tw * (c < m ? (double)yv[c] : 0.0);
        cd = fma(cy, (double)dp[src * 2 + cc], cd);
#pragma unroll
        for (int i = 0; i < RB; ++i) {
          const int r = r0 + i;
          b[i] = fma(cy, r < m ? (double)yv[r] : 0.0, b[i]);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < RB; ++i)
    if (r0 + i == c) b[i] += c < m ? I.alpha : 1.0;

  // ---- V0: stored FP32 basis (ms x ms, row-major), identity beyond ms ----
  const float *U = I.basis + (size_t)pid * ms * ms;
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    const int r = r0 + i;
    M0[r * LD + c] = b[i];                                       // A
    M1[r * LD + c] = (r < ms && c < ms) ? (double)U[r * ms + c] : (r == c ? 1.0 : 0.0);
  }
  __syncthreads();
  // Newton-Schulz: V <- V (3I - V^T V) / 2; G = V^T V in M2
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    const int j = r0 + i;
    double g = 0.0;
    for (int k = 0; k < MP; ++k) g = fma(M1[k * LD + j], M1[k * LD + c], g);
    M2[j * LD + c] = g;
  }
  __syncthreads();
  double v[RB];
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    const int r = r0 + i;
    double t = 0.0;
    for (int j = 0; j < MP; ++j) t = fma(M1[r * LD + j], M2[j * LD + c], t);
    v[i] = fma(-0.5, t, 1.5 * M1[r * LD + c]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < RB; ++i) M1[(r0 + i) * LD + c] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < RB; ++i) {                                // B = A V
    const int r = r0 + i;
    double t = 0.0;
    for (int k = 0; k < MP; ++k) t = fma(M0[r * LD + k], M1[k * LD + c], t);
    b[i] = t;
  }
  __syncthreads();                     // M0 / M1 are reused as the exchange buffer

  // ---- B-only sweeps, pairs (c, c ^ t) for t = 1 .. 63 ----
  // Per step: B to shared memory, partner rows read back, partial dots summed
  // over the row blocks by the 64 threads of block 0 (thread = column), which
  // compute the rotation and the new tracked norm; every thread then applies
  // the rotation to its rows. Three barriers per step.
  if (stop < tol) stop = tol;
  double *Bx = M0;
  double *rot = vec;                   // [2][64]: c, signed s
  double *nrm_s = vec + 2 * MP;        // [64] tracked squared norms
  const bool lead = tid < MP;          // block 0: thread = column
  int sweep = 0;
  bool converged = false;
  for (; sweep < max_sweeps; ++sweep) {
    double part = 0.0;
#pragma unroll
    for (int i = 0; i < RB; ++i) part = fma(b[i], b[i], part);
    const double nb = colsum_w(part, red, buf);
    if (lead) nrm_s[c] = nb;
    __syncthreads();
    int flags = 0;
    for (int t = 1; t < MP; ++t) {
#pragma unroll
      for (int i = 0; i < RB; ++i) Bx[(r0 + i) * LD + c] = b[i];
      __syncthreads();
      double pb[RB], pd = 0.0;
      const int pc = c ^ t;
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        pb[i] = Bx[(r0 + i) * LD + pc];
        pd = fma(b[i], pb[i], pd);
      }
      red[rb * MP + c] = pd;
      __syncthreads();
      double nnew = 0.0;
      if (lead) {
        double dot = 0.0;
        for (int q = 0; q < NB; ++q) dot += red[q * MP + c];
        const double mine = nrm_s[c], other = nrm_s[pc];
        const bool isp = c < pc;
        const double app = isp ? mine : other, aqq = isp ? other : mine;
        double cs = 1.0, sn = 0.0, tr = 0.0;
        if (fabs(dot) > tol * sqrt(app * aqq)) {
          // the tangent in FP32 from x = aqq - app and y = 2 dot formed in FP64,
          // then c = (1 + t^2)^-1/2 and s = c t in FP64 (orthogonal to FP64 rounding)
          const float x = (float)(aqq - app), y = (float)(2.0 * dot);
          const float rh = lk_rsqrt_normal(fmaxf(fmaf(x, x, y * y), 1e-37f));
          const float c2 = fmaf(0.5f * fabsf(x), rh, 0.5f);
          const float tt = (x >= 0.f ? y : -y) * (0.5f * rh) / c2;
          tr = (double)tt;
          cs = rsqrt(fma(tr, tr, 1.0));
          sn = cs * tr;
          flags |= fabs(dot) > stop * sqrt(app * aqq) ? 3 : 1;
        }
        nnew = isp ? (app - tr * dot) : (aqq + tr * dot);
        rot[c] = cs;
        rot[MP + c] = isp ? -sn : sn;  // p' = c p - s q ; q' = s p + c q
      }
      __syncthreads();
      const double cs = rot[c], sg = rot[MP + c];
#pragma unroll
      for (int i = 0; i < RB; ++i) b[i] = fma(sg, pb[i], cs * b[i]);
      if (lead) nrm_s[c] = nnew;       // read again only after the next step's first barrier
    }
    if (!__syncthreads_or(flags & 2)) {
      converged = true;
      break;
    }
  }
  if (tid == 0) {
    atomicMax(&counters[2], converged ? sweep + 1 : sweep);
    atomicAdd(&counters[3], converged ? sweep + 1 : sweep);
    if (!converged) atomicOr(&counters[0], LK_BIT_NOCONVERGE);
  }

  // ---- eigenpairs, transform and apply ----
  double part = 0.0;
#pragma unroll
  for (int i = 0; i < RB; ++i) part = fma(b[i], b[i], part);
  const double nb = colsum_w(part, red, buf);
  const double lam = nb > 0.0 ? sqrt(nb) : 1.0;
  const double il = 1.0 / lam;
#pragma unroll
  for (int i = 0; i < RB; ++i) b[i] *= il;                     // q = b / lambda
  float *xrow = static_cast<float *>(I.X) + (size_t)pid * 2 * m;
  double *cdv = vec + 3 * MP, *xs0 = cdv + MP, *xs1 = xs0 + MP;
  double *gz0 = xs1 + MP, *gz1 = gz0 + MP, *gs0 = gz1 + MP, *gs1 = gs0 + MP;
  if (rb == 0) {
    cdv[c] = cd;
    xs0[c] = c < m ? (double)xrow[c] : 0.0;
    xs1[c] = c < m ? (double)xrow[m + c] : 0.0;
  }
  __syncthreads();
  double xb0 = 0.0, xb1 = 0.0;
  for (int j = 0; j < MP; ++j) {
    xb0 += xs0[j];
    xb1 += xs1[j];
  }
  const double inv_m = 1.0 / m;
  xb0 *= inv_m;
  xb1 *= inv_m;
  double pu = 0.0, p0 = 0.0, p1 = 0.0;
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    const int r = r0 + i;
    pu = fma(b[i], cdv[r], pu);                               // (Q^T C d)_c
    p0 = fma(b[i], r < m ? xs0[r] - xb0 : 0.0, p0);           // (X'_0 Q)_c
    p1 = fma(b[i], r < m ? xs1[r] - xb1 : 0.0, p1);
  }
  const double u = colsum_w(pu, red, buf);
  const double g0 = colsum_w(p0, red, buf);
  const double g1 = colsum_w(p1, red, buf);
  // every eigenvector gets its root (a warm start leaves the padding's unit
  // eigenvectors in arbitrary columns; their g0, g1 are zero)
  const double z = u / lam, sroot = sqrt((m - 1) / lam);
  if (rb == 0) {
    gz0[c] = g0 * z;
    gz1[c] = g1 * z;
    gs0[c] = g0 * sroot;
    gs1[c] = g1 * sroot;
  }
  __syncthreads();
  // (X'_r W)_j = sum_c Q[j][c] g_r,c sroot_c: the terms, then a row sum per member
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    const int r = r0 + i;
    M1[r * LD + c] = b[i] * gs0[c];
    M2[r * LD + c] = b[i] * gs1[c];
  }
  __syncthreads();
  double xa0 = 0.0, xa1 = 0.0;
  const bool mem = tid < m;
  if (tid < MP) {
    const int j = tid;
    double q0 = 0.0, q1 = 0.0, P0 = 0.0, P1 = 0.0;
    for (int k = 0; k < MP; ++k) {
      q0 += M1[j * LD + k];
      q1 += M2[j * LD + k];
      P0 += gz0[k];                                           // X'_r wbar
      P1 += gz1[k];
    }
    xa0 = xb0 + P0 + q0;
    xa1 = xb1 + P1 + q1;
    if (mem) {
      xrow[j] = (float)xa0;
      xrow[m + j] = (float)xa1;
    }
  }
  // mean and spread over the members (threads 0 .. 63: two warps)
  double *sm4 = vec + 10 * MP;         // [4] warp partial sums
  const int wp = tid >> 5, ln = tid & 31;
  double s0 = lk_warp_sum(mem ? xa0 : 0.0), s1 = lk_warp_sum(mem ? xa1 : 0.0);
  if (ln == 0 && wp < 2) {
    sm4[2 * wp] = s0;
    sm4[2 * wp + 1] = s1;
  }
  __syncthreads();
  const double mu0 = (sm4[0] + sm4[2]) * inv_m, mu1 = (sm4[1] + sm4[3]) * inv_m;
  __syncthreads();
  const double e0 = mem ? xa0 - mu0 : 0.0, e1 = mem ? xa1 - mu1 : 0.0;
  s0 = lk_warp_sum(e0 * e0);
  s1 = lk_warp_sum(e1 * e1);
  if (ln == 0 && wp < 2) {
    sm4[2 * wp] = s0;
    sm4[2 * wp + 1] = s1;
  }
  __syncthreads();
  if (tid == 0) {
    const double sp0 = sqrt((sm4[0] + sm4[2]) / (m - 1)), sp1 = sqrt((sm4[1] + sm4[3]) / (m - 1));
    if (mean_out) {
      mean_out[0] = (float)mu0;
      mean_out[1] = (float)mu1;
    }
    if (spread_out) {
      spread_out[0] = (float)sp0;
      spread_out[1] = (float)sp1;
    }
    if (!isfinite(mu0) || !isfinite(mu1) || !isfinite(sp0) || !isfinite(sp1))
      atomicOr(&counters[0], LK_BIT_NONFINITE);
  }
}

// The wide class's queue (MP = 48 and 64 nodes of FP32 handles): a fixed grid
// of CTAs walking it.
__global__ void __launch_bounds__(N64W_THREADS)
    node64w_list_kernel(const LkInst *__restrict__ insts, const int2 *__restrict__ worklist,
                        const int *__restrict__ queue_len, float *__restrict__ mean,
                        float *__restrict__ spread, double tol, int max_sweeps,
                        int *__restrict__ counters) {
  extern __shared__ __align__(16) double n64_smem[];
  lk_pdl_wait();   // no early trigger (long kernel): dependents launch as its CTAs exit
  const int qn = *queue_len;
  for (int idx = blockIdx.x; idx < qn; idx += gridDim.x) {
    const int2 it = worklist[idx];
    const LkInst &I = insts[it.x];
    const long long row = I.node_off + it.y;
    node64w(I, it.y, mean ? mean + 2 * row : nullptr, spread ? spread + 2 * row : nullptr, tol,
            LK_WARM_STOP64, max_sweeps, counters, n64_smem);
    __syncthreads();                       // shared memory is reused by the next node
  }
}

// SM count of the handle's device (read once per device; handles on several
// host threads may race to fill the cache, with the same value).
int n64_sm_count(int device) {
  static std::atomic<int> cache[64];
  const int d = device >= 0 && device < 64 ? device : 0;
  int n = cache[d].load(std::memory_order_relaxed);
  if (n == 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0)
      n = 1;
    cache[d].store(n, std::memory_order_relaxed);
  }
  return n;
}

template <int MP>
cudaError_t launch_node64(letkf_ctx *h, void *mean, void *spread) {
  const size_t smem = n64_smem_doubles<MP>() * sizeof(double);
  if (h->fp64_warm)
    return lk_launch_pdl(node64_kernel<MP, double, true>, (unsigned)h->n_pts_total, N64_THREADS,
                         smem, h->stream, h->d_inst, h->node_items, (double *)mean,
                         (double *)spread, h->tol64, h->max_sweeps, h->counters, h->keep_basis);
  return lk_launch_pdl(node64_kernel<MP, double, false>, (unsigned)h->n_pts_total, N64_THREADS,
                       smem, h->stream, h->d_inst, h->node_items, (double *)mean, (double *)spread,
                       h->tol64, h->max_sweeps, h->counters, h->keep_basis);
}

template <int MP>
cudaError_t launch_list64(letkf_ctx *h, int cls, void *mean, void *spread) {
  long long n = 0;
  for (const LkInst &I : h->inst)
    if (I.mp == MP) n += I.n_pts;
  if (n == 0) return cudaSuccess;
  const long long cap = 4LL * n64_sm_count(h->device);
  const unsigned blocks = (unsigned)(n < cap ? n : cap);
  const size_t smem = n64_smem_doubles<MP>() * sizeof(double);
  return lk_launch_pdl(node64_list_kernel<MP>, blocks, N64_THREADS, smem, h->stream, h->d_inst,
                       h->worklist + (size_t)cls * h->n_pts_total, h->counters + 4 + cls,
                       (float *)mean, (float *)spread, h->tol64, h->max_sweeps, h->counters);
}

cudaError_t launch_list64w(letkf_ctx *h, void *mean, void *spread) {
  long long n = 0;
  for (const LkInst &I : h->inst)
    if (I.mp > 32) n += I.n_pts;
  if (n == 0) return cudaSuccess;
  const long long cap = n64_sm_count(h->device);        // one CTA per SM (216 registers)
  const unsigned blocks = (unsigned)(n < cap ? n : cap);
  return lk_launch_pdl(node64w_list_kernel, blocks, N64W_THREADS,
                       n64w_smem_doubles() * sizeof(double), h->stream, h->d_inst,
                       h->worklist + (size_t)2 * h->n_pts_total, h->counters + 6, (float *)mean,
                       (float *)spread, h->tol64, h->max_sweeps, h->counters);
}

}  // namespace

cudaError_t lk_setup_node64w() {
  return cudaFuncSetAttribute(node64w_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(n64w_smem_doubles() * sizeof(double)));
}

cudaError_t lk_launch_node64(letkf_ctx *h, int cls, void *mean, void *spread) {
  return cls == 0 ? launch_node64<16>(h, mean, spread) : launch_node64<32>(h, mean, spread);
}

cudaError_t lk_launch_list64(letkf_ctx *h, int cls, void *mean, void *spread) {
  if (cls == 2) return launch_list64w(h, mean, spread);
  return cls == 0 ? launch_list64<16>(h, cls, mean, spread)
                  : launch_list64<32>(h, cls, mean, spread);
}
