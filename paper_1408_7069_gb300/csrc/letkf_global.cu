// The global ETKF (Section 3.1.1: one domain observing every slope, partition
// 1) for ensembles of more than 64 members (the paper's global curves reach
// m ~ 626, Section 5.1; from m = 101 on this path is faster than the one-CTA
// Jacobi, which also stops at 128 columns). The transform needs only
// A^-1/2 and A^-1 c, so the eigendecomposition is replaced by matrix products:
//   Gram     A = (m-1)/rho I + S^T S, c = S^T s in FP64 (the split-K Gram of
//            letkf_domains.cu), s_A = |A|_F >= lambda_max
//   root     coupled Newton-Schulz on Y0 = A / s_A, Z0 = I:
//            T = (3 I - Z Y) / 2, Y <- Y T, Z <- T Z, converging to
//            Y -> (A/s_A)^1/2 and Z -> (A/s_A)^-1/2 (the spectrum of A / s_A
//            lies in (0, 1]); at most a fixed number of iterations (converged
//            ones skipped on the device), FP32 matrix products in 32 x 32
//            tiles, and a check of |I - Z Y|
//   mean     wbar = A^-1 c by iterative refinement: residual c - A wbar in
//            FP64, correction Z (Z r) / s_A in FP32
//   apply    T = wbar 1^T + sqrt((m-1) / s_A) Z, Xa = xbar + X' T (the same
//            matrix-product kernel over all state rows), mean and spread
#include <math.h>

#include <vector>

#include "letkf_device.cuh"

namespace {

constexpr int NS_TILE = 64, NS_KT = 32, NS_THREADS = 256;

// C = alpha A B + beta I (beta on the diagonal only), all row-major, M, N, K
// multiples of 64, leading dimensions multiples of 4 floats. A 64 x 64 tile
// per CTA, 4 x 4 outputs per thread; the next 32-deep slice of A and B is
// loaded into registers (float4) while the current one, in shared memory (A
// transposed), is multiplied.
__global__ void __launch_bounds__(NS_THREADS)
    ns_gemm_kernel(int K, const float *__restrict__ A, int lda, const float *__restrict__ B,
                   int ldb, float *__restrict__ C, int ldc, float alpha, float beta) {
  __shared__ __align__(16) float As[NS_KT][NS_TILE + 4];
  __shared__ __align__(16) float Bs[NS_KT][NS_TILE + 4];
  lk_pdl_wait();
  const int tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
  const int row0 = blockIdx.y * NS_TILE, col0 = blockIdx.x * NS_TILE;
  // slice loads: A 64 x 32 (two float4 per thread: row ar + 32 q, columns ak .. ak+3),
  // B 32 x 64 (two float4 per thread: row bk + 16 q, columns bc .. bc+3)
  const int ar = tid / 8, ak = (tid % 8) * 4;
  const int bk = tid / 16, bc = (tid % 16) * 4;
  float4 ra[2], rb[2];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      ra[q] = *reinterpret_cast<const float4 *>(A + (size_t)(row0 + ar + 32 * q) * lda + k0 + ak);
      rb[q] = *reinterpret_cast<const float4 *>(B + (size_t)(k0 + bk + 16 * q) * ldb + col0 + bc);
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int r = ar + 32 * q;
      As[ak + 0][r] = ra[q].x;
      As[ak + 1][r] = ra[q].y;
      As[ak + 2][r] = ra[q].z;
      As[ak + 3][r] = ra[q].w;
      *reinterpret_cast<float4 *>(&Bs[bk + 16 * q][bc]) = rb[q];
    }
  };
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  load(0);
  for (int k0 = 0; k0 < K; k0 += NS_KT) {
    store();
    __syncthreads();
    if (k0 + NS_KT < K) load(k0 + NS_KT);
#pragma unroll
    for (int k = 0; k < NS_KT; ++k) {
      const float4 a = *reinterpret_cast<const float4 *>(&As[k][tr * 4]);
      const float4 b = *reinterpret_cast<const float4 *>(&Bs[k][tc * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + tr * 4 + i;
    float4 o;
    float *ov = &o.x;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tc * 4 + j;
      ov[j] = alpha * acc[i][j] + (r == c ? beta : 0.f);
    }
    *reinterpret_cast<float4 *>(C + (size_t)r * ldc + col0 + tc * 4) = o;
  }
}

// The Newton-Schulz products: C = alpha A B + beta I, n x n, in 32 x 32 tiles
// of 64 threads (4 x 4 outputs per thread): 400 CTAs at m = 626 instead of 100
// CTAs of 64 x 64 tiles on 152 SMs. (Forming only the upper triangle of these
// products of commuting symmetric matrices and mirroring it would halve the
// flops, but it breaks the coupling of the iteration: in FP32 at the prior
// draw's kappa ~ 1.5e5, m = 200, the symmetrised iteration overflows after 20
// steps where the full one converges to |I - Z Y| ~ 3e-6.)
//
// Early exit: the first product of iteration it (T = 1.5 I - 0.5 Z Y) records
// max |Z Y - I| of its tiles in res[it] (non-negative floats compare as their
// bit patterns); an iteration whose predecessors include one with
// res <= NS_DONE is skipped, its three products turning into T = I, U = Y and
// Y' = Z (what they give for T = I), so the buffers' rotation on the host stays
// right. The iteration that reached NS_DONE still runs, and takes the residual
// from about 1e-4 to FP32 rounding (it converges quadratically there).
constexpr int NSS_TILE = 32, NSS_KT = 32, NSS_SPLIT = 4, NSS_GROUP = 64;
constexpr int NSS_THREADS = NSS_SPLIT * NSS_GROUP, NSS_LD = NSS_TILE + 4;
constexpr float NS_DONE = 1e-4f;
enum { NSG_PLAIN = 0, NSG_T = 1, NSG_SKIP_COPY_A = 2, NSG_SKIP_COPY_B = 3 };

__device__ __forceinline__ bool ns_skip(const unsigned *res, int it) {
  for (int i = 0; i < it; ++i)
    if (__uint_as_float(res[i]) <= NS_DONE) return true;
  return false;
}

// One 32 x 32 output tile per CTA, the K dimension split over four groups of
// 64 threads (group q takes the 32-deep slices q, q + 4, ...; 4 x 4 outputs
// per thread), whose partial tiles are added in group order through shared
// memory: 400 CTAs of 8 warps at m = 626.
__global__ void __launch_bounds__(NSS_THREADS)
    ns_sq_gemm_kernel(int n, const float *__restrict__ A, const float *__restrict__ B,
                      float *__restrict__ C, float alpha, float beta, int mode,
                      unsigned *__restrict__ res, int it) {
  __shared__ __align__(16) float As[NSS_SPLIT][NSS_KT][NSS_LD];
  __shared__ __align__(16) float Bs[NSS_SPLIT][NSS_KT][NSS_LD];
  lk_pdl_wait();
  const int row0 = blockIdx.y * NSS_TILE, col0 = blockIdx.x * NSS_TILE;
  const int tid = threadIdx.x;
  const int orow = tid / 8, ocol = (tid % 8) * 4;   // this thread's output float4
  if (mode != NSG_PLAIN && ns_skip(res, it)) {
    // skipped iteration: T = I, or a copy of the operand that is not T
    const int r = row0 + orow, c = col0 + ocol;
    float4 o;
    if (mode == NSG_T)
      o = make_float4(r == c ? 1.f : 0.f, r == c + 1 ? 1.f : 0.f, r == c + 2 ? 1.f : 0.f,
                      r == c + 3 ? 1.f : 0.f);
    else
      o = *reinterpret_cast<const float4 *>((mode == NSG_SKIP_COPY_A ? A : B) + (size_t)r * n + c);
    *reinterpret_cast<float4 *>(C + (size_t)r * n + c) = o;
    return;
  }
  const int q = tid / NSS_GROUP, lt = tid % NSS_GROUP, tr = lt / 8, tc = lt % 8;
  float(*as)[NSS_LD] = As[q];
  float(*bs)[NSS_LD] = Bs[q];
  // slice loads: A 32 x 32 (rows ar + 8j, columns ak .. ak+3), B 32 x 32
  // (rows ar + 8j, columns ak .. ak+3), four float4 each per thread of the group
  const int ar = lt / 8, ak = (lt % 8) * 4;
  const int nk = n / NSS_KT, steps = (nk + NSS_SPLIT - 1) / NSS_SPLIT;
  float4 ra[4], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      ra[j] = *reinterpret_cast<const float4 *>(A + (size_t)(row0 + ar + 8 * j) * n + k0 + ak);
      rb[j] = *reinterpret_cast<const float4 *>(B + (size_t)(k0 + ar + 8 * j) * n + col0 + ak);
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ar + 8 * j;
      as[ak + 0][r] = ra[j].x;
      as[ak + 1][r] = ra[j].y;
      as[ak + 2][r] = ra[j].z;
      as[ak + 3][r] = ra[j].w;
      *reinterpret_cast<float4 *>(&bs[r][ak]) = rb[j];
    }
  };
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  // every group runs `steps` rounds (the barriers are the CTA's); a group
  // whose slice index runs past nk idles in that round
  if (q < nk) load(q * NSS_KT);
  for (int s = 0; s < steps; ++s) {
    const int kt = q + NSS_SPLIT * s;
    const bool valid = kt < nk;
    if (valid) store();
    __syncthreads();
    if (kt + NSS_SPLIT < nk) load((kt + NSS_SPLIT) * NSS_KT);
    if (valid) {
#pragma unroll
      for (int k = 0; k < NSS_KT; ++k) {
        const float4 a = *reinterpret_cast<const float4 *>(&as[k][tr * 4]);
        const float4 b = *reinterpret_cast<const float4 *>(&bs[k][tc * 4]);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  // the groups' partial tiles, added in group order (As is free now)
#pragma unroll
  for (int i = 0; i < 4; ++i)
    *reinterpret_cast<float4 *>(&As[q][tr * 4 + i][tc * 4]) =
        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  __syncthreads();
  float4 t = *reinterpret_cast<const float4 *>(&As[0][orow][ocol]);
#pragma unroll
  for (int g = 1; g < NSS_SPLIT; ++g) {
    const float4 u = *reinterpret_cast<const float4 *>(&As[g][orow][ocol]);
    t = make_float4(t.x + u.x, t.y + u.y, t.z + u.z, t.w + u.w);
  }
  const int r = row0 + orow, c = col0 + ocol;
  const float tv[4] = {t.x, t.y, t.z, t.w};
  float ov[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) ov[j] = alpha * tv[j] + (r == c + j ? beta : 0.f);
  *reinterpret_cast<float4 *>(C + (size_t)r * n + c) = make_float4(ov[0], ov[1], ov[2], ov[3]);
  if (mode == NSG_T) {                     // max |Z Y - I| of the tile, Z Y = the sum
    float mx = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      mx = fmaxf(mx, fabsf(tv[j] - (r == c + j ? 1.f : 0.f)));
      if (!(tv[j] == tv[j])) mx = __int_as_float(0x7fc00000);   // NaN stays
    }
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      const float v = __shfl_xor_sync(FULL, mx, o2);
      mx = (v != v || mx != mx) ? __int_as_float(0x7fc00000) : fmaxf(mx, v);
    }
    if ((tid & 31) == 0) atomicMax(res + it, __float_as_uint(mx));
  }
}

// A (FP64) = (m-1)/rho I + the Gram partials, and the row sums of squares;
// a CTA per row.
__global__ void __launch_bounds__(256)
    ns_assemble_kernel(const LkInst *__restrict__ insts, const double *__restrict__ gpart,
                       const double *__restrict__ cpart, int kchunks, int mpt,
                       double *__restrict__ A64, double *__restrict__ c64,
                       double *__restrict__ rowsq) {
  lk_pdl_wait();
  const LkInst &I = insts[0];
  const int i = blockIdx.x;
  double sq = 0.0;
  for (int j = threadIdx.x; j < mpt; j += blockDim.x) {
    const int a = i <= j ? i : j, b = i <= j ? j : i;
    double s = 0.0;
    for (int k = 0; k < kchunks; ++k) s += gpart[((size_t)k * mpt + a) * mpt + b];
    // (m-1)/rho on the diagonal, the padding included: the padding's
    // eigenvalues then sit with the smallest real ones instead of at 1, far
    // below |A|_F, where the iteration would need the most steps to reach them
    if (i == j) s += I.alpha;
    A64[(size_t)i * mpt + j] = s;
    sq = fma(s, s, sq);
  }
  __shared__ double red[8];
  sq = lk_warp_sum(sq);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    rowsq[i] = t;
    double c = 0.0;
    for (int k = 0; k < kchunks; ++k) c += cpart[(size_t)k * mpt + i];
    c64[i] = c;
  }
}

// s_A = |A|_F from the row sums of squares, one warp in a fixed order; clears
// the iterations' residual words.
__global__ void __launch_bounds__(32)
    ns_scale_kernel(int mpt, const double *__restrict__ rowsq, double *__restrict__ scale,
                    unsigned *__restrict__ res, int iters) {
  lk_pdl_wait();
  double t = 0.0;
  for (int i = threadIdx.x; i < mpt; i += 32) t += rowsq[i];
  t = lk_warp_sum(t);
  if (threadIdx.x == 0) *scale = sqrt(t);
  for (int i = threadIdx.x; i < iters; i += 32) res[i] = 0u;
}

// Y = A / s_A, Z = I; wbar = 0.
__global__ void __launch_bounds__(256)
    ns_start_kernel(int mpt, const double *__restrict__ A64, const double *__restrict__ scale,
                    float *__restrict__ Y, float *__restrict__ Z, double *__restrict__ w64) {
  lk_pdl_wait();
  const double inv = 1.0 / *scale;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)mpt * mpt;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / mpt), j = (int)(e % mpt);
    Y[e] = (float)(A64[e] * inv);
    Z[e] = i == j ? 1.f : 0.f;
    if (e < mpt) w64[e] = 0.0;
  }
}

// max |I - Z Y| of the converged iteration (R = Z Y given) into the status
// word: NOCONVERGE above 1e-3.
__global__ void __launch_bounds__(256)
    ns_check_kernel(int mpt, const float *__restrict__ R, int *__restrict__ counters) {
  lk_pdl_wait();
  float mx = 0.f;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)mpt * mpt;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / mpt), j = (int)(e % mpt);
    mx = fmaxf(mx, fabsf((i == j ? 1.f : 0.f) - R[e]));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
  if ((threadIdx.x & 31) == 0 && !(mx <= 1e-3f)) atomicOr(&counters[0], LK_BIT_NOCONVERGE);
}

// r = c - A w (FP64), warp per row (lanes over the row, a fixed-order sum).
__global__ void __launch_bounds__(128)
    ns_residual_kernel(int mpt, const double *__restrict__ A64, const double *__restrict__ c64,
                       const double *__restrict__ w64, float *__restrict__ r) {
  lk_pdl_wait();
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= mpt) return;
  double s = 0.0;
  for (int j = lane; j < mpt; j += 32) s = fma(A64[(size_t)i * mpt + j], w64[j], s);
  s = lk_warp_sum(s);
  if (lane == 0) r[i] = (float)(c64[i] - s);
}

// out = Z v (FP32), warp per row; with `w`, w += out / s_A (FP64).
__global__ void __launch_bounds__(128)
    ns_matvec_kernel(int mpt, const float *__restrict__ Z, const float *__restrict__ v,
                     float *__restrict__ out, double *__restrict__ w,
                     const double *__restrict__ scale) {
  lk_pdl_wait();
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= mpt) return;
  float s = 0.f;
  for (int j = lane; j < mpt; j += 32) s = fmaf(Z[(size_t)i * mpt + j], v[j], s);
  s = lk_warp_sum(s);
  if (lane != 0) return;
  if (w)
    w[i] += (double)s / *scale;
  else
    out[i] = s;
}

// T = wbar 1^T + sqrt((m-1) / s_A) Z on the m x m block, zero elsewhere.
__global__ void __launch_bounds__(256)
    ns_transform_kernel(const LkInst *__restrict__ insts, int mpt, const float *__restrict__ Z,
                        const double *__restrict__ w64, const double *__restrict__ scale,
                        float *__restrict__ T) {
  lk_pdl_wait();
  const LkInst &I = insts[0];
  const float f = (float)sqrt((I.m - 1) / *scale);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)mpt * mpt;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / mpt), j = (int)(e % mpt);
    T[e] = (i < I.m && j < I.m) ? (float)w64[i] + f * Z[e] : 0.f;
  }
}

// Anomalies of every state row into Xp [n_pad][mpt] (zero padding), means into xm.
__global__ void __launch_bounds__(LK_WARP_CTA)
    ns_anom_kernel(const LkInst *__restrict__ insts, int mpt, long long n_pad,
                   float *__restrict__ Xp, float *__restrict__ xm) {
  lk_pdl_wait();
  const LkInst &I = insts[0];
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, m = I.m;
  if (r >= n_pad) return;
  const bool real = r < 2LL * I.n_pts;
  const float *x = static_cast<const float *>(I.X) + r * m;
  float s = 0.f;
  if (real)
    for (int j = lane; j < m; j += 32) s += x[j];
  s = lk_warp_sum(s) / float(m);
  for (int j = lane; j < mpt; j += 32) Xp[r * mpt + j] = (real && j < m) ? x[j] - s : 0.f;
  if (lane == 0) xm[r] = s;
}

// Xa = xbar + (X' T), mean and spread, warp per state row.
__global__ void __launch_bounds__(LK_WARP_CTA)
    ns_finish_kernel(const LkInst *__restrict__ insts, int mpt, const float *__restrict__ P,
                     const float *__restrict__ xm, float *__restrict__ mean,
                     float *__restrict__ spread, int *__restrict__ counters) {
  lk_pdl_wait();
  const LkInst &I = insts[0];
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, m = I.m;
  if (r >= 2LL * I.n_pts) return;
  float *x = static_cast<float *>(I.X) + r * m;
  float sum = 0.f;
  for (int j = lane; j < m; j += 32) {
    const float xa = xm[r] + P[r * mpt + j];
    x[j] = xa;
    sum += xa;
  }
  const float mu = lk_warp_sum(sum) / float(m);
  float sq = 0.f;
  for (int j = lane; j < m; j += 32) {
    const float d = x[j] - mu;
    sq = fmaf(d, d, sq);
  }
  const float sp = sqrtf(lk_warp_sum(sq) / float(m - 1));
  if (lane == 0) {
    if (mean) mean[r] = mu;
    if (spread) spread[r] = sp;
    if (!isfinite(mu) || !isfinite(sp)) atomicOr(&counters[0], LK_BIT_NONFINITE);
  }
}

cudaError_t gemm(cudaStream_t st, int M, int N, int K, const float *A, int lda, const float *B,
                 int ldb, float *C, int ldc, float alpha, float beta) {
  return lk_launch_pdl(ns_gemm_kernel, dim3(N / NS_TILE, M / NS_TILE), NS_THREADS, 0, st, K, A,
                       lda, B, ldb, C, ldc, alpha, beta);
}

cudaError_t sq_gemm(cudaStream_t st, int n, const float *A, const float *B, float *C, float alpha,
                    float beta, int mode = NSG_PLAIN, unsigned *res = nullptr, int it = 0) {
  const unsigned nt = (unsigned)(n / NSS_TILE);
  return lk_launch_pdl(ns_sq_gemm_kernel, dim3(nt, nt), NSS_THREADS, 0, st, n, A, B, C, alpha,
                       beta, mode, res, it);
}

}  // namespace

int lk_ns_tile() { return NS_TILE; }

// Workspace (one allocation): A64, c64, w64, rowsq, scale (FP64); Y, Z, T, U
// (FP32 [mpt][mpt]); r, v (FP32 [mpt]); Xp and the product (FP32 [n_pad][mpt]),
// xm [n_pad].
// (the FP32 part starts 256-byte aligned: the matrix products load float4)
static size_t ns_fp64_bytes(int mpt) {
  return (((size_t)mpt * mpt * 8 + 3 * (size_t)mpt * 8 + 8) + 255) & ~size_t(255);
}

size_t lk_ns_workspace_bytes(int mpt, long long n_pad) {
  const size_t f = 4 * (size_t)mpt * mpt * 4 + 2 * (size_t)mpt * 4 +
                   2 * (size_t)n_pad * mpt * 4 + (size_t)n_pad * 4;
  return ns_fp64_bytes(mpt) + f + 64 * sizeof(unsigned) + 1024;
}

cudaError_t lk_launch_ns_global(letkf_ctx *h, const double *gpart, const double *cpart,
                                int kchunks, int mpt, int iters, void *ws, void *mean,
                                void *spread) {
  const LkInst &I = h->inst[0];
  const long long n_pad = ((2LL * I.n_pts + NS_TILE - 1) / NS_TILE) * NS_TILE;
  unsigned char *b = static_cast<unsigned char *>(ws);
  double *A64 = reinterpret_cast<double *>(b);
  double *c64 = A64 + (size_t)mpt * mpt, *w64 = c64 + mpt, *rowsq = w64 + mpt;
  double *scale = rowsq + mpt;
  float *Y = reinterpret_cast<float *>(b + ns_fp64_bytes(mpt));
  float *Z = Y + (size_t)mpt * mpt, *T = Z + (size_t)mpt * mpt, *U = T + (size_t)mpt * mpt;
  float *rv = U + (size_t)mpt * mpt, *vv = rv + mpt;
  float *Xp = vv + mpt, *Pr = Xp + (size_t)n_pad * mpt, *xm = Pr + (size_t)n_pad * mpt;
  unsigned *res = reinterpret_cast<unsigned *>(xm + n_pad);   // [iters] residuals (early exit)
  cudaStream_t st = h->stream;
  cudaError_t e = lk_launch_pdl(ns_assemble_kernel, (unsigned)mpt, 256, 0, st,
                                (const LkInst *)h->d_inst, gpart, cpart, kchunks, mpt, A64, c64,
                                rowsq);
  const unsigned eb = (unsigned)(((long long)mpt * mpt + 255) / 256 < 2048
                                     ? ((long long)mpt * mpt + 255) / 256
                                     : 2048);
  if (e == cudaSuccess)
    e = lk_launch_pdl(ns_scale_kernel, 1u, 32, 0, st, mpt, (const double *)rowsq, scale, res,
                      iters);
  if (e == cudaSuccess)
    e = lk_launch_pdl(ns_start_kernel, eb, 256, 0, st, mpt, (const double *)A64,
                      (const double *)scale, Y, Z, w64);
  // Newton-Schulz, buffers rotating: T = 1.5 I - 0.5 Z Y; U = Y T; Y' = U;
  // Z' = T Z written into the old Y
  for (int it = 0; it < iters && e == cudaSuccess; ++it) {
    e = sq_gemm(st, mpt, Z, Y, T, -0.5f, 1.5f, NSG_T, res, it);
    if (e == cudaSuccess) e = sq_gemm(st, mpt, Y, T, U, 1.f, 0.f, NSG_SKIP_COPY_A, res, it);
    if (e == cudaSuccess) e = sq_gemm(st, mpt, T, Z, Y, 1.f, 0.f, NSG_SKIP_COPY_B, res, it);
    float *nY = U, *nZ = Y;
    U = Z;
    Y = nY;
    Z = nZ;
  }
  if (e == cudaSuccess) e = sq_gemm(st, mpt, Z, Y, T, 1.f, 0.f);
  if (e == cudaSuccess)
    e = lk_launch_pdl(ns_check_kernel, eb, 256, 0, st, mpt, (const float *)T, h->counters);
  // wbar = A^-1 c by refinement with A^-1 ~ Z Z / s_A
  const unsigned vb = (unsigned)((mpt * 32 + 127) / 128);
  for (int it = 0; it < 4 && e == cudaSuccess; ++it) {
    e = lk_launch_pdl(ns_residual_kernel, vb, 128, 0, st, mpt, (const double *)A64,
                      (const double *)c64, (const double *)w64, rv);
    if (e == cudaSuccess)
      e = lk_launch_pdl(ns_matvec_kernel, vb, 128, 0, st, mpt, (const float *)Z,
                        (const float *)rv, vv, (double *)nullptr, (const double *)scale);
    if (e == cudaSuccess)
      e = lk_launch_pdl(ns_matvec_kernel, vb, 128, 0, st, mpt, (const float *)Z,
                        (const float *)vv, rv, w64, (const double *)scale);
  }
  if (e == cudaSuccess)
    e = lk_launch_pdl(ns_transform_kernel, eb, 256, 0, st, (const LkInst *)h->d_inst, mpt,
                      (const float *)Z, (const double *)w64, (const double *)scale, T);
  const unsigned rb = (unsigned)((n_pad * 32 + LK_WARP_CTA - 1) / LK_WARP_CTA);
  if (e == cudaSuccess)
    e = lk_launch_pdl(ns_anom_kernel, rb, LK_WARP_CTA, 0, st, (const LkInst *)h->d_inst, mpt,
                      n_pad, Xp, xm);
  if (e == cudaSuccess) e = gemm(st, (int)n_pad, mpt, mpt, Xp, mpt, T, mpt, Pr, mpt, 1.f, 0.f);
  const unsigned fb = (unsigned)((2LL * I.n_pts * 32 + LK_WARP_CTA - 1) / LK_WARP_CTA);
  if (e == cudaSuccess)
    e = lk_launch_pdl(ns_finish_kernel, fb, LK_WARP_CTA, 0, st, (const LkInst *)h->d_inst, mpt,
                      (const float *)Pr, (const float *)xm, static_cast<float *>(mean),
                      static_cast<float *>(spread), h->counters);
  return e;
}
