// Device building blocks shared by the analysis and adjoint kernels: vector
// loads, dot products, the Gram matrix of a node's window and the one-sided
// Jacobi eigensolver. Included by each translation unit (internal linkage).
#pragma once

#include "letkf_common.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__device__ __forceinline__ void ld4(const float *p, float &a, float &b, float &c, float &d) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void ld4(const float *p, double &a, double &b, double &c, double &d) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void ld4(const double *p, double &a, double &b, double &c, double &d) {
  const double2 u = *reinterpret_cast<const double2 *>(p);
  const double2 v = *reinterpret_cast<const double2 *>(p + 2);
  a = u.x; b = u.y; c = v.x; d = v.y;
}

// Reciprocal square root of a positive normal float: the approximate PTX
// instruction with subnormals flushed, which needs no range fix-up. The Jacobi
// rotations of the node kernels call it on max(x^2 + y^2, 1e-37), on c^2 in
// [1/2, 1] and on 1 + t^2.
__device__ __forceinline__ float lk_rsqrt_normal(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lk_rsqrt(float x) { return lk_rsqrt_normal(x); }
__device__ __forceinline__ double lk_rsqrt(double x) { return rsqrt(x); }

// Dot product of two register columns with four independent FMA chains (the
// grouping is the same on both lanes of a pair, so both get the same bits).
template <int MP, typename T>
__device__ __forceinline__ T dot4(const T (&a)[MP], const T (&b)[MP]) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
  for (int k = 0; k < MP; k += 4) {
    s0 = fma(a[k], b[k], s0);
    s1 = fma(a[k + 1], b[k + 1], s1);
    s2 = fma(a[k + 2], b[k + 2], s2);
    s3 = fma(a[k + 3], b[k + 3], s3);
  }
  return (s0 + s1) + (s2 + s3);
}

// Row `lane` of A = (m-1)/rho I + sum_j c_j y_j y_j^T (identity on the padding),
// plus (C d)_lane and G_lane,lane. win / dwin: the node's window in shared memory,
// cell (ds, dt) at row stride `stride` cells.
template <int MP, typename S, typename T>
__device__ __forceinline__ void gram(const S *__restrict__ win, const S *__restrict__ dwin,
                                     int stride, const T *__restrict__ tap, int w, int m, T alpha,
                                     T (&b)[MP], T &diag, T &cd) {
  const int lane = threadIdx.x & 31;
  const bool col = lane < MP;
#pragma unroll
  for (int k = 0; k < MP; ++k) b[k] = T(0);
  diag = T(0);
  cd = T(0);
  for (int ds = 0; ds < w; ++ds) {
    for (int dt = 0; dt < w; ++dt) {
      const int cell = ds * stride + dt;
      const S *cy2 = win + (size_t)cell * 2 * MP;
      const T tw = tap[ds * w + dt];
      if (tw == T(0)) continue;                      // outside the taper's support
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const S *yv = cy2 + c * MP;
        const T yl = col ? T(yv[lane]) : T(0);
        const T cy = tw * yl;
        diag = fma(cy, yl, diag);
        cd = fma(cy, T(dwin[cell * 2 + c]), cd);
#pragma unroll
        for (int k = 0; k < MP; k += 4) {
          T y0, y1, y2, y3;
          ld4(yv + k, y0, y1, y2, y3);
          b[k] = fma(cy, y0, b[k]);
          b[k + 1] = fma(cy, y1, b[k + 1]);
          b[k + 2] = fma(cy, y2, b[k + 2]);
          b[k + 3] = fma(cy, y3, b[k + 3]);
        }
      }
    }
  }
  const T dval = lane < m ? alpha : T(1);
#pragma unroll
  for (int k = 0; k < MP; ++k)
    if (k == lane) b[k] += dval;
}

// One Hestenes rotation step for pair (lane, lane ^ t) on column b (and v when
// ACCUM). nrm = |b|^2 of this lane's column. Returns bit 0: it rotated (cosine
// above tol), bit 1: the cosine was above stop.
template <int MP, typename T, bool ACCUM>
__device__ __forceinline__ int jacobi_step(T (&b)[MP], T (&v)[MP], T &nrm, int t, T tol,
                                           T stop) {
  const int lane = threadIdx.x & 31;
  T pb[MP];
#pragma unroll
  for (int k = 0; k < MP; ++k) pb[k] = __shfl_xor_sync(FULL, b[k], t);
  const T dot = dot4<MP, T>(b, pb);
  const T pn = __shfl_xor_sync(FULL, nrm, t);
  const bool isp = lane < (lane ^ t);  // this lane holds column p of the pair (p < q)
  const T app = isp ? nrm : pn;
  const T aqq = isp ? pn : nrm;
  T cs = T(1), sn = T(0), tr = T(0);
  int rot = 0;
  const T scale = sqrt(app * aqq);
  if (fabs(dot) > tol * scale) {
    if constexpr (sizeof(T) == 8) {
      // FP64: the tangent in FP32 from x = aqq - app and y = 2 dot formed in
      // FP64 (cos 2theta = |x|/h, c^2 = (1 + cos 2theta)/2, t = sin 2theta / (2 c^2)),
      // then c = (1 + t^2)^-1/2 and s = c t in FP64: an orthogonal rotation whose
      // FP32-accurate angle leaves the pair's cosine at ~1e-7 of its value
      const float x = (float)(aqq - app), y = (float)(T(2) * dot);
      const float rh = lk_rsqrt_normal(fmaxf(fmaf(x, x, y * y), 1e-37f));
      const float c2 = fmaf(0.5f * fabsf(x), rh, 0.5f);
      tr = (T)((x >= 0.f ? y : -y) * (0.5f * rh) / c2);
    } else {
      const T zeta = (aqq - app) / (T(2) * dot);
      const T az = fabs(zeta);
      tr = az > T(1e15) ? T(0.5) / zeta : copysign(T(1), zeta) / (az + sqrt(T(1) + zeta * zeta));
    }
    cs = lk_rsqrt(T(1) + tr * tr);
    sn = cs * tr;
    rot = fabs(dot) > stop * scale ? 3 : 1;
  }
  const T sg = isp ? -sn : sn;  // p' = c p - s q ; q' = s p + c q
#pragma unroll
  for (int k = 0; k < MP; ++k) b[k] = fma(sg, pb[k], cs * b[k]);
  nrm = isp ? (app - tr * dot) : (aqq + tr * dot);
  if (ACCUM) {
#pragma unroll
    for (int k = 0; k < MP; ++k) pb[k] = __shfl_xor_sync(FULL, v[k], t);
#pragma unroll
    for (int k = 0; k < MP; ++k) v[k] = fma(sg, pb[k], cs * v[k]);
  }
  return rot;
}

// Start of an accumulated FP64 sweep from a stored FP32 eigenbasis U
// (row-major MP x MP, lane = column) instead of the identity. One Newton-Schulz
// step V <- V (3 I - V^T V) / 2 makes the columns orthonormal to FP64 rounding
// (it squares their orthogonality error), then b = A v_lane. On entry b holds
// row lane of the symmetric A; As and Vs are [MP][MP+1] warp scratch.
template <int MP, typename T>
__device__ __forceinline__ void warm_basis(T (&b)[MP], T (&v)[MP], const float *__restrict__ U,
                                           T *__restrict__ As, T *__restrict__ Vs) {
  constexpr int LD = MP + 1;
  const int lane = threadIdx.x & 31;
  const bool col = lane < MP;
#pragma unroll
  for (int k = 0; k < MP; ++k) v[k] = col ? T(U[k * MP + lane]) : T(0);
  __syncwarp();
  if (col) {
#pragma unroll
    for (int k = 0; k < MP; ++k) {
      As[k * LD + lane] = b[k];
      Vs[k * LD + lane] = v[k];
    }
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < MP; ++i) {                  // b <- V^T v_lane
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < MP; ++k) acc = fma(Vs[k * LD + i], v[k], acc);
    b[i] = acc;
  }
#pragma unroll
  for (int k = 0; k < MP; ++k) {                  // v_lane <- 1.5 v_lane - 0.5 V b
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < MP; ++i) acc = fma(Vs[k * LD + i], b[i], acc);
    v[k] = fma(T(-0.5), acc, T(1.5) * v[k]);
  }
#pragma unroll
  for (int k = 0; k < MP; ++k) {                  // b <- A v_lane
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < MP; ++i) acc = fma(As[k * LD + i], v[i], acc);
    b[k] = acc;
  }
  __syncwarp();
}

// Sweeps until a full sweep makes no rotation or, with stop > 0, until a sweep
// whose rotations all had cosines <= stop (sweeps converge quadratically, so
// the next one would rotate by about stop^2, except inside clusters of nearly
// equal eigenvalues, whose mixing leaves functions of A unchanged). Records
// the sweep count and a non-convergence flag.
template <int MP, typename T, bool ACCUM>
__device__ __forceinline__ void jacobi(T (&b)[MP], T (&v)[MP], T tol, int max_sweeps,
                                       int *__restrict__ counters, T stop = T(0)) {
  int sweep = 0;
  bool converged = false;
  if (stop < tol) stop = tol;
  for (; sweep < max_sweeps; ++sweep) {
    T nrm = dot4<MP, T>(b, b);
    int rotated = 0;
    for (int t = 1; t < MP; ++t) rotated |= jacobi_step<MP, T, ACCUM>(b, v, nrm, t, tol, stop);
    if (!__any_sync(FULL, rotated & 2)) {
      converged = true;
      break;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&counters[2], converged ? sweep + 1 : sweep);
    atomicAdd(&counters[3], converged ? sweep + 1 : sweep);
    if (!converged) atomicOr(&counters[0], LK_BIT_NOCONVERGE);
  }
}

}  // namespace
