// Internal declarations shared by the translation units of libletkf.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "letkf.h"

// Device status word bits (set with atomicOr by kernels, read by letkf_sync).
enum : int {
  LK_BIT_NOCONVERGE = 1,
  LK_BIT_NONFINITE = 2,
  LK_BIT_TIMEOUT = 4,
};

// Node tile processed by one analysis CTA: TI x TJ nodes.
constexpr int LK_TILE_I = 2;
constexpr int LK_TILE_J = 4;
// Extra padding of the slope-anomaly grid so that every tile's halo is in bounds.
constexpr int LK_TILE_MAX = 8;
// CTAs of the residual reduction (fixed, so the sum order is fixed).
constexpr int LK_RES_BLOCKS = 128;

// Everything a frame's kernels need. Device pointers unless noted. The real
// type of X, Yb, d, y, truth, taper and the outputs is float (precision 0) or
// double (precision 1).
struct LkGeom {
  int nsub, m, w, h;       // h = w / 2
  int n_pts, n_sap, p;
  int gs_rows, gs_cols;    // padded subaperture grid (cells); cell (s+h, t+h) holds subap (s, t)
  const int *pid_map;      // [(nsub+1)^2] node -> point id or -1
  const int2 *pts;         // [n_pts] (i, j)
  const int2 *saps;        // [n_sap] (s, t)
};

struct letkf_ctx {
  letkf_config cfg;        // host copy, host pointers cleared
  cudaStream_t stream = nullptr;
  int device = 0;
  int precision = 0;
  size_t rsz = 4;          // bytes of the real type
  int mp = 32;             // padded ensemble width of the kernels (16 or 32)
  LkGeom g{};
  double alpha = 0, tol32 = 0, tol64 = 0;
  int max_sweeps = 12;

  // device buffers
  void *X = nullptr;       // [n_pts][2][m]
  void *Ybp = nullptr;     // [gs_rows][gs_cols][2][m]
  void *dp = nullptr;      // [gs_rows][gs_cols][2]
  void *taper = nullptr;   // [w*w] tau / sigma2
  int *pid_map = nullptr;
  int2 *pts = nullptr;
  int2 *saps = nullptr;
  int2 *tiles = nullptr;   // analysis tile origins (node coordinates)
  int n_tiles = 0;
  float *bank = nullptr;
  int bank_B = 0, bank_G = 0;
  int *counters = nullptr; // [0] status bits, [1] fp64 list length, [2] max sweeps
  int *worklist = nullptr; // [n_pts] FP64 fallback point ids
  float *basis = nullptr;  // [n_pts][mp][mp] each node's last eigenbasis (warm start)
  double2 *partial = nullptr;   // [LK_RES_BLOCKS] residual partial sums
  long long *frame = nullptr;   // [0] forecast counter, [1] index within letkf_run
  double *zero_scalar = nullptr;

  // host copies
  std::vector<int32_t> pts_host, wslopes_host;
  long long frame_host = 0;

  // graph of one closed-loop frame (letkf_run)
  cudaGraphExec_t graph = nullptr;
  const void *graph_y = nullptr, *graph_truth = nullptr;
  const double *graph_resvar = nullptr;

  std::string err;
};

// Launchers (defined in letkf_kernels.cu / letkf_analysis.cu). All enqueue on
// h->stream and return the launch status. run_idx (device) selects element
// *run_idx of a sequence (y, truth, resvar); NULL means element 0.
cudaError_t lk_launch_obs(letkf_ctx *h, const void *y, const long long *run_idx);
cudaError_t lk_launch_analysis(letkf_ctx *h, void *mean, void *spread);
cudaError_t lk_launch_forecast(letkf_ctx *h, const void *noise);
cudaError_t lk_launch_residual(letkf_ctx *h, const void *truth, double *resvar, const long long *run_idx);
cudaError_t lk_launch_tick(letkf_ctx *h);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
template <typename T>
__device__ __forceinline__ T lk_warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// SplitMix64 output after the state advanced counter + 1 steps from seed
// (Steele, Lea & Flood 2014).
__device__ __forceinline__ unsigned long long lk_splitmix64(unsigned long long seed,
                                                            unsigned long long counter) {
  unsigned long long z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
#endif
