// Local ensemble transform analysis (Section 4.2 with Section 3.1 and Appendix A):
// the per-width-class dispatch of letkf_analyze, and the allocation-free
// analysis of letkf_analyze_noalloc.
//
// Per node, with column l of the m x m problem zero-padded to MP = 16 or 32
// columns (identity on the padding):
//   Gram     A = (m-1)/rho I + sum_j tau_j/sigma2 Yb_j Yb_j^T,  C d = sum_j tau_j/sigma2 d_j Yb_j
//   EVD      one-sided (Hestenes) Jacobi on the columns of B = A V0: rotations J make
//            the columns of B J orthogonal, so A (V0 J) = (V0 J) Lambda
//   weights  wbar = V Lambda^-1 V^T C d,  W = V ((m-1) Lambda^-1)^(1/2) V^T
//   apply    Xa_r = xbar_r + X'_r wbar + X'_r W for the node's two rows
//
// FP32 handles run the analysis in letkf_pair.cu (two columns per lane). Nodes
// whose kappa_hat = 1 + rho tr(G)/(m-1) exceeds the threshold still take that
// FP32 eigensolve, but their mean solve wbar = A^-1 C d would amplify the FP32
// Gram's rounding by kappa: they are queued and redone in FP64 (Gram and
// sweep, started from the FP32 eigenbasis) by letkf_node64.cu, which also
// analyses every node of FP64 handles (one CTA of four warps per node).
//
// The allocation-free analysis below keeps the earlier tile layout: one warp
// per node (lane = column, eigenvectors accumulated from the identity, pairs
// by the xor tournament: step t pairs column l with l ^ t), a CTA per tile of
// nodes staging the tile's window halo in shared memory once.
#include <math.h>
#include <stdio.h>

#include <mutex>
#include <type_traits>

#include "letkf_device.cuh"

namespace {

// Per-warp scratch: V staging [MP][MP+1] + 3 vectors, or A staging [MP][MP+4].
template <int MP, typename T>
__host__ __device__ constexpr size_t scratch_elems() {
  return (size_t)MP * (MP + 1) + 3 * MP > (size_t)MP * (MP + 4) ? (size_t)MP * (MP + 1) + 3 * MP
                                                                 : (size_t)MP * (MP + 4);
}

// Shared-memory layout of the tile kernel (offsets in bytes).
struct TileLayout {
  size_t halo, dh, tap, scr, total;
};
template <int MP, typename S, typename T, int TI, int TJ>
__host__ __device__ TileLayout tile_layout(int w) {
  TileLayout L;
  const size_t ncell = (size_t)(TI + w - 1) * (TJ + w - 1);
  L.halo = 0;
  L.dh = align16(ncell * 2 * MP * sizeof(S));
  L.tap = align16(L.dh + ncell * 2 * sizeof(S));
  L.scr = align16(L.tap + (size_t)w * w * sizeof(T));
  L.total = L.scr + (size_t)TI * TJ * scratch_elems<MP, T>() * sizeof(T);
  return L;
}

// wbar, W from the eigenpairs (lane j: eigenvector column v, eigenvalue lam) and
// the update of the node's two rows; writes Xa, the mean and the spread.
template <int MP, typename S, typename T>
__device__ __forceinline__ void transform_apply(const T (&v)[MP], T lam, T cd, int m,
                                                S *__restrict__ xrow, S *__restrict__ mean_out,
                                                S *__restrict__ spread_out, T *__restrict__ scr,
                                                int *__restrict__ counters) {
  const int lane = threadIdx.x & 31;
  const bool col = lane < MP;
  const bool mem = lane < m;
  T *vt = scr;                      // vt[i*(MP+1)+j] = V[i][j]
  T *vec = scr + MP * (MP + 1);     // [3][MP]
  const T x0 = mem ? T(xrow[lane]) : T(0);
  const T x1 = mem ? T(xrow[m + lane]) : T(0);
  const T inv_m = T(1) / T(m);
  const T xb0 = lk_warp_sum(x0) * inv_m;
  const T xb1 = lk_warp_sum(x1) * inv_m;
  const T xp0 = mem ? x0 - xb0 : T(0);
  const T xp1 = mem ? x1 - xb1 : T(0);
  __syncwarp();
  if (col) {
    vec[lane] = cd;
    vec[MP + lane] = xp0;
    vec[2 * MP + lane] = xp1;
#pragma unroll
    for (int k = 0; k < MP; ++k) vt[k * (MP + 1) + lane] = v[k];
  }
  __syncwarp();
  T u = T(0), g0 = T(0), g1 = T(0);
#pragma unroll
  for (int k = 0; k < MP; ++k) {
    u = fma(v[k], vec[k], u);               // (V^T C d)_lane
    g0 = fma(v[k], vec[MP + k], g0);        // (X'_0 V)_lane
    g1 = fma(v[k], vec[2 * MP + k], g1);    // (X'_1 V)_lane
  }
  const T z = u / lam;
  const T P0 = lk_warp_sum(g0 * z);           // X'_0 wbar
  const T P1 = lk_warp_sum(g1 * z);
  // every eigenvector gets its root: a warm-started sweep leaves the padding's
  // unit eigenvectors (lambda = 1) in arbitrary columns, and their projections
  // g0, g1 of the zero-padded anomalies are exactly zero
  const T sroot = col ? sqrt(T(m - 1) / lam) : T(0);
  __syncwarp();
  if (col) {
    vec[MP + lane] = g0 * sroot;
    vec[2 * MP + lane] = g1 * sroot;
  }
  __syncwarp();
  T q0 = T(0), q1 = T(0);
  if (col) {
    const T *vr = vt + lane * (MP + 1);
#pragma unroll
    for (int j = 0; j < MP; ++j) {
      q0 = fma(vr[j], vec[MP + j], q0);        // (X'_0 W)_lane
      q1 = fma(vr[j], vec[2 * MP + j], q1);
    }
  }
  const T xa0 = xb0 + P0 + q0;
  const T xa1 = xb1 + P1 + q1;
  if (mem) {
    xrow[lane] = S(xa0);
    xrow[m + lane] = S(xa1);
  }
  const T mu0 = lk_warp_sum(mem ? xa0 : T(0)) * inv_m;
  const T mu1 = lk_warp_sum(mem ? xa1 : T(0)) * inv_m;
  const T e0 = mem ? xa0 - mu0 : T(0);
  const T e1 = mem ? xa1 - mu1 : T(0);
  const T sp0 = sqrt(lk_warp_sum(e0 * e0) / T(m - 1));
  const T sp1 = sqrt(lk_warp_sum(e1 * e1) / T(m - 1));
  if (lane == 0) {
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

// Stores the node's eigenbasis (column `lane` = v) for the next analysis; a
// non-finite basis is replaced by the identity.
template <int MP, typename T>
__device__ __forceinline__ void store_basis(const T (&v)[MP], float *__restrict__ U) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < MP; ++k) ok = ok && isfinite(v[k]);
  ok = __all_sync(FULL, ok);
  if (lane < MP) {
#pragma unroll
    for (int k = 0; k < MP; ++k) U[k * MP + lane] = ok ? float(v[k]) : (k == lane ? 1.f : 0.f);
  }
}

// FP64 (or accumulate-V) analysis of one node, starting from the identity.
template <int MP, typename S, typename T>
__device__ __forceinline__ void analyze_node_accum(const S *__restrict__ win,
                                                   const S *__restrict__ dwin, int stride,
                                                   const T *__restrict__ tap, int w, int m,
                                                   T alpha, T tol, int max_sweeps,
                                                   S *__restrict__ xrow, S *__restrict__ mean_out,
                                                   S *__restrict__ spread_out,
                                                   T *__restrict__ scr, int *__restrict__ counters,
                                                   float *__restrict__ U, T kappa_thr = T(0)) {
  const int lane = threadIdx.x & 31;
  T b[MP], diag, cd;
  gram<MP, S, T>(win, dwin, stride, tap, w, m, alpha, b, diag, cd);
  if (kappa_thr > T(0)) {
    // kappa_hat = 1 + tr(G) / alpha bounds the condition number of A: above the
    // threshold the FP32 mean solve may miss the stated accuracy; count the node
    const T trg = lk_warp_sum(lane < MP ? diag : T(0));
    if (lane == 0 && T(1) + trg / alpha > kappa_thr) atomicAdd(&counters[1], 1);
  }
  T v[MP];
#pragma unroll
  for (int k = 0; k < MP; ++k) v[k] = (k == lane) ? T(1) : T(0);
  jacobi<MP, T, true>(b, v, tol, max_sweeps, counters);
  const T nrm = dot4<MP, T>(b, b);
  const T lam = (lane < MP && nrm > T(0)) ? sqrt(nrm) : T(1);   // |A v_j| = lambda_j
  transform_apply<MP, S, T>(v, lam, cd, m, xrow, mean_out, spread_out, scr, counters);
  if (U) store_basis<MP, T>(v, U);
}

// Stages a tile's halo (slope anomalies and innovations of the padded grid)
// and the taper table in shared memory.
template <int MP, typename S, typename T, int TI, int TJ>
__device__ __forceinline__ void stage_tile(const LkInst &I, int i0, int j0, S *halo, S *dh, T *tap) {
  const int w = I.w, m = I.m;
  const int HJ = TJ + w - 1;
  const int ncell = (TI + w - 1) * HJ;
  const S *Ybp = static_cast<const S *>(I.Ybp);
  const S *dp = static_cast<const S *>(I.dp);
  const S *taper = static_cast<const S *>(I.taper);
  for (int e = threadIdx.x; e < ncell * 2 * MP; e += blockDim.x) {
    const int cell = e / (2 * MP);
    const int r = e - cell * 2 * MP;
    const int c = r / MP;
    const int mm = r - c * MP;
    const int hi = cell / HJ, hj = cell - (cell / HJ) * HJ;
    const size_t src = (size_t)(i0 + hi) * I.gs_cols + (j0 + hj);
    halo[e] = mm < m ? Ybp[(src * 2 + c) * m + mm] : S(0);
  }
  for (int e = threadIdx.x; e < ncell * 2; e += blockDim.x) {
    const int cell = e >> 1;
    const int hi = cell / HJ, hj = cell - (cell / HJ) * HJ;
    const size_t src = (size_t)(i0 + hi) * I.gs_cols + (j0 + hj);
    dh[e] = dp[src * 2 + (e & 1)];
  }
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) tap[e] = T(taper[e]);
}

// One width class: FP64 handles run the FP32 basis pass of the pair kernel
// (unless switched off) and one CTA per node (letkf_node64.cu); FP32 handles
// the two-columns-per-lane kernel (letkf_pair.cu), then the FP64 analysis of
// the nodes it queued.
template <int MP>
cudaError_t launch_class(letkf_ctx *h, int cls, void *mean, void *spread) {
  if (h->n_tiles[cls] == 0) return cudaSuccess;
  if (h->precision == 1) {
    if (h->fp64_warm) {
      const cudaError_t e = lk_launch_pair_basis(h, cls);
      if (e != cudaSuccess) return e;
    }
    return lk_launch_node64(h, cls, mean, spread);
  }
  cudaError_t e = lk_launch_pair(h, cls, mean, spread);
  if (e != cudaSuccess || h->fp64_kappa <= 0) return e;
  return lk_launch_list64(h, cls, mean, spread);
}

}  // namespace

int lk_num_tile_shapes() { return LK_NUM_SHAPES; }

void lk_tile_shape(int s, int *ti, int *tj) {
  switch (s) {
#define LK_CASE(id, a, b) \
  case id:                \
    *ti = a;              \
    *tj = b;              \
    return;
    LK_FOR_SHAPES(LK_CASE)
#undef LK_CASE
  }
  *ti = LK_TILE_I;
  *tj = LK_TILE_J;
}

int lk_width_class(int m) { return m <= 16 ? 0 : (m <= 32 ? 1 : 2); }

// Raises the dynamic shared-memory limit of the analysis kernels this handle uses.
cudaError_t lk_setup_analysis(letkf_ctx *h) {
  cudaError_t e = lk_setup_pair(h);
  bool wide = false;
  for (const LkInst &I : h->inst) wide = wide || I.mp > 32;
  if (e == cudaSuccess && wide && h->precision == 0) e = lk_setup_node64w();
  return e;
}

cudaError_t lk_launch_analysis_class(letkf_ctx *h, int cls, void *mean, void *spread) {
  cudaError_t e = cudaMemsetAsync(h->counters + 1, 0, 7 * sizeof(int), h->stream);
  if (e != cudaSuccess) return e;
  if (cls == 0) return launch_class<16>(h, 0, mean, spread);
  if (cls == 1) return launch_class<32>(h, 1, mean, spread);
  return launch_class<64>(h, 2, mean, spread);
}

// Every caller launches the observation kernel just before; it zeroes the
// counters this analysis counts into (no memset node breaks the launch chain).
cudaError_t lk_launch_analysis(letkf_ctx *h, void *mean, void *spread) {
  if (h->dom) return lk_launch_domains(h, mean, spread);
  cudaError_t e = launch_class<16>(h, 0, mean, spread);
  if (e == cudaSuccess) e = launch_class<32>(h, 1, mean, spread);
  if (e == cudaSuccess) e = launch_class<64>(h, 2, mean, spread);
  return e;
}

// ===========================================================================
// Allocation-free analysis (letkf_analyze_noalloc)
//
// For callers that cannot allocate device memory at run time (for example a
// real-time controller whose memory is fixed at start-up, or code running
// where cudaMalloc is not permitted), this entry point analyses one frame
// without creating a handle: its scratch (instance descriptor, work lists,
// node tables, slope-anomaly grid, innovations, counters) is the file-scope
// array below, which every GPU that loads the library holds until the process
// exits.
// ===========================================================================
namespace {

constexpr int NA_MAX_NSUB = 128;
constexpr int NA_MAX_W = 15;
constexpr int NA_MAX_M = 32;
constexpr int NA_TI = 2, NA_TJ = 4;
constexpr int NA_NN = NA_MAX_NSUB + 1;
constexpr int NA_GS = ((NA_NN + LK_TILE_MAX - 1) / LK_TILE_MAX) * LK_TILE_MAX + NA_MAX_W;
constexpr size_t NA_CELLS = (size_t)NA_GS * NA_GS;
constexpr int NA_MAX_TILES = ((NA_NN + NA_TI - 1) / NA_TI) * ((NA_NN + NA_TJ - 1) / NA_TJ);
// byte offsets inside the scratch array (each 256-aligned)
constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t NA_OFF_YBP = 0;
constexpr size_t NA_OFF_DP = al256(NA_OFF_YBP + NA_CELLS * 2 * NA_MAX_M * sizeof(float));
constexpr size_t NA_OFF_PID = al256(NA_OFF_DP + NA_CELLS * 2 * sizeof(float));
constexpr size_t NA_OFF_SAPS = al256(NA_OFF_PID + (size_t)NA_NN * NA_NN * sizeof(int));
constexpr size_t NA_OFF_PTS = al256(NA_OFF_SAPS + (size_t)NA_MAX_NSUB * NA_MAX_NSUB * sizeof(int2));
constexpr size_t NA_OFF_OBS = al256(NA_OFF_PTS + (size_t)NA_NN * NA_NN * sizeof(int2));
constexpr size_t NA_OFF_TILES = al256(NA_OFF_OBS + (size_t)NA_MAX_NSUB * NA_MAX_NSUB * sizeof(int2));
constexpr size_t NA_OFF_TAPER = al256(NA_OFF_TILES + (size_t)NA_MAX_TILES * sizeof(LkTile));
constexpr size_t NA_OFF_INST = al256(NA_OFF_TAPER + (size_t)NA_MAX_W * NA_MAX_W * sizeof(float));
constexpr size_t NA_OFF_COUNTERS = al256(NA_OFF_INST + sizeof(LkInst));
constexpr size_t NA_BYTES = al256(NA_OFF_COUNTERS + 8 * sizeof(int));

// The scratch. Host code must not pass this name to a kernel: it is a host-side
// stand-in; the device address comes from cudaGetSymbolAddress (na_scratch_address).
__device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Host-side tables, built under g_na_mutex and copied into the scratch.
std::mutex g_na_mutex;
int g_na_pid[NA_NN * NA_NN];
int2 g_na_saps[NA_MAX_NSUB * NA_MAX_NSUB];
int2 g_na_pts[NA_NN * NA_NN];
int2 g_na_obs[NA_MAX_NSUB * NA_MAX_NSUB];
LkTile g_na_tiles[NA_MAX_TILES];
float g_na_taper[NA_MAX_W * NA_MAX_W];
void *g_na_addr[256];          // scratch address per device, set once

void na_error(char *buf, size_t len, const char *msg) {
  if (buf && len) snprintf(buf, len, "%s", msg);
}

// Gaspari & Cohn (1999) 5th-order piecewise rational function of z = r / c.
double na_gaspari_cohn(double z) {
  z = fabs(z);
  if (z <= 1.0) return (((-0.25 * z + 0.5) * z + 0.625) * z - 5.0 / 3.0) * z * z + 1.0;
  if (z < 2.0)
    return ((((z / 12.0 - 0.5) * z + 0.625) * z + 5.0 / 3.0) * z - 5.0) * z + 4.0 - (2.0 / 3.0) / z;
  return 0.0;
}

// Variant of the analysis tile kernel for the allocation-free path: FP32,
// eigenvectors accumulated from the identity (no per-node basis store, no FP64
// queue), descriptor, tables and scratch read from the static array.
template <int MP>
__global__ void __launch_bounds__(NA_TI *NA_TJ * 32)
    analysis_noalloc_kernel(const LkInst *__restrict__ insts, const LkTile *__restrict__ tiles,
                            float *__restrict__ mean, float *__restrict__ spread, float tol,
                            int max_sweeps, float kappa_thr, int *__restrict__ counters) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LkTile tl = tiles[blockIdx.x];
  const LkInst &I = insts[tl.inst];
  const int w = I.w;
  const TileLayout L = tile_layout<MP, float, float, NA_TI, NA_TJ>(w);
  const int HJ = NA_TJ + w - 1;
  float *halo = reinterpret_cast<float *>(smem + L.halo);
  float *dh = reinterpret_cast<float *>(smem + L.dh);
  float *tap = reinterpret_cast<float *>(smem + L.tap);
  float *scr = reinterpret_cast<float *>(smem + L.scr);
  stage_tile<MP, float, float, NA_TI, NA_TJ>(I, tl.i0, tl.j0, halo, dh, tap);
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  const int ti = warp / NA_TJ, tj = warp - (warp / NA_TJ) * NA_TJ;
  const int i = tl.i0 + ti, j = tl.j0 + tj;
  if (i > I.nsub || j > I.nsub) return;
  const int pid = I.pid_map[i * (I.nsub + 1) + j];
  if (pid < 0) return;
  const int off = ti * HJ + tj;
  const int m = I.m;
  analyze_node_accum<MP, float, float>(halo + (size_t)off * 2 * MP, dh + off * 2, HJ, tap, w, m,
                                       float(I.alpha), tol, max_sweeps,
                                       static_cast<float *>(I.X) + (size_t)pid * 2 * m,
                                       mean ? mean + 2 * pid : nullptr,
                                       spread ? spread + 2 * pid : nullptr,
                                       scr + (size_t)warp * scratch_elems<MP, float>(), counters,
                                       nullptr, kappa_thr);
}

// Device address of the scratch on the current device; looked up once per device.
cudaError_t na_scratch_address(int dev, unsigned char **out) {
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  if (!g_na_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_addr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_na_addr[dev]);
  return cudaSuccess;
}

template <int MP>
cudaError_t na_setup_kernel(size_t smem_bytes) {
  return cudaFuncSetAttribute(analysis_noalloc_kernel<MP>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

}  // namespace

extern "C" letkf_status letkf_analyze_noalloc(const letkf_config *cfg, void *X_dev,
                                              const void *y_dev, void *mean_dev, void *spread_dev,
                                              void *stream, char *errbuf, size_t errlen) {
  if (!cfg || !cfg->subap_mask || !X_dev || !y_dev) {
    na_error(errbuf, errlen, "cfg, cfg->subap_mask, X_dev and y_dev are required");
    return LETKF_ERR_ARG;
  }
  const letkf_config &c = *cfg;
  if (c.nsub < 1 || c.nsub > NA_MAX_NSUB || c.m < 2 || c.m > NA_MAX_M || c.window < 1 ||
      c.window > NA_MAX_W) {
    na_error(errbuf, errlen,
             "size beyond the allocation-free maximum: nsub 1..128, m 2..32, window 1..15");
    return LETKF_ERR_ARG;
  }
  if (c.partition != 0) {
    na_error(errbuf, errlen, "the allocation-free analysis is per node (partition must be 0)");
    return LETKF_ERR_ARG;
  }
  if (c.precision != 0 || (c.taper != 0 && c.taper != 1) || !(c.rho > 0) || !(c.sigma2 > 0) ||
      !isfinite(c.rho) || !isfinite(c.sigma2)) {
    na_error(errbuf, errlen, "precision must be 0, taper 0 or 1, rho and sigma2 finite and > 0");
    return LETKF_ERR_ARG;
  }
  // The tables below are copied from host memory that the next call reuses: a
  // graph captured from this call would keep those host pointers, so capture
  // is refused (the status query cannot be captured either: it synchronises).
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess ||
      cap != cudaStreamCaptureStatusNone) {
    (void)cudaGetLastError();
    na_error(errbuf, errlen, "letkf_analyze_noalloc cannot be captured into a CUDA graph");
    return LETKF_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  unsigned char *base = nullptr;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (e == cudaSuccess) e = na_scratch_address(dev, &base);
  const int mp = c.m <= 16 ? 16 : 32;
  const size_t smem = mp == 16 ? tile_layout<16, float, float, NA_TI, NA_TJ>(c.window).total
                               : tile_layout<32, float, float, NA_TI, NA_TJ>(c.window).total;
  if (e == cudaSuccess) e = mp == 16 ? na_setup_kernel<16>(smem) : na_setup_kernel<32>(smem);
  if (e != cudaSuccess) {
    na_error(errbuf, errlen, cudaGetErrorString(e));
    return LETKF_ERR_CUDA;
  }

  // ---- node and window tables (host, static storage) ----
  const int ns = c.nsub, nn = ns + 1, w = c.window, hw = w / 2;
  for (int k = 0; k < nn * nn; ++k) g_na_pid[k] = -1;
  int n_sap = 0;
  for (int s = 0; s < ns; ++s)
    for (int t = 0; t < ns; ++t)
      if (c.subap_mask[(size_t)s * ns + t]) {
        g_na_obs[n_sap] = make_int2(0, n_sap);
        g_na_saps[n_sap++] = make_int2(s, t);
        g_na_pid[s * nn + t] = g_na_pid[(s + 1) * nn + t] = 0;
        g_na_pid[s * nn + t + 1] = g_na_pid[(s + 1) * nn + t + 1] = 0;
      }
  if (n_sap == 0) {
    na_error(errbuf, errlen, "subap_mask has no valid subaperture");
    return LETKF_ERR_ARG;
  }
  int n_pts = 0;
  for (int i = 0; i < nn; ++i)
    for (int j = 0; j < nn; ++j)
      if (g_na_pid[i * nn + j] == 0) {
        g_na_pid[i * nn + j] = n_pts;
        g_na_pts[n_pts++] = make_int2(i, j);
      }
  int n_tiles = 0;
  for (int i0 = 0; i0 < nn; i0 += NA_TI)
    for (int j0 = 0; j0 < nn; j0 += NA_TJ) {
      bool any = false;
      for (int di = 0; di < NA_TI; ++di)
        for (int dj = 0; dj < NA_TJ; ++dj) {
          const int i = i0 + di, j = j0 + dj;
          any = any || (i < nn && j < nn && g_na_pid[i * nn + j] >= 0);
        }
      if (any) g_na_tiles[n_tiles++] = LkTile{0, i0, j0, 0};
    }
  const double cl = c.loc_len > 0 ? c.loc_len : w / 4.0;
  for (int ds = 0; ds < w; ++ds)
    for (int dt = 0; dt < w; ++dt) {
      const double tau =
          c.taper == 1 ? na_gaspari_cohn(hypot(ds - hw + 0.5, dt - hw + 0.5) / cl) : 1.0;
      g_na_taper[ds * w + dt] = (float)(tau / c.sigma2);
    }
  const int gs = ((nn + LK_TILE_MAX - 1) / LK_TILE_MAX) * LK_TILE_MAX + w;
  LkInst inst;
  memset(&inst, 0, sizeof(inst));
  inst.nsub = ns;
  inst.m = c.m;
  inst.w = w;
  inst.h = hw;
  inst.mp = mp;
  inst.n_pts = n_pts;
  inst.n_sap = n_sap;
  inst.p = 2 * n_sap;
  inst.gs_rows = gs;
  inst.gs_cols = gs;
  inst.pid_map = reinterpret_cast<const int *>(base + NA_OFF_PID);
  inst.pts = reinterpret_cast<const int2 *>(base + NA_OFF_PTS);
  inst.saps = reinterpret_cast<const int2 *>(base + NA_OFF_SAPS);
  inst.X = X_dev;
  inst.Ybp = base + NA_OFF_YBP;
  inst.dp = base + NA_OFF_DP;
  inst.taper = base + NA_OFF_TAPER;
  inst.alpha = (c.m - 1) / c.rho;
  inst.a_ar1 = c.a_ar1;
  inst.noise_std = c.noise_std;

  // ---- scratch: tables in, grids cleared (cells outside the pupil must read 0) ----
  cudaStream_t st = (cudaStream_t)stream;
  const size_t cells = (size_t)gs * gs;
  struct Copy {
    size_t off;
    const void *src;
    size_t bytes;
  } copies[] = {{NA_OFF_PID, g_na_pid, (size_t)nn * nn * sizeof(int)},
                {NA_OFF_SAPS, g_na_saps, (size_t)n_sap * sizeof(int2)},
                {NA_OFF_PTS, g_na_pts, (size_t)n_pts * sizeof(int2)},
                {NA_OFF_OBS, g_na_obs, (size_t)n_sap * sizeof(int2)},
                {NA_OFF_TILES, g_na_tiles, (size_t)n_tiles * sizeof(LkTile)},
                {NA_OFF_TAPER, g_na_taper, (size_t)w * w * sizeof(float)},
                {NA_OFF_INST, &inst, sizeof(LkInst)}};
  for (const Copy &cp : copies)
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(base + cp.off, cp.src, cp.bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + NA_OFF_YBP, 0, cells * 2 * c.m * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + NA_OFF_DP, 0, cells * 2 * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + NA_OFF_COUNTERS, 0, 8 * sizeof(int), st);

  // ---- observation (shared kernel) and analysis (variant kernel) ----
  letkf_ctx tmp;
  tmp.stream = st;
  tmp.precision = 0;
  tmp.n_inst = 1;
  tmp.d_inst = reinterpret_cast<LkInst *>(base + NA_OFF_INST);
  tmp.obs_items = reinterpret_cast<int2 *>(base + NA_OFF_OBS);
  tmp.sap_total = n_sap;
  tmp.p_total = 2 * n_sap;
  tmp.counters = reinterpret_cast<int *>(base + NA_OFF_COUNTERS);
  if (e == cudaSuccess) e = lk_launch_obs(&tmp, y_dev, nullptr);
  const int sweeps = c.max_sweeps > 0 ? c.max_sweeps : 20;
  const float kthr = c.fp64_kappa > 0 ? (float)c.fp64_kappa : 0.f;
  if (e == cudaSuccess) {
    const LkTile *tiles = reinterpret_cast<const LkTile *>(base + NA_OFF_TILES);
    if (mp == 16)
      analysis_noalloc_kernel<16><<<n_tiles, NA_TI * NA_TJ * 32, smem, st>>>(
          tmp.d_inst, tiles, (float *)mean_dev, (float *)spread_dev, 4e-6f, sweeps, kthr, tmp.counters);
    else
      analysis_noalloc_kernel<32><<<n_tiles, NA_TI * NA_TJ * 32, smem, st>>>(
          tmp.d_inst, tiles, (float *)mean_dev, (float *)spread_dev, 4e-6f, sweeps, kthr, tmp.counters);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    na_error(errbuf, errlen, cudaGetErrorString(e));
    return LETKF_ERR_CUDA;
  }
  return LETKF_OK;
}

extern "C" letkf_status letkf_noalloc_status(void *stream, int32_t *kappa_nodes) {
  if (kappa_nodes) *kappa_nodes = 0;
  int dev = 0;
  unsigned char *base = nullptr;
  cudaError_t e = cudaGetDevice(&dev);
  int c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (e == cudaSuccess) e = na_scratch_address(dev, &base);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemcpy(c, base + NA_OFF_COUNTERS, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return LETKF_ERR_CUDA;
  if (kappa_nodes) *kappa_nodes = c[1];
  if (c[0] & LK_BIT_NONFINITE) return LETKF_ERR_NONFINITE;
  if (c[0] & LK_BIT_NOCONVERGE) return LETKF_ERR_NOCONVERGE;
  return LETKF_OK;
}
