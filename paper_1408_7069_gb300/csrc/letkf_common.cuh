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

// Default node tile of one analysis CTA (TI x TJ nodes, one warp each); the
// autotuner may choose another of the compiled shapes.
constexpr int LK_TILE_I = 2;
constexpr int LK_TILE_J = 4;
// Padding of the slope-anomaly grid: tiles up to this many nodes per side keep
// their halo in bounds.
constexpr int LK_TILE_MAX = 8;
// The compiled analysis tile shapes (id, TI, TJ: nodes per CTA side), for the
// FP32 pair kernel and the FP64 tile kernel alike; letkf_tile_shape enumerates
// them. Each side divides LK_TILE_MAX, so the padded grid covers every halo.
#define LK_FOR_SHAPES(X) X(0, 2, 4) X(1, 4, 4) X(2, 2, 2) X(3, 1, 8) X(4, 1, 2) X(5, 1, 1)
constexpr int LK_NUM_SHAPES = 6;
// CTAs of the residual reduction per instance (fixed, so the sum order is fixed).
constexpr int LK_RES_BLOCKS = 128;
// Threads per CTA of the warp-per-item kernels (observation, forecast, reverse
// gathers): small CTAs spread a 16 m system's few hundred items over all SMs.
constexpr int LK_WARP_CTA = 64;
// Stop cosine of the FP64 sweeps that start from a stored FP32 eigenbasis
// (queued nodes of FP32 handles): the next sweep would rotate by about its
// square, far below what the FP32 outputs resolve.
constexpr double LK_WARM_STOP64 = 1e-8;

// One AO instance, as the kernels see it (device pointers, by-value copy in a
// device array). The real type of X, Yb, d, y, truth, taper and the outputs is
// float (precision 0) or double (precision 1).
struct LkInst {
  int nsub, m, w, h;        // h = w / 2
  int mp;                   // padded ensemble width of the kernels (16, 32, 48 or 64)
  int n_pts, n_sap, p;
  int gs_rows, gs_cols;     // padded subaperture grid: cell (s+h, t+h) holds subap (s, t)
  const int *pid_map;       // [(nsub+1)^2] node -> point id or -1
  const int2 *pts;          // [n_pts] (i, j)
  const int2 *saps;         // [n_sap] (s, t)
  void *X;                  // [n_pts][2][m]
  void *Ybp;                // [gs_rows][gs_cols][2][m]
  void *dp;                 // [gs_rows][gs_cols][2]
  const void *taper;        // [w*w] tau / sigma2
  float *basis;             // [n_pts][mp][mp] last eigenbasis (FP32 warm start)
  double *basis64;          // FP64 handles: [n_pts][mp][mp] FP64 eigenbasis the reverse mode records
  const float *bank;        // [bank_B][bank_G][bank_G] or NULL
  int bank_B, bank_G;
  double alpha;             // (m - 1) / rho
  double a_ar1, noise_std;
  unsigned long long seed;
  long long y_off;          // offset of this instance in concatenated slopes
  long long node_off;       // ... in concatenated node arrays (truth, mean/spread rows)
  long long noise_off;      // ... in concatenated [n_pts][m] noise
  long long state_off;      // ... in the concatenated ensemble
  // Deformable mirror (letkf_set_dm; dm = 0: none, the pseudo-open-loop form):
  // influence matrix N, command matrix P and D1 N as CSR over the nodes, the
  // commands u [3][n_pts] (slot f % 3 holds the command computed after
  // forecast number f, f the forecast counter *fcount), the predicted phase
  // pmean [n_pts] (written by the forecast) and the correction cor = N u_{k-1}.
  int dm;
  const int *n_ptr, *n_idx, *p_ptr, *p_idx, *dn_ptr, *dn_idx;
  const void *n_val, *p_val, *dn_val;
  void *u, *pmean, *cor;
  const long long *fcount;
};

// Work items.
struct LkTile {             // one analysis CTA: instance, tile origin (node coordinates)
  int inst, i0, j0, cost;
};

struct LkAdjWork;           // reverse-mode workspace (letkf_adjoint.cu)
struct LkDom;               // local-domain tables (letkf_domains.cu)

struct letkf_ctx {
  letkf_config cfg;         // first instance's config (host pointers cleared)
  std::vector<letkf_config> cfgs;   // every instance's config (host pointers cleared)
  cudaStream_t stream = nullptr;
  int device = 0;
  int precision = 0;
  size_t rsz = 4;           // bytes of the real type
  double tol32 = 4e-6, tol64 = 1e-13, fp64_kappa = 300;
  double stop32 = 1e-3;             // FP32 Jacobi stops after a sweep with all cosines <= this
  int max_sweeps = 20;
  int keep_basis = 0;               // store every node's eigenbasis (reverse mode needs it)

  int n_inst = 0;
  std::vector<LkInst> inst;         // host copies of the descriptors
  LkInst *d_inst = nullptr;         // device copies
  long long n_pts_total = 0, p_total = 0, state_total = 0, noise_total = 0;
  long long sap_total = 0;

  // work lists (device)
  int2 *obs_items = nullptr;        // [sap_total] (inst, subap)
  int2 *node_items = nullptr;       // [n_pts_total] (inst, point)
  LkTile *tiles[3] = {nullptr, nullptr, nullptr};   // per width class 16 / 32 / 64
  int n_tiles[3] = {0, 0, 0};
  int tile_shape[3] = {0, 0, 0};    // index into the compiled tile shapes, per class
  int tile_split[3] = {0, 0, 0};    // class 2: leading tiles of MP = 64 instances (MP = 48 after)
  int row_split[3] = {1, 1, 1};     // 2: each column's rows on two lanes (classes 0 and 1, FP32)
  int fp64_warm = 1;                // FP64 handles: FP32 basis pass, then the FP64 sweep from it
  std::vector<LkTile> tiles_host[3];

  // device buffers (single allocations sliced per instance)
  void *X = nullptr, *Ybp = nullptr, *dp = nullptr, *taper = nullptr;
  int *pid_map = nullptr;
  int2 *pts = nullptr, *saps = nullptr;
  float *bank = nullptr, *basis = nullptr;
  double *basis64 = nullptr;        // FP64 handles: the FP64 eigenbases the reverse mode records
  int *counters = nullptr;          // [0] status bits, [1] FP64 queue length, [2] max sweeps, [3] total sweeps
  int2 *worklist = nullptr;         // [n_pts_total] (inst, point) queued for FP64
  long long *frame = nullptr;       // [0] forecast counter, [1] frame index within letkf_run
  double2 *partial = nullptr;       // [n_inst][LK_RES_BLOCKS] residual partial sums
  void *noise_pre = nullptr;        // [noise_total] the frame's forecast noise, drawn ahead
  int *tickets = nullptr;           // [n_inst + 1] last-CTA counters: residual per instance, forecast

  // host copies
  std::vector<int32_t> pts_host, wslopes_host;
  long long frame_host = 0;

  // graph of one closed-loop frame (letkf_run)
  cudaGraphExec_t graph = nullptr;
  const void *graph_y = nullptr, *graph_truth = nullptr;
  const double *graph_resvar = nullptr;
  // graph of a whole run of frames (letkf_run_graph)
  cudaGraphExec_t mgraph = nullptr;
  int mgraph_frames = 0;
  const void *mgraph_y = nullptr, *mgraph_truth = nullptr;
  const double *mgraph_resvar = nullptr;
  const unsigned long long *mgraph_stamps = nullptr;

  LkAdjWork *adj = nullptr;         // letkf_grad buffers and graph, built on first use
  // multi-actuator local domains (cfg.partition > 0): tables, and the host
  // geometry they are rebuilt from when sigma2 or the taper changes
  LkDom *dom = nullptr;
  std::vector<int> dom_pid;
  std::vector<int2> dom_pts, dom_saps;

  // letkf_step: pinned staging and device copies of one frame's inputs and
  // outputs (y, truth, mean, resvar), and its graphs without / with truth
  unsigned char *step_pin = nullptr, *step_dev = nullptr;
  size_t step_off[4] = {0, 0, 0, 0};
  cudaGraphExec_t step_graph[2] = {nullptr, nullptr};

  // Second stream of a handle on a user stream: the residual runs on it beside
  // the observation kernel (fork / join events); ev_out marks a step's
  // downloads, so that letkf_step returns while its forecast still runs.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_out = nullptr;

  // deformable-mirror buffers (letkf_set_dm), single allocation per kind
  void *dm_buf = nullptr;           // N, P, D1 N (CSR) and u, pmean, cor
  unsigned char *dm_wfs_y = nullptr;   // letkf_run_dm: the simulated measurement [p]

  std::string err;
};

// Launchers (letkf_kernels.cu / letkf_analysis.cu). All enqueue on h->stream.
// run_idx (device) selects element *run_idx of a sequence (y, truth, resvar);
// NULL means element 0. y, truth, mean, spread and noise are concatenated over
// the instances in instance order.
cudaError_t lk_launch_obs(letkf_ctx *h, const void *y, const long long *run_idx);
// Observation of one frame with, in the same launch, its residual (truth and
// resvar given) and the model noise of the frame's forecast (noise_out given,
// [n_pts][m] at each instance's noise_off). Not with a deformable mirror, whose
// residual needs N u first, nor without subapertures.
cudaError_t lk_launch_obs_residual(letkf_ctx *h, const void *y, const void *truth,
                                   double *resvar, const long long *run_idx, void *noise_out);
cudaError_t lk_launch_analysis(letkf_ctx *h, void *mean, void *spread);
cudaError_t lk_launch_analysis_class(letkf_ctx *h, int cls, void *mean, void *spread);
// The forecast also advances the forecast counter and the run index (frame[0..1]).
cudaError_t lk_launch_forecast(letkf_ctx *h, const void *noise);
cudaError_t lk_launch_residual(letkf_ctx *h, const void *truth, double *resvar,
                               const long long *run_idx, double *piston = nullptr);
// The same on another stream of the handle's device.
cudaError_t lk_launch_residual_on(letkf_ctx *h, cudaStream_t stream, const void *truth,
                                  double *resvar, const long long *run_idx, double *piston);
cudaError_t lk_launch_basis_reset(letkf_ctx *h);   // warm-start eigenbases -> identity
// Deformable mirror (letkf_dm.cu): cor = N u_{k-1} on `stream` (before a
// residual), u_k = P pmean (after a forecast), and the simulated measurement
// y_k = D1 (phi_prev - N u_{k-2}) + w_k of a closed loop (phi_prev NULL: zero).
cudaError_t lk_launch_dm_cor(letkf_ctx *h, cudaStream_t stream);
cudaError_t lk_launch_dm_control(letkf_ctx *h);
cudaError_t lk_launch_dm_wfs(letkf_ctx *h, const void *truth_seq, const void *wnoise_seq,
                             const long long *run_idx, void *y_out);
cudaError_t lk_launch_dm_get(letkf_ctx *h, void *out);
// Writes the global timer (ns) into *dst once the preceding work has completed.
cudaError_t lk_launch_stamp(letkf_ctx *h, unsigned long long *dst);
cudaError_t lk_setup_analysis(letkf_ctx *h);
// FP32 analysis of width class cls, two columns per lane (letkf_pair.cu).
cudaError_t lk_launch_pair(letkf_ctx *h, int cls, void *mean, void *spread);
cudaError_t lk_setup_pair(letkf_ctx *h);
// FP64 analysis with one CTA of four warps per node (letkf_node64.cu): every
// node of width class cls (0: MP 16, 1: MP 32) of an FP64 handle, or the nodes
// the pair kernel queued in class cls of an FP32 handle.
cudaError_t lk_launch_node64(letkf_ctx *h, int cls, void *mean, void *spread);
cudaError_t lk_launch_list64(letkf_ctx *h, int cls, void *mean, void *spread);
// Shared-memory limit of the wide class's FP64 list kernel (MP = 48 / 64 queue).
cudaError_t lk_setup_node64w();

// Whether width class cls of the handle can take tile shape `shape`: FP32
// handles need whole warps of nodes and, in class 2 (one node per warp), at
// most 8 nodes per tile. (FP64 handles take any shape, which they ignore.)
bool lk_shape_ok(const letkf_ctx *h, int cls, int shape);
bool lk_shape_split_ok(const letkf_ctx *h, int cls, int shape, int split);
cudaError_t lk_launch_pair_basis(letkf_ctx *h, int cls);
int lk_num_tile_shapes();
void lk_tile_shape(int s, int *ti, int *tj);
int lk_width_class(int m);          // 0: m <= 16, 1: m <= 32, 2: m <= 64
void lk_adjoint_release(letkf_ctx *h);  // frees the letkf_grad workspace (and its graph)
// Gaspari & Cohn (1999) 5th-order piecewise rational function of z = r / c.
double lk_gaspari_cohn(double z);
// Local domains (letkf_domains.cu): build / rebuild the tables of a
// single-instance handle with cfg.partition > 0, free them, analyse.
letkf_status lk_domains_build(letkf_ctx *h, const letkf_config &c, const std::vector<int> &pid,
                              const std::vector<int2> &pts, const std::vector<int2> &saps,
                              std::string &err);
letkf_status lk_domains_set_params(letkf_ctx *h, const letkf_config &c,
                                   const std::vector<int> &pid, const std::vector<int2> &pts,
                                   const std::vector<int2> &saps, std::string &err);
void lk_domains_release(letkf_ctx *h);
int lk_domain_count(const letkf_ctx *h);
int lk_domain_of_nodes(const letkf_ctx *h, int *node_dom_host);
int lk_domain_obs_counts(const letkf_ctx *h, int *obs_host);
cudaError_t lk_launch_domains(letkf_ctx *h, void *mean, void *spread);
// The global ETKF for m > 128 (letkf_global.cu): Newton-Schulz root, refined
// mean, matrix-product apply, from the FP64 Gram partials.
int lk_ns_tile();
size_t lk_ns_workspace_bytes(int mpt, long long n_pad);
cudaError_t lk_launch_ns_global(letkf_ctx *h, const double *gpart, const double *cpart,
                                int kchunks, int mpt, int iters, void *ws, void *mean,
                                void *spread);

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

// Programmatic dependent launch of the per-frame kernels: each is launched
// with lk_launch_pdl, so that it can be scheduled while its predecessor on the
// stream drains; its first statement is lk_pdl_wait(), which returns once the
// predecessor grid has completed and its writes are visible (a no-op for a
// kernel launched without the attribute). The residual and forecast kernels
// then call lk_pdl_trigger(), letting the next kernel launch at once. The
// observation and analysis kernels do not: an analysis launched early has its
// CTAs placed on SMs that are still busy, several to an SM, which doubles the
// time of a latency-bound analysis that does not fill the GPU (measured on the
// 16 m system); their dependents launch as their CTAs exit.
__device__ __forceinline__ void lk_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void lk_pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t lk_launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
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
