// Host implementation of the C ABI declared in include/letkf.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "letkf_common.cuh"

cudaError_t lk_setup_analysis(letkf_ctx *h);

namespace {

thread_local std::string g_create_error;

letkf_status fail(letkf_ctx *h, letkf_status st, const std::string &msg) {
  if (h)
    h->err = msg;
  else
    g_create_error = msg;
  return st;
}

letkf_status cuda_fail(letkf_ctx *h, cudaError_t e, const char *what) {
  return fail(h, LETKF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LK_CUDA(h, call)                                  \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

// Gaspari & Cohn (1999) compactly supported 5th-order piecewise rational
// function of z = r / c (their Eq. 4.10): 1 at z = 0, 0 for z >= 2.
double gaspari_cohn(double z) {
  z = fabs(z);
  if (z <= 1.0) {
    const double z2 = z * z, z3 = z2 * z;
    return ((-0.25 * z + 0.5) * z + 0.625) * z3 - (5.0 / 3.0) * z2 + 1.0;
  }
  if (z < 2.0) {
    const double z2 = z * z;
    return (((z / 12.0 - 0.5) * z + 0.625) * z + 5.0 / 3.0) * z2 - 5.0 * z + 4.0 - (2.0 / 3.0) / z;
  }
  return 0.0;
}

template <typename T>
letkf_status upload(letkf_ctx *h, T **dst, const void *src, size_t bytes) {
  cudaError_t e = cudaMalloc((void **)dst, bytes ? bytes : 16);
  if (e != cudaSuccess) return fail(h, LETKF_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  if (src && bytes) {
    e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy");
  }
  return LETKF_OK;
}

void release(letkf_ctx *h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  void *bufs[] = {h->X,        h->Ybp,      h->dp,       h->taper,    h->pid_map,
                  h->pts,      h->saps,     h->tiles,    h->bank,     h->counters,
                  h->worklist, h->frame,    h->basis,    h->partial,  h->zero_scalar};
  for (void *p : bufs)
    if (p) cudaFree(p);
}

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      return;
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

letkf_status enqueue_frame(letkf_ctx *h, const void *y_seq, const void *truth_seq,
                           double *resvar) {
  const long long *ridx = h->frame + 1;
  if (truth_seq && resvar) LK_CUDA(h, lk_launch_residual(h, truth_seq, resvar, ridx));
  LK_CUDA(h, lk_launch_obs(h, y_seq, ridx));
  LK_CUDA(h, lk_launch_analysis(h, nullptr, nullptr));
  LK_CUDA(h, lk_launch_forecast(h, nullptr));
  LK_CUDA(h, lk_launch_tick(h));
  return LETKF_OK;
}

}  // namespace

extern "C" {

letkf_status letkf_create(const letkf_config *cfg, void *stream, letkf_t *out) {
  if (!out) return fail(nullptr, LETKF_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, LETKF_ERR_ARG, "cfg is NULL");
  const letkf_config &c = *cfg;
  if (c.nsub < 1 || c.nsub > 1024) return fail(nullptr, LETKF_ERR_ARG, "nsub must be in 1..1024");
  if (!c.subap_mask) return fail(nullptr, LETKF_ERR_ARG, "subap_mask is NULL");
  if (c.m < 2 || c.m > 32) return fail(nullptr, LETKF_ERR_ARG, "m must be in 2..32");
  if (c.window < 1 || c.window > 31) return fail(nullptr, LETKF_ERR_ARG, "window must be in 1..31");
  if (c.taper != 0 && c.taper != 1) return fail(nullptr, LETKF_ERR_ARG, "taper must be 0 or 1");
  if (!(c.rho > 0) || !(c.sigma2 > 0) || !isfinite(c.rho) || !isfinite(c.sigma2))
    return fail(nullptr, LETKF_ERR_ARG, "rho and sigma2 must be finite and > 0");
  if (!isfinite(c.a_ar1) || !isfinite(c.noise_std))
    return fail(nullptr, LETKF_ERR_ARG, "a_ar1 and noise_std must be finite");
  if (c.precision != 0 && c.precision != 1) return fail(nullptr, LETKF_ERR_ARG, "precision must be 0 or 1");
  if (c.noise_bank && (c.bank_B < 1 || c.bank_G < 1))
    return fail(nullptr, LETKF_ERR_ARG, "bank_B and bank_G must be >= 1 with a noise bank");

  letkf_ctx *h = new (std::nothrow) letkf_ctx();
  if (!h) return fail(nullptr, LETKF_ERR_NOMEM, "host allocation failed");
  h->cfg = c;
  h->cfg.subap_mask = nullptr;
  h->cfg.noise_bank = nullptr;
  h->stream = (cudaStream_t)stream;
  h->precision = c.precision;
  h->rsz = c.precision ? sizeof(double) : sizeof(float);
  h->mp = c.m <= 16 ? 16 : 32;
  h->max_sweeps = c.max_sweeps > 0 ? c.max_sweeps : 20;
  h->alpha = (c.m - 1) / c.rho;
  h->tol32 = 4e-6;
  h->tol64 = 1e-13;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return fail(nullptr, LETKF_ERR_CUDA, "no CUDA device");
  }

  // ---- geometry (host) ----
  const int ns = c.nsub, nn = ns + 1, w = c.window, hw = w / 2;
  std::vector<uint8_t> mask(c.subap_mask, c.subap_mask + (size_t)ns * ns);
  std::vector<int> pid((size_t)nn * nn, -1);
  std::vector<int2> saps;
  for (int s = 0; s < ns; ++s)
    for (int t = 0; t < ns; ++t)
      if (mask[(size_t)s * ns + t]) {
        saps.push_back(make_int2(s, t));
        pid[(size_t)s * nn + t] = pid[(size_t)(s + 1) * nn + t] = 0;
        pid[(size_t)s * nn + t + 1] = pid[(size_t)(s + 1) * nn + t + 1] = 0;
      }
  if (saps.empty()) {
    delete h;
    return fail(nullptr, LETKF_ERR_ARG, "subap_mask has no valid subaperture");
  }
  std::vector<int2> pts;
  for (int i = 0; i < nn; ++i)
    for (int j = 0; j < nn; ++j)
      if (pid[(size_t)i * nn + j] == 0) {
        pid[(size_t)i * nn + j] = (int)pts.size();
        pts.push_back(make_int2(i, j));
      }
  h->g.nsub = ns;
  h->g.m = c.m;
  h->g.w = w;
  h->g.h = hw;
  h->g.n_pts = (int)pts.size();
  h->g.n_sap = (int)saps.size();
  h->g.p = 2 * h->g.n_sap;
  const int tiles_i = (nn + LK_TILE_I - 1) / LK_TILE_I, tiles_j = (nn + LK_TILE_J - 1) / LK_TILE_J;
  h->g.gs_rows = tiles_i * LK_TILE_I + w;
  h->g.gs_cols = tiles_j * LK_TILE_J + w;
  h->pts_host.resize(2 * pts.size());
  h->wslopes_host.resize(pts.size());
  for (size_t k = 0; k < pts.size(); ++k) {
    h->pts_host[2 * k] = pts[k].x;
    h->pts_host[2 * k + 1] = pts[k].y;
    int cnt = 0;
    for (int s = pts[k].x - hw; s < pts[k].x - hw + w; ++s)
      for (int t = pts[k].y - hw; t < pts[k].y - hw + w; ++t)
        if (s >= 0 && s < ns && t >= 0 && t < ns && mask[(size_t)s * ns + t]) cnt += 2;
    h->wslopes_host[k] = cnt;
  }
  // taper weights tau / sigma2 by window offset: the subaperture (s, t) =
  // (i - h + ds, j - h + dt) has its centre at (ds - h + 0.5, dt - h + 0.5) pitches from node (i, j)
  const double cl = c.loc_len > 0 ? c.loc_len : w / 4.0;
  std::vector<double> tap64((size_t)w * w);
  for (int ds = 0; ds < w; ++ds)
    for (int dt = 0; dt < w; ++dt) {
      const double dist = hypot(ds - hw + 0.5, dt - hw + 0.5);
      const double tau = c.taper == 1 ? gaspari_cohn(dist / cl) : 1.0;
      tap64[(size_t)ds * w + dt] = tau / c.sigma2;
    }
  std::vector<float> tap32(tap64.begin(), tap64.end());
  std::vector<int2> tiles;
  for (int a = 0; a < tiles_i; ++a)
    for (int b = 0; b < tiles_j; ++b) {
      bool any = false;
      for (int di = 0; di < LK_TILE_I && !any; ++di)
        for (int dj = 0; dj < LK_TILE_J && !any; ++dj) {
          const int i = a * LK_TILE_I + di, j = b * LK_TILE_J + dj;
          if (i < nn && j < nn && pid[(size_t)i * nn + j] >= 0) any = true;
        }
      if (any) tiles.push_back(make_int2(a * LK_TILE_I, b * LK_TILE_J));
    }
  h->n_tiles = (int)tiles.size();

  // ---- device state ----
  letkf_status st;
  const size_t npt = (size_t)h->g.n_pts, m = (size_t)c.m;
  const size_t ncell = (size_t)h->g.gs_rows * h->g.gs_cols;
#define LK_TRY(x)    \
  do {               \
    st = (x);        \
    if (st != LETKF_OK) { \
      g_create_error = h->err; \
      release(h);    \
      delete h;      \
      return st;     \
    }                \
  } while (0)
  LK_TRY(upload(h, &h->X, nullptr, npt * 2 * m * h->rsz));
  LK_TRY(upload(h, &h->Ybp, nullptr, ncell * 2 * m * h->rsz));
  LK_TRY(upload(h, &h->dp, nullptr, ncell * 2 * h->rsz));
  LK_TRY(upload(h, &h->taper, c.precision ? (const void *)tap64.data() : (const void *)tap32.data(),
                (size_t)w * w * h->rsz));
  LK_TRY(upload(h, &h->pid_map, pid.data(), pid.size() * sizeof(int)));
  LK_TRY(upload(h, &h->pts, pts.data(), pts.size() * sizeof(int2)));
  LK_TRY(upload(h, &h->saps, saps.data(), saps.size() * sizeof(int2)));
  LK_TRY(upload(h, &h->tiles, tiles.data(), tiles.size() * sizeof(int2)));
  LK_TRY(upload(h, &h->counters, nullptr, 4 * sizeof(int)));
  LK_TRY(upload(h, &h->worklist, nullptr, npt * sizeof(int)));
  LK_TRY(upload(h, &h->frame, nullptr, 2 * sizeof(long long)));
  LK_TRY(upload(h, &h->partial, nullptr, LK_RES_BLOCKS * sizeof(double2)));
  {
    // every node's eigenbasis starts as the identity
    const size_t mp = (size_t)h->mp;
    std::vector<float> eye(npt * mp * mp, 0.f);
    for (size_t g = 0; g < npt; ++g)
      for (size_t k = 0; k < mp; ++k) eye[(g * mp + k) * mp + k] = 1.f;
    LK_TRY(upload(h, &h->basis, eye.data(), eye.size() * sizeof(float)));
  }
  if (c.noise_bank) {
    h->bank_B = c.bank_B;
    h->bank_G = c.bank_G;
    LK_TRY(upload(h, &h->bank, c.noise_bank, (size_t)c.bank_B * c.bank_G * c.bank_G * sizeof(float)));
  }
#undef LK_TRY
  h->g.pid_map = h->pid_map;
  h->g.pts = h->pts;
  h->g.saps = h->saps;
  cudaError_t e = cudaMemset(h->X, 0, npt * 2 * m * h->rsz);
  if (e == cudaSuccess) e = cudaMemset(h->Ybp, 0, ncell * 2 * m * h->rsz);
  if (e == cudaSuccess) e = cudaMemset(h->dp, 0, ncell * 2 * h->rsz);
  if (e == cudaSuccess) e = cudaMemset(h->counters, 0, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->frame, 0, 2 * sizeof(long long));
  if (e == cudaSuccess) e = lk_setup_analysis(h);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    g_create_error = std::string("device set-up: ") + cudaGetErrorString(e);
    release(h);
    delete h;
    return LETKF_ERR_CUDA;
  }
  *out = h;
  return LETKF_OK;
}

letkf_status letkf_destroy(letkf_t h) {
  if (!h) return LETKF_OK;
  DeviceGuard dg(h->device);
  cudaStreamSynchronize(h->stream);
  release(h);
  delete h;
  return LETKF_OK;
}

letkf_status letkf_query(letkf_t h, int32_t *n_pts, int32_t *p, int32_t *m) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (n_pts) *n_pts = h->g.n_pts;
  if (p) *p = h->g.p;
  if (m) *m = h->g.m;
  return LETKF_OK;
}

letkf_status letkf_query_points(letkf_t h, int32_t *ij_host, int32_t *window_slopes_host) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (ij_host) memcpy(ij_host, h->pts_host.data(), h->pts_host.size() * sizeof(int32_t));
  if (window_slopes_host)
    memcpy(window_slopes_host, h->wslopes_host.data(), h->wslopes_host.size() * sizeof(int32_t));
  return LETKF_OK;
}

letkf_status letkf_get_state(letkf_t h, void *X_dev) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (!X_dev) return fail(h, LETKF_ERR_ARG, "X_dev is NULL");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaMemcpyAsync(X_dev, h->X, (size_t)h->g.n_pts * 2 * h->g.m * h->rsz,
                             cudaMemcpyDeviceToDevice, h->stream));
  return LETKF_OK;
}

letkf_status letkf_set_state(letkf_t h, const void *X_dev) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (!X_dev) return fail(h, LETKF_ERR_ARG, "X_dev is NULL");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaMemcpyAsync(h->X, X_dev, (size_t)h->g.n_pts * 2 * h->g.m * h->rsz,
                             cudaMemcpyDeviceToDevice, h->stream));
  return LETKF_OK;
}

letkf_status letkf_forecast(letkf_t h, const void *noise_dev) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (!noise_dev && !h->bank)
    return fail(h, LETKF_ERR_STATE, "no noise given and the handle has no noise bank");
  DeviceGuard dg(h->device);
  LK_CUDA(h, lk_launch_forecast(h, noise_dev));
  LK_CUDA(h, lk_launch_tick(h));
  h->frame_host += 1;
  return LETKF_OK;
}

letkf_status letkf_analyze(letkf_t h, const void *y_dev, void *mean_dev, void *spread_dev) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (!y_dev) return fail(h, LETKF_ERR_ARG, "y_dev is NULL");
  DeviceGuard dg(h->device);
  LK_CUDA(h, lk_launch_obs(h, y_dev, nullptr));
  LK_CUDA(h, lk_launch_analysis(h, mean_dev, spread_dev));
  return LETKF_OK;
}

letkf_status letkf_residual(letkf_t h, const void *truth_dev, double *resvar_dev) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (!truth_dev || !resvar_dev) return fail(h, LETKF_ERR_ARG, "truth_dev and resvar_dev are required");
  DeviceGuard dg(h->device);
  LK_CUDA(h, lk_launch_residual(h, truth_dev, resvar_dev, nullptr));
  return LETKF_OK;
}

letkf_status letkf_run(letkf_t h, int32_t frames, const void *y_seq_dev, const void *truth_seq_dev,
                       double *resvar_dev, int32_t use_graph) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (frames < 0) return fail(h, LETKF_ERR_ARG, "frames < 0");
  if (!y_seq_dev) return fail(h, LETKF_ERR_ARG, "y_seq_dev is NULL");
  if (!h->bank) return fail(h, LETKF_ERR_STATE, "letkf_run needs a noise bank");
  if (use_graph && h->stream == nullptr)
    return fail(h, LETKF_ERR_STATE, "graph capture needs a non-default stream");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaMemsetAsync(h->frame + 1, 0, sizeof(long long), h->stream));
  if (frames == 0) return LETKF_OK;
  if (use_graph) {
    if (!h->graph || h->graph_y != y_seq_dev || h->graph_truth != truth_seq_dev ||
        h->graph_resvar != resvar_dev) {
      if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
      }
      LK_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      letkf_status st = enqueue_frame(h, y_seq_dev, truth_seq_dev, resvar_dev);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
      if (st != LETKF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&h->graph, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
      h->graph_y = y_seq_dev;
      h->graph_truth = truth_seq_dev;
      h->graph_resvar = resvar_dev;
    }
    for (int k = 0; k < frames; ++k) LK_CUDA(h, cudaGraphLaunch(h->graph, h->stream));
  } else {
    for (int k = 0; k < frames; ++k) {
      letkf_status st = enqueue_frame(h, y_seq_dev, truth_seq_dev, resvar_dev);
      if (st != LETKF_OK) return st;
    }
  }
  h->frame_host += frames;
  return LETKF_OK;
}

letkf_status letkf_sync(letkf_t h) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaStreamSynchronize(h->stream));
  int bits = 0;
  LK_CUDA(h, cudaMemcpy(&bits, h->counters, sizeof(int), cudaMemcpyDeviceToHost));
  LK_CUDA(h, cudaMemset(h->counters, 0, sizeof(int)));
  if (bits & LK_BIT_NONFINITE) return fail(h, LETKF_ERR_NONFINITE, "non-finite slopes or ensemble");
  if (bits & LK_BIT_TIMEOUT) return fail(h, LETKF_ERR_TIMEOUT, "a bounded device wait gave up");
  if (bits & LK_BIT_NOCONVERGE)
    return fail(h, LETKF_ERR_NOCONVERGE, "a Jacobi eigensolve reached its sweep limit");
  return LETKF_OK;
}

letkf_status letkf_stats(letkf_t h, int32_t *fp64_points, int32_t *max_sweeps,
                         int32_t *total_sweeps) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaStreamSynchronize(h->stream));
  int c[4];
  LK_CUDA(h, cudaMemcpy(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost));
  if (fp64_points) *fp64_points = c[1];
  if (max_sweeps) *max_sweeps = c[2];
  if (total_sweeps) *total_sweeps = c[3];
  return LETKF_OK;
}

const char *letkf_last_error(letkf_t h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
