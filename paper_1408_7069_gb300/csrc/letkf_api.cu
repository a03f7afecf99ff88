// Host implementation of the C ABI declared in include/letkf.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "letkf_common.cuh"

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

#define LK_CUDA(h, call)                                      \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);  \
  } while (0)

double gaspari_cohn(double z) { return lk_gaspari_cohn(z); }

template <typename T>
letkf_status dalloc(letkf_ctx *h, T **dst, size_t bytes) {
  cudaError_t e = cudaMalloc((void **)dst, bytes ? bytes : 16);
  if (e != cudaSuccess)
    return fail(h, LETKF_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  return LETKF_OK;
}

letkf_status upload(letkf_ctx *h, void *dst, const void *src, size_t bytes) {
  if (!bytes) return LETKF_OK;
  cudaError_t e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  return e == cudaSuccess ? LETKF_OK : cuda_fail(h, e, "cudaMemcpy");
}

// Drops every captured graph of the handle (they hold kernel arguments and
// tile lists that a call is about to change).
void drop_graphs(letkf_ctx *h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  if (h->mgraph) cudaGraphExecDestroy(h->mgraph);
  h->mgraph = nullptr;
  for (cudaGraphExec_t &g : h->step_graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
  lk_adjoint_release(h);
}

void release(letkf_ctx *h) {
  drop_graphs(h);
  lk_domains_release(h);
  if (h->dm_buf) cudaFree(h->dm_buf);
  h->dm_buf = nullptr;
  for (cudaEvent_t ev : {h->ev_fork, h->ev_join, h->ev_out})
    if (ev) cudaEventDestroy(ev);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->step_pin) cudaFreeHost(h->step_pin);
  if (h->step_dev) cudaFree(h->step_dev);
  void *bufs[] = {h->X,          h->Ybp,      h->dp,       h->taper,    h->pid_map,
                  h->pts,        h->saps,     h->bank,     h->basis,    h->basis64,  h->counters,
                  h->worklist,   h->frame,    h->partial,  h->tickets,  h->d_inst,   h->obs_items,
                  h->node_items, h->tiles[0], h->tiles[1], h->tiles[2], h->noise_pre};
  for (void *p : bufs)
    if (p) cudaFree(p);
}

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

letkf_status check_config(const letkf_config &c) {
  if (c.nsub < 1 || c.nsub > 1024) return fail(nullptr, LETKF_ERR_ARG, "nsub must be in 1..1024");
  if (!c.subap_mask) return fail(nullptr, LETKF_ERR_ARG, "subap_mask is NULL");
  if (c.partition < 0 || c.partition > 64)
    return fail(nullptr, LETKF_ERR_ARG, "partition must be in 0..64");
  if (c.partition > 1 && (c.m < 2 || c.m > 128))
    return fail(nullptr, LETKF_ERR_ARG, "m must be in 2..128 with local domains");
  if (c.partition == 1 && (c.m < 2 || c.m > 1024))
    return fail(nullptr, LETKF_ERR_ARG, "m must be in 2..1024 for the global ETKF");
  if (c.partition > 0 && c.precision != 0)
    return fail(nullptr, LETKF_ERR_ARG, "local domains are analysed in FP32 (precision 0)");
  if (c.partition == 0 && (c.m < 2 || c.m > 64))
    return fail(nullptr, LETKF_ERR_ARG, "m must be in 2..64");
  if (c.precision == 1 && c.m > 32)
    return fail(nullptr, LETKF_ERR_ARG, "m must be in 2..32 with precision 1");
  if (c.window < 1 || c.window > 31) return fail(nullptr, LETKF_ERR_ARG, "window must be in 1..31");
  if (c.taper != 0 && c.taper != 1) return fail(nullptr, LETKF_ERR_ARG, "taper must be 0 or 1");
  if (!(c.rho > 0) || !(c.sigma2 > 0) || !isfinite(c.rho) || !isfinite(c.sigma2))
    return fail(nullptr, LETKF_ERR_ARG, "rho and sigma2 must be finite and > 0");
  if (!isfinite(c.a_ar1) || !isfinite(c.noise_std))
    return fail(nullptr, LETKF_ERR_ARG, "a_ar1 and noise_std must be finite");
  if (c.precision != 0 && c.precision != 1)
    return fail(nullptr, LETKF_ERR_ARG, "precision must be 0 or 1");
  if (c.noise_bank && (c.bank_B < 1 || c.bank_G < 1))
    return fail(nullptr, LETKF_ERR_ARG, "bank_B and bank_G must be >= 1 with a noise bank");
  return LETKF_OK;
}

// Per-instance host geometry before upload.
struct HostInst {
  std::vector<int> pid;
  std::vector<int2> pts, saps;
  std::vector<int32_t> wslopes;
  std::vector<double> taper;
};

// Taper weights tau / sigma2 by window offset: subaperture (s, t) = (i - h + ds, j - h + dt)
// has its centre at (ds - h + 0.5, dt - h + 0.5) pitches from node (i, j).
void taper_table(const letkf_config &c, std::vector<double> &tap) {
  const int w = c.window, hw = w / 2;
  const double cl = c.loc_len > 0 ? c.loc_len : w / 4.0;
  tap.resize((size_t)w * w);
  for (int ds = 0; ds < w; ++ds)
    for (int dt = 0; dt < w; ++dt) {
      const double tau = c.taper == 1 ? gaspari_cohn(hypot(ds - hw + 0.5, dt - hw + 0.5) / cl) : 1.0;
      tap[(size_t)ds * w + dt] = tau / c.sigma2;
    }
}

letkf_status upload_taper(letkf_ctx *h, const LkInst &I, const std::vector<double> &tap) {
  if (h->precision) return upload(h, (void *)I.taper, tap.data(), tap.size() * sizeof(double));
  std::vector<float> t32(tap.begin(), tap.end());
  return upload(h, (void *)I.taper, t32.data(), t32.size() * sizeof(float));
}

void build_geometry(const letkf_config &c, HostInst &g) {
  const int ns = c.nsub, nn = ns + 1, w = c.window, hw = w / 2;
  g.pid.assign((size_t)nn * nn, -1);
  g.saps.clear();
  g.pts.clear();
  for (int s = 0; s < ns; ++s)
    for (int t = 0; t < ns; ++t)
      if (c.subap_mask[(size_t)s * ns + t]) {
        g.saps.push_back(make_int2(s, t));
        g.pid[(size_t)s * nn + t] = g.pid[(size_t)(s + 1) * nn + t] = 0;
        g.pid[(size_t)s * nn + t + 1] = g.pid[(size_t)(s + 1) * nn + t + 1] = 0;
      }
  for (int i = 0; i < nn; ++i)
    for (int j = 0; j < nn; ++j)
      if (g.pid[(size_t)i * nn + j] == 0) {
        g.pid[(size_t)i * nn + j] = (int)g.pts.size();
        g.pts.push_back(make_int2(i, j));
      }
  g.wslopes.resize(g.pts.size());
  for (size_t k = 0; k < g.pts.size(); ++k) {
    int cnt = 0;
    for (int s = g.pts[k].x - hw; s < g.pts[k].x - hw + w; ++s)
      for (int t = g.pts[k].y - hw; t < g.pts[k].y - hw + w; ++t)
        if (s >= 0 && s < ns && t >= 0 && t < ns && c.subap_mask[(size_t)s * ns + t]) cnt += 2;
    g.wslopes[k] = cnt;
  }
  taper_table(c, g.taper);
}

int padded_grid(int nsub, int w) {
  return ((nsub + 1 + LK_TILE_MAX - 1) / LK_TILE_MAX) * LK_TILE_MAX + w;
}

// Analysis tiles of one width class for its current tile shape, most
// expensive first (cost: slopes in the tile's windows times mp^2).
letkf_status build_tiles(letkf_ctx *h, int cls, const std::vector<std::vector<int>> &pids) {
  int ti, tj;
  lk_tile_shape(h->tile_shape[cls], &ti, &tj);
  std::vector<LkTile> &tl = h->tiles_host[cls];
  tl.clear();
  for (int k = 0; k < h->n_inst; ++k) {
    const LkInst &I = h->inst[k];
    const int nn = I.nsub + 1;
    if (lk_width_class(I.m) != cls) continue;
    const std::vector<int> &pid = pids[k];
    for (int i0 = 0; i0 < nn; i0 += ti)
      for (int j0 = 0; j0 < nn; j0 += tj) {
        long long cost = 0;
        bool any = false;
        for (int di = 0; di < ti; ++di)
          for (int dj = 0; dj < tj; ++dj) {
            const int i = i0 + di, j = j0 + dj;
            if (i < nn && j < nn && pid[(size_t)i * nn + j] >= 0) {
              any = true;
              cost += h->wslopes_host[I.node_off + pid[(size_t)i * nn + j]];
            }
          }
        if (any) tl.push_back(LkTile{k, i0, j0, (int)(cost * I.mp * I.mp / 32)});
      }
  }
  // class 2 runs as two launches (MP = 64, then MP = 48), and class 1 of FP32
  // handles in the whole-column form too (ensembles of at most 24 members on
  // 24 columns, then the rest on 32): group by width first
  const bool narrow24 = cls == 1 && h->precision == 0 && h->row_split[1] == 1;
  auto first = [h, cls, narrow24](const LkTile &t) {
    const LkInst &I = h->inst[t.inst];
    return cls == 2 ? I.mp == 64 : (narrow24 && I.m <= 24);
  };
  std::stable_sort(tl.begin(), tl.end(), [&](const LkTile &a, const LkTile &b) {
    if (first(a) != first(b)) return first(a);
    return a.cost > b.cost;
  });
  h->tile_split[cls] = (int)std::count_if(tl.begin(), tl.end(), first);
  if (h->tiles[cls]) cudaFree(h->tiles[cls]);
  h->tiles[cls] = nullptr;
  letkf_status st = dalloc(h, &h->tiles[cls], tl.size() * sizeof(LkTile));
  if (st != LETKF_OK) return st;
  h->n_tiles[cls] = (int)tl.size();
  drop_graphs(h);          // they hold the old tile list
  return upload(h, h->tiles[cls], tl.data(), tl.size() * sizeof(LkTile));
}

letkf_status rebuild_tiles(letkf_ctx *h, int cls) {
  std::vector<std::vector<int>> pids(h->n_inst);
  for (int k = 0; k < h->n_inst; ++k) {
    const LkInst &I = h->inst[k];
    if (lk_width_class(I.m) != cls) continue;
    pids[k].resize((size_t)(I.nsub + 1) * (I.nsub + 1));
    cudaError_t e = cudaMemcpy(pids[k].data(), I.pid_map, pids[k].size() * sizeof(int),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy");
  }
  return build_tiles(h, cls, pids);
}

letkf_status build_handle(const letkf_config *cfgs, int n, void *stream, letkf_t *out) {
  if (!out) return fail(nullptr, LETKF_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfgs || n < 1) return fail(nullptr, LETKF_ERR_ARG, "need at least one configuration");
  for (int k = 0; k < n; ++k) {
    letkf_status st = check_config(cfgs[k]);
    if (st != LETKF_OK) return st;
    if (cfgs[k].precision != cfgs[0].precision)
      return fail(nullptr, LETKF_ERR_ARG, "all instances of a batch share one precision");
    if (cfgs[k].partition > 0 && n > 1)
      return fail(nullptr, LETKF_ERR_ARG, "local domains take a single-instance handle");
  }
  letkf_ctx *h = new (std::nothrow) letkf_ctx();
  if (!h) return fail(nullptr, LETKF_ERR_NOMEM, "host allocation failed");
  h->cfgs.assign(cfgs, cfgs + n);
  for (letkf_config &c : h->cfgs) {
    c.subap_mask = nullptr;
    c.noise_bank = nullptr;
  }
  h->cfg = h->cfgs[0];
  h->stream = (cudaStream_t)stream;
  h->precision = cfgs[0].precision;
  h->rsz = h->precision ? sizeof(double) : sizeof(float);
  h->max_sweeps = cfgs[0].max_sweeps > 0 ? cfgs[0].max_sweeps : 20;
  h->fp64_kappa = cfgs[0].fp64_kappa;
  h->n_inst = n;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return fail(nullptr, LETKF_ERR_CUDA, "no CUDA device");
  }
  std::vector<HostInst> geo(n);
  for (int k = 0; k < n; ++k) {
    build_geometry(cfgs[k], geo[k]);
    if (geo[k].saps.empty()) {
      delete h;
      return fail(nullptr, LETKF_ERR_ARG, "subap_mask has no valid subaperture");
    }
  }
  // ---- sizes and offsets ----
  h->inst.resize(n);
  size_t n_ybp = 0, n_dp = 0, n_tap = 0, n_pid = 0, n_basis = 0, n_bank = 0;
  for (int k = 0; k < n; ++k) {
    const letkf_config &c = cfgs[k];
    LkInst &I = h->inst[k];
    memset(&I, 0, sizeof(I));
    I.nsub = c.nsub;
    I.m = c.m;
    I.w = c.window;
    I.h = c.window / 2;
    // (domain handles use no per-node kernel and keep the smallest basis store)
    I.mp = c.partition > 0 ? 16 : c.m <= 16 ? 16 : (c.m <= 32 ? 32 : (c.m <= 48 ? 48 : 64));
    I.n_pts = (int)geo[k].pts.size();
    I.n_sap = (int)geo[k].saps.size();
    I.p = 2 * I.n_sap;
    I.gs_rows = padded_grid(c.nsub, c.window);
    I.gs_cols = padded_grid(c.nsub, c.window);
    I.alpha = (c.m - 1) / c.rho;
    I.a_ar1 = c.a_ar1;
    I.noise_std = c.noise_std;
    I.seed = c.seed;
    I.y_off = h->p_total;
    I.node_off = h->n_pts_total;
    I.noise_off = h->noise_total;
    I.state_off = h->state_total;
    h->p_total += I.p;
    h->n_pts_total += I.n_pts;
    h->noise_total += (long long)I.n_pts * I.m;
    h->state_total += 2LL * I.n_pts * I.m;
    h->sap_total += I.n_sap;
    n_ybp += (size_t)I.gs_rows * I.gs_cols * 2 * I.m;
    n_dp += (size_t)I.gs_rows * I.gs_cols * 2;
    n_tap += (size_t)I.w * I.w;
    n_pid += (size_t)(c.nsub + 1) * (c.nsub + 1);
    n_basis += (size_t)I.n_pts * I.mp * I.mp;
    if (c.noise_bank) n_bank += (size_t)c.bank_B * c.bank_G * c.bank_G;
  }
  letkf_status st = LETKF_OK;
#define LK_TRY(x)               \
  do {                          \
    st = (x);                   \
    if (st != LETKF_OK) {       \
      g_create_error = h->err;  \
      release(h);               \
      delete h;                 \
      return st;                \
    }                           \
  } while (0)
  LK_TRY(dalloc(h, &h->X, h->state_total * h->rsz));
  LK_TRY(dalloc(h, &h->Ybp, n_ybp * h->rsz));
  LK_TRY(dalloc(h, &h->dp, n_dp * h->rsz));
  LK_TRY(dalloc(h, &h->taper, n_tap * h->rsz));
  LK_TRY(dalloc(h, &h->pid_map, n_pid * sizeof(int)));
  LK_TRY(dalloc(h, &h->pts, h->n_pts_total * sizeof(int2)));
  LK_TRY(dalloc(h, &h->saps, h->sap_total * sizeof(int2)));
  LK_TRY(dalloc(h, &h->basis, n_basis * sizeof(float)));
  if (h->precision == 1) LK_TRY(dalloc(h, &h->basis64, n_basis * sizeof(double)));
  LK_TRY(dalloc(h, &h->bank, n_bank * sizeof(float)));
  LK_TRY(dalloc(h, &h->counters, 8 * sizeof(int)));
  LK_TRY(dalloc(h, &h->worklist, 3 * h->n_pts_total * sizeof(int2)));
  LK_TRY(dalloc(h, &h->frame, 2 * sizeof(long long)));
  LK_TRY(dalloc(h, &h->partial, (size_t)n * LK_RES_BLOCKS * sizeof(double2)));
  LK_TRY(dalloc(h, &h->noise_pre, (size_t)h->noise_total * h->rsz));
  LK_TRY(dalloc(h, &h->tickets, (size_t)(n + 1) * sizeof(int)));
  LK_TRY(dalloc(h, &h->d_inst, (size_t)n * sizeof(LkInst)));
  LK_TRY(dalloc(h, &h->obs_items, h->sap_total * sizeof(int2)));
  LK_TRY(dalloc(h, &h->node_items, h->n_pts_total * sizeof(int2)));
  if (h->stream) {
    cudaError_t es = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
    if (es == cudaSuccess) es = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (es == cudaSuccess) es = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
    if (es == cudaSuccess) es = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
    if (es != cudaSuccess) LK_TRY(cuda_fail(h, es, "stream / event creation"));
  }
  // ---- slice buffers, upload tables ----
  size_t o_ybp = 0, o_dp = 0, o_tap = 0, o_pid = 0, o_basis = 0, o_bank = 0, o_pts = 0, o_sap = 0;
  std::vector<int2> obs_items, node_items;
  std::vector<std::vector<int>> pids(n);
  for (int k = 0; k < n; ++k) {
    const letkf_config &c = cfgs[k];
    LkInst &I = h->inst[k];
    const HostInst &G = geo[k];
    I.X = static_cast<char *>(h->X) + I.state_off * h->rsz;
    I.Ybp = static_cast<char *>(h->Ybp) + o_ybp * h->rsz;
    I.dp = static_cast<char *>(h->dp) + o_dp * h->rsz;
    I.taper = static_cast<char *>(h->taper) + o_tap * h->rsz;
    I.pid_map = h->pid_map + o_pid;
    I.pts = h->pts + o_pts;
    I.saps = h->saps + o_sap;
    I.basis = h->basis + o_basis;
    I.basis64 = h->basis64 ? h->basis64 + o_basis : nullptr;
    LK_TRY(upload_taper(h, I, G.taper));
    LK_TRY(upload(h, (void *)I.pid_map, G.pid.data(), G.pid.size() * sizeof(int)));
    LK_TRY(upload(h, (void *)I.pts, G.pts.data(), G.pts.size() * sizeof(int2)));
    LK_TRY(upload(h, (void *)I.saps, G.saps.data(), G.saps.size() * sizeof(int2)));
    {
      const size_t mp = (size_t)I.mp;
      std::vector<float> eye((size_t)I.n_pts * mp * mp, 0.f);
      for (size_t g = 0; g < (size_t)I.n_pts; ++g)
        for (size_t q = 0; q < mp; ++q) eye[(g * mp + q) * mp + q] = 1.f;
      LK_TRY(upload(h, I.basis, eye.data(), eye.size() * sizeof(float)));
    }
    if (c.noise_bank) {
      I.bank = h->bank + o_bank;
      I.bank_B = c.bank_B;
      I.bank_G = c.bank_G;
      LK_TRY(upload(h, (void *)I.bank, c.noise_bank,
                    (size_t)c.bank_B * c.bank_G * c.bank_G * sizeof(float)));
      o_bank += (size_t)c.bank_B * c.bank_G * c.bank_G;
    }
    for (int q = 0; q < I.n_sap; ++q) obs_items.push_back(make_int2(k, q));
    for (int q = 0; q < I.n_pts; ++q) node_items.push_back(make_int2(k, q));
    for (size_t q = 0; q < G.pts.size(); ++q) {
      h->pts_host.push_back(G.pts[q].x);
      h->pts_host.push_back(G.pts[q].y);
      h->wslopes_host.push_back(G.wslopes[q]);
    }
    pids[k] = G.pid;
    o_ybp += (size_t)I.gs_rows * I.gs_cols * 2 * I.m;
    o_dp += (size_t)I.gs_rows * I.gs_cols * 2;
    o_tap += (size_t)I.w * I.w;
    o_pid += (size_t)(c.nsub + 1) * (c.nsub + 1);
    o_basis += (size_t)I.n_pts * I.mp * I.mp;
    o_pts += G.pts.size();
    o_sap += G.saps.size();
  }
  LK_TRY(upload(h, h->d_inst, h->inst.data(), (size_t)n * sizeof(LkInst)));
  LK_TRY(upload(h, h->obs_items, obs_items.data(), obs_items.size() * sizeof(int2)));
  LK_TRY(upload(h, h->node_items, node_items.data(), node_items.size() * sizeof(int2)));
  cudaError_t e = cudaMemset(h->X, 0, h->state_total * h->rsz);
  if (e == cudaSuccess) e = cudaMemset(h->Ybp, 0, n_ybp * h->rsz);
  if (e == cudaSuccess) e = cudaMemset(h->dp, 0, n_dp * h->rsz);
  if (e == cudaSuccess) e = cudaMemset(h->counters, 0, 8 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->frame, 0, 2 * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(h->tickets, 0, (size_t)(n + 1) * sizeof(int));
  if (e != cudaSuccess) LK_TRY(cuda_fail(h, e, "cudaMemset"));
  if (n == 1) {
    h->dom_pid = geo[0].pid;
    h->dom_pts = geo[0].pts;
    h->dom_saps = geo[0].saps;
  }
  if (cfgs[0].partition > 0) {
    letkf_status ds = lk_domains_build(h, cfgs[0], h->dom_pid, h->dom_pts, h->dom_saps, h->err);
    if (ds != LETKF_OK && h->err.empty()) h->err = "local-domain set-up failed";
    LK_TRY(ds);
  } else {
    for (int cls = 0; cls < 3; ++cls) LK_TRY(build_tiles(h, cls, pids));
  }
  e = lk_setup_analysis(h);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) LK_TRY(cuda_fail(h, e, "device set-up"));
#undef LK_TRY
  *out = h;
  return LETKF_OK;
}

bool all_have_banks(const letkf_ctx *h);

// Residual and observation of a frame. Both read the prediction ensemble
// only, so they share one launch (the residual's CTAs first), which also
// draws the frame's forecast noise when every instance has a bank (*drawn is
// set: the forecast then reads h->noise_pre). With a deformable mirror, whose
// residual needs N u first, the residual runs on a side stream beside the
// observation kernel and rejoins before the analysis overwrites the ensemble.
letkf_status enqueue_head(letkf_ctx *h, const void *y, const void *truth, double *resvar,
                          const long long *ridx, bool *drawn) {
  const bool res = truth && resvar;
  *drawn = false;
  if (!h->inst[0].dm && h->sap_total > 0) {
    *drawn = all_have_banks(h);
    LK_CUDA(h, lk_launch_obs_residual(h, y, res ? truth : nullptr, res ? resvar : nullptr, ridx,
                                      *drawn ? h->noise_pre : nullptr));
    return LETKF_OK;
  }
  const bool fork = res && h->side && h->stream;
  if (fork) {
    LK_CUDA(h, cudaEventRecord(h->ev_fork, h->stream));
    LK_CUDA(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    LK_CUDA(h, lk_launch_residual_on(h, h->side, truth, resvar, ridx, nullptr));
    LK_CUDA(h, cudaEventRecord(h->ev_join, h->side));
  } else if (res) {
    LK_CUDA(h, lk_launch_residual(h, truth, resvar, ridx));
  }
  LK_CUDA(h, lk_launch_obs(h, y, ridx));
  if (fork) LK_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  return LETKF_OK;
}

letkf_status enqueue_frame(letkf_ctx *h, const void *y_seq, const void *truth_seq,
                           double *resvar) {
  const long long *ridx = h->frame + 1;
  bool drawn;
  letkf_status st = enqueue_head(h, y_seq, truth_seq, resvar, ridx, &drawn);
  if (st != LETKF_OK) return st;
  LK_CUDA(h, lk_launch_analysis(h, nullptr, nullptr));
  LK_CUDA(h, lk_launch_forecast(h, drawn ? h->noise_pre : nullptr));
  return LETKF_OK;
}

// One frame from the step staging buffers: upload, (residual beside the)
// observation, analysis (mean into staging), download, then the forecast.
// ev_out is recorded after the downloads (an event node of the step graph),
// so that the caller can return its outputs while the forecast still runs.
letkf_status enqueue_step(letkf_ctx *h, bool with_truth) {
  unsigned char *yd = h->step_dev + h->step_off[0], *td = h->step_dev + h->step_off[1];
  unsigned char *md = h->step_dev + h->step_off[2], *rd = h->step_dev + h->step_off[3];
  unsigned char *yp = h->step_pin + h->step_off[0], *mp = h->step_pin + h->step_off[2];
  // y and truth are adjacent in the staging buffers: one upload covers both
  const size_t up = with_truth ? h->step_off[1] + h->n_pts_total * h->rsz : h->p_total * h->rsz;
  LK_CUDA(h, cudaMemcpyAsync(yd, yp, up, cudaMemcpyHostToDevice, h->stream));
  bool drawn;
  letkf_status st = enqueue_head(h, yd, with_truth ? td : nullptr,
                                 with_truth ? reinterpret_cast<double *>(rd) : nullptr, nullptr,
                                 &drawn);
  if (st != LETKF_OK) return st;
  LK_CUDA(h, lk_launch_analysis(h, md, nullptr));
  // mean and resvar are adjacent too: one download
  const size_t down = with_truth ? h->step_off[3] + h->n_inst * sizeof(double) - h->step_off[2]
                                 : 2 * h->n_pts_total * h->rsz;
  LK_CUDA(h, cudaMemcpyAsync(mp, md, down, cudaMemcpyDeviceToHost, h->stream));
  if (h->ev_out)
    LK_CUDA(h, cudaEventRecordWithFlags(h->ev_out, h->stream, cudaEventRecordExternal));
  LK_CUDA(h, lk_launch_forecast(h, drawn ? h->noise_pre : nullptr));
  return LETKF_OK;
}

// One frame of the simulated closed loop with a deformable mirror: residual
// against the correction, measurement of the residual phase, analysis of the
// pseudo-open-loop slopes, forecast and command.
letkf_status enqueue_frame_dm(letkf_ctx *h, const void *truth_seq, const void *wnoise_seq,
                              double *resvar) {
  const long long *ridx = h->frame + 1;
  if (resvar) LK_CUDA(h, lk_launch_residual(h, truth_seq, resvar, ridx));
  LK_CUDA(h, lk_launch_dm_wfs(h, truth_seq, wnoise_seq, ridx, h->dm_wfs_y));
  LK_CUDA(h, lk_launch_obs(h, h->dm_wfs_y, nullptr));
  LK_CUDA(h, lk_launch_analysis(h, nullptr, nullptr));
  LK_CUDA(h, lk_launch_forecast(h, nullptr));
  return LETKF_OK;
}

bool all_have_banks(const letkf_ctx *h) {
  for (const LkInst &I : h->inst)
    if (!I.bank) return false;
  return true;
}

}  // namespace

extern "C" {

letkf_status letkf_create(const letkf_config *cfg, void *stream, letkf_t *out) {
  if (!cfg) {
    if (out) *out = nullptr;
    return fail(nullptr, LETKF_ERR_ARG, "cfg is NULL");
  }
  return build_handle(cfg, 1, stream, out);
}

letkf_status letkf_create_batch(const letkf_config *cfgs, int32_t n, void *stream, letkf_t *out) {
  return build_handle(cfgs, n, stream, out);
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
  if (n_pts) *n_pts = (int32_t)h->n_pts_total;
  if (p) *p = (int32_t)h->p_total;
  if (m) *m = h->n_inst == 1 ? h->inst[0].m : 0;
  return LETKF_OK;
}

letkf_status letkf_query_instance(letkf_t h, int32_t i, int32_t *n_pts, int32_t *p, int32_t *m,
                                  int32_t *n_inst) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (n_inst) *n_inst = h->n_inst;
  if (i < 0 || i >= h->n_inst) return fail(h, LETKF_ERR_ARG, "instance index out of range");
  if (n_pts) *n_pts = h->inst[i].n_pts;
  if (p) *p = h->inst[i].p;
  if (m) *m = h->inst[i].m;
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
  LK_CUDA(h, cudaMemcpyAsync(X_dev, h->X, h->state_total * h->rsz, cudaMemcpyDeviceToDevice,
                             h->stream));
  return LETKF_OK;
}

letkf_status letkf_set_state(letkf_t h, const void *X_dev) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (!X_dev) return fail(h, LETKF_ERR_ARG, "X_dev is NULL");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaMemcpyAsync(h->X, X_dev, h->state_total * h->rsz, cudaMemcpyDeviceToDevice,
                             h->stream));
  LK_CUDA(h, lk_launch_basis_reset(h));
  return LETKF_OK;
}

letkf_status letkf_forecast(letkf_t h, const void *noise_dev) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (!noise_dev && !all_have_banks(h))
    return fail(h, LETKF_ERR_STATE, "no noise given and an instance has no noise bank");
  DeviceGuard dg(h->device);
  LK_CUDA(h, lk_launch_forecast(h, noise_dev));
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
  if (!truth_dev || !resvar_dev)
    return fail(h, LETKF_ERR_ARG, "truth_dev and resvar_dev are required");
  DeviceGuard dg(h->device);
  LK_CUDA(h, lk_launch_residual(h, truth_dev, resvar_dev, nullptr));
  return LETKF_OK;
}

letkf_status letkf_run(letkf_t h, int32_t frames, const void *y_seq_dev, const void *truth_seq_dev,
                       double *resvar_dev, int32_t use_graph) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (frames < 0) return fail(h, LETKF_ERR_ARG, "frames < 0");
  if (!y_seq_dev) return fail(h, LETKF_ERR_ARG, "y_seq_dev is NULL");
  if (!all_have_banks(h))
    return fail(h, LETKF_ERR_STATE, "letkf_run needs a noise bank for every instance");
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

letkf_status letkf_run_graph(letkf_t h, int32_t frames, const void *y_seq_dev,
                             const void *truth_seq_dev, double *resvar_dev,
                             uint64_t *stamps_dev) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (frames < 1 || frames > (1 << 16)) return fail(h, LETKF_ERR_ARG, "frames must be 1..65536");
  if (!y_seq_dev) return fail(h, LETKF_ERR_ARG, "y_seq_dev is NULL");
  if (!all_have_banks(h))
    return fail(h, LETKF_ERR_STATE, "letkf_run_graph needs a noise bank for every instance");
  if (h->stream == nullptr)
    return fail(h, LETKF_ERR_STATE, "graph capture needs a non-default stream");
  DeviceGuard dg(h->device);
  unsigned long long *stamps = reinterpret_cast<unsigned long long *>(stamps_dev);
  if (!h->mgraph || h->mgraph_frames != frames || h->mgraph_y != y_seq_dev ||
      h->mgraph_truth != truth_seq_dev || h->mgraph_resvar != resvar_dev ||
      h->mgraph_stamps != stamps) {
    if (h->mgraph) {
      cudaGraphExecDestroy(h->mgraph);
      h->mgraph = nullptr;
    }
    LK_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    letkf_status st = LETKF_OK;
    cudaError_t ce = stamps ? lk_launch_stamp(h, stamps) : cudaSuccess;
    if (ce != cudaSuccess) st = cuda_fail(h, ce, "stamp launch");
    for (int k = 0; k < frames && st == LETKF_OK; ++k) {
      st = enqueue_frame(h, y_seq_dev, truth_seq_dev, resvar_dev);
      if (st == LETKF_OK && stamps) {
        ce = lk_launch_stamp(h, stamps + k + 1);
        if (ce != cudaSuccess) st = cuda_fail(h, ce, "stamp launch");
      }
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (st != LETKF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->mgraph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    h->mgraph_frames = frames;
    h->mgraph_y = y_seq_dev;
    h->mgraph_truth = truth_seq_dev;
    h->mgraph_resvar = resvar_dev;
    h->mgraph_stamps = stamps;
  }
  LK_CUDA(h, cudaMemsetAsync(h->frame + 1, 0, sizeof(long long), h->stream));
  LK_CUDA(h, cudaGraphLaunch(h->mgraph, h->stream));
  h->frame_host += frames;
  return LETKF_OK;
}

letkf_status letkf_set_dm(letkf_t h, int32_t n, const int32_t *n_ptr, const int32_t *n_idx,
                          const double *n_val, const int32_t *p_ptr, const int32_t *p_idx,
                          const double *p_val) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (h->n_inst != 1 || h->dom)
    return fail(h, LETKF_ERR_ARG, "a deformable mirror takes a single-instance per-node handle");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaStreamSynchronize(h->stream));
  LkInst &I = h->inst[0];
  if (!n_ptr) {                                  // back to the pseudo-open-loop form
    if (h->dm_buf) cudaFree(h->dm_buf);
    h->dm_buf = nullptr;
    h->dm_wfs_y = nullptr;
    I.dm = 0;
    drop_graphs(h);
    return upload(h, h->d_inst, &I, sizeof(LkInst));
  }
  if (n != I.n_pts || !n_idx || !n_val || !p_ptr || !p_idx || !p_val)
    return fail(h, LETKF_ERR_ARG, "N and P must be n_pts x n_pts CSR matrices");
  auto valid = [n](const int32_t *ptr, const int32_t *idx) {
    if (ptr[0] != 0) return false;
    for (int r = 0; r < n; ++r)
      if (ptr[r + 1] < ptr[r]) return false;
    for (int q = 0; q < ptr[n]; ++q)
      if (idx[q] < 0 || idx[q] >= n) return false;
    return true;
  };
  if (!valid(n_ptr, n_idx) || !valid(p_ptr, p_idx))
    return fail(h, LETKF_ERR_ARG, "malformed CSR (row pointers or column indices)");
  // D1 N: the Fried slopes of every row of N (Appendix B)
  const int nn = I.nsub + 1, ns = I.n_sap;
  std::vector<int32_t> dn_ptr{0}, dn_idx;
  std::vector<double> dn_val, acc(n, 0.0);
  std::vector<int> touched;
  std::vector<char> mark(n, 0);
  for (int r = 0; r < 2 * ns; ++r) {
    const int2 st = h->dom_saps[r % ns];
    const int q00 = h->dom_pid[(size_t)st.x * nn + st.y];
    const int q10 = h->dom_pid[(size_t)(st.x + 1) * nn + st.y];
    const int q01 = h->dom_pid[(size_t)st.x * nn + st.y + 1];
    const int q11 = h->dom_pid[(size_t)(st.x + 1) * nn + st.y + 1];
    const int rows[4] = {q00, q10, q01, q11};
    const double wx[4] = {-0.5, 0.5, -0.5, 0.5}, wy[4] = {-0.5, -0.5, 0.5, 0.5};
    for (int c = 0; c < 4; ++c) {
      const double wc = r < ns ? wx[c] : wy[c];
      for (int q = n_ptr[rows[c]]; q < n_ptr[rows[c] + 1]; ++q) {
        const int a = n_idx[q];
        if (!mark[a]) {
          mark[a] = 1;
          touched.push_back(a);
        }
        acc[a] += wc * n_val[q];
      }
    }
    std::sort(touched.begin(), touched.end());
    for (int a : touched) {
      if (acc[a] != 0.0) {
        dn_idx.push_back(a);
        dn_val.push_back(acc[a]);
      }
      acc[a] = 0.0;
      mark[a] = 0;
    }
    touched.clear();
    dn_ptr.push_back((int32_t)dn_idx.size());
  }
  // one allocation: int arrays, then real arrays (each 256-byte aligned)
  const size_t rs = h->rsz, nzN = n_ptr[n], nzP = p_ptr[n], nzD = dn_idx.size();
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off = 0;
  const size_t o_nptr = off; off = al(off + (n + 1) * 4);
  const size_t o_nidx = off; off = al(off + nzN * 4);
  const size_t o_pptr = off; off = al(off + (n + 1) * 4);
  const size_t o_pidx = off; off = al(off + nzP * 4);
  const size_t o_dptr = off; off = al(off + (2 * ns + 1) * 4);
  const size_t o_didx = off; off = al(off + nzD * 4);
  const size_t o_nval = off; off = al(off + nzN * rs);
  const size_t o_pval = off; off = al(off + nzP * rs);
  const size_t o_dval = off; off = al(off + nzD * rs);
  const size_t o_u = off; off = al(off + 3 * (size_t)n * rs);
  const size_t o_pm = off; off = al(off + (size_t)n * rs);
  const size_t o_cor = off; off = al(off + (size_t)n * rs);
  const size_t o_y = off; off = al(off + (size_t)2 * ns * rs);
  if (h->dm_buf) cudaFree(h->dm_buf);
  h->dm_buf = nullptr;
  LK_CUDA(h, cudaMalloc(&h->dm_buf, off));
  unsigned char *b = static_cast<unsigned char *>(h->dm_buf);
  auto put_real = [&](size_t o, const double *v, size_t cnt) -> cudaError_t {
    if (h->precision == 1) return cudaMemcpy(b + o, v, cnt * 8, cudaMemcpyHostToDevice);
    std::vector<float> f(v, v + cnt);
    return cudaMemcpy(b + o, f.data(), cnt * 4, cudaMemcpyHostToDevice);
  };
  LK_CUDA(h, cudaMemcpy(b + o_nptr, n_ptr, (n + 1) * 4, cudaMemcpyHostToDevice));
  LK_CUDA(h, cudaMemcpy(b + o_nidx, n_idx, nzN * 4, cudaMemcpyHostToDevice));
  LK_CUDA(h, cudaMemcpy(b + o_pptr, p_ptr, (n + 1) * 4, cudaMemcpyHostToDevice));
  LK_CUDA(h, cudaMemcpy(b + o_pidx, p_idx, nzP * 4, cudaMemcpyHostToDevice));
  LK_CUDA(h, cudaMemcpy(b + o_dptr, dn_ptr.data(), dn_ptr.size() * 4, cudaMemcpyHostToDevice));
  LK_CUDA(h, cudaMemcpy(b + o_didx, dn_idx.data(), nzD * 4, cudaMemcpyHostToDevice));
  LK_CUDA(h, put_real(o_nval, n_val, nzN));
  LK_CUDA(h, put_real(o_pval, p_val, nzP));
  LK_CUDA(h, put_real(o_dval, dn_val.data(), nzD));
  LK_CUDA(h, cudaMemset(b + o_u, 0, 3 * (size_t)n * rs));
  LK_CUDA(h, cudaMemset(b + o_pm, 0, (size_t)n * rs));
  LK_CUDA(h, cudaMemset(b + o_cor, 0, (size_t)n * rs));
  I.dm = 1;
  I.n_ptr = reinterpret_cast<const int *>(b + o_nptr);
  I.n_idx = reinterpret_cast<const int *>(b + o_nidx);
  I.p_ptr = reinterpret_cast<const int *>(b + o_pptr);
  I.p_idx = reinterpret_cast<const int *>(b + o_pidx);
  I.dn_ptr = reinterpret_cast<const int *>(b + o_dptr);
  I.dn_idx = reinterpret_cast<const int *>(b + o_didx);
  I.n_val = b + o_nval;
  I.p_val = b + o_pval;
  I.dn_val = b + o_dval;
  I.u = b + o_u;
  I.pmean = b + o_pm;
  I.cor = b + o_cor;
  I.fcount = h->frame;
  h->dm_wfs_y = b + o_y;
  drop_graphs(h);
  return upload(h, h->d_inst, &I, sizeof(LkInst));
}

letkf_status letkf_get_command(letkf_t h, void *u_dev) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (!u_dev) return fail(h, LETKF_ERR_ARG, "u_dev is NULL");
  if (!h->inst[0].dm) return fail(h, LETKF_ERR_STATE, "no deformable mirror (letkf_set_dm)");
  DeviceGuard dg(h->device);
  LK_CUDA(h, lk_launch_dm_get(h, u_dev));
  return LETKF_OK;
}

letkf_status letkf_run_dm(letkf_t h, int32_t frames, const void *truth_seq_dev,
                          const void *wnoise_seq_dev, double *resvar_dev, int32_t use_graph) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (frames < 0) return fail(h, LETKF_ERR_ARG, "frames < 0");
  if (!truth_seq_dev || !wnoise_seq_dev)
    return fail(h, LETKF_ERR_ARG, "truth_seq_dev and wnoise_seq_dev are required");
  if (!h->inst[0].dm) return fail(h, LETKF_ERR_STATE, "no deformable mirror (letkf_set_dm)");
  if (!all_have_banks(h)) return fail(h, LETKF_ERR_STATE, "letkf_run_dm needs a noise bank");
  if (use_graph && h->stream == nullptr)
    return fail(h, LETKF_ERR_STATE, "graph capture needs a non-default stream");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaMemsetAsync(h->frame + 1, 0, sizeof(long long), h->stream));
  if (frames == 0) return LETKF_OK;
  if (use_graph) {
    if (h->graph) {                              // the one-frame graph of this call's form
      cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
    }
    LK_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    letkf_status st = enqueue_frame_dm(h, truth_seq_dev, wnoise_seq_dev, resvar_dev);
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
    h->graph_y = h->graph_truth = nullptr;       // not letkf_run's graph
    h->graph_resvar = nullptr;
    for (int k = 0; k < frames; ++k) LK_CUDA(h, cudaGraphLaunch(h->graph, h->stream));
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  } else {
    for (int k = 0; k < frames; ++k) {
      letkf_status st = enqueue_frame_dm(h, truth_seq_dev, wnoise_seq_dev, resvar_dev);
      if (st != LETKF_OK) return st;
    }
  }
  h->frame_host += frames;
  return LETKF_OK;
}

letkf_status letkf_query_domains(letkf_t h, int32_t *n_dom, int32_t *node_dom_host,
                                 int32_t *obs_count_host) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (n_dom) *n_dom = lk_domain_count(h);
  if (h->dom && (node_dom_host || obs_count_host)) {
    DeviceGuard dg(h->device);
    if (node_dom_host && !lk_domain_of_nodes(h, node_dom_host))
      return fail(h, LETKF_ERR_CUDA, "cudaMemcpy");
    if (obs_count_host && !lk_domain_obs_counts(h, obs_count_host))
      return fail(h, LETKF_ERR_CUDA, "cudaMemcpy");
  }
  return LETKF_OK;
}

letkf_status letkf_set_params(letkf_t h, int32_t i, double rho, double sigma2, double loc_len) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (i < 0 || i >= h->n_inst) return fail(h, LETKF_ERR_ARG, "no such instance");
  if (!(rho > 0) || !(sigma2 > 0) || !isfinite(rho) || !isfinite(sigma2) || !isfinite(loc_len))
    return fail(h, LETKF_ERR_ARG, "rho and sigma2 must be finite and > 0, loc_len finite");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaStreamSynchronize(h->stream));
  letkf_config &c = h->cfgs[i];
  c.rho = rho;
  c.sigma2 = sigma2;
  c.loc_len = loc_len;
  if (i == 0) h->cfg = c;
  LkInst &I = h->inst[i];
  I.alpha = (c.m - 1) / rho;
  std::vector<double> tap;
  taper_table(c, tap);
  letkf_status st = upload_taper(h, I, tap);
  if (st == LETKF_OK) st = upload(h, h->d_inst + i, &I, sizeof(LkInst));
  if (st == LETKF_OK && h->dom)
    st = lk_domains_set_params(h, c, h->dom_pid, h->dom_pts, h->dom_saps, h->err);
  drop_graphs(h);          // the reverse mode's graph holds rho and sigma2 as kernel arguments
  return st;
}

letkf_status letkf_set_jacobi(letkf_t h, double rotate_tol, double stop_cos) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (!(rotate_tol > 0) || !(rotate_tol < 1) || !(stop_cos >= 0) || !(stop_cos < 1))
    return fail(h, LETKF_ERR_ARG, "rotate_tol must be in (0, 1) and stop_cos in [0, 1)");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaStreamSynchronize(h->stream));
  h->tol32 = rotate_tol;
  h->stop32 = stop_cos > rotate_tol ? stop_cos : rotate_tol;
  drop_graphs(h);                    // captured launches hold the old values
  return LETKF_OK;
}

letkf_status letkf_set_frame(letkf_t h, int64_t frame) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (frame < 0) return fail(h, LETKF_ERR_ARG, "frame < 0");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaStreamSynchronize(h->stream));
  const long long f = frame;
  LK_CUDA(h, cudaMemcpy(h->frame, &f, sizeof(long long), cudaMemcpyHostToDevice));
  h->frame_host = frame;
  return LETKF_OK;
}

letkf_status letkf_step(letkf_t h, const void *y_host, const void *truth_host, void *mean_host,
                        double *resvar_host) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (!y_host) return fail(h, LETKF_ERR_ARG, "y_host is NULL");
  if (!all_have_banks(h))
    return fail(h, LETKF_ERR_STATE, "letkf_step needs a noise bank for every instance");
  DeviceGuard dg(h->device);
  if (!h->step_pin) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    h->step_off[0] = 0;
    h->step_off[1] = al(h->p_total * h->rsz);
    h->step_off[2] = h->step_off[1] + al(h->n_pts_total * h->rsz);
    h->step_off[3] = h->step_off[2] + al(2 * h->n_pts_total * h->rsz);
    const size_t total = h->step_off[3] + al(h->n_inst * sizeof(double));
    LK_CUDA(h, cudaMallocHost((void **)&h->step_pin, total));
    cudaError_t e = cudaMalloc((void **)&h->step_dev, total);
    if (e != cudaSuccess) {
      cudaFreeHost(h->step_pin);
      h->step_pin = nullptr;
      return fail(h, LETKF_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  const bool wt = truth_host != nullptr;
  // the staging is free once the previous step's downloads are done (its
  // forecast may still run: the next graph is ordered after it on the stream)
  LK_CUDA(h, h->ev_out ? cudaEventSynchronize(h->ev_out) : cudaStreamSynchronize(h->stream));
  memcpy(h->step_pin + h->step_off[0], y_host, h->p_total * h->rsz);
  if (wt) memcpy(h->step_pin + h->step_off[1], truth_host, h->n_pts_total * h->rsz);
  if (h->stream) {
    cudaGraphExec_t &g = h->step_graph[wt ? 1 : 0];
    if (!g) {
      LK_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      letkf_status st = enqueue_step(h, wt);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
      if (st != LETKF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&g, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    }
    LK_CUDA(h, cudaGraphLaunch(g, h->stream));
  } else {
    letkf_status st = enqueue_step(h, wt);
    if (st != LETKF_OK) return st;
  }
  LK_CUDA(h, h->ev_out ? cudaEventSynchronize(h->ev_out) : cudaStreamSynchronize(h->stream));
  h->frame_host += 1;
  if (mean_host)
    memcpy(mean_host, h->step_pin + h->step_off[2], 2 * h->n_pts_total * h->rsz);
  if (wt && resvar_host)
    memcpy(resvar_host, h->step_pin + h->step_off[3], h->n_inst * sizeof(double));
  return LETKF_OK;
}

letkf_status letkf_tile_shape(int32_t shape, int32_t *tile_i, int32_t *tile_j) {
  if (shape < 0 || shape >= lk_num_tile_shapes())
    return fail(nullptr, LETKF_ERR_ARG, "no such tile shape");
  int a, b;
  lk_tile_shape(shape, &a, &b);
  if (tile_i) *tile_i = a;
  if (tile_j) *tile_j = b;
  return LETKF_OK;
}

letkf_status letkf_set_tile_shape(letkf_t h, int32_t width_class, int32_t shape) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (width_class < 0 || width_class > 2 || shape < 0 || shape >= lk_num_tile_shapes())
    return fail(h, LETKF_ERR_ARG, "width class or tile shape out of range");
  if (!lk_shape_ok(h, width_class, shape))
    return fail(h, LETKF_ERR_ARG,
                "FP32 tiles hold whole warps of nodes (4 per warp for m <= 16, 2 for m <= 32; "
                "2 and 1 with the row split) and ensembles of 33..64 members at most 8 nodes");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaStreamSynchronize(h->stream));
  h->tile_shape[width_class] = shape;
  return rebuild_tiles(h, width_class);
}

letkf_status letkf_set_fp64_start(letkf_t h, int32_t warm) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (h->precision != 1 || h->dom || (warm != 0 && warm != 1))
    return fail(h, LETKF_ERR_ARG, "an FP64 per-node handle and warm = 0 or 1 are required");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->fp64_warm != warm) drop_graphs(h);     // they hold the other launch sequence
  h->fp64_warm = warm;
  return LETKF_OK;
}

letkf_status letkf_set_row_split(letkf_t h, int32_t width_class, int32_t split) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (width_class < 0 || width_class > 2 || (split != 1 && split != 2))
    return fail(h, LETKF_ERR_ARG, "width class out of range or split not 1 or 2");
  if (h->dom || !lk_shape_split_ok(h, width_class, h->tile_shape[width_class], split))
    return fail(h, LETKF_ERR_ARG,
                "the row split needs an FP32 per-node handle, width class 0 or 1, and a tile "
                "of whole warps (an even node count in class 0)");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->row_split[width_class] == split) return LETKF_OK;
  h->row_split[width_class] = split;
  return rebuild_tiles(h, width_class);    // class 1 groups its tiles by width only unsplit
}

letkf_status letkf_autotune(letkf_t h, const void *y_dev, int32_t reps, int32_t *shapes_out,
                            float *us_out) {
  if (!h) return fail(nullptr, LETKF_ERR_ARG, "handle is NULL");
  if (!y_dev || reps < 1) return fail(h, LETKF_ERR_ARG, "y_dev and reps >= 1 are required");
  DeviceGuard dg(h->device);
  LK_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->precision == 1 || h->dom) {      // one CTA per node or domain: no tile shape
    for (int cls = 0; cls < 3; ++cls) {
      if (shapes_out) shapes_out[cls] = h->tile_shape[cls];
      if (us_out) us_out[cls] = 0.f;
    }
    return LETKF_OK;
  }
  const int ns = lk_num_tile_shapes();
  // every timed analysis starts from the same ensemble and eigenbases
  size_t n_basis = 0;
  for (const LkInst &I : h->inst) n_basis += (size_t)I.n_pts * I.mp * I.mp;
  void *x_save = nullptr;
  float *b_save = nullptr;
  LK_CUDA(h, cudaMalloc(&x_save, h->state_total * h->rsz));
  cudaError_t e = cudaMalloc((void **)&b_save, n_basis * sizeof(float) + 16);
  if (e != cudaSuccess) {
    cudaFree(x_save);
    return cuda_fail(h, e, "cudaMalloc");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  letkf_status st = LETKF_OK;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(x_save, h->X, h->state_total * h->rsz, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b_save, h->basis, n_basis * sizeof(float), cudaMemcpyDeviceToDevice,
                        h->stream);
  for (int cls = 0; cls < 3 && e == cudaSuccess && st == LETKF_OK; ++cls) {
    if (shapes_out) shapes_out[cls] = h->tile_shape[cls];
    if (us_out) us_out[cls] = 0.f;
    if (h->n_tiles[cls] == 0) continue;
    int best = h->tile_shape[cls];
    float best_ms = 1e30f;
    for (int s = 0; s < ns && e == cudaSuccess && st == LETKF_OK; ++s) {
      if (!lk_shape_ok(h, cls, s)) continue;
      h->tile_shape[cls] = s;
      st = rebuild_tiles(h, cls);
      float total = 0.f;
      for (int r = 0; r <= reps && e == cudaSuccess && st == LETKF_OK; ++r) {  // r = 0 warms up
        e = cudaMemcpyAsync(h->X, x_save, h->state_total * h->rsz, cudaMemcpyDeviceToDevice,
                            h->stream);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(h->basis, b_save, n_basis * sizeof(float), cudaMemcpyDeviceToDevice,
                              h->stream);
        if (e == cudaSuccess) e = lk_launch_obs(h, y_dev, nullptr);
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
        if (e == cudaSuccess) e = lk_launch_analysis_class(h, cls, nullptr, nullptr);
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) total += ms;
      }
      if (e == cudaSuccess && st == LETKF_OK && total < best_ms) {
        best_ms = total;
        best = s;
      }
    }
    if (shapes_out) shapes_out[cls] = best;
    if (us_out) us_out[cls] = 1e3f * best_ms / reps;
    h->tile_shape[cls] = best;
    if (st == LETKF_OK && e == cudaSuccess) st = rebuild_tiles(h, cls);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->X, x_save, h->state_total * h->rsz, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->basis, b_save, n_basis * sizeof(float), cudaMemcpyDeviceToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(x_save);
  cudaFree(b_save);
  if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
  return st;
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
  int c[8];
  LK_CUDA(h, cudaMemcpy(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost));
  if (fp64_points) *fp64_points = c[1];
  if (max_sweeps) *max_sweeps = c[2];
  if (total_sweeps) *total_sweeps = c[3];
  return LETKF_OK;
}

const char *letkf_last_error(letkf_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

// Gaspari & Cohn (1999) compactly supported 5th-order piecewise rational
// function of z = r / c (their Eq. 4.10): 1 at z = 0, 0 for z >= 2.
double lk_gaspari_cohn(double z) {
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
