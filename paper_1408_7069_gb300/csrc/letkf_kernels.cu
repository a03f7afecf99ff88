// Per-frame kernels around the analysis: observation of the background
// ensemble (means, slope anomalies, innovations), the AR(1) forecast, the
// residual criterion and the frame counter.
#include "letkf_common.cuh"

namespace {

// One warp per valid subaperture (s, t); lane = member.
// Background mean and anomalies of the phi_{k-1} row at the four corners
// (Section 3.1, Eq. Cov_emp), Fried slopes of the anomalies Yb = D1 X'
// (Appendix B) into the padded grid cell (s+h, t+h), and the innovation
// d = y - D1 xbar (Section 3.1.1, with the correction known exactly).
template <typename S>
__global__ void __launch_bounds__(256) obs_kernel(LkGeom g, const S *__restrict__ X,
                                                  const S *__restrict__ y,
                                                  const long long *__restrict__ run_idx,
                                                  S *__restrict__ Ybp, S *__restrict__ dp,
                                                  int *__restrict__ counters) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= g.n_sap) return;
  if (run_idx) y += (*run_idx) * (long long)g.p;
  const int m = g.m;
  const int nn = g.nsub + 1;
  const int2 st = g.saps[k];
  const int q00 = g.pid_map[st.x * nn + st.y];
  const int q10 = g.pid_map[(st.x + 1) * nn + st.y];
  const int q01 = g.pid_map[st.x * nn + st.y + 1];
  const int q11 = g.pid_map[(st.x + 1) * nn + st.y + 1];
  const bool act = lane < m;
  const S v00 = act ? X[(size_t)(2 * q00 + 1) * m + lane] : S(0);
  const S v10 = act ? X[(size_t)(2 * q10 + 1) * m + lane] : S(0);
  const S v01 = act ? X[(size_t)(2 * q01 + 1) * m + lane] : S(0);
  const S v11 = act ? X[(size_t)(2 * q11 + 1) * m + lane] : S(0);
  const S inv_m = S(1) / S(m);
  const S u00 = lk_warp_sum(v00) * inv_m;
  const S u10 = lk_warp_sum(v10) * inv_m;
  const S u01 = lk_warp_sum(v01) * inv_m;
  const S u11 = lk_warp_sum(v11) * inv_m;
  const S a00 = act ? v00 - u00 : S(0);
  const S a10 = act ? v10 - u10 : S(0);
  const S a01 = act ? v01 - u01 : S(0);
  const S a11 = act ? v11 - u11 : S(0);
  const size_t cell = (size_t)(st.x + g.h) * g.gs_cols + (st.y + g.h);
  if (act) {
    Ybp[(cell * 2 + 0) * m + lane] = S(0.5) * ((a10 + a11) - (a00 + a01));
    Ybp[(cell * 2 + 1) * m + lane] = S(0.5) * ((a01 + a11) - (a00 + a10));
  }
  if (lane == 0) {
    const S ybx = S(0.5) * ((u10 + u11) - (u00 + u01));
    const S yby = S(0.5) * ((u01 + u11) - (u00 + u10));
    const S dx = y[k] - ybx;
    const S dy = y[g.n_sap + k] - yby;
    dp[cell * 2 + 0] = dx;
    dp[cell * 2 + 1] = dy;
    if (!isfinite(dx) || !isfinite(dy)) atomicOr(&counters[0], LK_BIT_NONFINITE);
  }
}

// One thread per (node, member): phi_{k+1} = a phi_k + v, phi_k -> row 1
// (Section 2.2, A1 = [[a I, 0], [I, 0]]; Section 3.1.2, Eq. Mem_pre).
template <typename S>
__global__ void __launch_bounds__(256) forecast_kernel(S *__restrict__ X, int n_pts, int m, S a, S q,
                                                       const S *__restrict__ noise,
                                                       const float *__restrict__ bank, int B, int G,
                                                       const int2 *__restrict__ pts,
                                                       unsigned long long seed,
                                                       const long long *__restrict__ frame) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_pts * m) return;
  const int gpt = (int)(idx / m);
  const int i = (int)(idx - (long long)gpt * m);
  S *row0 = X + (size_t)gpt * 2 * m;
  const S x0 = row0[i];
  S v;
  if (noise) {
    v = noise[idx];
  } else {
    const unsigned long long hsh =
        lk_splitmix64(seed, ((unsigned long long)frame[0] << 16) | (unsigned long long)i);
    const int b = (int)(hsh % (unsigned long long)B);
    const int ox = (int)((hsh >> 16) % (unsigned long long)G);
    const int oy = (int)((hsh >> 40) % (unsigned long long)G);
    const int2 ij = pts[gpt];
    v = q * S(bank[((size_t)b * G + (ij.x + ox) % G) * G + (ij.y + oy) % G]);
  }
  row0[m + i] = x0;
  row0[i] = a * x0 + v;
}

// Spatial variance of truth - mean(row 0) over the nodes, piston removed
// (Section 2.1, Eq. Crit_Opt; Section 5). Warp per node (lane = member), FP64
// partial sums per CTA, then one warp adds the partials in a fixed order.
template <typename S>
__global__ void __launch_bounds__(256) residual_partial_kernel(const S *__restrict__ X, int n_pts,
                                                               int m, const S *__restrict__ truth,
                                                               const long long *__restrict__ run_idx,
                                                               double2 *__restrict__ partial) {
  const long long k = run_idx ? *run_idx : 0;
  truth += k * n_pts;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  double s1 = 0.0, s2 = 0.0;
  for (int gpt = blockIdx.x * nw + wid; gpt < n_pts; gpt += gridDim.x * nw) {
    const double x = lane < m ? (double)X[(size_t)gpt * 2 * m + lane] : 0.0;
    const double r = (double)truth[gpt] - lk_warp_sum(x) / m;
    s1 += r;
    s2 += r * r;
  }
  __shared__ double sh1[32], sh2[32];
  if (lane == 0) {
    sh1[wid] = s1;
    sh2[wid] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nw; ++i) {
      a += sh1[i];
      b += sh2[i];
    }
    partial[blockIdx.x] = make_double2(a, b);
  }
}

__global__ void residual_final_kernel(const double2 *__restrict__ partial, int nparts, int n_pts,
                                      const long long *__restrict__ run_idx,
                                      double *__restrict__ resvar) {
  const long long k = run_idx ? *run_idx : 0;
  double s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 32) {
    s1 += partial[i].x;
    s2 += partial[i].y;
  }
  s1 = lk_warp_sum(s1);
  s2 = lk_warp_sum(s2);
  if (threadIdx.x == 0) {
    const double mu = s1 / n_pts;
    resvar[k] = s2 / n_pts - mu * mu;
  }
}

__global__ void tick_kernel(long long *frame) {
  frame[0] += 1;
  frame[1] += 1;
}

}  // namespace

cudaError_t lk_launch_obs(letkf_ctx *h, const void *y, const long long *run_idx) {
  const int threads = 256;
  const int blocks = (h->g.n_sap * 32 + threads - 1) / threads;
  if (h->precision == 1)
    obs_kernel<double><<<blocks, threads, 0, h->stream>>>(
        h->g, (const double *)h->X, (const double *)y, run_idx, (double *)h->Ybp, (double *)h->dp,
        h->counters);
  else
    obs_kernel<float><<<blocks, threads, 0, h->stream>>>(
        h->g, (const float *)h->X, (const float *)y, run_idx, (float *)h->Ybp, (float *)h->dp,
        h->counters);
  return cudaGetLastError();
}

cudaError_t lk_launch_forecast(letkf_ctx *h, const void *noise) {
  const long long n = (long long)h->g.n_pts * h->g.m;
  const int threads = 256;
  const int blocks = (int)((n + threads - 1) / threads);
  if (h->precision == 1)
    forecast_kernel<double><<<blocks, threads, 0, h->stream>>>(
        (double *)h->X, h->g.n_pts, h->g.m, h->cfg.a_ar1, h->cfg.noise_std, (const double *)noise,
        h->bank, h->bank_B, h->bank_G, h->pts, h->cfg.seed, h->frame);
  else
    forecast_kernel<float><<<blocks, threads, 0, h->stream>>>(
        (float *)h->X, h->g.n_pts, h->g.m, (float)h->cfg.a_ar1, (float)h->cfg.noise_std,
        (const float *)noise, h->bank, h->bank_B, h->bank_G, h->pts, h->cfg.seed, h->frame);
  return cudaGetLastError();
}

cudaError_t lk_launch_residual(letkf_ctx *h, const void *truth, double *resvar,
                               const long long *run_idx) {
  if (h->precision == 1)
    residual_partial_kernel<double><<<LK_RES_BLOCKS, 256, 0, h->stream>>>(
        (const double *)h->X, h->g.n_pts, h->g.m, (const double *)truth, run_idx, h->partial);
  else
    residual_partial_kernel<float><<<LK_RES_BLOCKS, 256, 0, h->stream>>>(
        (const float *)h->X, h->g.n_pts, h->g.m, (const float *)truth, run_idx, h->partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  residual_final_kernel<<<1, 32, 0, h->stream>>>(h->partial, LK_RES_BLOCKS, h->g.n_pts, run_idx,
                                                 resvar);
  return cudaGetLastError();
}

cudaError_t lk_launch_tick(letkf_ctx *h) {
  tick_kernel<<<1, 1, 0, h->stream>>>(h->frame);
  return cudaGetLastError();
}
