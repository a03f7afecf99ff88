// Per-frame kernels around the analysis, over every instance of a handle:
// observation of the background ensemble (means, slope anomalies,
// innovations), the AR(1) forecast, the residual criterion and the frame counter.
#include <stdint.h>

#include "letkf_common.cuh"

namespace {

// One warp per (instance, valid subaperture); lane = member (m <= 64: two passes).
// Background mean and anomalies of the phi_{k-1} row at the four corners
// (Section 3.1, Eq. Cov_emp), Fried slopes of the anomalies Yb = D1 X'
// (Appendix B) into the padded grid cell (s+h, t+h), and the innovation
// d = y - D1 xbar (Section 3.1.1, with the correction known exactly).
// The observation's part of CTA `bx`.
template <typename S>
__device__ __forceinline__ void obs_block(const LkInst *__restrict__ insts,
                                          const int2 *__restrict__ items, long long n_items,
                                          long long p_total, const S *__restrict__ y,
                                          const long long *__restrict__ run_idx,
                                          int *__restrict__ counters, int bx) {
  lk_pdl_wait();   // no early trigger: an analysis launched early would have its CTAs
                   // packed onto the SMs this kernel still occupies
  // the analysis that follows counts into counters[1..7] (queue lengths, sweeps)
  if (bx == 0 && threadIdx.x < 7) counters[1 + threadIdx.x] = 0;
  const long long wi = ((long long)bx * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wi >= n_items) return;
  const int2 it = items[wi];
  const LkInst &I = insts[it.x];
  const int k = it.y;
  if (run_idx) y += (*run_idx) * p_total;
  y += I.y_off;
  const S *X = static_cast<const S *>(I.X);
  S *Ybp = static_cast<S *>(I.Ybp);
  S *dp = static_cast<S *>(I.dp);
  const int m = I.m;
  const int nn = I.nsub + 1;
  const int2 st = I.saps[k];
  const int q00 = I.pid_map[st.x * nn + st.y];
  const int q10 = I.pid_map[(st.x + 1) * nn + st.y];
  const int q01 = I.pid_map[st.x * nn + st.y + 1];
  const int q11 = I.pid_map[(st.x + 1) * nn + st.y + 1];
  // means over members
  S s00 = 0, s10 = 0, s01 = 0, s11 = 0;
  for (int i = lane; i < m; i += 32) {
    s00 += X[(size_t)(2 * q00 + 1) * m + i];
    s10 += X[(size_t)(2 * q10 + 1) * m + i];
    s01 += X[(size_t)(2 * q01 + 1) * m + i];
    s11 += X[(size_t)(2 * q11 + 1) * m + i];
  }
  const S inv_m = S(1) / S(m);
  const S u00 = lk_warp_sum(s00) * inv_m;
  const S u10 = lk_warp_sum(s10) * inv_m;
  const S u01 = lk_warp_sum(s01) * inv_m;
  const S u11 = lk_warp_sum(s11) * inv_m;
  const size_t cell = (size_t)(st.x + I.h) * I.gs_cols + (st.y + I.h);
  for (int i = lane; i < m; i += 32) {
    const S a00 = X[(size_t)(2 * q00 + 1) * m + i] - u00;
    const S a10 = X[(size_t)(2 * q10 + 1) * m + i] - u10;
    const S a01 = X[(size_t)(2 * q01 + 1) * m + i] - u01;
    const S a11 = X[(size_t)(2 * q11 + 1) * m + i] - u11;
    Ybp[(cell * 2 + 0) * m + i] = S(0.5) * ((a10 + a11) - (a00 + a01));
    Ybp[(cell * 2 + 1) * m + i] = S(0.5) * ((a01 + a11) - (a00 + a10));
  }
  if (lane == 0) {
    const S ybx = S(0.5) * ((u10 + u11) - (u00 + u01));
    const S yby = S(0.5) * ((u01 + u11) - (u00 + u10));
    S yx = y[k], yy = y[I.n_sap + k];
    if (I.dm) {
      // the measurement sees the residual phase: the analysis takes the
      // pseudo-open-loop slopes y + D1 N u_{k-2} (Section 3.1.1, ybar)
      const S *u2 = static_cast<const S *>(I.u) + (size_t)((*I.fcount + 1) % 3) * I.n_pts;
      const S *dv = static_cast<const S *>(I.dn_val);
      for (int q = I.dn_ptr[k]; q < I.dn_ptr[k + 1]; ++q) yx += dv[q] * u2[I.dn_idx[q]];
      for (int q = I.dn_ptr[I.n_sap + k]; q < I.dn_ptr[I.n_sap + k + 1]; ++q)
        yy += dv[q] * u2[I.dn_idx[q]];
    }
    const S dx = yx - ybx;
    const S dy = yy - yby;
    dp[cell * 2 + 0] = dx;
    dp[cell * 2 + 1] = dy;
    if (!isfinite(dx) || !isfinite(dy)) atomicOr(&counters[0], LK_BIT_NONFINITE);
  }
}

template <typename S>
__global__ void __launch_bounds__(LK_WARP_CTA) obs_kernel(const LkInst *__restrict__ insts,
                                                  const int2 *__restrict__ items, long long n_items,
                                                  long long p_total, const S *__restrict__ y,
                                                  const long long *__restrict__ run_idx,
                                                  int *__restrict__ counters) {
  obs_block<S>(insts, items, n_items, p_total, y, run_idx, counters, blockIdx.x);
}

// Member i's model noise at node point ij for forecast number f (Section 3.1.2,
// Eq. Mem_pre): a bank screen and a wrapped offset chosen by SplitMix64,
// scaled by q.
template <typename S>
__device__ __forceinline__ S bank_draw(const LkInst &I, int2 ij, int i, long long f) {
  const unsigned long long hsh =
      lk_splitmix64(I.seed, ((unsigned long long)f << 16) | (unsigned long long)i);
  const int B = I.bank_B, G = I.bank_G;
  const int b = (int)(hsh % (unsigned long long)B);
  const int ox = (int)((hsh >> 16) % (unsigned long long)G);
  const int oy = (int)((hsh >> 40) % (unsigned long long)G);
  return S(I.noise_std) * S(I.bank[((size_t)b * G + (ij.x + ox) % G) * G + (ij.y + oy) % G]);
}

template <typename S>
__device__ __forceinline__ void forecast_node(const LkInst *__restrict__ insts, int2 it, int lane,
                                              const S *__restrict__ noise,
                                              const long long *__restrict__ frame) {
  const LkInst &I = insts[it.x];
  const int gpt = it.y, m = I.m;
  S *row0 = static_cast<S *>(I.X) + (size_t)gpt * 2 * m;
  const S a = S(I.a_ar1);
  const int2 ij = I.pts[gpt];
  S psum = S(0);
  for (int i = lane; i < m; i += 32) {
    const S x0 = row0[i];
    const S v = noise ? noise[I.noise_off + (long long)gpt * m + i] : bank_draw<S>(I, ij, i, frame[0]);
    row0[m + i] = x0;
    row0[i] = a * x0 + v;
    psum += row0[i];
  }
  if (I.dm) {                       // the predicted phase, for the command u = P phihat
    psum = lk_warp_sum(psum);
    if (lane == 0) static_cast<S *>(I.pmean)[gpt] = psum / S(m);
  }
}

// One warp per (instance, node), lane = member: phi_{k+1} = a phi_k + v,
// phi_k -> row 1 (Section 2.2, A1 = [[a I, 0], [I, 0]]; Section 3.1.2, Eq. Mem_pre).
// v is the caller's noise, or a bank screen chosen per member by SplitMix64.
template <typename S>
__global__ void __launch_bounds__(LK_WARP_CTA) forecast_kernel(const LkInst *__restrict__ insts,
                                                       const int2 *__restrict__ items,
                                                       long long n_items, const S *__restrict__ noise,
                                                       long long *__restrict__ frame,
                                                       int *__restrict__ ticket) {
  lk_pdl_wait();
  lk_pdl_trigger();
  const long long wi = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wi < n_items) forecast_node<S>(insts, items[wi], lane, noise, frame);
  // the last CTA to finish advances the forecast counter and the run index
  // (every CTA has read the counter by then)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ticket, 1) == (int)gridDim.x - 1) {
      frame[0] += 1;
      frame[1] += 1;
      *ticket = 0;
    }
  }
}

// Spatial variance of truth - mean(row 0) over one instance's nodes, piston
// removed (Section 2.1, Eq. Crit_Opt; Section 5): the part of CTA rb of nrb of
// instance `inst`. Thread per node, FP64 partial sums per CTA; the last CTA of
// an instance to finish (ticket counter, reset by it) adds the partials in a
// fixed order and writes the variance and, when piston is given, the piston
// (the mean).
template <typename S>
__device__ __forceinline__ void residual_block(const LkInst &I, int inst, int rb, int nrb,
                                               long long n_pts_total, const S *__restrict__ truth,
                                               const long long *__restrict__ run_idx,
                                               double2 *__restrict__ partial,
                                               int *__restrict__ tickets, int n_inst,
                                               double *__restrict__ resvar,
                                               double *__restrict__ piston) {
  const long long k = run_idx ? *run_idx : 0;
  const S *tr = truth + k * n_pts_total + I.node_off;
  const S *X = static_cast<const S *>(I.X);
  const int m = I.m;
  const double inv_m = 1.0 / m;
  const bool vec = sizeof(S) == 4 && (m & 3) == 0 &&
                   (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  double s1 = 0.0, s2 = 0.0;
  for (int g = rb * blockDim.x + threadIdx.x; g < I.n_pts; g += nrb * blockDim.x) {
    const S *row = X + (size_t)g * 2 * m;
    double x = 0.0;
    if (vec) {
      // FP32 storage: the member sum in FP32 (four chains; its rounding is far
      // below the FP32 state's own), the residual and its moments in FP64
      const float4 *r4 = reinterpret_cast<const float4 *>(row);
      float a = 0.f, b = 0.f, c = 0.f, d = 0.f;
      for (int i = 0; i < m / 4; ++i) {
        const float4 v = r4[i];
        a += v.x;
        b += v.y;
        c += v.z;
        d += v.w;
      }
      x = (double)((a + b) + (c + d));
    } else {
      for (int i = 0; i < m; ++i) x += (double)row[i];
    }
    // with a deformable mirror the residual phase is phi^tur_k - N u_{k-1}
    // (Section 2.1, Eq. Eq_Cor); without, the prediction is the correction
    const double r = (double)tr[g] - (I.dm ? (double)static_cast<const S *>(I.cor)[g] : x * inv_m);
    s1 += r;
    s2 += r * r;
  }
  s1 = lk_warp_sum(s1);
  s2 = lk_warp_sum(s2);
  __shared__ double sh1[2], sh2[2];
  __shared__ int last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh1[wid] = s1;
    sh2[wid] = s2;
  }
  __syncthreads();
  double2 *pp = partial + (size_t)inst * nrb;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a += sh1[i];
      b += sh2[i];
    }
    pp[rb] = make_double2(a, b);
    __threadfence();
    last = atomicAdd(&tickets[inst], 1) == nrb - 1;
  }
  __syncthreads();
  if (last && threadIdx.x < 32) {
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nrb; i += 32) {
      const double2 v = __ldcg(pp + i);
      a += v.x;
      b += v.y;
    }
    a = lk_warp_sum(a);
    b = lk_warp_sum(b);
    if (threadIdx.x == 0) {
      const double n = I.n_pts;
      const double mu = a / n;
      resvar[k * n_inst + inst] = b / n - mu * mu;
      if (piston) piston[k * n_inst + inst] = mu;
      tickets[inst] = 0;
    }
  }
}

// The residual alone. Grid (LK_RES_BLOCKS, n_inst), 64 threads.
template <typename S>
__global__ void __launch_bounds__(64) residual_kernel(const LkInst *__restrict__ insts,
                                                       long long n_pts_total,
                                                       const S *__restrict__ truth,
                                                       const long long *__restrict__ run_idx,
                                                       double2 *__restrict__ partial,
                                                       int *__restrict__ tickets, int n_inst,
                                                       double *__restrict__ resvar,
                                                       double *__restrict__ piston) {
  lk_pdl_wait();
  lk_pdl_trigger();
  residual_block<S>(insts[blockIdx.y], blockIdx.y, blockIdx.x, gridDim.x, n_pts_total, truth,
                    run_idx, partial, tickets, n_inst, resvar, piston);
}

// Residual, observation and the coming forecast's model noise of a frame in one
// launch (all read only the prediction ensemble, the noise not even that): the
// first res_blocks CTAs (LK_RES_BLOCKS per instance) take the residual, the
// next noise_blocks draw the noise (warp per node, the draws the forecast would
// make, into noise_out), the others the observation, 64 threads each.
template <typename S>
__global__ void __launch_bounds__(LK_WARP_CTA)
    obs_residual_kernel(const LkInst *__restrict__ insts, const int2 *__restrict__ items,
                        long long n_items, long long p_total, const S *__restrict__ y,
                        const long long *__restrict__ run_idx, int *__restrict__ counters,
                        int res_blocks, long long n_pts_total, const S *__restrict__ truth,
                        double2 *__restrict__ partial, int *__restrict__ tickets, int n_inst,
                        double *__restrict__ resvar, int noise_blocks,
                        const int2 *__restrict__ node_items, const long long *__restrict__ frame,
                        S *__restrict__ noise_out) {
  if ((int)blockIdx.x < res_blocks) {
    lk_pdl_wait();
    const int inst = blockIdx.x / LK_RES_BLOCKS, rb = blockIdx.x - inst * LK_RES_BLOCKS;
    residual_block<S>(insts[inst], inst, rb, LK_RES_BLOCKS, n_pts_total, truth, run_idx, partial,
                      tickets, n_inst, resvar, nullptr);
    return;
  }
  if ((int)blockIdx.x < res_blocks + noise_blocks) {
    lk_pdl_wait();                  // the previous forecast advanced frame[0]
    const long long wi =
        ((long long)(blockIdx.x - res_blocks) * blockDim.x + threadIdx.x) >> 5;
    if (wi >= n_pts_total) return;
    const int lane = threadIdx.x & 31;
    const int2 it = node_items[wi];
    const LkInst &I = insts[it.x];
    const int2 ij = I.pts[it.y];
    const long long f = frame[0];
    S *out = noise_out + I.noise_off + (long long)it.y * I.m;
    for (int i = lane; i < I.m; i += 32) out[i] = bank_draw<S>(I, ij, i, f);
    return;
  }
  obs_block<S>(insts, items, n_items, p_total, y, run_idx, counters,
               blockIdx.x - res_blocks - noise_blocks);
}

// Every node's warm-start eigenbasis back to the identity (grid.y = instance).
__global__ void basis_reset_kernel(const LkInst *__restrict__ insts) {
  const LkInst &I = insts[blockIdx.y];
  const long long mp = I.mp, n = (long long)I.n_pts * mp * mp;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % (mp * mp);
    I.basis[e] = (r / mp == r % mp) ? 1.f : 0.f;
  }
}


int warp_blocks(long long warps) {
  return (int)((warps * 32 + LK_WARP_CTA - 1) / LK_WARP_CTA);
}

}  // namespace

cudaError_t lk_launch_obs(letkf_ctx *h, const void *y, const long long *run_idx) {
  // no subaperture, no kernel: the analysis counters are zeroed here instead
  if (h->sap_total == 0) return cudaMemsetAsync(h->counters + 1, 0, 7 * sizeof(int), h->stream);
  const int blocks = warp_blocks(h->sap_total);
  if (h->precision == 1)
    return lk_launch_pdl(obs_kernel<double>, blocks, LK_WARP_CTA, 0, h->stream, h->d_inst,
                         h->obs_items, h->sap_total, h->p_total, (const double *)y, run_idx,
                         h->counters);
  return lk_launch_pdl(obs_kernel<float>, blocks, LK_WARP_CTA, 0, h->stream, h->d_inst,
                       h->obs_items, h->sap_total, h->p_total, (const float *)y, run_idx,
                       h->counters);
}

cudaError_t lk_launch_obs_residual(letkf_ctx *h, const void *y, const void *truth,
                                   double *resvar, const long long *run_idx, void *noise_out) {
  if (h->sap_total == 0 || h->inst[0].dm) return cudaErrorInvalidValue;
  const int rblocks = (truth && resvar) ? LK_RES_BLOCKS * h->n_inst : 0;
  const int nblocks = noise_out ? warp_blocks(h->n_pts_total) : 0;
  const int blocks = rblocks + nblocks + warp_blocks(h->sap_total);
  if (h->precision == 1)
    return lk_launch_pdl(obs_residual_kernel<double>, blocks, LK_WARP_CTA, 0, h->stream,
                         h->d_inst, h->obs_items, h->sap_total, h->p_total, (const double *)y,
                         run_idx, h->counters, rblocks, h->n_pts_total, (const double *)truth,
                         h->partial, h->tickets, h->n_inst, resvar, nblocks, h->node_items,
                         h->frame, (double *)noise_out);
  return lk_launch_pdl(obs_residual_kernel<float>, blocks, LK_WARP_CTA, 0, h->stream, h->d_inst,
                       h->obs_items, h->sap_total, h->p_total, (const float *)y, run_idx,
                       h->counters, rblocks, h->n_pts_total, (const float *)truth, h->partial,
                       h->tickets, h->n_inst, resvar, nblocks, h->node_items, h->frame,
                       (float *)noise_out);
}

cudaError_t lk_launch_forecast(letkf_ctx *h, const void *noise) {
  const int blocks = warp_blocks(h->n_pts_total);
  int *ticket = h->tickets + h->n_inst;
  cudaError_t e;
  if (h->precision == 1)
    e = lk_launch_pdl(forecast_kernel<double>, blocks, LK_WARP_CTA, 0, h->stream, h->d_inst,
                      h->node_items, h->n_pts_total, (const double *)noise, h->frame, ticket);
  else
    e = lk_launch_pdl(forecast_kernel<float>, blocks, LK_WARP_CTA, 0, h->stream, h->d_inst,
                      h->node_items, h->n_pts_total, (const float *)noise, h->frame, ticket);
  // with a deformable mirror, the command of the new prediction
  if (e == cudaSuccess && h->inst[0].dm) e = lk_launch_dm_control(h);
  return e;
}

cudaError_t lk_launch_residual(letkf_ctx *h, const void *truth, double *resvar,
                               const long long *run_idx, double *piston) {
  return lk_launch_residual_on(h, h->stream, truth, resvar, run_idx, piston);
}

cudaError_t lk_launch_residual_on(letkf_ctx *h, cudaStream_t stream, const void *truth,
                                  double *resvar, const long long *run_idx, double *piston) {
  const dim3 grid(LK_RES_BLOCKS, h->n_inst);
  if (h->inst[0].dm) {              // the correction N u_{k-1} the residual is taken against
    cudaError_t e = lk_launch_dm_cor(h, stream);
    if (e != cudaSuccess) return e;
  }
  if (h->precision == 1)
    return lk_launch_pdl(residual_kernel<double>, grid, 64, 0, stream, h->d_inst, h->n_pts_total,
                         (const double *)truth, run_idx, h->partial, h->tickets, h->n_inst,
                         resvar, piston);
  return lk_launch_pdl(residual_kernel<float>, grid, 64, 0, stream, h->d_inst, h->n_pts_total,
                       (const float *)truth, run_idx, h->partial, h->tickets, h->n_inst, resvar,
                       piston);
}

cudaError_t lk_launch_basis_reset(letkf_ctx *h) {
  basis_reset_kernel<<<dim3(152, h->n_inst), 256, 0, h->stream>>>(h->d_inst);
  return cudaGetLastError();
}

// Frame stamp of a multi-frame graph: the global timer (ns) once the frame's
// last kernel has completed (a plain launch waits for the whole forecast grid).
__global__ void stamp_kernel(unsigned long long *__restrict__ dst) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *dst = t;
}

cudaError_t lk_launch_stamp(letkf_ctx *h, unsigned long long *dst) {
  stamp_kernel<<<1, 1, 0, h->stream>>>(dst);
  return cudaGetLastError();
}
