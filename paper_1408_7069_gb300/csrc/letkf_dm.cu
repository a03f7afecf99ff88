// Deformable mirror and the true closed loop (Section 2.1, Eqs. Eq_Obs and
// Eq_Cor; Section 2.2; Section 3.1.1; Appendix B.3).
//
// With a DM (letkf_set_dm: the caller's influence matrix N and command matrix
// P over the instance's nodes, CSR; the library forms D1 N), a frame is
//   residual   of phi^tur_k - N u_{k-1}                          (cor kernel)
//   analysis   of the pseudo-open-loop slopes y_k + D1 N u_{k-2}  (observation kernel)
//   forecast   and the predicted phase phihat_{k+1/k}            (forecast kernel)
//   command    u_k = P phihat_{k+1/k}                            (control kernel)
// the commands kept in a ring of three indexed by the forecast counter f
// (slot f % 3 = the command computed after forecast f), so that every launch
// finds u_{k-1} and u_{k-2} on the device and a frame can be captured in a
// CUDA graph. letkf_run_dm simulates the measurement of a closed loop,
// y_k = D1 (phi^tur_{k-1} - N u_{k-2}) + w_k (wfs kernel).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "letkf_device.cuh"

namespace {

// cor = N u_{k-1}: thread per node (u_{k-1} in slot (f + 2) % 3).
template <typename S>
__global__ void __launch_bounds__(128) dm_cor_kernel(const LkInst *__restrict__ insts) {
  lk_pdl_wait();
  const LkInst &I = insts[0];
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= I.n_pts) return;
  const S *u1 = static_cast<const S *>(I.u) + (size_t)((*I.fcount + 2) % 3) * I.n_pts;
  const S *nv = static_cast<const S *>(I.n_val);
  S s = S(0);
  for (int q = I.n_ptr[b]; q < I.n_ptr[b + 1]; ++q) s += nv[q] * u1[I.n_idx[q]];
  static_cast<S *>(I.cor)[b] = s;
}

// u_k = P phihat_{k+1/k}: warp per actuator, after the forecast (which has
// advanced the counter to f + 1: the new command goes to slot f % 3).
template <typename S>
__global__ void __launch_bounds__(LK_WARP_CTA) dm_control_kernel(const LkInst *__restrict__ insts) {
  lk_pdl_wait();
  const LkInst &I = insts[0];
  const int a = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (a >= I.n_pts) return;
  const S *pv = static_cast<const S *>(I.p_val);
  const S *ph = static_cast<const S *>(I.pmean);
  S s = S(0);
  for (int q = I.p_ptr[a] + lane; q < I.p_ptr[a + 1]; q += 32) s += pv[q] * ph[I.p_idx[q]];
  s = lk_warp_sum(s);
  if (lane == 0)
    static_cast<S *>(I.u)[(size_t)((*I.fcount + 2) % 3) * I.n_pts + a] = s;
}

// y_k = D1 (phi_prev - N u_{k-2}) + w_k, thread per slope (sx of every valid
// subaperture, then sy); phi_prev = truth_seq[run_idx - 1], zero for the first
// frame of a run.
template <typename S>
__global__ void __launch_bounds__(128)
    dm_wfs_kernel(const LkInst *__restrict__ insts, const S *__restrict__ truth_seq,
                  const S *__restrict__ wnoise_seq, const long long *__restrict__ run_idx,
                  S *__restrict__ y) {
  lk_pdl_wait();
  const LkInst &I = insts[0];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= I.p) return;
  const long long k = *run_idx;
  const int sub = r < I.n_sap ? r : r - I.n_sap;
  const int nn = I.nsub + 1;
  const int2 st = I.saps[sub];
  S d1 = S(0);
  if (k > 0) {
    const S *ph = truth_seq + (k - 1) * I.n_pts;
    const S p00 = ph[I.pid_map[st.x * nn + st.y]], p10 = ph[I.pid_map[(st.x + 1) * nn + st.y]];
    const S p01 = ph[I.pid_map[st.x * nn + st.y + 1]];
    const S p11 = ph[I.pid_map[(st.x + 1) * nn + st.y + 1]];
    d1 = r < I.n_sap ? S(0.5) * ((p10 + p11) - (p00 + p01)) : S(0.5) * ((p01 + p11) - (p00 + p10));
  }
  const S *u2 = static_cast<const S *>(I.u) + (size_t)((*I.fcount + 1) % 3) * I.n_pts;
  const S *dv = static_cast<const S *>(I.dn_val);
  S dn = S(0);
  for (int q = I.dn_ptr[r]; q < I.dn_ptr[r + 1]; ++q) dn += dv[q] * u2[I.dn_idx[q]];
  y[r] = d1 - dn + wnoise_seq[k * I.p + r];
}

// The latest command u_{k-1} (slot (f + 2) % 3) into out, thread per actuator.
template <typename S>
__global__ void __launch_bounds__(128) dm_get_kernel(const LkInst *__restrict__ insts,
                                                     S *__restrict__ out) {
  lk_pdl_wait();
  const LkInst &I = insts[0];
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < I.n_pts)
    out[a] = static_cast<const S *>(I.u)[(size_t)((*I.fcount + 2) % 3) * I.n_pts + a];
}

}  // namespace

cudaError_t lk_launch_dm_get(letkf_ctx *h, void *out) {
  const unsigned blocks = (unsigned)((h->inst[0].n_pts + 127) / 128);
  if (h->precision == 1)
    return lk_launch_pdl(dm_get_kernel<double>, blocks, 128, 0, h->stream,
                         (const LkInst *)h->d_inst, (double *)out);
  return lk_launch_pdl(dm_get_kernel<float>, blocks, 128, 0, h->stream, (const LkInst *)h->d_inst,
                       (float *)out);
}

cudaError_t lk_launch_dm_cor(letkf_ctx *h, cudaStream_t stream) {
  const unsigned blocks = (unsigned)((h->inst[0].n_pts + 127) / 128);
  if (h->precision == 1)
    return lk_launch_pdl(dm_cor_kernel<double>, blocks, 128, 0, stream, (const LkInst *)h->d_inst);
  return lk_launch_pdl(dm_cor_kernel<float>, blocks, 128, 0, stream, (const LkInst *)h->d_inst);
}

cudaError_t lk_launch_dm_control(letkf_ctx *h) {
  const unsigned blocks = (unsigned)(((long long)h->inst[0].n_pts * 32 + LK_WARP_CTA - 1) / LK_WARP_CTA);
  if (h->precision == 1)
    return lk_launch_pdl(dm_control_kernel<double>, blocks, LK_WARP_CTA, 0, h->stream,
                         (const LkInst *)h->d_inst);
  return lk_launch_pdl(dm_control_kernel<float>, blocks, LK_WARP_CTA, 0, h->stream,
                       (const LkInst *)h->d_inst);
}

cudaError_t lk_launch_dm_wfs(letkf_ctx *h, const void *truth_seq, const void *wnoise_seq,
                             const long long *run_idx, void *y_out) {
  const unsigned blocks = (unsigned)((h->inst[0].p + 127) / 128);
  if (h->precision == 1)
    return lk_launch_pdl(dm_wfs_kernel<double>, blocks, 128, 0, h->stream,
                         (const LkInst *)h->d_inst, (const double *)truth_seq,
                         (const double *)wnoise_seq, run_idx, (double *)y_out);
  return lk_launch_pdl(dm_wfs_kernel<float>, blocks, 128, 0, h->stream, (const LkInst *)h->d_inst,
                       (const float *)truth_seq, (const float *)wnoise_seq, run_idx,
                       (float *)y_out);
}
