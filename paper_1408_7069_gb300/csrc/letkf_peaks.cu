// Arithmetic peaks of the GPU the library runs on, measured: the denominators
// of the analysis roofline. The analysis (Section 4.2's Gram, eigensolve and
// transform) is bound by FP32 arithmetic, and the FP64 fallback by FP64
// arithmetic; the nominal rates assume the maximum SM clock, which a GPU under
// load need not hold. Each kernel runs independent FMA chains in every thread of
// a grid that fills the device (a multiple of the SM count), long enough for the
// clocks to settle, and records the SM clock cycles and the global timer of
// every CTA, from which the clock the arithmetic actually ran at follows.
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>

#include "letkf.h"

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CTAS_PER_SM = 4;      // 32 warps per SM
constexpr int PK_CHAINS = 8;           // independent FMA chains per thread

__device__ __forceinline__ unsigned long long pk_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// a <- a b + c in PK_CHAINS chains; b < 1 keeps every chain bounded.
template <typename T>
__device__ __forceinline__ void pk_step(T (&a)[PK_CHAINS], T b, T c) {
#pragma unroll
  for (int i = 0; i < PK_CHAINS; ++i) a[i] = fma(a[i], b, c);
}
__device__ __forceinline__ void pk_step(float2 (&a)[PK_CHAINS], float2 b, float2 c) {
#pragma unroll
  for (int i = 0; i < PK_CHAINS; ++i) a[i] = __ffma2_rn(a[i], b, c);
}

template <typename T>
__device__ __forceinline__ T pk_init(int i) {
  return T(threadIdx.x * 1e-3 + i);
}
template <>
__device__ __forceinline__ float2 pk_init<float2>(int i) {
  return make_float2(threadIdx.x * 1e-3f + i, threadIdx.x * 2e-3f + i);
}
__device__ __forceinline__ float pk_sum(float x) { return x; }
__device__ __forceinline__ double pk_sum(double x) { return x; }
__device__ __forceinline__ float pk_sum(float2 x) { return x.x + x.y; }

// stamps[4 * cta + 0..3]: clock64 and globaltimer at the start and the end.
template <typename T>
__global__ void __launch_bounds__(PK_THREADS)
    fma_peak_kernel(int iters, T b, T c, float *__restrict__ sink,
                    unsigned long long *__restrict__ stamps) {
  __syncthreads();
  const unsigned long long c0 = clock64(), g0 = pk_globaltimer();
  T a[PK_CHAINS];
#pragma unroll
  for (int i = 0; i < PK_CHAINS; ++i) a[i] = pk_init<T>(i);
  for (int it = 0; it < iters; ++it) {
    pk_step(a, b, c);
    pk_step(a, b, c);
    pk_step(a, b, c);
    pk_step(a, b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < PK_CHAINS; ++i) s += (float)pk_sum(a[i]);
  sink[blockIdx.x * PK_THREADS + threadIdx.x] = s;   // keeps the chains live
  __syncthreads();
  if (threadIdx.x == 0) {
    stamps[4 * blockIdx.x + 0] = c0;
    stamps[4 * blockIdx.x + 1] = clock64();
    stamps[4 * blockIdx.x + 2] = g0;
    stamps[4 * blockIdx.x + 3] = pk_globaltimer();
  }
}

// Runs one kernel: a warm-up launch, then a timed one. flops per FMA-chain step
// per thread: 2 (4 for the packed float2 form). Returns TFLOP/s and the mean
// SM clock of its CTAs in MHz.
template <typename T>
cudaError_t run_peak(int ctas, int iters, int flops_per_fma, T b, T c, float *sink,
                     unsigned long long *stamps, unsigned long long *stamps_host, double *tflops,
                     double *mhz) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    fma_peak_kernel<T><<<ctas, PK_THREADS>>>(iters / 4, b, c, sink, stamps);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  if (e == cudaSuccess) {
    fma_peak_kernel<T><<<ctas, PK_THREADS>>>(iters, b, c, sink, stamps);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess)
    e = cudaMemcpy(stamps_host, stamps, (size_t)ctas * 4 * sizeof(unsigned long long),
                   cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    const double fmas = (double)ctas * PK_THREADS * PK_CHAINS * 4.0 * iters;
    *tflops = fmas * flops_per_fma / (ms * 1e-3) / 1e12;
    double cyc = 0.0, ns = 0.0;
    for (int i = 0; i < ctas; ++i) {
      cyc += (double)(stamps_host[4 * i + 1] - stamps_host[4 * i + 0]);
      ns += (double)(stamps_host[4 * i + 3] - stamps_host[4 * i + 2]);
    }
    *mhz = ns > 0 ? 1e3 * cyc / ns : 0.0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" letkf_status letkf_fma_peaks(double *out) {
  if (!out) return LETKF_ERR_ARG;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || sms <= 0) return LETKF_ERR_CUDA;
  const int ctas = sms * PK_CTAS_PER_SM;
  float *sink = nullptr;
  unsigned long long *stamps = nullptr;
  unsigned long long *host = new (std::nothrow) unsigned long long[(size_t)ctas * 4];
  if (!host) return LETKF_ERR_NOMEM;
  e = cudaMalloc((void **)&sink, (size_t)ctas * PK_THREADS * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void **)&stamps, (size_t)ctas * 4 * sizeof(unsigned long long));
  for (int i = 0; i < 7; ++i) out[i] = 0.0;
  out[6] = sms;
  // about 30 ms of FP32 work at 80 TFLOP/s; FP64 runs at a small fraction of that rate
  if (e == cudaSuccess)
    e = run_peak<float>(ctas, 1 << 18, 2, 0.999999f, 1e-6f, sink, stamps, host, &out[0], &out[1]);
  if (e == cudaSuccess)
    e = run_peak<float2>(ctas, 1 << 17, 4, make_float2(0.999999f, 0.999999f),
                         make_float2(1e-6f, 1e-6f), sink, stamps, host, &out[2], &out[3]);
  if (e == cudaSuccess)
    e = run_peak<double>(ctas, 1 << 12, 2, 0.999999, 1e-6, sink, stamps, host, &out[4], &out[5]);
  if (sink) cudaFree(sink);
  if (stamps) cudaFree(stamps);
  delete[] host;
  return e == cudaSuccess ? LETKF_OK : LETKF_ERR_CUDA;
}
