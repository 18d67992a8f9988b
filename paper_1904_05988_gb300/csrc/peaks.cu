// Measured arithmetic peaks for the roofline of kernels bound by the FP64 or
// FP32 pipe (diagnostic; no counterpart in the paper).
//
// Every thread runs kChains independent FMA recurrences x <- x*a + b for
// `iters` steps (2 flops each); the grid holds `blocks_per_sm` blocks of 256
// threads on every SM, enough independent work to cover the pipe latency.
// The kernel is timed with CUDA events around repeated launches on a private
// stream; the best of `reps` launches gives the rate.
#include "internal.cuh"

namespace pfsh {

constexpr int kChains = 8;

__device__ double g_fma_sink;   // external linkage: the store below cannot be dropped

template <typename R>
__global__ void __launch_bounds__(256) k_fma_loop(int iters, R a, R b) {
  R x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (R)(threadIdx.x * 1e-3 + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  R s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (R)-1.0) g_fma_sink = (double)s;   // never true (x stays positive): keeps the loop alive
}

template <typename R>
static int fma_peak(double *tflops) {
  int dev = 0, sms = 0;
  PFSH_CUDA(cudaGetDevice(&dev));
  PFSH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = sizeof(R) == 8 ? 1 << 12 : 1 << 15, reps = 5;
  cudaStream_t s;
  cudaEvent_t e0, e1;
  PFSH_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  PFSH_CUDA(cudaEventCreate(&e0));
  PFSH_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int rc = PFSH_OK;
  for (int r = 0; r < reps + 1 && rc == PFSH_OK; ++r) {
    cudaEventRecord(e0, s);
    {
      PFSH_LAUNCH("k_fma_loop", s);
      k_fma_loop<R><<<blocks, threads, 0, s>>>(iters, (R)0.999999, (R)1e-7);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "k_fma_loop");
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (rc == PFSH_OK && e != cudaSuccess) rc = cuda_fail(e, "k_fma_loop sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms < best) best = ms;   // the first launch warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (rc) return rc;
  const double flops = 2.0 * kChains * (double)iters * blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return PFSH_OK;
}

}  // namespace pfsh

extern "C" int pfsh_alu_peak(int prec, double *tflops) {
  if (!tflops || (prec != PFSH_FP64 && prec != PFSH_FP32))
    return pfsh::fail(PFSH_EINVAL, "pfsh_alu_peak: prec must be PFSH_FP64 or PFSH_FP32, tflops non-NULL");
  return prec == PFSH_FP64 ? pfsh::fma_peak<double>(tflops) : pfsh::fma_peak<float>(tflops);
}
