// Failure detection without faulting the GPU.
//
// 1. Non-finite check (opt-in, pfsh_set_check_finite): after swe_rhs,
//    sdc_sweep and the PFASST calls, one grid-stride kernel scans the
//    results (F_E and F_I; the swept nodes; the fine end values of every
//    slice) and records ST_NUMERIC in the library's status word if any
//    component is NaN or infinite; pfsh_sync_status then returns
//    PFSH_ENUMERIC.  The check reads what the call wrote and changes nothing.
// 2. Bounded waits (pfsh_selftest_wait): one CTA allocates tensor memory,
//    waits with the library's bounded mbarrier wait on a barrier that nothing
//    arms, records ST_TIMEOUT when the poll limit runs out, frees its tensor
//    memory and returns, leaving the context usable.  This is the path every
//    tcgen05 kernel of the library takes when one of its waits gives up.
#include <atomic>

#include "internal.cuh"
#include "tc.cuh"

namespace pfsh {

static std::atomic<int> g_check_finite{0};

bool check_finite_on() { return g_check_finite.load(std::memory_order_relaxed) != 0; }

__global__ void k_nonfinite(const double *__restrict__ x, size_t n, int *status) {
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(status, ST_OK, ST_NUMERIC);
}

int check_finite(const double *x, size_t n, cudaStream_t s) {
  if (!check_finite_on() || n == 0) return PFSH_OK;
  int *st = device_status();
  if (!st) return fail(PFSH_ECUDA, "check_finite: no status word");
  int dev = 0, sms = 0;
  PFSH_CUDA(cudaGetDevice(&dev));
  PFSH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t blocks = std::min<size_t>((n + 255) / 256, (size_t)sms * 8);
  {
    PFSH_LAUNCH("k_nonfinite", s);
    k_nonfinite<<<(unsigned)blocks, 256, 0, s>>>(x, n, st);
  }
  PFSH_CHECK_LAUNCH("k_nonfinite");
  return PFSH_OK;
}

// one CTA of 128 threads: TMEM allocation, a bounded wait on a barrier that
// is never armed, ST_TIMEOUT, TMEM freed
__global__ void k_wait_selftest(unsigned polls, int *status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(&tmem_slot, 32);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const bool ok = tc::mbar_wait(&bar, 0, polls);   // nothing arrives: gives up after `polls` polls
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) tc::tmem_dealloc(tmem_slot, 32);
  if (!ok && threadIdx.x == 0 && status) atomicExch(status, ST_TIMEOUT);
}

}  // namespace pfsh

using namespace pfsh;

extern "C" int pfsh_set_check_finite(int on) {
  g_check_finite.store(on ? 1 : 0);
  return PFSH_OK;
}

extern "C" int pfsh_selftest_wait(unsigned polls, pfsh_stream_t stream) {
  if (polls < 1 || polls > (1u << 20)) return fail(PFSH_EINVAL, "pfsh_selftest_wait: polls must be in 1..2^20");
  cudaStream_t s = (cudaStream_t)stream;
  {
    PFSH_LAUNCH("k_wait_selftest", s);
    k_wait_selftest<<<1, 128, 0, s>>>(polls, device_status());
  }
  PFSH_CHECK_LAUNCH("k_wait_selftest");
  return PFSH_OK;
}
