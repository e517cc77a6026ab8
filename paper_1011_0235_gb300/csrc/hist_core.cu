// hist_core.cu -- one-shot kernels (hist_plain, hist_adaptive), the device-side
// binning pattern and degeneracy, error handling.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "hist.h"
#include "hist_device.cuh"
#include "hist_internal.h"

using namespace histdev;

namespace {

thread_local int g_last_cuda_error = 0;

// One-shot histogram of [in, in+n) into out (zeroed beforehand by the caller).
// pat == nullptr selects the per-warp (PLAIN) layout.  One CTA of 1024
// threads per SM with four loads in flight per thread: as many bytes in
// flight as two CTAs with two loads each, without two CTAs on one SM
// finishing their ranges apart (1 GiB, full table: 6.05 -> 6.25 TB/s
// uniform, 6.14 -> 6.41 TB/s N(128, 8); per-warp tables unchanged).
__global__ void __launch_bounds__(kThreads, 1)
    oneshot_kernel(const uint8_t* __restrict__ in, size_t n, const hist_pattern* __restrict__ pat,
                   uint32_t* __restrict__ out) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* table = smem;
  uint32_t* lut = smem + kTableWords;
  __shared__ CtaShared cs;

  zero_table(table);
  if (pat) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(pat);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&cs.pat);
    for (int i = threadIdx.x; i < (int)(sizeof(hist_pattern) / 4); i += kThreads) dst[i] = src[i];
    __syncthreads();
    classify_pattern(cs.pat, lut, cs);
  } else {
    if (threadIdx.x == 0) {
      cs.path = PATH_PLAIN;
      cs.lk = 0;
    }
    __syncthreads();
  }
  const Split sp = split_bytes(in, n);
  const uint4* body = reinterpret_cast<const uint4*>(in + sp.head);
  const size_t begin = part_begin(sp.nvec, gridDim.x, blockIdx.x);
  const size_t end = part_begin(sp.nvec, gridDim.x, blockIdx.x + 1);
  count_range_dispatch<4>(cs.path, cs.lk, body, begin, end, table, lut, threadIdx.x, kThreads);
  flush_table(cs.path, cs.lk, table, cs.pat, lut, cs);
  if (blockIdx.x == 0) {
    count_edges(in, sp, cs);
    __syncthreads();
  }
  if (threadIdx.x < HIST_BINS && cs.res[threadIdx.x]) atomicAdd(out + threadIdx.x, cs.res[threadIdx.x]);
}

// Change detection between two uint64 histograms (256 threads).
__global__ void __launch_bounds__(HIST_BINS) change_kernel(const unsigned long long* __restrict__ acc,
                                                          const unsigned long long* __restrict__ win,
                                                          uint32_t tau_milli, hist_change_result* __restrict__ res) {
  __shared__ ChangeShared sh;
  const int t = threadIdx.x;
  const hist_change_result r = change_eval(acc[t], win[t], tau_milli, sh);
  if (t == 0) *res = r;
}

// One warp: the binning pattern of h (or the default pattern if h is null).
__global__ void __launch_bounds__(32) pattern_kernel(const uint32_t* __restrict__ h, uint32_t budget,
                                                     hist_pattern* __restrict__ out) {
  __shared__ hist_pattern P;
  __shared__ uint32_t hs[HIST_BINS];
  for (int i = threadIdx.x; i < HIST_BINS; i += 32) hs[i] = h ? h[i] : 0u;
  __syncwarp();
  warp_epilogue(hs, budget, HIST_THETA_MILLI_DEFAULT, P);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&P);
  uint32_t* dst = reinterpret_cast<uint32_t*>(out);
  for (int i = threadIdx.x; i < (int)(sizeof(hist_pattern) / 4); i += 32) dst[i] = src[i];
}

// One warp: the degeneracy of h.
template <class T>
__global__ void __launch_bounds__(32) degeneracy_kernel(const T* __restrict__ h, uint32_t theta,
                                                        hist_degeneracy_result* __restrict__ res) {
  __shared__ hist_pattern P;
  __shared__ T hs[HIST_BINS];
  for (int i = threadIdx.x; i < HIST_BINS; i += 32) hs[i] = h[i];
  __syncwarp();
  const hist_degeneracy_result r = warp_epilogue(hs, HIST_BUDGET_MAX, theta, P);
  if (threadIdx.x == 0) *res = r;
}

}  // namespace

namespace histlib {

int cuda_fail(cudaError_t e) {
  g_last_cuda_error = (int)e;
  return HIST_ECUDA;
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 148;
  return sms;
}

int ensure_smem_attr(const void* fn, int* done) { return ensure_smem_attr_bytes(fn, done, kSmemBytes); }

int ensure_smem_attr_bytes(const void* fn, int* done, size_t bytes) {
  // Kernels using more than 48 KiB of dynamic shared memory need the opt-in,
  // once per (kernel, device); `done` is the caller's per-kernel array of
  // kMaxDevices.
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev >= 0 && dev < kMaxDevices && done[dev]) return HIST_OK;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev >= 0 && dev < kMaxDevices) done[dev] = 1;
  return HIST_OK;
}

int oneshot(const uint8_t* d_in, size_t n, const hist_pattern* d_pat, uint32_t* d_out, cudaStream_t s) {
  if (!d_out || (!d_in && n) || n >= ((size_t)1 << 32)) return HIST_EINVAL;
  cudaError_t e = cudaMemsetAsync(d_out, 0, HIST_BINS * sizeof(uint32_t), s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (n == 0) return HIST_OK;
  static int attr_done[kMaxDevices];
  int rc = ensure_smem_attr((const void*)oneshot_kernel, attr_done);
  if (rc) return rc;
  const Split sp = split_bytes(d_in, n);
  const size_t want = (sp.nvec + 4 * kThreads - 1) / (4 * kThreads);
  const size_t cap = 1 * (size_t)sm_count();
  const int grid = (int)(want < 1 ? 1 : (want > cap ? cap : want));
  oneshot_kernel<<<grid, kThreads, kSmemBytes, s>>>(d_in, n, d_pat, d_out);
  e = cudaGetLastError();
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

}  // namespace histlib

using namespace histlib;

extern "C" {

const char* hist_strerror(int code) {
  switch (code) {
    case HIST_OK: return "ok";
    case HIST_EINVAL: return "invalid argument";
    case HIST_ENOMEM: return "out of memory";
    case HIST_EBUDGET: return "request exceeds the admission budget";
    case HIST_ETIMEDOUT: return "bounded wait timed out";
    case HIST_ECUDA: return "CUDA error";
    case HIST_EBUSY: return "no free slot";
    case HIST_ESTATE: return "object in the wrong state";
    default: return "unknown error";
  }
}

int hist_last_cuda_error(void) { return g_last_cuda_error; }

int hist_device_sms(void) { return sm_count(); }

int hist_pattern_check(const hist_pattern* p) {
  if (!p) return HIST_EINVAL;
  if (p->budget < HIST_BUDGET_MIN || p->budget > HIST_BUDGET_MAX) return HIST_EINVAL;
  uint8_t seen[HIST_BUDGET_MAX];
  memset(seen, 0, sizeof(seen));
  uint32_t used = 0;
  for (int b = 0; b < HIST_BINS; ++b) {
    if (p->log2k[b] > 5) return HIST_EINVAL;
    const uint32_t k = 1u << p->log2k[b];
    const uint32_t o = p->off[b];
    if (o % k != 0 || o + k > p->budget) return HIST_EINVAL;
    for (uint32_t j = 0; j < k; ++j) {
      if (seen[o + j]) return HIST_EINVAL;
      seen[o + j] = 1;
    }
    used += k;
  }
  return used == p->used ? HIST_OK : HIST_EINVAL;
}

int hist_plain(const uint8_t* d_in, size_t n, uint32_t* d_out, hist_cuda_stream s) {
  return oneshot(d_in, n, nullptr, d_out, (cudaStream_t)s);
}

int hist_adaptive(const uint8_t* d_in, size_t n, const hist_pattern* d_pat, uint32_t* d_out,
                  hist_cuda_stream s) {
  if (!d_pat) return HIST_EINVAL;
  return oneshot(d_in, n, d_pat, d_out, (cudaStream_t)s);
}

int binning_pattern(const uint32_t* d_prev_hist, uint32_t budget, hist_pattern* d_pat, hist_cuda_stream s) {
  if (!d_prev_hist || !d_pat || budget < HIST_BUDGET_MIN || budget > HIST_BUDGET_MAX) return HIST_EINVAL;
  pattern_kernel<<<1, 32, 0, (cudaStream_t)s>>>(d_prev_hist, budget, d_pat);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int default_pattern(uint32_t budget, hist_pattern* d_pat, hist_cuda_stream s) {
  if (!d_pat || budget < HIST_BUDGET_MIN || budget > HIST_BUDGET_MAX) return HIST_EINVAL;
  pattern_kernel<<<1, 32, 0, (cudaStream_t)s>>>(nullptr, budget, d_pat);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int degeneracy(const uint32_t* d_hist, uint32_t theta_milli, hist_degeneracy_result* d_res,
               hist_cuda_stream s) {
  if (!d_hist || !d_res || theta_milli > 1000) return HIST_EINVAL;
  degeneracy_kernel<uint32_t><<<1, 32, 0, (cudaStream_t)s>>>(d_hist, theta_milli, d_res);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int hist_change(const uint64_t* d_acc, const uint64_t* d_win, uint32_t tau_milli, hist_change_result* d_res,
                hist_cuda_stream s) {
  if (!d_acc || !d_win || !d_res || tau_milli > 1000) return HIST_EINVAL;
  change_kernel<<<1, HIST_BINS, 0, (cudaStream_t)s>>>(reinterpret_cast<const unsigned long long*>(d_acc),
                                                      reinterpret_cast<const unsigned long long*>(d_win), tau_milli,
                                                      d_res);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int degeneracy_u64(const uint64_t* d_hist, uint32_t theta_milli, hist_degeneracy_result* d_res,
                   hist_cuda_stream s) {
  if (!d_hist || !d_res || theta_milli > 1000) return HIST_EINVAL;
  degeneracy_kernel<unsigned long long><<<1, 32, 0, (cudaStream_t)s>>>(
      reinterpret_cast<const unsigned long long*>(d_hist), theta_milli, d_res);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

}  // extern "C"
