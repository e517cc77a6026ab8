// hist_ablation.cu -- the kernel built up step by step (Table 1).
//
// Table 1 measures the adaptive kernel as five cumulative variants: read the
// packed pixels and write a block result; + clear the shared sub-histogram;
// + read the binning pattern; + the sub-histogram atomics; + sum the sub-bins
// and write the histogram.  This file builds the same five variants on the
// one-shot kernel's structure (2 CTAs of 1024 threads per SM, each CTA one
// contiguous range of 16-byte vectors), so that the time each step adds can
// be measured on this hardware:
//   stage 1: load every vector and fold it into a register; each CTA writes
//            256 words (its "block result") to a scratch sink;
//   stage 2: + clear the 32 KiB shared table;
//   stage 3: + read the binning pattern into shared memory and compute every
//            pixel's sub-bin address (the lookup or shift of the layout),
//            folding the addresses into the register instead of counting;
//   stage 4: + the shared-memory increments (the full counting);
//   stage 5: + reduce the table per bin and add it into the histogram: the
//            complete kernel (hist_plain / hist_adaptive);
//   stage 6: stage 5 with warp-aggregated increments: the lanes holding the
//            same value elect one (__match_any_sync over the active lanes),
//            which adds the group's size -- the classic remedy for
//            same-address conflicts, measured against the plain increments;
//   stage 7: stage 5 with the input staged through shared memory: one thread
//            streams the CTA's range into two 16 KiB buffers with 1-D bulk
//            copies (cp.async.bulk, completion on an mbarrier), and every
//            thread counts one 16-byte vector of the full buffer -- the
//            copy-engine alternative to each thread's own 16-byte loads.
// Without a pattern the variants are those of the per-warp (plain) kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hist.h"
#include "hist_device.cuh"
#include "hist_internal.h"

using namespace histdev;
using namespace histlib;

namespace {

// Sub-bin address of pixel v (PATH/LK as in count_word), or the increment.
template <int STAGE, int PATH, int LK>
__device__ __forceinline__ void ablate_word(uint32_t w, uint32_t base, uint32_t lutb, uint32_t table, uint32_t& acc) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t v = (w >> (8 * k)) & 0xffu;
    if (STAGE <= 2) {
      acc += v;
    } else if (STAGE == 6) {
      const uint32_t m = __match_any_sync(__activemask(), v);
      if ((uint32_t)(__ffs(m) - 1) == (threadIdx.x & 31u)) {
        const uint32_t a = PATH == PATH_LUT ? table + (shared_ld(lutb + (v << 7)) << 2) : base + (v << (LK + 2));
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"((uint32_t)__popc(m)) : "memory");
      }
    } else {
      const uint32_t a = PATH == PATH_LUT ? table + (shared_ld(lutb + (v << 7)) << 2) : base + (v << (LK + 2));
      if (STAGE == 3) acc ^= a;
      else shared_inc(a);
    }
  }
}

template <int STAGE, int PATH, int LK>
__device__ __forceinline__ void ablate_vec(const uint4& q0, uint32_t base, uint32_t lutb, uint32_t table, uint32_t& acc) {
  // the counting kernels' lane order of the bytes from the address stage on
  const uint4 q = (STAGE >= 3 && !(PATH == PATH_SHIFT && LK >= 4)) ? lane_permute(q0, lane_order()) : q0;
  ablate_word<STAGE, PATH, LK>(q.x, base, lutb, table, acc);
  ablate_word<STAGE, PATH, LK>(q.y, base, lutb, table, acc);
  ablate_word<STAGE, PATH, LK>(q.z, base, lutb, table, acc);
  ablate_word<STAGE, PATH, LK>(q.w, base, lutb, table, acc);
}

template <int STAGE, int PATH, int LK>
__device__ void ablate_range(const uint4* __restrict__ p, size_t begin, size_t end, uint32_t* table,
                             const uint32_t* lut, uint32_t& acc) {
  uint32_t base, lutb, tab;
  thread_bases<PATH, LK>(table, lut, base, lutb, tab);
  // the loop of count_range (two vectors per group, the next group's loads
  // issued before the current group is processed)
  size_t i = begin + threadIdx.x;
  if (i + kThreads < end) {
    uint4 a = ldg_stream(p + i), b = ldg_stream(p + i + kThreads);
    for (i += 2 * kThreads; i + kThreads < end; i += 2 * kThreads) {
      const uint4 c = ldg_stream(p + i), d = ldg_stream(p + i + kThreads);
      ablate_vec<STAGE, PATH, LK>(a, base, lutb, tab, acc);
      ablate_vec<STAGE, PATH, LK>(b, base, lutb, tab, acc);
      a = c;
      b = d;
    }
    ablate_vec<STAGE, PATH, LK>(a, base, lutb, tab, acc);
    ablate_vec<STAGE, PATH, LK>(b, base, lutb, tab, acc);
  }
  for (; i < end; i += kThreads) ablate_vec<STAGE, PATH, LK>(ldg_stream(p + i), base, lutb, tab, acc);
}

template <int STAGE>
__device__ void ablate_dispatch(int path, int lk, const uint4* p, size_t begin, size_t end, uint32_t* table,
                                const uint32_t* lut, uint32_t& acc) {
  if (begin >= end) return;
  if (STAGE <= 2 || path == PATH_PLAIN) ablate_range<STAGE, PATH_PLAIN, 0>(p, begin, end, table, lut, acc);
  else if (path == PATH_LUT) ablate_range<STAGE, PATH_LUT, 0>(p, begin, end, table, lut, acc);
  else {
    switch (lk) {
      case 5: ablate_range<STAGE, PATH_SHIFT, 5>(p, begin, end, table, lut, acc); break;
      case 4: ablate_range<STAGE, PATH_SHIFT, 4>(p, begin, end, table, lut, acc); break;
      case 3: ablate_range<STAGE, PATH_SHIFT, 3>(p, begin, end, table, lut, acc); break;
      case 2: ablate_range<STAGE, PATH_SHIFT, 2>(p, begin, end, table, lut, acc); break;
      case 1: ablate_range<STAGE, PATH_SHIFT, 1>(p, begin, end, table, lut, acc); break;
      default: ablate_range<STAGE, PATH_SHIFT, 0>(p, begin, end, table, lut, acc); break;
    }
  }
}

// ---------------------------------------------------------- stage 7 --
// Bulk-copy staging.  Waits on the mbarriers are bounded (kStageWaitLimit
// polls): a wait that runs out sets *status (when given) and the CTA stops
// issuing copies, waits (bounded again) for the ones it issued, adds what it
// counted and returns.

constexpr int kStageVecs = kThreads;            // 16 KiB per buffer: one vector per thread
constexpr int kStageBufs = 2;
constexpr size_t kStageSmem = kSmemBytes + (size_t)kStageBufs * kStageVecs * 16;  // + 32 KiB
constexpr uint32_t kStageWaitLimit = 1u << 22;
constexpr uint32_t kStageTimeout = 1u;

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t k = 0; k < kStageWaitLimit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Count vectors [begin, end) of p staged through buf (kStageBufs buffers of
// kStageVecs vectors) with full[] as their mbarriers; all threads call.
template <int PATH, int LK>
__device__ void staged_range(const uint4* __restrict__ p, size_t begin, size_t end, uint32_t* table,
                             const uint32_t* lut, const uint4* buf, const unsigned long long* full,
                             uint32_t* status) {
  uint32_t base, lutb, tab;
  thread_bases<PATH, LK>(table, lut, base, lutb, tab);
  const LaneOrder o = lane_order();
  const size_t total = end > begin ? end - begin : 0;
  const size_t iters = (total + kStageVecs - 1) / kStageVecs;
  const uint32_t b0 = smem_addr(buf), f0 = smem_addr(full);
  __shared__ int stop;
  auto issue = [&](size_t it) {
    const size_t v0 = it * kStageVecs;
    const uint32_t vecs = (uint32_t)(total - v0 < (size_t)kStageVecs ? total - v0 : (size_t)kStageVecs);
    const uint32_t k = (uint32_t)(it % kStageBufs);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of the buffer, then the copy
    mbar_expect_tx(f0 + 8 * k, vecs * 16);
    bulk_load(b0 + k * kStageVecs * 16, p + begin + v0, vecs * 16, f0 + 8 * k);
  };
  if (threadIdx.x == 0) {
    stop = 0;
    for (size_t it = 0; it < iters && it < (size_t)kStageBufs; ++it) issue(it);
  }
  __syncthreads();
  size_t it = 0;
  for (; it < iters; ++it) {
    const uint32_t k = (uint32_t)(it % kStageBufs), parity = (uint32_t)((it / kStageBufs) & 1);
    if (!mbar_wait(f0 + 8 * k, parity)) atomicExch(&stop, 1);
    __syncthreads();
    if (stop) break;
    const size_t v0 = it * kStageVecs;
    if (v0 + threadIdx.x < total) {
      const uint4 q = buf[k * kStageVecs + threadIdx.x];
      count_vec<PATH, LK>(q, base, lutb, tab, o);
    }
    __syncthreads();  // every thread is done with buffer k
    if (threadIdx.x == 0 && it + kStageBufs < iters) issue(it + kStageBufs);
  }
  if (it < iters) {
    // a wait ran out: report it, and wait (bounded) for the copies issued
    if (threadIdx.x == 0) {
      if (status) atomicOr(status, kStageTimeout);
      for (size_t j = it; j < iters && j < it + kStageBufs; ++j)
        mbar_wait(f0 + 8 * (uint32_t)(j % kStageBufs), (uint32_t)((j / kStageBufs) & 1));
    }
    __syncthreads();
  }
}

__device__ void staged_dispatch(int path, int lk, const uint4* p, size_t begin, size_t end, uint32_t* table,
                                const uint32_t* lut, const uint4* buf, const unsigned long long* full,
                                uint32_t* status) {
  if (path == PATH_PLAIN) staged_range<PATH_PLAIN, 0>(p, begin, end, table, lut, buf, full, status);
  else if (path == PATH_LUT) staged_range<PATH_LUT, 0>(p, begin, end, table, lut, buf, full, status);
  else {
    switch (lk) {
      case 5: staged_range<PATH_SHIFT, 5>(p, begin, end, table, lut, buf, full, status); break;
      case 4: staged_range<PATH_SHIFT, 4>(p, begin, end, table, lut, buf, full, status); break;
      case 3: staged_range<PATH_SHIFT, 3>(p, begin, end, table, lut, buf, full, status); break;
      case 2: staged_range<PATH_SHIFT, 2>(p, begin, end, table, lut, buf, full, status); break;
      case 1: staged_range<PATH_SHIFT, 1>(p, begin, end, table, lut, buf, full, status); break;
      default: staged_range<PATH_SHIFT, 0>(p, begin, end, table, lut, buf, full, status); break;
    }
  }
}

template <int STAGE>
__global__ void __launch_bounds__(kThreads, 2)
    ablation_kernel(const uint8_t* __restrict__ in, size_t n, const hist_pattern* __restrict__ pat,
                    uint32_t* __restrict__ out, uint32_t* __restrict__ sink) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* table = smem;
  uint32_t* lut = smem + kTableWords;
  __shared__ CtaShared cs;
  __shared__ uint32_t wacc[kWarps];

  if (STAGE >= 2) zero_table(table);
  if (STAGE >= 3 && pat) {
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
  uint32_t acc = 0;
  if (STAGE == 7) {
    __shared__ __align__(8) unsigned long long full[kStageBufs];
    if (threadIdx.x == 0) {
      for (int k = 0; k < kStageBufs; ++k) mbar_init(smem_addr(&full[k]), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    staged_dispatch(cs.path, cs.lk, body, begin, end, table, lut,
                    reinterpret_cast<const uint4*>(smem + kTableWords + kLutWords), full, sink);
  } else {
    ablate_dispatch<STAGE>(cs.path, cs.lk, body, begin, end, table, lut, acc);
  }
  if (STAGE >= 5) {
    flush_table(cs.path, cs.lk, table, cs.pat, lut, cs);
    if (blockIdx.x == 0) {
      count_edges(in, sp, cs);
      __syncthreads();
    }
    if (threadIdx.x < HIST_BINS && cs.res[threadIdx.x]) atomicAdd(out + threadIdx.x, cs.res[threadIdx.x]);
  } else {
    // the block result: 256 words per CTA, built from every thread's register
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) wacc[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < HIST_BINS) sink[(size_t)blockIdx.x * HIST_BINS + threadIdx.x] = wacc[threadIdx.x & 31] ^ threadIdx.x;
  }
}

const void* ablation_fn(uint32_t stage) {
  switch (stage) {
    case 1: return (const void*)ablation_kernel<1>;
    case 2: return (const void*)ablation_kernel<2>;
    case 3: return (const void*)ablation_kernel<3>;
    case 4: return (const void*)ablation_kernel<4>;
    case 5: return (const void*)ablation_kernel<5>;
    case 6: return (const void*)ablation_kernel<6>;
    default: return (const void*)ablation_kernel<7>;
  }
}

}  // namespace

extern "C" {

int hist_ablation_grid(size_t n) {
  const size_t nvec = n / 16 + 1;
  const size_t want = (nvec + 4 * kThreads - 1) / (4 * kThreads);
  const size_t cap = 2 * (size_t)sm_count();
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

int hist_ablation(const uint8_t* d_in, size_t n, const hist_pattern* d_pat, uint32_t stage, uint32_t* d_out,
                  uint32_t* d_sink, hist_cuda_stream s) {
  if ((!d_in && n) || n >= ((size_t)1 << 32) || stage < 1 || stage > 7) return HIST_EINVAL;
  if (stage >= 5 && !d_out) return HIST_EINVAL;
  if (stage < 5 && !d_sink) return HIST_EINVAL;
  static int attr_done[7][kMaxDevices];
  const void* fn = ablation_fn(stage);
  const size_t smem = stage == 7 ? kStageSmem : kSmemBytes;
  int rc = ensure_smem_attr_bytes(fn, attr_done[stage - 1], smem);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  if (stage >= 5) e = cudaMemsetAsync(d_out, 0, HIST_BINS * sizeof(uint32_t), (cudaStream_t)s);
  if (e == cudaSuccess && stage == 7 && d_sink) e = cudaMemsetAsync(d_sink, 0, sizeof(uint32_t), (cudaStream_t)s);
  if (e != cudaSuccess) return cuda_fail(e);
  const int grid = hist_ablation_grid(n);
  void* args[] = {(void*)&d_in, (void*)&n, (void*)&d_pat, (void*)&d_out, (void*)&d_sink};
  e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kThreads), args, smem, (cudaStream_t)s);
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

}  // extern "C"
