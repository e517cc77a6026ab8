// hist_batch.cu -- many histograms in one launch (Sec. III.B: small slices or
// packets batched into one call that returns many histograms).
//
// One kernel takes up to kBatchMaxImages images.  Each CTA computes the
// images' size prefix in shared memory, then counts an equal contiguous range
// of the concatenated bytes: the part of each image that falls in its range is
// counted into the CTA's table and added into that image's output at the
// image boundary.  The kernel needs no scratch memory, so a batch is a memset
// of the outputs plus one kernel, and captures into a CUDA graph as such.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "hist.h"
#include "hist_device.cuh"
#include "hist_internal.h"

using namespace histdev;
using namespace histlib;

namespace {

constexpr uint32_t kBatchMaxImages = HIST_BATCH_MAX_IMAGES;
// dynamic shared memory: the table, then the size prefix (u64 per image + 1)
constexpr size_t kBatchSmem = (size_t)kTableWords * 4 + (size_t)(kBatchMaxImages + 1) * 8;

struct BatchImgArgs {
  const uint8_t* const* ptrs;
  const size_t* sizes;
  uint32_t* out;
  uint32_t count;
  uint32_t small_bytes;  // images below this size use small_lk
  uint32_t small_lk;
  uint32_t large_lk;
};

// Exclusive prefix of the image sizes into pre[0..count] (all threads).
__device__ void size_prefix(const size_t* sizes, uint32_t count, unsigned long long* pre) {
  __shared__ unsigned long long wsum[kWarps];
  const int t = threadIdx.x, nt = blockDim.x;
  const uint32_t per = (count + nt - 1) / nt;  // images per thread, consecutive
  const uint32_t b0 = t * per;
  unsigned long long local = 0;
  for (uint32_t i = 0; i < per && b0 + i < count; ++i) local += sizes[b0 + i];
  // inclusive scan of `local` over the block
  unsigned long long x = local;
  const int lane = t & 31, w = t >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  unsigned long long before = 0;
  for (int i = 0; i < w; ++i) before += wsum[i];
  unsigned long long run = before + x - local;  // exclusive start of this thread's images
  for (uint32_t i = 0; i < per && b0 + i < count; ++i) {
    pre[b0 + i] = run;
    run += sizes[b0 + i];
  }
  if (t == nt - 1) pre[count] = before + x;
  __syncthreads();
}

template <int UNROLL, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) batch_images_kernel(BatchImgArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* table = smem;
  unsigned long long* pre = reinterpret_cast<unsigned long long*>(smem + kTableWords);
  __shared__ CtaShared cs;
  __shared__ uint32_t part[kThreads];

  zero_table(table);
  size_prefix(a.sizes, a.count, pre);
  const unsigned long long total = pre[a.count];
  const unsigned long long lo0 = total * blockIdx.x / gridDim.x;
  const unsigned long long hi = total * (blockIdx.x + 1) / gridDim.x;
  if (lo0 >= hi) return;
  // first image whose bytes reach past lo0
  uint32_t lo_i = 0, hi_i = a.count;
  while (lo_i + 1 < hi_i) {
    const uint32_t mid = (lo_i + hi_i) >> 1;
    if (pre[mid] <= lo0) lo_i = mid;
    else hi_i = mid;
  }
  uint32_t i = lo_i;
  unsigned long long lo = lo0;
  while (lo < hi && i < a.count) {
    const unsigned long long img_end = pre[i + 1];
    if (img_end <= lo) {
      ++i;
      continue;
    }
    const unsigned long long seg_end = img_end < hi ? img_end : hi;
    const size_t off = (size_t)(lo - pre[i]);
    const size_t len = (size_t)(seg_end - lo);
    const uint8_t* base = a.ptrs[i] + off;
    const int lk = a.sizes[i] < a.small_bytes ? (int)a.small_lk : (int)a.large_lk;
    const Split sp = split_bytes(base, len);
    count_range_dispatch<UNROLL>(PATH_SHIFT, lk, reinterpret_cast<const uint4*>(base + sp.head), 0, sp.nvec, table,
                                 part, threadIdx.x, blockDim.x);
    flush_table(PATH_SHIFT, lk, table, cs.pat, part, cs);  // the pattern is not read for SHIFT
    count_edges(base, sp, cs);
    __syncthreads();
    if (threadIdx.x < HIST_BINS && cs.res[threadIdx.x])
      atomicAdd(a.out + (size_t)i * HIST_BINS + threadIdx.x, cs.res[threadIdx.x]);
    // clear the slots this layout used
    const int words = HIST_BINS << lk;
    uint4* t4 = reinterpret_cast<uint4*>(table);
    for (int w = threadIdx.x; w < (words >> 2); w += blockDim.x) t4[w] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    lo = seg_end;
    ++i;
  }
}

int launch_batch_images(const hist_batch_tuning& tu, const uint8_t* const* d_ptrs, const size_t* d_sizes,
                        uint32_t count, uint32_t* d_out, cudaStream_t s) {
  // one CTA per SM with 64 registers (2 or 4 loads in flight), or two with 32
  // registers (2 loads in flight)
  static int attr21[kMaxDevices], attr41[kMaxDevices], attr22[kMaxDevices];
  const void* fn;
  int* done;
  if (tu.ctas_per_sm == 2) {
    fn = (const void*)batch_images_kernel<2, 2>;
    done = attr22;
  } else if (tu.unroll == 4) {
    fn = (const void*)batch_images_kernel<4, 1>;
    done = attr41;
  } else {
    fn = (const void*)batch_images_kernel<2, 1>;
    done = attr21;
  }
  int rc = ensure_smem_attr_bytes(fn, done, kBatchSmem);
  if (rc) return rc;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, kBatchSmem);
  if (e != cudaSuccess) return cuda_fail(e);
  if (per_sm < 1) per_sm = 1;
  const int want = (int)(tu.ctas_per_sm ? tu.ctas_per_sm : 1);
  const int grid = sm_count() * (want < per_sm ? want : per_sm);
  for (uint32_t first = 0; first < count; first += kBatchMaxImages) {
    BatchImgArgs a;
    a.ptrs = d_ptrs + first;
    a.sizes = d_sizes + first;
    a.out = d_out + (size_t)first * HIST_BINS;
    a.count = count - first < kBatchMaxImages ? count - first : kBatchMaxImages;
    a.small_bytes = tu.small_bytes;
    a.small_lk = tu.small_log2k;
    a.large_lk = 5;
    void* params[] = {&a};
    e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kThreads), params, kBatchSmem, s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return HIST_OK;
}

bool tuning_ok(const hist_batch_tuning* t) {
  return t && (t->unroll == 2 || t->unroll == 4) && t->ctas_per_sm >= 1 && t->ctas_per_sm <= 2 &&
         !(t->ctas_per_sm == 2 && t->unroll == 4) && t->small_log2k <= 5;
}

}  // namespace

extern "C" {

void hist_batch_tuning_init(hist_batch_tuning* t) {
  if (!t) return;
  memset(t, 0, sizeof(*t));
  // the setting the autotuner picks on GB300 for every batch measured
  t->ctas_per_sm = 2;
  t->unroll = 2;
  t->small_bytes = 0;
  t->small_log2k = 5;
}

int hist_batch(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t* d_out,
               const hist_batch_tuning* tuning, hist_cuda_stream s) {
  hist_batch_tuning tu;
  if (tuning) tu = *tuning;
  else hist_batch_tuning_init(&tu);
  if (!tuning_ok(&tu) || (count && (!d_ptrs || !d_sizes || !d_out))) return HIST_EINVAL;
  if (count == 0) return HIST_OK;
  cudaError_t e = cudaMemsetAsync(d_out, 0, (size_t)count * HIST_BINS * sizeof(uint32_t), (cudaStream_t)s);
  if (e != cudaSuccess) return cuda_fail(e);
  return launch_batch_images(tu, d_ptrs, d_sizes, count, d_out, (cudaStream_t)s);
}

int hist_batch_capture(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t* d_out,
                       const hist_batch_tuning* tuning, hist_batch_graph** out) {
  if (!out) return HIST_EINVAL;
  *out = nullptr;
  hist_batch_tuning tu;
  if (tuning) tu = *tuning;
  else hist_batch_tuning_init(&tu);
  if (!tuning_ok(&tu) || count == 0 || !d_ptrs || !d_sizes || !d_out) return HIST_EINVAL;
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e);
  // attributes and occupancy are set up outside the capture
  int rc = launch_batch_images(tu, d_ptrs, d_sizes, 0, d_out, cs);
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  if (rc == HIST_OK) {
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rc = hist_batch(d_ptrs, d_sizes, count, d_out, &tu, (hist_cuda_stream)cs);
      cudaError_t e2 = cudaStreamEndCapture(cs, &g);
      if (rc == HIST_OK && e2 != cudaSuccess) rc = cuda_fail(e2);
    } else {
      rc = cuda_fail(e);
    }
  }
  if (rc == HIST_OK) {
    e = cudaGraphInstantiate(&ge, g, 0);
    if (e != cudaSuccess) rc = cuda_fail(e);
  }
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (rc) return rc;
  *out = reinterpret_cast<hist_batch_graph*>(ge);
  return HIST_OK;
}

int hist_batch_graph_launch(hist_batch_graph* g, hist_cuda_stream s) {
  if (!g) return HIST_EINVAL;
  cudaError_t e = cudaGraphLaunch(reinterpret_cast<cudaGraphExec_t>(g), (cudaStream_t)s);
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int hist_batch_graph_destroy(hist_batch_graph* g) {
  if (!g) return HIST_EINVAL;
  cudaError_t e = cudaGraphExecDestroy(reinterpret_cast<cudaGraphExec_t>(g));
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int hist_batch_autotune(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t* d_out,
                        uint32_t repeats, hist_batch_tuning* best, float* best_ms) {
  if (!best || count == 0 || !d_ptrs || !d_sizes || !d_out) return HIST_EINVAL;
  if (repeats == 0) repeats = 3;
  cudaStream_t s;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // candidates: CTAs per SM, loads in flight, and the sub-bins of small images
  std::vector<hist_batch_tuning> cands;
  const uint32_t smalls[][2] = {{0, 5}, {1u << 16, 2}, {1u << 16, 3}, {1u << 18, 3}, {1u << 20, 4}};
  for (uint32_t cps = 1; cps <= 2; ++cps)
    for (uint32_t un : {2u, 4u})
      for (const auto& sm : smalls) {
        if (cps == 2 && un == 4) continue;
        hist_batch_tuning t;
        hist_batch_tuning_init(&t);
        t.ctas_per_sm = cps;
        t.unroll = un;
        t.small_bytes = sm[0];
        t.small_log2k = sm[1];
        cands.push_back(t);
      }
  float bms = 1e30f;
  int rc = HIST_OK;
  for (const auto& t : cands) {
    rc = hist_batch(d_ptrs, d_sizes, count, d_out, &t, (hist_cuda_stream)s);  // warm-up
    if (rc) break;
    float tot = 0;
    for (uint32_t r = 0; r < repeats && rc == HIST_OK; ++r) {
      cudaEventRecord(e0, s);
      rc = hist_batch(d_ptrs, d_sizes, count, d_out, &t, (hist_cuda_stream)s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      tot += ms;
    }
    if (rc) break;
    const float avg = tot / repeats;
    if (avg < bms) {
      bms = avg;
      *best = t;
    }
  }
  e = cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e);
  if (best_ms) *best_ms = bms;
  return HIST_OK;
}

}  // extern "C"
