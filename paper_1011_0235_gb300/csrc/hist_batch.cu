// hist_batch.cu -- many histograms in one launch (Sec. III.B: small slices or
// packets batched into one call that returns many histograms).
//
// One kernel takes up to kBatchMaxImages images.  Each CTA computes the
// images' size prefix in shared memory, then counts a contiguous range of the
// concatenated bytes, an equal share of the batch's cost (the bytes plus a
// fixed cost per image): the part of each image that falls in its range is
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

constexpr uint32_t kPerWarp = HIST_LAYOUT_PER_WARP;

// The layout of an image: per regime (index 0 for every image when the
// launch has no regimes) a layout, and a second one below a size.
struct RegimeLayouts {
  uint32_t layout[HIST_REGIMES];
  uint32_t small_bytes[HIST_REGIMES];
  uint32_t small_layout[HIST_REGIMES];
};

struct BatchImgArgs {
  const uint8_t* const* ptrs;
  const size_t* sizes;
  uint32_t* out;
  const uint8_t* regime;  // per image, or null: every image takes entry 0
  uint32_t count;
  RegimeLayouts lay;
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

// The CTAs split the batch by cost: an image costs kImageCost before its
// bytes (its table reduction and output adds) plus one per byte, so a CTA
// whose range holds many small images takes fewer bytes.  The 4096-image
// batch (9.83 GB, one graph launch): 6.51 TB/s with no fixed cost, 6.63 at
// 32 KiB, 6.64 - 6.69 at 64 KiB, 6.65 at 128 KiB, 6.49 at 256 KiB.
constexpr unsigned long long kImageCost = 64ull << 10;

// The cut at cost position x, as a position in the concatenated bytes: the
// start of the image whose fixed cost holds x, else x's byte moved to a 32
// KiB boundary of its image's memory (split_point; not past the image's
// end).  Both CTAs of the cut compute it from the same x.
__device__ unsigned long long batch_cut(const BatchImgArgs& a, const unsigned long long* pre, unsigned long long x) {
  const unsigned long long W = pre[a.count] + (unsigned long long)a.count * kImageCost;
  if (x >= W) return pre[a.count];
  uint32_t i = 0, hi = a.count;  // the last image whose cost starts at or before x
  while (i + 1 < hi) {
    const uint32_t mid = (i + hi) >> 1;
    if (pre[mid] + (unsigned long long)mid * kImageCost <= x) i = mid;
    else hi = mid;
  }
  const unsigned long long c0 = pre[i] + (unsigned long long)i * kImageCost + kImageCost;
  const unsigned long long n = pre[i + 1] - pre[i];
  if (x <= c0) return pre[i];
  const unsigned long long c = split_point(a.ptrs[i], x - c0);
  return pre[i] + (c < n ? c : n);
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
  const unsigned long long W = pre[a.count] + (unsigned long long)a.count * kImageCost;
  const unsigned long long lo0 = batch_cut(a, pre, W * blockIdx.x / gridDim.x);
  const unsigned long long hi = batch_cut(a, pre, W * (blockIdx.x + 1) / gridDim.x);
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
    const uint32_t r = a.regime ? a.regime[i] : 0u;
    // selects rather than an index, so the parameters stay out of local memory
    const uint32_t big = r == 0 ? a.lay.layout[0] : (r == 1 ? a.lay.layout[1] : a.lay.layout[2]);
    const uint32_t cut = r == 0 ? a.lay.small_bytes[0] : (r == 1 ? a.lay.small_bytes[1] : a.lay.small_bytes[2]);
    const uint32_t sml = r == 0 ? a.lay.small_layout[0] : (r == 1 ? a.lay.small_layout[1] : a.lay.small_layout[2]);
    const uint32_t lay = a.sizes[i] < cut ? sml : big;
    const int path = lay == kPerWarp ? PATH_PLAIN : PATH_SHIFT;
    const int lk = lay == kPerWarp ? 0 : (int)(lay > 5u ? 5u : lay);
    const Split sp = split_bytes(base, len);
    count_range_dispatch<UNROLL>(path, lk, reinterpret_cast<const uint4*>(base + sp.head), 0, sp.nvec, table,
                                 part, threadIdx.x, blockDim.x);
    // the pattern is not read for SHIFT or PLAIN
    const bool cleared = flush_table(path, lk, table, cs.pat, part, cs, true);
    count_edges(base, sp, cs);
    __syncthreads();
    if (threadIdx.x < HIST_BINS && cs.res[threadIdx.x])
      atomicAdd(a.out + (size_t)i * HIST_BINS + threadIdx.x, cs.res[threadIdx.x]);
    if (!cleared) {
      // clear the slots this layout used (the per-warp tables fill the table)
      const int words = path == PATH_PLAIN ? kTableWords : (HIST_BINS << lk);
      uint4* t4 = reinterpret_cast<uint4*>(table);
      for (int w = threadIdx.x; w < (words >> 2); w += blockDim.x) t4[w] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    lo = seg_end;
    ++i;
  }
}

// The regime of image blockIdx.x (rule in hist.h): 256 threads; thread t
// takes run t of the sample (16 consecutive pixels from floor(t n / 256)),
// or pixels t, t + 256, ... of an image of at most 4096 pixels, loading all
// 16 bytes before counting them in shared memory; then the largest bin and
// the sum of squares (below 2^25: m <= 4096).
__global__ void __launch_bounds__(HIST_BINS) regime_kernel(const uint8_t* const* ptrs, const size_t* sizes,
                                                           uint32_t theta, uint8_t* regime) {
  __shared__ uint32_t h[HIST_BINS];
  __shared__ uint32_t wmax[HIST_BINS / 32], wsq[HIST_BINS / 32];
  const int t = threadIdx.x;
  const uint32_t i = blockIdx.x;
  const unsigned long long n = sizes[i];
  const uint8_t* x = ptrs[i];
  h[t] = 0;
  uint32_t v[16];
  const bool runs = n > HIST_REGIME_SAMPLE;
  const unsigned long long start = runs ? ((unsigned long long)t * n) >> 8 : (unsigned long long)t;
  const unsigned long long step = runs ? 1ull : (unsigned long long)HIST_BINS;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const unsigned long long at = start + (unsigned long long)u * step;
    v[u] = at < n ? (uint32_t)__ldg(x + at) : 0xffffffffu;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 16; ++u)
    if (v[u] != 0xffffffffu) atomicAdd(&h[v[u]], 1u);
  __syncthreads();
  const uint32_t c = h[t];
  const uint32_t mx = __reduce_max_sync(0xffffffffu, c);
  const uint32_t sq = __reduce_add_sync(0xffffffffu, c * c);
  if ((t & 31) == 0) {
    wmax[t >> 5] = mx;
    wsq[t >> 5] = sq;
  }
  __syncthreads();
  if (t == 0) {
    const unsigned long long m = n < HIST_REGIME_SAMPLE ? n : HIST_REGIME_SAMPLE;
    uint32_t M = 0, S = 0;
    for (int w = 0; w < HIST_BINS / 32; ++w) {
      M = wmax[w] > M ? wmax[w] : M;
      S += wsq[w];
    }
    uint8_t r = (uint8_t)HIST_REGIME_WIDE;
    if (m == 0) r = (uint8_t)HIST_REGIME_WIDE;
    else if ((unsigned long long)M * 1000ull >= (unsigned long long)theta * m) r = (uint8_t)HIST_REGIME_DEGENERATE;
    else if (64ull * S >= m * m) r = (uint8_t)HIST_REGIME_PEAKED;
    regime[i] = r;
  }
}

int launch_regimes(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t theta,
                   uint8_t* d_regime, cudaStream_t s) {
  for (uint32_t first = 0; first < count; first += 65535u) {
    const uint32_t c = count - first < 65535u ? count - first : 65535u;
    regime_kernel<<<c, HIST_BINS, 0, s>>>(d_ptrs + first, d_sizes + first, theta, d_regime + first);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return HIST_OK;
}

RegimeLayouts layouts_of(const hist_batch_tuning& tu) {
  RegimeLayouts l;
  for (uint32_t r = 0; r < HIST_REGIMES; ++r) {
    l.layout[r] = 5;
    l.small_bytes[r] = tu.small_bytes;
    l.small_layout[r] = tu.small_log2k;
  }
  return l;
}

RegimeLayouts layouts_of(const hist_batch_table& tb) {
  RegimeLayouts l;
  for (uint32_t r = 0; r < HIST_REGIMES; ++r) {
    l.layout[r] = tb.regime[r].layout;
    l.small_bytes[r] = tb.regime[r].small_bytes;
    l.small_layout[r] = tb.regime[r].small_layout;
  }
  return l;
}

int launch_batch_images(const hist_batch_tuning& tu, const RegimeLayouts& lay, const uint8_t* regime,
                        const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t* d_out,
                        cudaStream_t s) {
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
    a.regime = regime ? regime + first : nullptr;
    a.count = count - first < kBatchMaxImages ? count - first : kBatchMaxImages;
    a.lay = lay;
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

bool layout_ok(uint32_t l) { return l <= 5 || l == kPerWarp; }

bool table_ok(const hist_batch_table* t) {
  if (!t || !(t->unroll == 2 || t->unroll == 4) || t->ctas_per_sm < 1 || t->ctas_per_sm > 2 ||
      (t->ctas_per_sm == 2 && t->unroll == 4) || t->theta_milli > 1000)
    return false;
  for (uint32_t r = 0; r < HIST_REGIMES; ++r)
    if (!layout_ok(t->regime[r].layout) || !layout_ok(t->regime[r].small_layout)) return false;
  return true;
}

hist_batch_tuning shape_of(const hist_batch_table& t) {
  hist_batch_tuning tu;
  memset(&tu, 0, sizeof(tu));
  tu.ctas_per_sm = t.ctas_per_sm;
  tu.unroll = t.unroll;
  return tu;
}

// The regimes call: memset, classification, counting.
int batch_regimes(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t* d_out,
                  uint8_t* d_regime, const hist_batch_table& tb, cudaStream_t s) {
  if (count == 0) return HIST_OK;
  cudaError_t e = cudaMemsetAsync(d_out, 0, (size_t)count * HIST_BINS * sizeof(uint32_t), s);
  if (e != cudaSuccess) return cuda_fail(e);
  int rc = launch_regimes(d_ptrs, d_sizes, count, tb.theta_milli, d_regime, s);
  if (rc) return rc;
  return launch_batch_images(shape_of(tb), layouts_of(tb), d_regime, d_ptrs, d_sizes, count, d_out, s);
}

// Capture `enqueue` (which enqueues on the stream it is given) into an
// instantiated graph; the kernels' attributes are set up by `prepare`
// outside the capture.
template <class Prep, class Enq>
int capture_graph(Prep prepare, Enq enqueue, hist_batch_graph** out) {
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e);
  int rc = prepare(cs);
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  if (rc == HIST_OK) {
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rc = enqueue(cs);
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
  return launch_batch_images(tu, layouts_of(tu), nullptr, d_ptrs, d_sizes, count, d_out, (cudaStream_t)s);
}

int hist_batch_capture(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t* d_out,
                       const hist_batch_tuning* tuning, hist_batch_graph** out) {
  if (!out) return HIST_EINVAL;
  *out = nullptr;
  hist_batch_tuning tu;
  if (tuning) tu = *tuning;
  else hist_batch_tuning_init(&tu);
  if (!tuning_ok(&tu) || count == 0 || !d_ptrs || !d_sizes || !d_out) return HIST_EINVAL;
  // attributes and occupancy are set up outside the capture (a launch of no images)
  return capture_graph(
      [&](cudaStream_t cs) { return launch_batch_images(tu, layouts_of(tu), nullptr, d_ptrs, d_sizes, 0, d_out, cs); },
      [&](cudaStream_t cs) { return hist_batch(d_ptrs, d_sizes, count, d_out, &tu, (hist_cuda_stream)cs); }, out);
}

void hist_batch_table_init(hist_batch_table* t) {
  if (!t) return;
  memset(t, 0, sizeof(*t));
  t->ctas_per_sm = 2;
  t->unroll = 2;
  t->theta_milli = HIST_THETA_MILLI_DEFAULT;
  for (uint32_t r = 0; r < HIST_REGIMES; ++r) {
    t->regime[r].layout = 5;
    t->regime[r].small_bytes = 0;
    t->regime[r].small_layout = 5;
  }
}

int hist_batch_classify(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t theta_milli,
                        uint8_t* d_regime, hist_cuda_stream s) {
  if (theta_milli > 1000 || (count && (!d_ptrs || !d_sizes || !d_regime))) return HIST_EINVAL;
  return launch_regimes(d_ptrs, d_sizes, count, theta_milli, d_regime, (cudaStream_t)s);
}

int hist_batch_regimes(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t* d_out,
                       uint8_t* d_regime, const hist_batch_table* table, hist_cuda_stream s) {
  hist_batch_table tb;
  if (table) tb = *table;
  else hist_batch_table_init(&tb);
  if (!table_ok(&tb) || (count && (!d_ptrs || !d_sizes || !d_out || !d_regime))) return HIST_EINVAL;
  return batch_regimes(d_ptrs, d_sizes, count, d_out, d_regime, tb, (cudaStream_t)s);
}

int hist_batch_regimes_capture(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count,
                               uint32_t* d_out, uint8_t* d_regime, const hist_batch_table* table,
                               hist_batch_graph** out) {
  if (!out) return HIST_EINVAL;
  *out = nullptr;
  hist_batch_table tb;
  if (table) tb = *table;
  else hist_batch_table_init(&tb);
  if (!table_ok(&tb) || count == 0 || !d_ptrs || !d_sizes || !d_out || !d_regime) return HIST_EINVAL;
  return capture_graph(
      [&](cudaStream_t cs) {
        return launch_batch_images(shape_of(tb), layouts_of(tb), d_regime, d_ptrs, d_sizes, 0, d_out, cs);
      },
      [&](cudaStream_t cs) { return batch_regimes(d_ptrs, d_sizes, count, d_out, d_regime, tb, cs); }, out);
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

namespace {

// Mean time of `enqueue` on `s` over `repeats` runs after one warm-up run
// (CUDA events), or a negative HIST_E* code.
template <class Enq>
float time_runs(Enq enqueue, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, uint32_t repeats, int* rc) {
  *rc = enqueue();
  if (*rc) return 0.0f;
  float tot = 0.0f;
  for (uint32_t r = 0; r < repeats; ++r) {
    cudaEventRecord(e0, s);
    *rc = enqueue();
    cudaEventRecord(e1, s);
    if (*rc) return 0.0f;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      *rc = cuda_fail(e);
      return 0.0f;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    tot += ms;
  }
  return tot / (float)repeats;
}

}  // namespace

extern "C" int hist_batch_autotune_regimes(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count,
                                           uint32_t* d_out, uint8_t* d_regime, uint32_t repeats,
                                           hist_batch_table* best, hist_regime_report* report) {
  if (!best || count == 0 || !d_ptrs || !d_sizes || !d_out || !d_regime) return HIST_EINVAL;
  if (repeats == 0) repeats = 3;
  hist_batch_table tb;
  hist_batch_table_init(&tb);
  tb.theta_milli = best->theta_milli <= 1000 && best->theta_milli ? best->theta_milli : HIST_THETA_MILLI_DEFAULT;
  hist_regime_report rep;
  memset(&rep, 0, sizeof(rep));
  cudaStream_t s;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // the images' regimes, pointers and sizes on the host
  std::vector<uint8_t> reg(count);
  std::vector<const uint8_t*> ptrs(count);
  std::vector<size_t> sizes(count);
  int rc = launch_regimes(d_ptrs, d_sizes, count, tb.theta_milli, d_regime, s);
  if (rc == HIST_OK) {
    e = cudaMemcpyAsync(reg.data(), d_regime, count, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ptrs.data(), d_ptrs, count * sizeof(void*), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sizes.data(), d_sizes, count * sizeof(size_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e);
  }
  // candidate settings: a layout, and none or one smaller layout for small images
  std::vector<hist_regime_setting> cands;
  const uint32_t layouts[] = {kPerWarp, 0, 1, 2, 3, 4, 5};
  const uint32_t smalls[][2] = {{0, 5}, {64u << 10, 0}, {64u << 10, kPerWarp}, {1u << 20, 2}};
  for (uint32_t l : layouts)
    for (const auto& sm : smalls) {
      if (sm[0] && sm[1] == l) continue;
      hist_regime_setting c;
      memset(&c, 0, sizeof(c));
      c.layout = l;
      c.small_bytes = sm[0];
      c.small_layout = sm[0] ? sm[1] : l;
      cands.push_back(c);
    }
  rep.candidates = (uint32_t)cands.size();
  // per regime: its images alone, every candidate (each image counted with
  // the setting in entry 0: no regime array)
  const hist_batch_tuning shape = shape_of(tb);
  for (uint32_t r = 0; r < HIST_REGIMES && rc == HIST_OK; ++r) {
    std::vector<const uint8_t*> rp;
    std::vector<size_t> rz;
    for (uint32_t i = 0; i < count; ++i)
      if (reg[i] == r) {
        rp.push_back(ptrs[i]);
        rz.push_back(sizes[i]);
        rep.bytes[r] += sizes[i];
      }
    rep.images[r] = (uint32_t)rp.size();
    if (rp.empty()) continue;
    const uint32_t rc_n = (uint32_t)rp.size();
    const uint8_t** dp = nullptr;
    size_t* dz = nullptr;
    uint32_t* dout = nullptr;
    e = cudaMalloc((void**)&dp, rc_n * sizeof(void*));
    if (e == cudaSuccess) e = cudaMalloc((void**)&dz, rc_n * sizeof(size_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&dout, (size_t)rc_n * HIST_BINS * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpy(dp, rp.data(), rc_n * sizeof(void*), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dz, rz.data(), rc_n * sizeof(size_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = e == cudaErrorMemoryAllocation ? HIST_ENOMEM : cuda_fail(e);
    float bms = 1e30f;
    for (size_t k = 0; k < cands.size() && rc == HIST_OK; ++k) {
      RegimeLayouts lay;
      for (uint32_t q = 0; q < HIST_REGIMES; ++q) {
        lay.layout[q] = cands[k].layout;
        lay.small_bytes[q] = cands[k].small_bytes;
        lay.small_layout[q] = cands[k].small_layout;
      }
      const float ms = time_runs(
          [&]() {
            cudaError_t me = cudaMemsetAsync(dout, 0, (size_t)rc_n * HIST_BINS * sizeof(uint32_t), s);
            if (me != cudaSuccess) return cuda_fail(me);
            return launch_batch_images(shape, lay, nullptr, dp, dz, rc_n, dout, s);
          },
          s, e0, e1, repeats, &rc);
      if (rc) break;
      if (cands[k].layout == 5 && cands[k].small_bytes == 0) rep.ms_default[r] = ms;
      if (ms < bms) {
        bms = ms;
        tb.regime[r] = cands[k];
      }
    }
    rep.ms[r] = bms < 1e30f ? bms : 0.0f;
    cudaFree(dp);
    cudaFree(dz);
    cudaFree(dout);
  }
  // the launch shape of the whole batch with the chosen settings
  const uint32_t shapes[][2] = {{2, 2}, {1, 2}, {1, 4}};
  float bms = 1e30f;
  hist_batch_table chosen = tb;
  for (const auto& sh : shapes) {
    if (rc) break;
    hist_batch_table t = tb;
    t.ctas_per_sm = sh[0];
    t.unroll = sh[1];
    const float ms = time_runs([&]() { return batch_regimes(d_ptrs, d_sizes, count, d_out, d_regime, t, s); }, s, e0,
                               e1, repeats, &rc);
    if (rc) break;
    if (ms < bms) {
      bms = ms;
      chosen = t;
    }
  }
  if (rc == HIST_OK) {
    rep.batch_ms = bms;
    hist_batch_table def;
    hist_batch_table_init(&def);
    def.theta_milli = tb.theta_milli;
    rep.batch_default_ms =
        time_runs([&]() { return batch_regimes(d_ptrs, d_sizes, count, d_out, d_regime, def, s); }, s, e0, e1,
                  repeats, &rc);
  }
  // leave d_out holding the batch under the chosen table
  if (rc == HIST_OK) rc = batch_regimes(d_ptrs, d_sizes, count, d_out, d_regime, chosen, s);
  e = cudaStreamSynchronize(s);
  if (rc == HIST_OK && e != cudaSuccess) rc = cuda_fail(e);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (rc) return rc;
  *best = chosen;
  if (report) *report = rep;
  return HIST_OK;
}
