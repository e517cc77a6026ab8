// hist_noalloc.cu -- a chunked-stream run that allocates nothing.
//
// hist_stream_create() allocates the stream's device state with cudaMalloc.
// Some callers cannot do that at the point where they need histograms:
// code running while a CUDA graph is being captured, real-time loops in
// which a cudaMalloc would stall on a device-wide synchronisation, and hosts
// whose device memory is owned by another allocator (a framework pool) that
// must see every allocation.  hist_stream_run_noalloc serves them: it runs a
// fresh stream over the chunks it is given -- the same per-chunk switch and
// pattern as the synchronised stream kernel -- and keeps its scratch in the
// file-scope device array below, which exists once per GPU that loads the
// library and lives until the process exits.
//
// Host code may not pass `g_noalloc_scratch` itself to a kernel: on the host
// that name is a stand-in, not a device address.  The device address is
// fetched with cudaGetSymbolAddress once per device (first call on that
// device) and passed to the kernel.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "hist.h"
#include "hist_device.cuh"
#include "hist_internal.h"

using namespace histdev;
using namespace histlib;

namespace {

constexpr int kNaReplicas = 4;
constexpr uint32_t kNaPollLimit = 1u << 22;  // bounded wait: about a second
constexpr uint32_t kNaStatusTimeout = 4;

// Partial sums of the three chunks in flight (chunk j uses buffer j mod 3)
// and their counters: CTAs that published (high 32 bits) and their pixels
// (low 32 bits).  A chunk is complete when every CTA has published and the
// pixels equal its size; the arrivals make sure that a CTA with no pixels is
// also past the steps before its publication.
struct NoAllocScratch {
  uint32_t rep[3][kNaReplicas][HIST_BINS];
  unsigned long long cnt[3][16];
  uint32_t abort;
  uint32_t status;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

struct NaChunk {
  const uint8_t* in;
  uint32_t* out;
  uint32_t n;
  uint32_t pad;
};

struct NaArgs {
  NoAllocScratch* sc;
  unsigned long long* totals;
  uint32_t* status_out;
  uint32_t count;
  uint32_t budget;
  uint32_t theta;
  uint32_t mode;
  NaChunk c[HIST_NOALLOC_MAX_CHUNKS];
};

__device__ __forceinline__ uint32_t na_kernel_for(uint32_t mode, uint32_t flag) {
  return mode == HIST_MODE_AUTO ? flag : (mode == HIST_MODE_PLAIN ? HIST_FLAG_PLAIN : HIST_FLAG_ADAPTIVE);
}

__device__ __forceinline__ unsigned long long na_ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t na_ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

struct NaGeo {
  const uint4* body;
  uint32_t begin, end;
};

__device__ __forceinline__ NaGeo na_geo(const NaChunk& d) {
  const Split sp = split_bytes(d.in, d.n);
  NaGeo g;
  g.body = reinterpret_cast<const uint4*>(d.in + sp.head);
  const uint32_t nvec = (uint32_t)sp.nvec;
  const uint32_t per = (nvec + gridDim.x - 1) / gridDim.x;
  const uint32_t b = per * blockIdx.x;
  g.end = b + per < nvec ? b + per : nvec;
  g.begin = b < g.end ? b : g.end;
  return g;
}

__device__ __forceinline__ void na_prefetch(const NaChunk& d) {
  if (threadIdx.x != 0) return;
  const NaGeo g = na_geo(d);
  const uint8_t* p = reinterpret_cast<const uint8_t*>(g.body + g.begin);
  size_t bytes = (size_t)(g.end - g.begin) * 16;
  while (bytes) {
    const uint32_t c = bytes > (1u << 20) ? (1u << 20) : (uint32_t)bytes;
    prefetch_l2(p, c);
    p += c;
    bytes -= c;
  }
}

// Wait (bounded) until every CTA has published chunk buffer b and it holds n
// pixels, then sum its replicas
// into cs.hist.  All threads call.
__device__ bool na_gather(NoAllocScratch* sc, uint32_t* status_out, uint32_t b, uint32_t n, uint32_t* part,
                          CtaShared& cs) {
  const int t = threadIdx.x;
  if (t == 0) {
    uint32_t state = 0;
    for (uint32_t it = 0;; ++it) {
      if (na_ld_acquire(&sc->cnt[b][0]) == (((unsigned long long)gridDim.x << 32) | n)) {
        state = 1;
        break;
      }
      if (it >= kNaPollLimit) {
        atomicExch(&sc->abort, 1u);
        atomicExch(&sc->status, kNaStatusTimeout);
        if (status_out) atomicExch(status_out, kNaStatusTimeout);
        break;
      }
      if ((it & 63) == 63 && na_ld_relaxed(&sc->abort)) break;
      __nanosleep(32);
    }
    cs.kernel = state;
  }
  __syncthreads();
  if (cs.kernel != 1u) return false;
  __threadfence();
  const int bin = t & 255, q = t >> 8;
  part[t] = q < kNaReplicas ? __ldcg(&sc->rep[b][q][bin]) : 0u;
  __syncthreads();
  if (t < HIST_BINS) {
    uint32_t h = 0;
    for (int r = 0; r < kNaReplicas; ++r) h += part[r * HIST_BINS + t];
    cs.hist[t] = h;
  }
  __syncthreads();
  return true;
}

// Chunk k's histogram (in cs.hist) to its output and the totals, a slice of
// the bins per CTA.
__device__ __forceinline__ void na_fold(const NaArgs& a, uint32_t k, const CtaShared& cs) {
  const uint32_t bin = blockIdx.x + threadIdx.x * gridDim.x;
  if (bin < HIST_BINS) {
    const uint32_t h = cs.hist[bin];
    if (a.c[k].out) a.c[k].out[bin] = h;
    a.totals[bin] += h;
  }
}

__global__ void __launch_bounds__(kThreads, 1) noalloc_stream_kernel(const __grid_constant__ NaArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* table = smem;
  uint32_t* lut = smem + kTableWords;
  __shared__ CtaShared cs;
  __shared__ EpiShared es;
  NoAllocScratch* sc = a.sc;

  // the totals start at zero; a CTA's slice is cleared before it publishes
  // its first chunk, so before anyone adds to it
  {
    const uint32_t bin = blockIdx.x + threadIdx.x * gridDim.x;
    if (bin < HIST_BINS) a.totals[bin] = 0;
  }
  na_prefetch(a.c[0]);
  zero_table(table);
  // first chunk: plain kernel, default pattern
  if (threadIdx.x < HIST_BINS) cs.hist[threadIdx.x] = 0;
  __syncthreads();
  block_epilogue(cs.hist, 0, a.budget, a.theta, cs.pat, es);
  if (threadIdx.x == 0) cs.flag = HIST_FLAG_PLAIN;
  __syncthreads();

  for (uint32_t j = 0; j < a.count; ++j) {
    const uint32_t b = j % 3;
    if (j > 0) {
      if (!na_gather(sc, a.status_out, (j - 1) % 3, a.c[j - 1].n, lut, cs)) return;
      const hist_degeneracy_result r = block_epilogue(cs.hist, a.c[j - 1].n, a.budget, a.theta, cs.pat, es);
      if (threadIdx.x == 0) cs.flag = r.flag;
      __syncthreads();
      na_fold(a, j - 1, cs);
      zero_table(table);
    }
    {
      // chunk j+1's buffer; its last readers gathered chunk j-2 before adding chunk j-1
      uint32_t* nb = &sc->rep[(b + 1) % 3][0][0];
      const uint32_t i = blockIdx.x + threadIdx.x * gridDim.x;
      if (i < kNaReplicas * HIST_BINS) nb[i] = 0;
      if (blockIdx.x == 0 && threadIdx.x == 0) sc->cnt[(b + 1) % 3][0] = 0;
    }
    if (na_kernel_for(a.mode, cs.flag) == HIST_FLAG_ADAPTIVE) {
      classify_pattern(cs.pat, lut, cs);
    } else {
      if (threadIdx.x == 0) {
        cs.path = PATH_PLAIN;
        cs.lk = 0;
      }
      __syncthreads();
    }
    if (j + 1 < a.count) na_prefetch(a.c[j + 1]);
    const NaGeo g = na_geo(a.c[j]);
    count_dispatch(cs.path, cs.lk, g.body, g.begin, g.end, table, lut);
    flush_table(cs.path, cs.lk, table, cs.pat, lut, cs);
    if (blockIdx.x == 0) {
      count_edges(a.c[j].in, split_bytes(a.c[j].in, a.c[j].n), cs);
      __syncthreads();
    }
    if (threadIdx.x < HIST_BINS) {
      if (cs.res[threadIdx.x]) atomicAdd(&sc->rep[b][blockIdx.x % kNaReplicas][threadIdx.x], cs.res[threadIdx.x]);
      __threadfence();  // this thread's sums, zeroing and totals writes before the count
    }
    uint32_t c = 0;
    if (threadIdx.x < 32) {
      for (int i = threadIdx.x; i < HIST_BINS; i += 32) c += cs.res[i];
      c = (uint32_t)warp_sum(c);
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&sc->cnt[b][0], (1ull << 32) | c);
  }
  // the last chunk
  const uint32_t last = a.count - 1;
  if (!na_gather(sc, a.status_out, last % 3, a.c[last].n, lut, cs)) return;
  na_fold(a, last, cs);
}

std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices];
int g_grid[kMaxDevices];

// Once per device, with that device current: the scratch's device address,
// the kernel's shared-memory opt-in and its grid (all CTAs resident).
int noalloc_setup(int dev, void** ptr, int* grid) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (dev < 0 || dev >= kMaxDevices) return HIST_EINVAL;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    e = cudaFuncSetAttribute((const void*)noalloc_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemBytes);
    if (e != cudaSuccess) return cuda_fail(e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, noalloc_stream_kernel, kThreads, kSmemBytes);
    if (e != cudaSuccess) return cuda_fail(e);
    const int sms = sm_count();
    g_grid[dev] = per_sm >= 1 ? sms : 0;
    if (!g_grid[dev]) return HIST_ECUDA;
    g_scratch_ptr[dev] = p;
  }
  *ptr = g_scratch_ptr[dev];
  *grid = g_grid[dev];
  return HIST_OK;
}

}  // namespace

extern "C" int hist_stream_run_noalloc(const uint8_t* const* d_chunks, const size_t* sizes, uint32_t count,
                                       const hist_config* cfg, uint32_t* d_chunk_outs, uint64_t* d_totals,
                                       uint32_t* d_status, hist_cuda_stream s) {
  if (!cfg || !d_totals || count == 0 || count > HIST_NOALLOC_MAX_CHUNKS || !d_chunks || !sizes) return HIST_EINVAL;
  if (cfg->budget < HIST_BUDGET_MIN || cfg->budget > HIST_BUDGET_MAX || cfg->theta_milli > 1000 ||
      cfg->mode > HIST_MODE_ADAPTIVE || cfg->window != 1)
    return HIST_EINVAL;
  for (uint32_t i = 0; i < count; ++i)
    if ((!d_chunks[i] && sizes[i]) || sizes[i] >= ((size_t)1 << 32)) return HIST_EINVAL;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  void* ptr = nullptr;
  int grid = 0;
  int rc = noalloc_setup(dev, &ptr, &grid);
  if (rc) return rc;

  NaArgs a;
  memset(&a, 0, sizeof(a));
  a.sc = static_cast<NoAllocScratch*>(ptr);
  a.totals = reinterpret_cast<unsigned long long*>(d_totals);
  a.status_out = d_status;
  a.count = count;
  a.budget = cfg->budget;
  a.theta = cfg->theta_milli;
  a.mode = cfg->mode;
  for (uint32_t i = 0; i < count; ++i) {
    a.c[i].in = d_chunks[i];
    a.c[i].n = (uint32_t)sizes[i];
    a.c[i].out = d_chunk_outs ? d_chunk_outs + (size_t)i * HIST_BINS : nullptr;
  }
  // the scratch keeps the previous call's contents: start from zero
  e = cudaMemsetAsync(ptr, 0, sizeof(NoAllocScratch), (cudaStream_t)s);
  if (e == cudaSuccess && d_status) e = cudaMemsetAsync(d_status, 0, sizeof(uint32_t), (cudaStream_t)s);
  if (e != cudaSuccess) return cuda_fail(e);
  void* params[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)noalloc_stream_kernel, dim3((unsigned)grid), dim3(kThreads), params,
                                  kSmemBytes, (cudaStream_t)s);
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}
