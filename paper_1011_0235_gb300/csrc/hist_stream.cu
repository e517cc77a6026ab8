// hist_stream.cu -- the chunked stream of Sec. III.B with the kernel switch of
// Sec. III.C, all on the device.
//
// One kernel launch per chunk, chained with programmatic dependent launch:
// chunk i+1's CTAs start while chunk i still runs, zero their tables and pull
// their slice of chunk i+1 into L2, then wait for chunk i to finish.  Each
// CTA then sums chunk i's partial histograms (16 replicas in global memory),
// derives chunk i+1's switch and binning pattern from them (every CTA computes
// the same values), and CTA 0 folds chunk i into the stream state (totals,
// last histogram, chunk output).  So chunk i's epilogue runs at the head of
// chunk i+1, and a finish kernel runs it for the last chunk on flush.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "hist.h"
#include "hist_device.cuh"
#include "hist_internal.h"

using namespace histdev;
using namespace histlib;

namespace {

// Device-resident stream state.
struct StreamDev {
  uint32_t rep[3][kReplicas][HIST_BINS];  // chunk partials, triple-buffered by launch
  unsigned long long totals[HIST_BINS];
  uint32_t last_hist[HIST_BINS];
  hist_pattern pattern;       // pattern for the next chunk
  hist_pattern last_pattern;  // pattern the last completed chunk was given
  unsigned long long chunks;  // completed chunks
  uint32_t flag;              // switch computed from the last completed chunk
  uint32_t last_kernel;       // kernel the last completed chunk ran
  uint32_t status;
  uint32_t pad;
};

struct ChunkArgs {
  StreamDev* st;
  const uint8_t* in;
  size_t n;
  uint32_t* prev_out;  // output of the pending previous chunk (nullable)
  uint32_t cur;        // replica buffer this chunk adds into
  uint32_t prev;       // replica buffer of the pending previous chunk
  uint32_t has_prev;   // the previous chunk's epilogue runs here
  uint32_t budget;
  uint32_t theta;
  uint32_t mode;
};

__device__ __forceinline__ uint32_t kernel_for(uint32_t mode, uint32_t flag) {
  return mode == HIST_MODE_AUTO ? flag : (mode == HIST_MODE_PLAIN ? HIST_FLAG_PLAIN : HIST_FLAG_ADAPTIVE);
}

__device__ __forceinline__ void copy_pattern(hist_pattern* dst, const hist_pattern* src) {
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(hist_pattern) / 4); i += blockDim.x) d[i] = s[i];
}

// Sum the replicas of buffer `buf` into cs.hist (all threads call; `part` is
// 1024 words of free shared memory).
__device__ void gather_partials(const StreamDev* st, uint32_t buf, uint32_t* part, CtaShared& cs) {
  const int b = threadIdx.x & 255, q = threadIdx.x >> 8;
  uint32_t s = 0;
  for (int r = q; r < kReplicas; r += (int)(blockDim.x >> 8)) s += __ldcg(&st->rep[buf][r][b]);
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < HIST_BINS) {
    uint32_t t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 8); ++k) t += part[k * HIST_BINS + threadIdx.x];
    cs.hist[threadIdx.x] = t;
  }
  __syncthreads();
}

// From the previous chunk's histogram in cs.hist: the next switch and pattern
// (into cs.flag / cs.pat).  With `writer`, also fold the previous chunk into
// the stream state.  All threads call.
__device__ void epilogue(StreamDev* st, uint32_t* prev_out, uint32_t budget, uint32_t theta,
                         uint32_t mode, bool writer, CtaShared& cs) {
  const hist_degeneracy_result r =
      degeneracy_block([&](int b) { return (unsigned long long)cs.hist[b]; }, theta, cs);
  binning_pattern_block([&](int b) { return cs.hist[b]; }, budget, cs.pat, cs);
  if (threadIdx.x == 0) cs.flag = r.flag;
  if (writer) {
    const uint32_t old_flag = st->flag;  // every thread reads before thread 0 writes (sync below)
    copy_pattern(&st->last_pattern, &st->pattern);
    __syncthreads();
    copy_pattern(&st->pattern, &cs.pat);
    if (threadIdx.x < HIST_BINS) {
      const uint32_t h = cs.hist[threadIdx.x];
      st->totals[threadIdx.x] += h;
      st->last_hist[threadIdx.x] = h;
      if (prev_out) prev_out[threadIdx.x] = h;
    }
    if (threadIdx.x == 0) {
      st->last_kernel = kernel_for(mode, old_flag);
      st->flag = r.flag;
      st->chunks += 1;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 2) chunk_kernel(ChunkArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* table = smem;
  uint32_t* lut = smem + kTableWords;
  __shared__ CtaShared cs;

  pdl_launch_dependents();
  // Before the previous chunk has finished: nothing read here depends on it.
  zero_table(table);
  const Split sp = split_bytes(a.in, a.n);
  const uint4* body = reinterpret_cast<const uint4*>(a.in + sp.head);
  const size_t per = (sp.nvec + gridDim.x - 1) / gridDim.x;
  const size_t begin = per * blockIdx.x;
  const size_t end = begin + per < sp.nvec ? begin + per : sp.nvec;
  if (threadIdx.x == 0 && end > begin) {
    // bulk L2 prefetch of this CTA's slice, in pieces of at most 1 MiB
    const uint8_t* p = reinterpret_cast<const uint8_t*>(body + begin);
    size_t bytes = (end - begin) * 16;
    while (bytes) {
      const uint32_t c = bytes > (1u << 20) ? (1u << 20) : (uint32_t)bytes;
      prefetch_l2(p, c);
      p += c;
      bytes -= c;
    }
  }
  pdl_wait();

  StreamDev* st = a.st;
  if (a.has_prev) {
    gather_partials(st, a.prev, lut, cs);
    epilogue(st, a.prev_out, a.budget, a.theta, a.mode, blockIdx.x == 0, cs);
  } else {
    copy_pattern(&cs.pat, &st->pattern);
    if (threadIdx.x == 0) cs.flag = st->flag;
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    // the buffer the next chunk adds into; its last reader finished before this launch
    uint32_t* nb = &st->rep[(a.cur + 1) % 3][0][0];
    for (int i = threadIdx.x; i < kReplicas * HIST_BINS; i += kThreads) nb[i] = 0;
  }
  const uint32_t kern = kernel_for(a.mode, cs.flag);
  if (kern == HIST_FLAG_ADAPTIVE) {
    classify_pattern(cs.pat, lut, cs);
  } else {
    if (threadIdx.x == 0) {
      cs.path = PATH_PLAIN;
      cs.lk = 0;
    }
    __syncthreads();
  }
  count_dispatch(cs.path, cs.lk, body, begin, end, table, lut);
  flush_table(cs.path, cs.lk, table, cs.pat, lut, cs);
  if (blockIdx.x == 0) {
    count_edges(a.in, sp, cs);
    __syncthreads();
  }
  if (threadIdx.x < HIST_BINS && cs.res[threadIdx.x])
    atomicAdd(&st->rep[a.cur][blockIdx.x % kReplicas][threadIdx.x], cs.res[threadIdx.x]);
}

// Epilogue of the last pushed chunk (one CTA).
__global__ void __launch_bounds__(kThreads) finish_kernel(StreamDev* st, uint32_t prev, uint32_t* prev_out,
                                                          uint32_t budget, uint32_t theta, uint32_t mode) {
  __shared__ uint32_t part[kThreads];
  __shared__ CtaShared cs;
  gather_partials(st, prev, part, cs);
  epilogue(st, prev_out, budget, theta, mode, true, cs);
}

__global__ void init_kernel(StreamDev* st, uint32_t budget) {
  __shared__ CtaShared cs;
  default_pattern_block(budget, cs.pat, cs);
  copy_pattern(&st->pattern, &cs.pat);
  copy_pattern(&st->last_pattern, &cs.pat);
}

}  // namespace

struct hist_stream {
  hist_config cfg;
  StreamDev* d;
  int sms;
  int grid;
  unsigned long long launches;
  bool pending;
  uint32_t* pending_out;
};

namespace {

int launch_chunk(hist_stream* st, const uint8_t* d_chunk, size_t n, uint32_t* d_out, cudaStream_t s) {
  static int attr_done[kMaxDevices];
  int rc = ensure_smem_attr((const void*)chunk_kernel, attr_done);
  if (rc) return rc;
  ChunkArgs a;
  a.st = st->d;
  a.in = d_chunk;
  a.n = n;
  a.prev_out = st->pending_out;
  a.cur = (uint32_t)(st->launches % 3);
  a.prev = (uint32_t)((st->launches + 2) % 3);
  a.has_prev = st->pending ? 1u : 0u;
  a.budget = st->cfg.budget;
  a.theta = st->cfg.theta_milli;
  a.mode = st->cfg.mode;

  cudaLaunchConfig_t lc;
  memset(&lc, 0, sizeof(lc));
  lc.gridDim = dim3((unsigned)st->grid);
  lc.blockDim = dim3(kThreads);
  lc.dynamicSmemBytes = kSmemBytes;
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&lc, chunk_kernel, a);
  if (e != cudaSuccess) return cuda_fail(e);
  st->launches += 1;
  st->pending = true;
  st->pending_out = d_out;
  return HIST_OK;
}

int do_flush(hist_stream* st, cudaStream_t s) {
  if (!st->pending) return HIST_OK;
  finish_kernel<<<1, kThreads, 0, s>>>(st->d, (uint32_t)((st->launches + 2) % 3), st->pending_out,
                                       st->cfg.budget, st->cfg.theta_milli, st->cfg.mode);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e);
  st->pending = false;
  st->pending_out = nullptr;
  return HIST_OK;
}

bool config_ok(const hist_config* c) {
  return c && c->budget >= HIST_BUDGET_MIN && c->budget <= HIST_BUDGET_MAX && c->theta_milli <= 1000 &&
         c->mode <= HIST_MODE_ADAPTIVE;
}

}  // namespace

extern "C" {

void hist_config_init(hist_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->budget = HIST_BUDGET_MAX;
  c->theta_milli = HIST_THETA_MILLI_DEFAULT;
  c->mode = HIST_MODE_AUTO;
  c->grid = 0;
}

int hist_stream_create(const hist_config* cfg, hist_stream** out) {
  if (!out || !config_ok(cfg)) return HIST_EINVAL;
  *out = nullptr;
  hist_stream* st = (hist_stream*)calloc(1, sizeof(hist_stream));
  if (!st) return HIST_ENOMEM;
  st->cfg = *cfg;
  st->sms = sm_count();
  st->grid = cfg->grid ? (int)cfg->grid : st->sms;
  cudaError_t e = cudaMalloc((void**)&st->d, sizeof(StreamDev));
  if (e != cudaSuccess) {
    free(st);
    return e == cudaErrorMemoryAllocation ? HIST_ENOMEM : cuda_fail(e);
  }
  e = cudaMemset(st->d, 0, sizeof(StreamDev));
  if (e == cudaSuccess) {
    init_kernel<<<1, 256>>>(st->d, cfg->budget);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(st->d);
    free(st);
    return cuda_fail(e);
  }
  *out = st;
  return HIST_OK;
}

int hist_stream_destroy(hist_stream* st) {
  if (!st) return HIST_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  cudaFree(st->d);
  free(st);
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int hist_stream_push(hist_stream* st, const uint8_t* d_chunk, size_t n, uint32_t* d_chunk_out,
                     hist_cuda_stream s) {
  if (!st || (!d_chunk && n) || n >= ((size_t)1 << 32)) return HIST_EINVAL;
  return launch_chunk(st, d_chunk, n, d_chunk_out, (cudaStream_t)s);
}

int hist_stream_push_many(hist_stream* st, uint32_t count, const uint8_t* const* d_chunks, const size_t* sizes,
                          uint32_t* const* d_chunk_outs, hist_cuda_stream s) {
  if (!st || (count && (!d_chunks || !sizes))) return HIST_EINVAL;
  for (uint32_t i = 0; i < count; ++i)
    if ((!d_chunks[i] && sizes[i]) || sizes[i] >= ((size_t)1 << 32)) return HIST_EINVAL;
  for (uint32_t i = 0; i < count; ++i) {
    int rc = launch_chunk(st, d_chunks[i], sizes[i], d_chunk_outs ? d_chunk_outs[i] : nullptr, (cudaStream_t)s);
    if (rc) return rc;
  }
  return HIST_OK;
}

int hist_stream_flush(hist_stream* st, hist_cuda_stream s) {
  if (!st) return HIST_EINVAL;
  return do_flush(st, (cudaStream_t)s);
}

int hist_stream_totals(hist_stream* st, uint64_t* d_totals, hist_cuda_stream s) {
  if (!st || !d_totals) return HIST_EINVAL;
  int rc = do_flush(st, (cudaStream_t)s);
  if (rc) return rc;
  const void* src = reinterpret_cast<const char*>(st->d) + offsetof(StreamDev, totals);
  cudaError_t e = cudaMemcpyAsync(d_totals, src, HIST_BINS * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)s);
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int hist_stream_get_state(hist_stream* st, hist_stream_state* h, hist_cuda_stream s) {
  if (!st || !h) return HIST_EINVAL;
  int rc = do_flush(st, (cudaStream_t)s);
  if (rc) return rc;
  StreamDev* tmp = (StreamDev*)malloc(sizeof(StreamDev));
  if (!tmp) return HIST_ENOMEM;
  cudaError_t e = cudaMemcpyAsync(tmp, st->d, sizeof(StreamDev), cudaMemcpyDeviceToHost, (cudaStream_t)s);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)s);
  if (e != cudaSuccess) {
    free(tmp);
    return cuda_fail(e);
  }
  memset(h, 0, sizeof(*h));
  memcpy(h->totals, tmp->totals, sizeof(h->totals));
  memcpy(h->last_hist, tmp->last_hist, sizeof(h->last_hist));
  h->pattern = tmp->pattern;
  h->last_pattern = tmp->last_pattern;
  h->chunks = tmp->chunks;
  h->flag = tmp->flag;
  h->last_kernel = tmp->last_kernel;
  h->status = tmp->status;
  free(tmp);
  return HIST_OK;
}

int hist_stream_set_state(hist_stream* st, const hist_stream_state* h, hist_cuda_stream s) {
  if (!st || !h) return HIST_EINVAL;
  if (hist_pattern_check(&h->pattern) != HIST_OK || hist_pattern_check(&h->last_pattern) != HIST_OK ||
      h->pattern.budget != st->cfg.budget || h->flag > HIST_FLAG_ADAPTIVE)
    return HIST_EINVAL;
  int rc = do_flush(st, (cudaStream_t)s);
  if (rc) return rc;
  StreamDev* tmp = (StreamDev*)calloc(1, sizeof(StreamDev));
  if (!tmp) return HIST_ENOMEM;
  memcpy(tmp->totals, h->totals, sizeof(tmp->totals));
  memcpy(tmp->last_hist, h->last_hist, sizeof(tmp->last_hist));
  tmp->pattern = h->pattern;
  tmp->last_pattern = h->last_pattern;
  tmp->chunks = h->chunks;
  tmp->flag = h->flag;
  tmp->last_kernel = h->last_kernel;
  tmp->status = 0;
  cudaError_t e = cudaMemcpyAsync(st->d, tmp, sizeof(StreamDev), cudaMemcpyHostToDevice, (cudaStream_t)s);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)s);
  free(tmp);
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

}  // extern "C"
