// hist_server.cu -- a serving loop for histogram requests on many streams.
//
// Each request is the next chunk of one of `streams` independent streams; a
// stream's adaptive state (the switch flag, the binning pattern and the
// layout derived from it, the totals and the last histogram) stays on the
// device, so a request runs the kernel and pattern chosen from its stream's
// previous request (Sec. III.B / III.C), exactly as hist_stream_push would.
//
// Continuous batching on the host: submitted requests wait in a FIFO queue;
// whenever a batch slot is free, the queued requests that fit the HBM byte
// budget and whose stream has no request on the GPU form a batch, launched
// on the slot's own CUDA stream, so batches overlap on the device.  A batch
// is one kernel with no device-side waits: the CTAs split the requests by a
// cost model (bytes plus a fixed cost per request), count each piece with
// its stream's layout and add it into the request's accumulator; the CTA
// that completes a request (a done-bytes counter) computes its degeneracy
// and next pattern and updates the stream's state.  A request counted whole
// by one CTA skips the accumulator.  Once a request's output is written, its
// epilogue writes the batch's sequence number into the request's completion
// word in pinned host memory, so the host sees each request complete without
// waiting for the rest of its batch; it then updates the stream's state and
// writes the number into the request's state word, which releases the stream
// to admission: the stream's next request may run in a batch that fills the
// SMs while this one drains.  The slot itself (its scratch and its bytes of
// the budget) is released when the slot's event shows the whole batch done.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <list>
#include <new>
#include <vector>

#include "hist.h"
#include "hist_device.cuh"
#include "hist_internal.h"

using namespace histdev;
using namespace histlib;

namespace {

constexpr uint32_t kSrvMaxBatch = HIST_SERVER_MAX_BATCH;  // <= kThreads (one prefix lane each)
constexpr uint32_t kSrvMaxSlots = HIST_SERVER_MAX_INFLIGHT;
// cost of a request beyond its bytes, in bytes: about what one CTA counts
// while it reduces its table, publishes its piece and runs a request's
// epilogue and completion (a burst of 4000 requests of 4 KiB..64 MiB on
// GB300: 3.64 TB/s at 64 KiB, 4.1 at 256 KiB, no better beyond)
constexpr unsigned long long kReqCost = 256ull << 10;
// cost units per CTA of a batch (the grid is at most every resident CTA)
constexpr unsigned long long kCtaCost = 64ull << 10;
// dynamic shared memory: table, slot table, request cost prefix (u64 per
// request + 1), each request's stream ctl word
constexpr size_t kSrvSmem = (size_t)(kTableWords + kLutWords) * 4 + (size_t)(kSrvMaxBatch + 1) * 8 +
                            (size_t)kSrvMaxBatch * 4;
// request-table capacities of the two kernel variants (the table travels in
// the launch's parameters: 24 bytes per request)
constexpr uint32_t kSmallCap = 32;

static_assert(kSrvMaxBatch <= (uint32_t)kThreads, "one prefix lane per request");

// Per-stream state on the device.  The two patterns sit in two slots: the
// next request's in pat[cur], the last request's in the other; a request's
// epilogue writes the new pattern over the older one and flips cur, so no
// pattern is ever copied.  ctl packs what a batch reads about a stream
// before counting: the switch (bit 0), whether pat[cur] is a uniform shift
// (bit 1), cur (bit 2) and the shift's log2 k (bits 8..15).
struct SrvStream {
  unsigned long long totals[HIST_BINS];
  uint32_t last_hist[HIST_BINS];
  hist_pattern pat[2];
  unsigned long long chunks;
  uint32_t ctl;
  uint32_t last_kernel;  // kernel the last request ran
};

__host__ __device__ __forceinline__ uint32_t srv_ctl(uint32_t flag, uint32_t shift, uint32_t cur, uint32_t lk) {
  return (flag & 1u) | ((shift & 1u) << 1) | ((cur & 1u) << 2) | ((lk & 0xffu) << 8);
}

struct SrvReq {
  const uint8_t* in;
  uint32_t* out;
  uint32_t n;
  uint32_t stream;
};

// Per batch slot, on the device.  acc and done return to zero when a
// request's epilogue has read them, so a slot needs clearing only once.
struct SrvSlot {
  uint32_t acc[kSrvMaxBatch][HIST_BINS];  // partial sums of split requests
  unsigned long long done[kSrvMaxBatch];  // bytes of each split request counted
};

struct SrvCommon {
  SrvStream* streams;
  SrvSlot* slot;
  // the slot's words in pinned, mapped host memory: request r's completion
  // word in done[r], its state word in done[kSrvMaxBatch + r]
  uint32_t* done;
  uint32_t seq;  // the batch's sequence number, written into both words of request r
  uint32_t count;
  uint32_t budget;
  uint32_t theta;
  uint32_t mode;
  uint32_t pad;
};

template <uint32_t CAP>
struct SrvArgs {
  SrvCommon c;
  SrvReq req[CAP];
};

__device__ __forceinline__ uint32_t srv_kernel_for(uint32_t mode, uint32_t flag) {
  return mode == HIST_MODE_AUTO ? flag : (mode == HIST_MODE_PLAIN ? HIST_FLAG_PLAIN : HIST_FLAG_ADAPTIVE);
}

// Whether P gives every bin the same k = 2^lk at off = b k (all threads call).
__device__ bool srv_is_shift(const hist_pattern& P) {
  const bool act = threadIdx.x < HIST_BINS;
  const uint32_t lk0 = P.log2k[0];
  const int ok = !act || (P.log2k[threadIdx.x] == lk0 && lk0 <= 5 &&
                          (uint32_t)P.off[threadIdx.x] == ((uint32_t)threadIdx.x << lk0));
  return __syncthreads_and(ok) != 0;
}

__device__ __forceinline__ void srv_copy_words(void* dst, const void* src, int words) {
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < words; i += blockDim.x) d[i] = s[i];
}

// The same from a stream's state in global memory, read at L2: the state is
// written by another batch's epilogue, possibly while an older batch that
// read it on this SM is still resident, so no line of it is taken from L1.
__device__ __forceinline__ void srv_copy_state_words(void* dst, const void* src, int words) {
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < words; i += blockDim.x) d[i] = __ldcg(s + i);
}

// pre[r] = sum over requests before r of (n + kReqCost); pre[count] = total;
// ctl[r] = request r's stream ctl word (its load overlaps the scan).  The
// request table sits in the kernel's parameters, read through the constant
// cache, which serves a warp's distinct addresses one after another: each
// warp first copies its requests' sizes and streams into pre[] and ctl[]
// with a warp-uniform index, and thread r then reads entry r from there.
__device__ void srv_cost_prefix(const SrvReq* req, uint32_t count, const SrvStream* streams,
                                unsigned long long* pre, uint32_t* ctl) {
  __shared__ unsigned long long wsum[kWarps];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (uint32_t r = (uint32_t)w; r < count; r += kWarps) {
    const uint32_t n = req[r].n, sid = req[r].stream;
    if (lane == 0) {
      pre[r] = n;
      ctl[r] = sid;
    }
  }
  __syncthreads();
  // thread t reads entry t and later overwrites only entry t (and pre[count])
  const uint32_t cw = t < (int)count ? __ldcg(&streams[ctl[t]].ctl) : 0u;
  const unsigned long long c = t < (int)count ? pre[t] + kReqCost : 0ull;
  unsigned long long x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  unsigned long long before = 0;
  for (int i = 0; i < w; ++i) before += wsum[i];
  if (t < (int)count) {
    pre[t] = before + x - c;
    ctl[t] = cw;
  }
  if (t == (int)count - 1) pre[count] = before + x;
  __syncthreads();
}

// Request r (q) is complete and cs.hist holds its histogram: write its
// output and publish the request's completion word, then advance its
// stream's state.  The state can follow the completion: the stream's next
// request is admitted only once the state word below has been seen.  All
// threads of the CTA call.
__device__ __noinline__ void srv_epilogue(const SrvCommon& a, uint32_t r, const SrvReq& q, uint32_t ctl,
                                          CtaShared& cs, EpiShared& es) {
  SrvStream* st = a.streams + q.stream;
  const uint32_t kernel = srv_kernel_for(a.mode, ctl & 1u), cur = (ctl >> 2) & 1u;
  __syncthreads();  // cs.hist is written
  if (threadIdx.x < HIST_BINS && q.out) q.out[threadIdx.x] = cs.hist[threadIdx.x];
  // the output precedes the completion word: the barrier orders the CTA's
  // writes before thread 0's system-scope release store, whose release is
  // cumulative (an explicit system fence before it measured 1.5 % slower on
  // a burst of 4000 requests and orders nothing more)
  __syncthreads();
  if (threadIdx.x == 0)
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(a.done + r), "r"(a.seq) : "memory");
  const hist_degeneracy_result d = block_epilogue(cs.hist, q.n, a.budget, a.theta, cs.pat, es);
  __syncthreads();
  if (threadIdx.x < HIST_BINS) {
    const uint32_t h = cs.hist[threadIdx.x];
    if (h) atomicAdd(&st->totals[threadIdx.x], (unsigned long long)h);
    st->last_hist[threadIdx.x] = h;
  }
  // the new pattern replaces the older of the two
  srv_copy_words(&st->pat[cur ^ 1u], &cs.pat, (int)(sizeof(hist_pattern) / 4));
  const bool shift = srv_is_shift(cs.pat);
  if (threadIdx.x == 0) {
    st->ctl = srv_ctl(d.flag, shift ? 1u : 0u, cur ^ 1u, shift ? cs.pat.log2k[0] : 0u);
    st->last_kernel = kernel;
    atomicAdd(&st->chunks, 1ull);  // at L2, like every other read of the state
  }
  // the stream's state is written: its state word releases the stream to
  // the host's admission, so that its next request may run in a batch that
  // starts while this one is still counting (the same release argument as
  // for the completion word)
  __syncthreads();
  if (threadIdx.x == 0)
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(a.done + kSrvMaxBatch + r), "r"(a.seq) : "memory");
}

// The slot table of a stream's pattern that is not a uniform shift (all
// threads call).
__device__ __noinline__ void srv_layout_general(const SrvStream* st, uint32_t cur, uint32_t* lut, CtaShared& cs) {
  __syncthreads();
  srv_copy_state_words(&cs.pat, &st->pat[cur], (int)(sizeof(hist_pattern) / 4));
  __syncthreads();
  classify_pattern(cs.pat, lut, cs);
}

// One CTA of 1024 threads per SM, four loads in flight per thread (as the
// stream's counting kernel): at 2k and 50k requests/s p50 19.7 -> 18.9 and
// 21.0 -> 19.6 us, p99 39.9 -> 35.6 and 52.4 -> 44.2 us against two CTAs
// per SM; burst capacity 2.53 -> 2.49 TB/s.
template <uint32_t CAP>
__global__ void __launch_bounds__(kThreads, 1) server_batch_kernel(const __grid_constant__ SrvArgs<CAP> args) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* table = smem;
  uint32_t* lut = smem + kTableWords;  // slot table while counting, then scratch of the reduction
  unsigned long long* pre = reinterpret_cast<unsigned long long*>(smem + kTableWords + kLutWords);
  uint32_t* ctl = reinterpret_cast<uint32_t*>(pre + kSrvMaxBatch + 1);
  __shared__ CtaShared cs;
  __shared__ EpiShared es;
  __shared__ int last;
  const SrvCommon& a = args.c;

  zero_table(table);
  srv_cost_prefix(args.req, a.count, a.streams, pre, ctl);
  const unsigned long long W = pre[a.count];
  const unsigned long long lo = W * blockIdx.x / gridDim.x;
  const unsigned long long hi = W * (blockIdx.x + 1) / gridDim.x;
  if (lo >= hi) return;
  // the request holding cost position lo
  uint32_t r = 0, rh = a.count;
  while (r + 1 < rh) {
    const uint32_t mid = (r + rh) >> 1;
    if (pre[mid] <= lo) r = mid;
    else rh = mid;
  }
  for (; r < a.count && pre[r] < hi; ++r) {
    const SrvReq q = args.req[r];
    const unsigned long long p0 = pre[r];
    if (q.n == 0) {
      // no bytes: the CTA holding the request's first cost position folds it
      if (p0 >= lo) {
        if (threadIdx.x < HIST_BINS) cs.hist[threadIdx.x] = 0;
        srv_epilogue(a, r, q, ctl[r], cs, es);
      }
      continue;
    }
    // this CTA's bytes of the request: its cost range cut to [0, n), each
    // cut moved to a 32 KiB boundary of the request's memory; a request of
    // at most a quarter of a CTA's range is not split (the range holding
    // its first cost position counts it whole, with no accumulator)
    unsigned long long b0 = lo > p0 ? split_point(q.in, lo - p0) : 0ull;
    unsigned long long e0 = split_point(q.in, hi - p0);
    if (e0 > (unsigned long long)q.n) e0 = q.n;
    if ((unsigned long long)q.n * 4 <= W / gridDim.x) {
      if (p0 < lo) continue;
      b0 = 0;
      e0 = q.n;
    }
    if (b0 >= e0) continue;
    const uint32_t c = ctl[r];
    int path = PATH_PLAIN, lk = 0;
    if (srv_kernel_for(a.mode, c & 1u) == HIST_FLAG_ADAPTIVE) {
      if ((c >> 1) & 1u) {
        path = PATH_SHIFT;
        lk = (int)((c >> 8) & 0xffu);
      } else {
        srv_layout_general(a.streams + q.stream, (c >> 2) & 1u, lut, cs);
        path = cs.path;
        lk = cs.lk;
      }
    }
    const uint8_t* base = q.in + b0;
    const uint32_t len = (uint32_t)(e0 - b0);
    const Split sp = split_bytes(base, len);
    count_call4(path, lk, reinterpret_cast<const uint4*>(base + sp.head), 0, sp.nvec, table, lut);
    const bool more = r + 1 < a.count && pre[r + 1] < hi;  // the CTA has another piece
    const bool cleared = flush_table(path, lk, table, cs.pat, lut, cs, more);
    count_edges(base, sp, cs);
    if (more && !cleared) zero_table(table);
    __syncthreads();
    if (b0 == 0 && e0 == q.n) {
      // the whole request
      if (threadIdx.x < HIST_BINS) cs.hist[threadIdx.x] = cs.res[threadIdx.x];
      srv_epilogue(a, r, q, ctl[r], cs, es);
      continue;
    }
    if (threadIdx.x < HIST_BINS && cs.res[threadIdx.x]) atomicAdd(&a.slot->acc[r][threadIdx.x], cs.res[threadIdx.x]);
    __syncthreads();
    if (threadIdx.x == 0) {
      // the barrier orders the CTA's adds before this fence, which publishes
      // them before the byte count
      __threadfence();
      last = atomicAdd(&a.slot->done[r], (unsigned long long)len) + len == q.n;
    }
    __syncthreads();
    if (last) {
      // every other piece of r was added (and fenced) before its done count
      __threadfence();
      if (threadIdx.x < HIST_BINS) {
        cs.hist[threadIdx.x] = __ldcg(&a.slot->acc[r][threadIdx.x]);
        a.slot->acc[r][threadIdx.x] = 0;
      }
      if (threadIdx.x == 0) a.slot->done[r] = 0;
      srv_epilogue(a, r, q, ctl[r], cs, es);
    }
  }
}

// Every stream starts with no chunks, the plain kernel and the default
// pattern (one CTA).
__global__ void server_init_kernel(SrvStream* s, uint32_t streams, uint32_t budget) {
  __shared__ CtaShared cs;
  __shared__ EpiShared es;
  if (threadIdx.x < HIST_BINS) cs.hist[threadIdx.x] = 0;
  __syncthreads();
  block_epilogue(cs.hist, 0, budget, HIST_THETA_MILLI_DEFAULT, cs.pat, es);
  __syncthreads();
  const bool shift = srv_is_shift(cs.pat);
  for (uint32_t i = 0; i < streams; ++i) {
    SrvStream* st = s + i;
    srv_copy_words(&st->pat[0], &cs.pat, (int)(sizeof(hist_pattern) / 4));
    srv_copy_words(&st->pat[1], &cs.pat, (int)(sizeof(hist_pattern) / 4));
    if (threadIdx.x == 0) {
      st->ctl = srv_ctl(HIST_FLAG_PLAIN, shift ? 1u : 0u, 0u, shift ? cs.pat.log2k[0] : 0u);
      st->last_kernel = HIST_FLAG_PLAIN;
    }
  }
}

uint64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

struct PendingReq {
  uint32_t stream;
  const uint8_t* in;
  size_t n;
  uint32_t* out;
  uint64_t tag;
  uint64_t submit_ns;
};

struct BatchSlot {
  bool busy = false;
  bool waited = false;  // completed by a host wait (its event could not be recorded)
  cudaStream_t cs = nullptr;
  cudaEvent_t done = nullptr;
  SrvSlot* d_slot = nullptr;
  // completion words of the batch's requests, then their state words
  // (pinned, mapped: 2 kSrvMaxBatch words)
  uint32_t* h_done = nullptr;
  uint32_t* d_done = nullptr;  // the same words as the device sees them
  uint32_t seq = 0;            // the running batch's sequence number
  std::vector<PendingReq> reqs;
  std::vector<uint8_t> reported;  // the request's completion has been returned
  std::vector<uint8_t> released;  // the request's stream has gone back to admission
  uint32_t n_reported = 0;
  uint32_t n_released = 0;
  uint32_t polls = 0;  // polls of the running batch
  uint64_t admit_ns = 0;
  uint64_t bytes = 0;
};

}  // namespace

struct hist_server {
  hist_server_config cfg;
  SrvStream* d_streams = nullptr;
  std::vector<uint8_t> stream_busy;  // a request of the stream is on the GPU
  std::vector<uint64_t> scan_mark;   // the stream was passed over in admission scan #mark
  uint64_t scan = 0;
  std::list<PendingReq> queue;  // FIFO; admission erases from the middle
  std::vector<std::list<PendingReq>::iterator> pick;  // the admission scan's requests
  BatchSlot slot[kSrvMaxSlots];
  uint64_t inflight_bytes = 0;
  uint32_t* h_done = nullptr;  // pinned: 2 kSrvMaxBatch words per batch slot
  uint32_t seq = 0;            // sequence number of the last batch launched
  int sms = 0;
  int max_grid = 0;                          // resident CTAs of the batch kernel
  SrvArgs<kSrvMaxBatch>* args = nullptr;     // parameter block of the next launch
  hist_server_stats stats;
};

namespace {

bool server_config_ok(const hist_server_config* c) {
  return c && c->streams >= 1 && c->streams <= HIST_SERVER_MAX_STREAMS && c->max_batch >= 1 &&
         c->max_batch <= kSrvMaxBatch && c->max_inflight >= 1 && c->max_inflight <= kSrvMaxSlots &&
         c->hbm_budget > 0 && c->theta_milli <= 1000 && c->pattern_budget >= HIST_BUDGET_MIN &&
         c->pattern_budget <= HIST_BUDGET_MAX && c->mode <= HIST_MODE_ADAPTIVE;
}

// Return the completions of finished requests -- those whose completion word
// holds their batch's sequence number, and every request of a batch whose
// event shows it done -- writing at most `cap` of them to `out` (out null:
// discard them); give a returned request's stream back to admission once its
// state word holds the number too, and release the slots of finished
// batches; returns how many completions were written or discarded.
uint32_t retire(hist_server* s, hist_completion* out, uint32_t cap, int* err) {
  uint32_t n = 0;
  for (uint32_t k = 0; k < s->cfg.max_inflight; ++k) {
    BatchSlot& f = s->slot[k];
    if (!f.busy) continue;
    const uint32_t count = (uint32_t)f.reqs.size();
    // the event is asked (a driver call) once every request's stream has
    // been released, and every 32nd poll before that, so that a failed batch
    // is still seen; the words themselves are plain reads of host memory
    cudaError_t q = cudaErrorNotReady;
    if (f.waited) q = cudaSuccess;
    else if (f.n_released == count || (++f.polls & 31u) == 0) q = cudaEventQuery(f.done);
    if (q != cudaSuccess && q != cudaErrorNotReady) {
      *err = cuda_fail(q);
      return n;
    }
    const bool all = q == cudaSuccess;
    for (uint32_t i = 0; i < count && f.n_released < count; ++i) {
      const PendingReq& r = f.reqs[i];
      if (!f.reported[i]) {
        // the acquire pairs with the epilogue's release: the request's
        // output is written before its completion word is
        if ((out && n >= cap) || (!all && __atomic_load_n(f.h_done + i, __ATOMIC_ACQUIRE) != f.seq)) continue;
        if (out) {
          hist_completion& c = out[n];
          c.tag = r.tag;
          c.stream = r.stream;
          c.status = 0;
          c.bytes = r.n;
          c.submit_ns = r.submit_ns;
          c.admit_ns = f.admit_ns;
          c.done_ns = now_ns();
        }
        ++n;
        f.reported[i] = 1;
        f.n_reported += 1;
        s->stats.completed += 1;
        s->stats.bytes += r.n;
      }
      // the stream's state is written before its state word is; a stream
      // goes back only after its request's completion has been returned, so
      // a stream's completions are returned in its order
      if (f.released[i] ||
          (!all && __atomic_load_n(f.h_done + kSrvMaxBatch + i, __ATOMIC_ACQUIRE) != f.seq))
        continue;
      s->stream_busy[r.stream] = 0;
      f.released[i] = 1;
      f.n_released += 1;
    }
    if (!all || f.n_released < count) continue;
    // the whole batch is done: its bytes go back to admission
    s->inflight_bytes -= f.bytes;
    f.reqs.clear();
    f.busy = false;
  }
  return n;
}

// Launch one batch if a slot is free and the queue holds admissible requests.
// FIFO order; only each stream's first queued request is a candidate, and
// only if the stream has no request on the GPU; the scan stops at the first
// candidate that does not fit the byte budget, so no request waits forever
// behind smaller later ones; it ends once every stream has been met.  A
// batch is launched whatever its size: one formed while the batches on the
// GPU hold every SM starts on the SMs their last CTAs leave (waiting for a
// quarter of a full batch instead measured no faster on a burst of 4000
// requests, and raised p99 at 50k requests/s from 44 to 55 us).
int admit(hist_server* s) {
  BatchSlot* f = nullptr;
  for (uint32_t k = 0; k < s->cfg.max_inflight; ++k)
    if (!s->slot[k].busy) {
      f = &s->slot[k];
      break;
    }
  if (!f || s->queue.empty()) return HIST_OK;
  s->pick.clear();
  uint64_t bytes = 0;
  uint32_t met = 0;  // streams met by the scan
  const uint64_t mark = ++s->scan;
  for (auto it = s->queue.begin();
       it != s->queue.end() && s->pick.size() < s->cfg.max_batch && met < s->cfg.streams; ++it) {
    const PendingReq& r = *it;
    if (s->scan_mark[r.stream] == mark) continue;  // not the stream's first: keep its order
    s->scan_mark[r.stream] = mark;
    ++met;
    if (s->stream_busy[r.stream]) continue;
    if (s->inflight_bytes + bytes + r.n > s->cfg.hbm_budget) {
      s->stats.deferred += 1;
      break;
    }
    bytes += r.n;
    s->pick.push_back(it);
  }
  if (s->pick.empty()) return HIST_OK;
  f->reqs.clear();
  f->bytes = bytes;
  for (const auto& it : s->pick) {
    s->stream_busy[it->stream] = 1;
    f->reqs.push_back(*it);
    s->queue.erase(it);
  }
  const uint32_t count = (uint32_t)f->reqs.size();
  // the launch's parameters: common fields, then the request table
  if (++s->seq == 0) s->seq = 1;  // completion words start at 0: never a batch's number
  f->seq = s->seq;
  f->reported.assign(count, 0);
  f->released.assign(count, 0);
  f->n_reported = 0;
  f->n_released = 0;
  f->polls = 0;
  SrvArgs<kSrvMaxBatch>* a = s->args;
  a->c.streams = s->d_streams;
  a->c.slot = f->d_slot;
  a->c.done = f->d_done;
  a->c.seq = f->seq;
  a->c.count = count;
  a->c.budget = s->cfg.pattern_budget;
  a->c.theta = s->cfg.theta_milli;
  a->c.mode = s->cfg.mode;
  unsigned long long cost = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const PendingReq& r = f->reqs[i];
    a->req[i].in = r.in;
    a->req[i].out = r.out;
    a->req[i].n = (uint32_t)r.n;
    a->req[i].stream = r.stream;
    cost += r.n + kReqCost;
  }
  unsigned long long grid = (cost + kCtaCost - 1) / kCtaCost;
  if (grid > (unsigned long long)s->max_grid) grid = (unsigned long long)s->max_grid;
  if (grid < 1) grid = 1;
  // the small variant's parameters are a prefix of the large one's
  static_assert(offsetof(SrvArgs<kSmallCap>, req) == offsetof(SrvArgs<kSrvMaxBatch>, req), "parameter layout");
  void* params[] = {a};
  const void* fn = count <= kSmallCap ? (const void*)server_batch_kernel<kSmallCap>
                                      : (const void*)server_batch_kernel<kSrvMaxBatch>;
  cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kThreads), params, kSrvSmem, f->cs);
  if (e != cudaSuccess) {
    // nothing was enqueued: the requests go back to the head of the queue
    for (const PendingReq& r : f->reqs) s->stream_busy[r.stream] = 0;
    s->queue.insert(s->queue.begin(), f->reqs.begin(), f->reqs.end());
    f->reqs.clear();
    return cuda_fail(e);
  }
  f->busy = true;
  e = cudaEventRecord(f->done, f->cs);
  f->waited = e != cudaSuccess;
  if (f->waited) {
    // no completion event: wait for the batch here so that it still retires
    cudaStreamSynchronize(f->cs);
    f->admit_ns = now_ns();
    s->inflight_bytes += f->bytes;
    s->stats.batches += 1;
    return cuda_fail(e);
  }
  f->admit_ns = now_ns();
  s->inflight_bytes += f->bytes;
  s->stats.batches += 1;
  return HIST_OK;
}

bool server_idle(const hist_server* s) {
  if (!s->queue.empty()) return false;
  for (uint32_t k = 0; k < s->cfg.max_inflight; ++k)
    if (s->slot[k].busy) return false;
  return true;
}

}  // namespace

extern "C" {

void hist_server_config_init(hist_server_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->streams = 256;
  c->max_batch = 256;
  c->max_inflight = 4;
  c->theta_milli = HIST_THETA_MILLI_DEFAULT;
  c->pattern_budget = HIST_BUDGET_MAX;
  c->mode = HIST_MODE_AUTO;
  c->hbm_budget = 32ull << 30;
}

int hist_server_create(const hist_server_config* cfg, hist_server** out) {
  if (!out || !server_config_ok(cfg)) return HIST_EINVAL;
  *out = nullptr;
  hist_server* s = new (std::nothrow) hist_server();
  if (!s) return HIST_ENOMEM;
  s->cfg = *cfg;
  s->stream_busy.assign(cfg->streams, 0);
  s->scan_mark.assign(cfg->streams, 0);
  s->sms = sm_count();
  memset(&s->stats, 0, sizeof(s->stats));
  static int attr_small[kMaxDevices], attr_large[kMaxDevices];
  int rc = s->sms > 0 ? HIST_OK : HIST_ECUDA;
  if (rc == HIST_OK) rc = ensure_smem_attr_bytes((const void*)server_batch_kernel<kSmallCap>, attr_small, kSrvSmem);
  if (rc == HIST_OK) rc = ensure_smem_attr_bytes((const void*)server_batch_kernel<kSrvMaxBatch>, attr_large, kSrvSmem);
  if (rc == HIST_OK) {
    int per_sm = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, (const void*)server_batch_kernel<kSrvMaxBatch>, kThreads, kSrvSmem);
    if (e != cudaSuccess) rc = cuda_fail(e);
    s->max_grid = s->sms * (per_sm > 0 ? per_sm : 1);
  }
  s->args = new (std::nothrow) SrvArgs<kSrvMaxBatch>();
  if (!s->args && rc == HIST_OK) rc = HIST_ENOMEM;
  if (rc == HIST_OK) {
    cudaError_t e = cudaMalloc((void**)&s->d_streams, sizeof(SrvStream) * cfg->streams);
    if (e == cudaSuccess) e = cudaMemset(s->d_streams, 0, sizeof(SrvStream) * cfg->streams);
    const size_t done_bytes = sizeof(uint32_t) * 2 * kSrvMaxBatch * kSrvMaxSlots;
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_done, done_bytes, cudaHostAllocMapped);
    if (e == cudaSuccess) memset(s->h_done, 0, done_bytes);
    for (uint32_t k = 0; e == cudaSuccess && k < cfg->max_inflight; ++k) {
      BatchSlot& f = s->slot[k];
      f.h_done = s->h_done + (size_t)k * 2 * kSrvMaxBatch;
      e = cudaHostGetDevicePointer((void**)&f.d_done, f.h_done, 0);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&f.cs, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaMalloc((void**)&f.d_slot, sizeof(SrvSlot));
      if (e == cudaSuccess) e = cudaMemset(f.d_slot, 0, sizeof(SrvSlot));
    }
    if (e == cudaSuccess) {
      server_init_kernel<<<1, 256>>>(s->d_streams, cfg->streams, cfg->pattern_budget);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = e == cudaErrorMemoryAllocation ? HIST_ENOMEM : cuda_fail(e);
  }
  if (rc) {
    hist_server_destroy(s);
    return rc;
  }
  *out = s;
  return HIST_OK;
}

int hist_server_destroy(hist_server* s) {
  if (!s) return HIST_EINVAL;
  cudaError_t e = cudaSuccess;
  for (uint32_t k = 0; k < kSrvMaxSlots; ++k) {
    BatchSlot& f = s->slot[k];
    if (f.cs) {
      const cudaError_t w = cudaStreamSynchronize(f.cs);
      if (e == cudaSuccess) e = w;
    }
  }
  for (uint32_t k = 0; k < kSrvMaxSlots; ++k) {
    BatchSlot& f = s->slot[k];
    if (f.d_slot) cudaFree(f.d_slot);
    if (f.done) cudaEventDestroy(f.done);
    if (f.cs) cudaStreamDestroy(f.cs);
  }
  if (s->d_streams) cudaFree(s->d_streams);
  if (s->h_done) cudaFreeHost(s->h_done);
  delete s->args;
  delete s;
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int hist_server_submit(hist_server* s, uint32_t stream, const uint8_t* d_in, size_t n, uint32_t* d_out,
                       uint64_t tag) {
  if (!s || stream >= s->cfg.streams || (!d_in && n) || n >= ((size_t)1 << 32)) return HIST_EINVAL;
  if (n > s->cfg.hbm_budget) return HIST_EBUDGET;
  s->queue.push_back(PendingReq{stream, d_in, n, d_out, tag, now_ns()});
  s->stats.submitted += 1;
  return HIST_OK;
}

int hist_server_poll(hist_server* s, hist_completion* out, uint32_t cap, uint32_t* n_out) {
  if (n_out) *n_out = 0;
  if (!s || (cap && !out)) return HIST_EINVAL;
  int err = HIST_OK;
  const uint32_t n = retire(s, cap ? out : nullptr, cap, &err);
  if (n_out && cap) *n_out = n;
  if (err) return err;
  return admit(s);
}

int hist_server_drain(hist_server* s, uint32_t timeout_ms) {
  if (!s) return HIST_EINVAL;
  const uint64_t t0 = now_ns();
  while (!server_idle(s)) {
    int err = HIST_OK;
    retire(s, nullptr, 0, &err);
    if (err) return err;
    const int rc = admit(s);
    if (rc) return rc;
    if (timeout_ms && now_ns() - t0 > (uint64_t)timeout_ms * 1000000ull) return HIST_ETIMEDOUT;
  }
  return HIST_OK;
}

int hist_server_stream_state(hist_server* s, uint32_t stream, hist_stream_state* h) {
  if (!s || !h || stream >= s->cfg.streams) return HIST_EINVAL;
  const int rc = hist_server_drain(s, 0);
  if (rc) return rc;
  SrvStream tmp;
  const cudaError_t e = cudaMemcpy(&tmp, s->d_streams + stream, sizeof(SrvStream), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e);
  memset(h, 0, sizeof(*h));
  memcpy(h->totals, tmp.totals, sizeof(h->totals));
  memcpy(h->last_hist, tmp.last_hist, sizeof(h->last_hist));
  const uint32_t cur = (tmp.ctl >> 2) & 1u;
  h->pattern = tmp.pat[cur];
  h->last_pattern = tmp.pat[cur ^ 1u];
  h->chunks = tmp.chunks;
  h->flag = tmp.ctl & 1u;
  h->last_kernel = tmp.last_kernel;
  return HIST_OK;
}

int hist_server_get_stats(hist_server* s, hist_server_stats* out) {
  if (!s || !out) return HIST_EINVAL;
  *out = s->stats;
  out->queued = s->queue.size();
  out->inflight_bytes = s->inflight_bytes;
  return HIST_OK;
}

int hist_server_replay(hist_server* s, const hist_request* reqs, uint32_t count, hist_completion* out,
                       uint32_t timeout_ms) {
  if (!s || (count && (!reqs || !out))) return HIST_EINVAL;
  for (uint32_t i = 0; i < count; ++i) {
    const hist_request& r = reqs[i];
    if (r.stream >= s->cfg.streams || (!r.d_in && r.n) || r.n >= (1ull << 32) ||
        (i && r.arrival_ns < reqs[i - 1].arrival_ns))
      return HIST_EINVAL;
    if (r.n > s->cfg.hbm_budget) return HIST_EBUDGET;
  }
  if (!server_idle(s)) return HIST_ESTATE;
  std::vector<hist_completion> buf((size_t)s->cfg.max_batch * s->cfg.max_inflight);
  uint32_t done = 0, next = 0;
  const uint64_t t0 = now_ns();
  while (done < count) {
    const uint64_t now = now_ns() - t0;
    if (timeout_ms && now > (uint64_t)timeout_ms * 1000000ull) return HIST_ETIMEDOUT;
    while (next < count && reqs[next].arrival_ns <= now) {
      const hist_request& r = reqs[next];
      s->queue.push_back(PendingReq{r.stream, r.d_in, (size_t)r.n, r.d_out, next, t0 + r.arrival_ns});
      s->stats.submitted += 1;
      ++next;
    }
    uint32_t n = 0;
    const int rc = hist_server_poll(s, buf.data(), (uint32_t)buf.size(), &n);
    if (rc) return rc;
    for (uint32_t i = 0; i < n; ++i) {
      hist_completion c = buf[i];
      const uint64_t idx = c.tag;
      c.tag = reqs[idx].tag;
      c.submit_ns -= t0;
      c.admit_ns -= t0;
      c.done_ns -= t0;
      out[idx] = c;
    }
    done += n;
  }
  // every request has completed; the last batches retire once their events fire
  while (!server_idle(s)) {
    if (timeout_ms && now_ns() - t0 > (uint64_t)timeout_ms * 1000000ull) return HIST_ETIMEDOUT;
    int err = HIST_OK;
    retire(s, nullptr, 0, &err);
    if (err) return err;
  }
  return HIST_OK;
}

}  // extern "C"
