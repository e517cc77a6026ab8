// hist_stream.cu -- the chunked stream of Sec. III.B with the kernel switch of
// Sec. III.C, all on the device.
//
// Every batch of chunks a stream is given (hist_stream_push / push_many) is
// counted by one launch of batch_flat_kernel, which needs no device-wide
// waits: a chunk's counts do not depend on the kernel or the layout that
// count it, so where those depend on the previous chunk's histogram (AUTO
// mode; the adaptive kernel below the full budget) predict_kernel derives
// them beforehand from a sample of the previous chunk, and the chunks'
// epilogues record the exact switches and patterns (see the comments above
// the kernels).
#include <cuda_runtime.h>
#include <stddef.h>
#include <mutex>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "hist.h"
#include "hist_device.cuh"
#include "hist_internal.h"

using namespace histdev;
using namespace histlib;

namespace {

constexpr uint32_t kMaxBatch = 1024;   // chunks per launch
constexpr uint32_t kSmallBatch = 128;  // chunks per launch of the smaller parameter block
constexpr uint32_t kPlanCtas = 160;    // largest grid whose ranges the host plans
constexpr uint32_t kChunkRing = 4 * kMaxBatch;  // flat scratch: chunk accumulators
constexpr uint32_t kLaunchRing = 8;             // flat scratch: per-launch records
constexpr uint32_t kPollLimit = 1u << 22;  // bounded wait: about a second
constexpr uint32_t kStatusTimeout = 4;     // device status: a wait ran out
constexpr uint32_t kStatusPattern = 8;     // device status: a layout differed from the rule's pattern

// Device-resident stream state.
struct StreamDev {
  // flat batches.  Launches of one stream overlap, so their scratch is in
  // rings: flat chunk g (counted from the stream's first flat chunk) sums
  // into slot g mod kChunkRing, which returns to zero in the chunk's
  // epilogue; flat launch L (from 1) keeps the switch and patterns of its
  // last chunks and its completed-chunk count in slot L mod kLaunchRing.
  uint32_t racc[kChunkRing][HIST_BINS];        // by flat chunk number mod kChunkRing
  unsigned long long rdone[kChunkRing];
  uint32_t rpred[kChunkRing];                  // AUTO flat batches: a chunk's predicted switch
  hist_pattern ppat[kChunkRing];               // below the full budget: the layout a chunk is counted with
  uint32_t rflag[kChunkRing];                  // AUTO flat batches: a chunk's switch
  uint32_t lredo_n[kLaunchRing];               // AUTO flat batches: chunks counted with the wrong kernel
  uint32_t lk0[kLaunchRing];                   // AUTO flat batches: the stream's switch before the launch
  // flat batches with a window of more than one chunk: every chunk's
  // histogram (by chunk number mod kChunkRing: a window of up to 256 chunks
  // plus a batch of 1024 fit), its sample histogram and sample size (AUTO),
  // and the window histogram after the last chunk of the last launch
  uint32_t whist[kChunkRing][HIST_BINS];
  uint32_t wsamp[kChunkRing][HIST_BINS];
  uint32_t wsn[kChunkRing];                    // pixels in chunk g's sample
  uint32_t wn[kChunkRing];                     // chunk g's size
  unsigned long long wmw[HIST_BINS];
  uint32_t lwin[kLaunchRing];                  // window switches written, by launch (window_flat_kernel)
  uint32_t lredo[kLaunchRing][kMaxBatch];
  unsigned long long lchunks[kLaunchRing];     // by flat launch number mod kLaunchRing
  hist_pattern lpat[kLaunchRing][2];
  uint32_t lflag[kLaunchRing];
  unsigned long long launches_done;            // flat launches whose stream state is written
  unsigned long long totals[HIST_BINS];
  uint32_t last_hist[HIST_BINS];
  hist_pattern pattern;       // pattern for the next chunk
  hist_pattern last_pattern;  // pattern the last completed chunk was given
  unsigned long long chunks;  // completed chunks
  uint32_t flag;              // switch computed from the last completed chunk
  uint32_t last_kernel;       // kernel the last completed chunk ran
  uint32_t status;            // 0, or kStatusTimeout
  uint32_t recounted;         // AUTO flat batches: chunks recounted after a misprediction
};

struct ChunkDesc {
  const uint8_t* in;
  uint32_t* out;
  uint32_t n;
  uint32_t pad;
};

// The launch parameters: the header and the chunk table.  Two capacities,
// so that a launch of a few chunks does not carry (and the driver does not
// copy) a 24 KiB table; the kernels are instantiated for both.
template <uint32_t CAP>
struct BatchArgs {
  static constexpr uint32_t kCap = CAP;
  StreamDev* st;
  uint32_t count;
  uint32_t budget;
  uint32_t theta;
  uint32_t mode;
  uint32_t trace_first;             // index of this batch's first chunk in the trace
  unsigned long long* trace;        // optional phase timestamps (see hist_stream_trace)
  uint32_t trace_cap;               // chunks the trace holds
  uint32_t chunk0_full;             // flat: the stream's pattern is known to be the full table
  unsigned long long first_chunk;   // flat: number of this batch's first chunk among the stream's flat chunks
  unsigned long long launch;        // flat: number of this launch among the stream's flat launches (from 1)
  uint32_t window;                  // chunks in the moving window
  uint32_t early;                   // flat: chunks may be read before the work before the launch completes
  // flat: the host splits the batch's cost into the CTAs' ranges, every
  // chunk of weight 1 (all modes but AUTO; AUTO with a window of one chunk
  // when every chunk is small), so a CTA reads its own range instead of
  // scanning the chunk table (see flat_plan)
  uint32_t planned;
  unsigned long long W;                        // the batch's total cost
  unsigned long long range;                    // W / grid
  unsigned long long plan_lo[kPlanCtas + 1];   // CTA b's range is [plan_lo[b], plan_lo[b + 1])
  unsigned long long plan_pre[kPlanCtas];      // cost position of its first chunk
  uint16_t plan_j[kPlanCtas];                  // its first chunk
  // CTA b with bit b of plan_groups set has only whole chunks for the
  // groups: chunks [plan_s[b], plan_s[b + 1]) start in its range, and any
  // chunk that overlaps the range from before is whole (an earlier CTA's)
  uint16_t plan_s[kPlanCtas + 1];
  uint32_t plan_groups[(kPlanCtas + 31) / 32];
  ChunkDesc c[CAP];
};
using SmallArgs = BatchArgs<kSmallBatch>;
using LargeArgs = BatchArgs<kMaxBatch>;
static_assert(sizeof(LargeArgs) <= 32764, "kernel parameters are limited to 32764 bytes");

// Phase timestamps (%globaltimer, ns) of chunk j by CTA slot k (0: the first
// CTA, 1: the middle one, 2: the last one), eight slots per chunk and CTA, of
// which the flat launch records phase 0 (start of the CTA's piece of the
// chunk), 5 (table reduced) and 7 (end).
constexpr int kTracePhases = 8;
constexpr int kTraceCtas = 3;

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void copy_pattern(hist_pattern* dst, const hist_pattern* src) {
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(hist_pattern) / 4); i += blockDim.x) d[i] = s[i];
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

struct Geo {
  const uint4* body;
  uint32_t begin, end;  // this CTA's 16-byte vectors (a chunk is below 2^32 bytes)
};

__device__ __forceinline__ Geo chunk_geo(const ChunkDesc& d) {
  const Split sp = split_bytes(d.in, d.n);
  Geo g;
  g.body = reinterpret_cast<const uint4*>(d.in + sp.head);
  g.begin = (uint32_t)part_begin(sp.nvec, gridDim.x, blockIdx.x);
  g.end = (uint32_t)part_begin(sp.nvec, gridDim.x, blockIdx.x + 1);
  return g;
}

__device__ void saturated_pattern(uint32_t prev_n, uint32_t budget, CtaShared& cs, EpiShared& es) {
  if (prev_n) {
    if (threadIdx.x < HIST_BINS) {
      cs.pat.off[threadIdx.x] = (uint16_t)(threadIdx.x * HIST_KMAX);
      cs.pat.log2k[threadIdx.x] = 5;
    }
    if (threadIdx.x == 0) {
      cs.pat.budget = budget;
      cs.pat.used = HIST_BINS * HIST_KMAX;
    }
  } else {
    if (threadIdx.x < HIST_BINS) cs.hist[threadIdx.x] = 0;
    __syncthreads();
    block_epilogue(cs.hist, 0, budget, HIST_THETA_MILLI_DEFAULT, cs.pat, es);
  }
  __syncthreads();
}

__device__ __forceinline__ bool same_pattern(const hist_pattern& x, const hist_pattern& y) {
  const uint32_t* a = reinterpret_cast<const uint32_t*>(&x);
  const uint32_t* b = reinterpret_cast<const uint32_t*>(&y);
  bool ok = true;
  for (int i = threadIdx.x; i < (int)(sizeof(hist_pattern) / 4); i += blockDim.x) ok &= a[i] == b[i];
  return __syncthreads_and(ok);
}

// ------------------------------------------------------------ flat batches --
//
// A chunk's counts do not depend on the kernel or the layout that count it,
// so the chunks of a batch need not be counted one after the other.  Where
// the layout does not depend on the previous chunk's histogram -- the plain
// mode (the plain kernel uses no pattern) and the adaptive mode at the full
// budget (the pattern rule then gives the full table after every non-empty
// chunk and the default pattern after an empty one) -- it is known before
// the launch; elsewhere predict_kernel derives each chunk's kernel and layout
// from a sample of the previous chunk, and the epilogues record the exact
// switch and pattern.  batch_flat_kernel splits the batch's chunks, placed end to end,
// into one contiguous range per CTA by a cost model (a chunk costs its bytes
// plus kFlatChunkCost, flat_cost), so a CTA counts one or two pieces of chunks and
// reduces its table only where its range crosses a chunk boundary.  A CTA
// adds a piece's per-bin sums into the chunk's accumulator and its bytes
// into the chunk's counter; the CTA whose bytes complete a chunk runs the
// chunk's epilogue (switch, pattern, output, totals, and the check that the
// layout the next chunk was counted with is the one the rule gives), and
// the CTA that completes the batch's last epilogue writes the stream state.
// No CTA waits for another, so the launch is not cooperative, and a chunk's
// accumulator returns to zero in its epilogue.

constexpr unsigned long long kFlatChunkCost = 64ull << 10;  // cost of a chunk beyond its bytes
constexpr uint32_t kGroupChunkMax = 256u << 10;  // largest chunk a group counts (flat_groups)
// The batch's last two chunks, when small, also cost kFlatTailCost, placed
// before their bytes: their epilogues derive the patterns the stream keeps,
// CTA-wide (about 5 us each), and in a launch of many small chunks the CTAs
// holding them should take fewer other chunks (1024 chunks of 64 KiB: 34.8
// -> 24.0 us per launch).  Beside 16 MiB chunks the epilogues are noise and
// the extra cost only shifts the split (AUTO, 64 chunks: 209 -> 220 us).
constexpr unsigned long long kFlatTailCost = 1ull << 20;
__host__ __device__ __forceinline__ unsigned long long flat_tail(unsigned long long n, uint32_t j, uint32_t count) {
  return j + 2 >= count && n <= kGroupChunkMax ? kFlatTailCost : 0ull;
}
// chunk j's cost: n bytes of weight w, then the fixed cost and the tail
// cost in `unit`s per byte (the weight of a byte of the full table)
__host__ __device__ __forceinline__ unsigned long long flat_cost(unsigned long long n, uint32_t w, uint32_t j,
                                                                 uint32_t count, uint32_t unit = 1) {
  return n * w + unit * (kFlatChunkCost + flat_tail(n, j, count));
}

// Whole small chunks are counted by groups of warps (flat_groups), thread b
// of a group holding bin b of its chunk.  Two groups take the table and the
// slot table as their tables; more groups need tables of their own.
constexpr int kGroups = 2;
constexpr int kGroupThreads = kThreads / kGroups;
constexpr int kGroupWarps = kGroupThreads / 32;
constexpr int kGroupOwnTables = kGroups > 2 ? kGroups : 0;
constexpr uint32_t kGroupPrefetch = 64;  // list entries whose pointers are read ahead
static_assert(kGroupThreads >= HIST_BINS, "one bin per thread of a group");
static_assert(kTableWords == kLutWords, "a group table in the slot table");

// dynamic shared memory: table, slot table, the groups' own tables, chunk
// cost prefix (u64 per chunk + 1)
template <class A>
constexpr size_t flat_smem_bytes() {
  return (size_t)(kTableWords + kLutWords + kGroupOwnTables * kTableWords) * 4 + (size_t)(A::kCap + 1) * 8;
}
static_assert(kMaxBatch <= (uint32_t)kThreads, "one prefix lane per chunk");

// pre[j] = sum over chunks before j of their costs (flat_cost); pre[count] = total.
// The kernel a flat launch runs chunk j with: the mode's, or in AUTO mode
// the predicted switch of chunk j-1 (chunk 0: the stream's switch, exact, as
// predict_kernel copied it before the launch; the launch rewrites the
// stream's switch at its end).
template <class A>
__device__ __forceinline__ uint32_t flat_kernel_of(const A& a, uint32_t j) {
  if (a.mode == HIST_MODE_PLAIN) return HIST_FLAG_PLAIN;
  if (a.mode == HIST_MODE_ADAPTIVE) return HIST_FLAG_ADAPTIVE;
  return j == 0 ? a.st->lk0[a.launch % kLaunchRing] : a.st->rpred[(a.first_chunk + j - 1) % kChunkRing];
}

// In AUTO mode (the launches whose ranges the host does not plan) a byte of
// a chunk predicted to run the plain kernel weighs kPlainWeight, a byte of
// the full table kFullWeight, and the fixed costs count kFullWeight per
// byte-equivalent; every other launch weighs every byte 1.  wt[j] holds
// chunk j's weight.
// The chunk table sits in the kernel's parameters, which are read through the
// constant cache: the distinct addresses of one warp's load are served one
// after another (4 us per launch when thread t read chunk t's size), so each
// warp reads its chunks' sizes with a warp-uniform index into shared memory
// (sz), where the rest of the launch reads them.
// The plain kernel counts wide data at well under half the full table's
// rate; on the degenerate workload (8 chunks of one value, 8 uniform, in
// turn) 5 : 2 measured best: 3.76 TB/s, against 3.54 at 2 : 1, 3.65 at
// 9 : 4 and 3.41 at 3 : 1.
constexpr uint32_t kFullWeight = 2, kPlainWeight = 5;
template <class A>
__device__ __forceinline__ uint32_t flat_unit(const A& a) {
  return a.mode == HIST_MODE_AUTO && !a.planned ? kFullWeight : 1u;
}

template <class A>
__device__ void flat_prefix(const A& a, unsigned long long* pre, uint32_t* wt, uint32_t* sz) {
  __shared__ unsigned long long wsum[kWarps];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (uint32_t j = (uint32_t)w; j < a.count; j += kWarps) {
    const uint32_t n = a.c[j].n;
    if (lane == 0) sz[j] = n;
  }
  __syncthreads();
  const uint32_t unit = flat_unit(a);
  uint32_t weight = unit;
  if (t < (int)a.count && a.mode == HIST_MODE_AUTO && flat_kernel_of(a, t) == HIST_FLAG_PLAIN) weight = kPlainWeight;
  if (t < (int)a.count) wt[t] = weight;
  const unsigned long long c = t < (int)a.count ? flat_cost(sz[t], weight, t, a.count, unit) : 0ull;
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
  if (t < (int)a.count) pre[t] = before + x - c;
  if (t == (int)a.count - 1) pre[a.count] = before + x;
  __syncthreads();
}

// Layout of chunk j (uniform over the CTA): the plain tables, the full table,
// or -- for chunk 0 (the stream's current pattern) and after an empty chunk
// (the default pattern) -- the pattern in cs.pat with its slot table.
__device__ __forceinline__ void copy_pattern_cg(hist_pattern* dst, const hist_pattern* src) {
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(hist_pattern) / 4); i += blockDim.x) d[i] = __ldcg(s + i);
}
template <class A>
__device__ __noinline__ void flat_layout_general(const A& a, uint32_t j, uint32_t* lut, CtaShared& cs,
                                                 EpiShared& es) {
  __syncthreads();
  if (a.budget < HIST_BUDGET_MAX) {
    // the pattern predict_kernel derived for the chunk (chunk 0: the stream's)
    copy_pattern_cg(&cs.pat, &a.st->ppat[(a.first_chunk + j) % kChunkRing]);
  } else if (j == 0) {
    pdl_wait();  // the previous launch writes the stream's pattern
    copy_pattern(&cs.pat, &a.st->pattern);
  } else {
    saturated_pattern(0, a.budget, cs, es);
  }
  __syncthreads();
  classify_pattern(cs.pat, lut, cs);
}

template <class A>
__device__ __forceinline__ uint32_t flat_check(const A& a);
template <class A>
__device__ __forceinline__ uint32_t flat_last_kernel(const A& a) {
  return a.mode == HIST_MODE_ADAPTIVE ? HIST_FLAG_ADAPTIVE : HIST_FLAG_PLAIN;  // AUTO: set by the last epilogue
}

template <class A>
__device__ __forceinline__ void flat_layout(const A& a, uint32_t j, bool adaptive, uint32_t* lut,
                                            CtaShared& cs, EpiShared& es, int& path, int& lk) {
  if (!adaptive) {
    path = PATH_PLAIN;
    lk = 0;
    return;
  }
  if (a.budget == HIST_BUDGET_MAX && (j > 0 ? a.c[j - 1].n > 0 : a.chunk0_full != 0)) {
    path = PATH_SHIFT;
    lk = 5;
    return;
  }
  flat_layout_general(a, j, lut, cs, es);
  path = cs.path;
  lk = cs.lk;
}


// AUTO flat launches: the chunks to count again.  Chunk i ran the kernel
// chunk i-1's predicted switch chose and had to run the one its exact switch
// chose (chunk 0: the stream's switch, which is exact); the list holds the
// chunks where the two differ, in order, one thread per chunk (a ballot and
// a prefix over the warps).  Returns the list's length and, in `kern`, the
// kernel the last chunk had to run.  All threads call.
__device__ __noinline__ uint32_t redo_list(StreamDev* st, unsigned long long g0, uint32_t count, uint32_t ls,
                                           uint32_t& kern) {
  __shared__ uint32_t wn[kWarps];
  __shared__ uint32_t base;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = (int)(blockDim.x >> 5);
  if (t == 0) base = 0;
  __syncthreads();
  for (uint32_t i0 = 0; i0 < count; i0 += blockDim.x) {
    const uint32_t i = i0 + (uint32_t)t;
    bool redo = false;
    if (i > 0 && i < count) {
      const uint32_t prev = (uint32_t)((g0 + i - 1) % kChunkRing);
      redo = __ldcg(&st->rflag[prev]) != __ldcg(&st->rpred[prev]);
    }
    const unsigned m = __ballot_sync(0xffffffffu, redo);
    if (lane == 0) wn[w] = __popc(m);
    __syncthreads();
    uint32_t off = base;
    for (int k = 0; k < w; ++k) off += wn[k];
    if (redo) st->lredo[ls][off + __popc(m & ((1u << lane) - 1u))] = i;
    __syncthreads();
    if (t == 0)
      for (int k = 0; k < nw; ++k) base += wn[k];
    __syncthreads();
  }
  kern = count > 1 ? __ldcg(&st->rflag[(uint32_t)((g0 + count - 2) % kChunkRing)]) : st->lk0[ls];
  return base;
}

// Chunk j is complete and cs.hist holds its histogram: its switch, pattern,
// output and totals; `check` says when chunk j+1 was counted with the full
// table that the rule must then give (0: never, 1: always, 2: when chunk j's
// switch chose the adaptive kernel); the CTA that completes the batch's last
// epilogue writes the stream state, `last_kernel` being the kernel the last
// chunk ran.  All threads call.
// kCheckPredicted (AUTO flat batches): chunk j+1 ran the full table when
// chunk j's predicted switch chose the adaptive kernel; the epilogue also
// records chunk j's switch, and the last one lists the chunks whose
// predicted kernel was not the one the switch chose (for a recount) and
// sets the last kernel itself.
constexpr uint32_t kCheckNever = 0, kCheckAlways = 1, kCheckPredicted = 3;
template <class A>
__device__ __forceinline__ uint32_t flat_check(const A& a) {
  return a.mode == HIST_MODE_PLAIN ? kCheckNever : (a.mode == HIST_MODE_ADAPTIVE ? kCheckAlways : kCheckPredicted);
}
// The switch of a chunk whose histogram is cs.hist (n pixels): its largest
// bin against theta (threads 0..255 hold the bins; all threads call; two
// barriers).  Returned to every thread.
__device__ __forceinline__ uint32_t block_flag(const uint32_t* hist, uint32_t n, uint32_t theta, EpiShared& es) {
  const int t = threadIdx.x;
  if (t < HIST_BINS) {
    const uint32_t m = __reduce_max_sync(0xffffffffu, hist[t]);
    if ((t & 31) == 0) es.wmax[t >> 5] = m;
  }
  __syncthreads();
  uint32_t mx = 0;
#pragma unroll
  for (int i = 0; i < HIST_BINS / 32; ++i) mx = es.wmax[i] > mx ? es.wmax[i] : mx;
  __syncthreads();
  return reaches_theta(mx, n, theta) ? HIST_FLAG_ADAPTIVE : HIST_FLAG_PLAIN;
}

template <class A>
__device__ __noinline__ void flat_epilogue(const A& a, uint32_t j, uint32_t check, hist_pattern& next,
                                           CtaShared& cs, EpiShared& es) {
  StreamDev* st = a.st;
  const int t = threadIdx.x;
  const uint32_t n = a.c[j].n;
  __syncthreads();
  // The stream state keeps the patterns of the launch's last two chunks and
  // the last chunk's switch; an AUTO launch records every chunk's switch.
  // At the full budget every other chunk's pattern is known without the
  // rule's arithmetic (the full table after a non-empty chunk, the default
  // pattern after an empty one: the layout the next chunk was counted
  // with), and below it the next chunk's layout came from its prediction,
  // so those patterns are not computed here.
  const bool want_pattern = j + 2 >= a.count;
  uint32_t flag = HIST_FLAG_PLAIN;
  if (want_pattern) {
    const hist_degeneracy_result r = block_epilogue(cs.hist, n, a.budget, a.theta, next, es);
    if (t == 0) cs.flag = r.flag;  // r is valid in threads 0..255 only
    __syncthreads();
    flag = cs.flag;
  } else if (check == kCheckPredicted) {
    flag = block_flag(cs.hist, n, a.theta, es);
  }
  if (t < HIST_BINS) {
    const uint32_t h = cs.hist[t];
    if (a.c[j].out) a.c[j].out[t] = h;
    if (h) atomicAdd(&st->totals[t], (unsigned long long)h);
    if (j + 1 == a.count) st->last_hist[t] = h;
  }
  const uint32_t rs = (uint32_t)((a.first_chunk + j) % kChunkRing);
  if (check == kCheckPredicted && t == 0) st->rflag[rs] = flag;
  if (a.window > 1 && t < HIST_BINS) st->whist[rs][t] = cs.hist[t];
  if (want_pattern && j + 1 < a.count && a.budget == HIST_BUDGET_MAX &&
      (check == kCheckAlways || (check == kCheckPredicted && __ldcg(&st->rpred[rs]) == HIST_FLAG_ADAPTIVE))) {
    // chunk j+1 was counted with the layout the rule gives after n pixels
    saturated_pattern(n, a.budget, cs, es);
    if (!same_pattern(next, cs.pat) && t == 0) atomicExch(&st->status, kStatusPattern);
  }
  const uint32_t ls = (uint32_t)(a.launch % kLaunchRing);
  if (want_pattern) copy_pattern(&st->lpat[ls][j + 1 == a.count ? 1 : 0], &next);
  if (j + 1 == a.count && t == 0) st->lflag[ls] = flag;
  __syncthreads();
}

// A CTA that ran `epis` chunk epilogues adds them to the launch's count once
// it is done (after a fence that publishes them); the CTA whose add completes
// the launch's chunks writes the stream state after the batch.  All threads
// call.
template <class A>
__device__ __noinline__ void flat_finish(const A& a, uint32_t epis, uint32_t check, uint32_t last_kernel,
                                         CtaShared& cs) {
  StreamDev* st = a.st;
  const int t = threadIdx.x;
  const uint32_t ls = (uint32_t)(a.launch % kLaunchRing);
  __syncthreads();
  if (t == 0) {
    // the barrier orders the CTA's epilogue writes before this fence
    __threadfence();
    cs.kernel = atomicAdd(&st->lchunks[ls], (unsigned long long)epis) + epis == a.count ? 1u : 0u;
  }
  __syncthreads();
  if (cs.kernel) {
    // every chunk's epilogue is done: the stream state after the batch
    __threadfence();
    if (a.count == 1) {
      copy_pattern(&st->last_pattern, &st->pattern);
      __syncthreads();
    } else {
      copy_pattern_cg(&st->last_pattern, &st->lpat[ls][0]);
    }
    copy_pattern_cg(&st->pattern, &st->lpat[ls][1]);
    if (check == kCheckPredicted && a.window == 1) {
      const uint32_t nr = redo_list(st, a.first_chunk, a.count, ls, last_kernel);
      if (t == 0) {
        st->lredo_n[ls] = nr;
        st->recounted += nr;
      }
    }
    if (t == 0) {
      if (a.window == 1) {  // with a window the window kernel sets both
        st->flag = __ldcg(&st->lflag[ls]);
        st->last_kernel = last_kernel;
      }
      st->chunks += a.count;
      st->lchunks[ls] = 0;
      __threadfence();
      st->launches_done = a.launch;
    }
  }
  __syncthreads();
}

// CTA-wide state of batch_flat_kernel (shared memory).
template <uint32_t CAP>
struct FlatShared {
  CtaShared cs;
  EpiShared es;
  hist_pattern next;
  uint32_t eh[HIST_BINS];  // unaligned edge bytes of the pieces in the table
  int cur;                 // chunk whose pieces the table holds, -1 if none
  int path, lk;            // its layout
  uint32_t bytes;          // its bytes in the table
  int last;
  int released;  // this CTA has waited for the previous launch
  int ring_ok;   // the chunk ring slots of this launch are free
  uint32_t epis; // chunk epilogues this CTA ran
  uint32_t wt[CAP];  // cost weight of each chunk (flat_prefix)
  uint32_t sz[CAP];  // size of each chunk (flat_prefix)
  uint16_t wl[CAP];  // whole chunks left to the groups, in batch order
  const uint8_t* gin[kGroupPrefetch];  // input and output of the first wl entries
  uint32_t* gout[kGroupPrefetch];
  uint32_t take;     // next entry of wl a group takes
  uint32_t gitem[kGroups];
  uint32_t gmax[kGroups][kGroupWarps];
  uint32_t gres[kGroups][HIST_BINS];  // each group's chunk histogram
};

template <class A>
__device__ __forceinline__ void flat_mark(const A& a, uint32_t j, int phase, bool lead) {
  const int tslot = blockIdx.x == 0 ? 0 : (blockIdx.x == gridDim.x / 2 ? 1 : (blockIdx.x == gridDim.x - 1 ? 2 : -1));
  if (a.trace && tslot >= 0 && lead && a.trace_first + j < a.trace_cap)
    a.trace[((size_t)(a.trace_first + j) * kTraceCtas + tslot) * kTracePhases + phase] = globaltimer();
}
template <class A>
__device__ __forceinline__ void flat_mark(const A& a, uint32_t j, int phase) {
  flat_mark(a, j, phase, threadIdx.x == 0);
}

// Launches of one stream overlap (programmatic dependent launch): every
// CTA lets the next launch start as soon as it starts, so the next launch's
// CTAs take the SM slots that this launch's CTAs free as they finish, clear
// their tables and split the work.  Unless the caller has declared every
// chunk complete when it was pushed (a.early, HIST_OVERLAP_PUSHES), a CTA
// then waits for the work before the launch on the CUDA stream to complete
// before it reads a chunk byte: that work may be the kernel that wrote the
// chunk, and only the wait makes its writes visible.  A CTA also waits for
// the previous launch to complete before its first epilogue, which reads
// and writes the stream state (flat_release), and before it first adds
// into a chunk ring slot, the last user of the slot -- a launch at least
// kChunkRing / kMaxBatch - 1 launches back -- must have written its state
// (flat_ring_ready, a bounded wait).  All threads call both.
template <class F>
__device__ __forceinline__ void flat_release(F& fs) {
  if (!fs.released) pdl_wait();
  __syncthreads();
  if (threadIdx.x == 0) fs.released = 1;
}

template <class A>
__device__ __noinline__ void flat_ring_ready(const A& a, FlatShared<A::kCap>& fs) {
  // fs.ring_ok is read between the first two barriers and written after the
  // second, so every thread takes the same branch
  __syncthreads();
  if (fs.ring_ok) return;
  constexpr unsigned long long back = kChunkRing / kMaxBatch - 1;
  if (threadIdx.x == 0) {
    uint32_t it = 0;
    while (a.launch > back && ld_acquire(&a.st->launches_done) < a.launch - back) {
      if (++it >= kPollLimit) {
        atomicOr(&a.st->status, kStatusTimeout);
        break;
      }
      __nanosleep(256);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) fs.ring_ok = 1;
}

// Reduce the table (the pieces of chunk fs.cur) and publish them: into the
// chunk's accumulator and byte counter, or, when the table holds the whole
// chunk, straight into the chunk's epilogue.  The CTA whose bytes complete
// the chunk runs the epilogue.  The CTA's last flush leaves the table as it
// is.  All threads call.
template <class A>
__device__ __noinline__ void flat_flush(const A& a, uint32_t* table, uint32_t* lut, FlatShared<A::kCap>& fs,
                                        bool last_flush = false) {
  __syncthreads();
  const int j = fs.cur;
  if (j < 0) return;
  StreamDev* st = a.st;
  const uint32_t slot = (uint32_t)((a.first_chunk + (unsigned)j) % kChunkRing);
  const int t = threadIdx.x;
  const bool cleared = flush_table(fs.path, fs.lk, table, fs.cs.pat, lut, fs.cs, !last_flush);
  if (t < HIST_BINS) {
    fs.cs.res[t] += fs.eh[t];
    fs.eh[t] = 0;
  }
  if (!last_flush && !cleared) zero_table(table);
  const uint32_t n = fs.sz[j], len = fs.bytes;
  __syncthreads();
  flat_mark(a, j, 5);
  if (t == 0) fs.cur = -1;
  if (len == n) {
    // the whole chunk
    if (t < HIST_BINS) fs.cs.hist[t] = fs.cs.res[t];
    flat_release(fs);
    flat_epilogue(a, j, flat_check(a), fs.next, fs.cs, fs.es);
    if (t == 0) fs.epis += 1;
    flat_mark(a, j, 7);
    return;
  }
  flat_ring_ready(a, fs);
  if (t < HIST_BINS && fs.cs.res[t]) atomicAdd(&st->racc[slot][t], fs.cs.res[t]);
  __syncthreads();
  if (t == 0) {
    // the barrier orders the CTA's adds before this fence, which publishes
    // them before the byte count
    __threadfence();
    fs.last = atomicAdd(&st->rdone[slot], (unsigned long long)len) + len == n;
  }
  __syncthreads();
  if (fs.last) {
    // every other piece of chunk j was added (and fenced) before its count
    __threadfence();
    if (t < HIST_BINS) {
      fs.cs.hist[t] = __ldcg(&st->racc[slot][t]);
      st->racc[slot][t] = 0;
    }
    if (t == 0) st->rdone[slot] = 0;
    flat_release(fs);
    flat_epilogue(a, j, flat_check(a), fs.next, fs.cs, fs.es);
    if (t == 0) fs.epis += 1;
  }
  flat_mark(a, j, 7);
  __syncthreads();
}

// Count bytes [b0, e0) of chunk j (not empty) into the table, reducing the
// table first if it holds another chunk.  All threads call.
template <class A>
__device__ __forceinline__ void flat_piece(const A& a, uint32_t j, uint32_t b0, uint32_t e0,
                                           uint32_t* table, uint32_t* lut, FlatShared<A::kCap>& fs) {
  if (fs.cur != (int)j) {
    flat_flush(a, table, lut, fs);
    flat_mark(a, j, 0);
    int path, lk;
    flat_layout(a, j, flat_kernel_of(a, j) == HIST_FLAG_ADAPTIVE, lut, fs.cs, fs.es, path, lk);
    __syncthreads();
    if (threadIdx.x == 0) {
      fs.cur = (int)j;
      fs.path = path;
      fs.lk = lk;
      fs.bytes = 0;
    }
    __syncthreads();
  }
  const uint8_t* base = a.c[j].in + b0;
  const Split sp = split_bytes(base, e0 - b0);
  count_call4(fs.path, fs.lk, reinterpret_cast<const uint4*>(base + sp.head), 0, sp.nvec, table, lut);
  count_edges_into(base, sp, fs.eh);
  if (threadIdx.x == 0) fs.bytes += e0 - b0;
}

// Whether a whole chunk j goes to the groups: not empty, at most
// kGroupChunkMax bytes, not one of the batch's last two chunks (their
// epilogues keep the stream's patterns), and counted with a layout known
// without a pattern -- the plain kernel's tables, or the full table at the
// full budget after a non-empty chunk.
template <class A>
__device__ __forceinline__ bool group_chunk(const A& a, uint32_t j, uint32_t n, uint32_t prev_n) {
  if (n == 0 || n > kGroupChunkMax || j + 2 >= a.count) return false;
  if (flat_kernel_of(a, j) != HIST_FLAG_ADAPTIVE) return true;
  return a.budget == HIST_BUDGET_MAX && prev_n > 0;
}

// Sizes of chunks [j0, j0 + kWarps) into sz, warp w reading chunk j0 + w's;
// returns the end of the chunks read.  All threads call (ends with a
// barrier).
template <class A>
__device__ __noinline__ uint32_t flat_sizes(const A& a, uint32_t j0, uint32_t* sz) {
  const uint32_t j = j0 + (threadIdx.x >> 5);
  if (j < a.count) {
    const uint32_t n = a.c[j].n;
    if ((threadIdx.x & 31) == 0) sz[j] = n;
  }
  __syncthreads();
  return j0 + kWarps;
}

// Count the cost range [x0, x1) of the batch.  Chunk j's byte b sits at
// cost pre[j] + b wt[j] (after the tail cost for the last two chunks); a
// range takes the bytes whose cost position it holds.  All threads call.
template <class A>
__device__ uint32_t flat_range(const A& a, const unsigned long long* pre, const uint32_t* wt,
                               unsigned long long x0, unsigned long long x1, unsigned long long range, uint32_t* table,
                               uint32_t* lut, FlatShared<A::kCap>& fs) {
  uint32_t nwl = 0;
  uint32_t j = 0;
  const uint32_t unit = flat_unit(a);
  unsigned long long p0;  // cost position of chunk j
  if (a.planned) {
    j = a.plan_j[blockIdx.x];
    p0 = a.plan_pre[blockIdx.x];
  } else {
    uint32_t jh = a.count;
    while (j + 1 < jh) {
      const uint32_t mid = (j + jh) >> 1;
      if (pre[mid] <= x0) j = mid;
      else jh = mid;
    }
    p0 = pre[j];
  }
  // A planned launch reads the sizes of the chunks it meets here, kWarps
  // at a time from chunk j-1 on, warp w one chunk's with a warp-uniform
  // index, so the warps' constant-cache misses overlap (chunk after chunk:
  // 0.5 us each).  Chunk weights are 1 there.
  uint32_t wend = 0;
  if (a.planned) wend = flat_sizes(a, j > 0 ? j - 1 : 0, fs.sz);
  // the size of chunk j-1 (before chunk 0: the stream's last chunk, known
  // to be non-empty when chunk0_full)
  uint32_t prev_n = j > 0 ? fs.sz[j - 1] : a.chunk0_full;
  unsigned long long p1 = 0;
  for (; j < a.count && p0 < x1; ++j, p0 = p1) {
    if (a.planned && j == wend) wend = flat_sizes(a, j, fs.sz);
    const uint32_t n = fs.sz[j], w = a.planned ? 1u : wt[j];
    p1 = p0 + flat_cost(n, w, j, a.count, unit);
    const uint32_t pn = prev_n;
    prev_n = n;
    if (n == 0) {
      // no bytes: the range holding the chunk's first cost position folds it
      if (p0 >= x0) {
        flat_flush(a, table, lut, fs);
        flat_mark(a, j, 0);
        if (threadIdx.x < HIST_BINS) fs.cs.hist[threadIdx.x] = 0;
        flat_release(fs);
        flat_epilogue(a, j, flat_check(a), fs.next, fs.cs, fs.es);
        if (threadIdx.x == 0) fs.epis += 1;
        flat_mark(a, j, 7);
      }
      continue;
    }
    if ((unsigned long long)n * w * 4 <= range) {
      // a chunk of at most a quarter of a CTA's range is not split: the
      // range holding its first cost position counts it whole, so it needs
      // no accumulator, byte counter or ring; a small one whose layout and
      // epilogue need no pattern is left to the groups
      if (p0 >= x0) {
        if (group_chunk(a, j, n, pn)) {
          if (threadIdx.x == 0) fs.wl[nwl] = (uint16_t)j;
          ++nwl;
        } else {
          flat_piece(a, j, 0, n, table, lut, fs);
        }
      }
      continue;
    }
    // byte b sits at cost q0 + b w, after the chunk's tail cost
    const unsigned long long q0 = p0 + unit * flat_tail(n, j, a.count);
    if (x1 <= q0) continue;
    const unsigned long long c0 = x0 > q0 ? split_point(a.c[j].in, (x0 - q0 + w - 1) / w) : 0ull;
    const unsigned long long c1 = split_point(a.c[j].in, (x1 - q0 + w - 1) / w);
    const unsigned long long e0 = c1 < (unsigned long long)n ? c1 : (unsigned long long)n;
    if (c0 < e0) flat_piece(a, j, (uint32_t)c0, (uint32_t)e0, table, lut, fs);
  }
  return nwl;
}

// ------------------------------------------------ whole small chunks --
//
// A CTA that counts a small chunk whole spends little of its time loading
// it: a 64 KiB chunk is one round of four loads per thread, after which the
// CTA reduces its table and runs the chunk's epilogue between CTA-wide
// barriers, with no load in flight.  So the CTA leaves such chunks to the
// end of its range and counts them with kGroups groups of warps.  Each
// group has its own table and named barrier and takes the next chunk from a
// shared counter, so one group's reduction and epilogue run while the other
// groups' loads are in flight.  A group chunk's epilogue is the part of
// flat_epilogue that such a chunk needs: its output, the totals, its window
// entry and, in AUTO mode, its exact switch.

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kGroupThreads) : "memory");
}

// Count vectors [0, nvec) of p with thread gt of a group into the group's
// table: the full table, or the per-warp tables of the group's warps (the
// plain layout indexes them by the CTA's warp number w, so they sit at
// words 256 w of the group's table, g kGroupWarps <= w < (g + 1) kGroupWarps).
static __device__ __noinline__ void group_count(bool adaptive, const uint4* p, size_t nvec, uint32_t* table,
                                                int gt) {
  if (adaptive) count_range<PATH_SHIFT, 5, 4>(p, 0, nvec, table, table, gt, kGroupThreads);
  else count_range<PATH_PLAIN, 0, 4>(p, 0, nvec, table, table, gt, kGroupThreads);
}

// All threads call (after a CTA barrier); returns after the CTA's groups
// have counted the nwl chunks listed in fs.wl and run their epilogues.
template <class A>
__device__ __noinline__ void flat_groups(const A& a, uint32_t nwl, uint32_t* gtables, FlatShared<A::kCap>& fs) {
  StreamDev* st = a.st;
  const int t = threadIdx.x, g = t / kGroupThreads, gt = t % kGroupThreads;
  const int gw = gt >> 5, lane = t & 31;
  uint32_t* table = gtables + (size_t)g * kTableWords;
  uint32_t* res = fs.gres[g];
  const uint32_t check = flat_check(a);
  bool released = fs.released != 0;
  uint32_t epis = 0;
  {
    uint4* t4 = reinterpret_cast<uint4*>(table);
    for (int i = gt; i < kTableWords / 4; i += kGroupThreads) t4[i] = make_uint4(0, 0, 0, 0);
    if (gt < HIST_BINS) res[gt] = 0;
  }
  for (;;) {
    group_sync(g);  // the table is clear and the last epilogue has read res
    if (gt == 0) fs.gitem[g] = atomicAdd(&fs.take, 1u);
    group_sync(g);
    const uint32_t i = fs.gitem[g];
    if (i >= nwl) break;
    const uint32_t j = fs.wl[i];
    const uint32_t n = fs.sz[j];
    const bool adaptive = flat_kernel_of(a, j) == HIST_FLAG_ADAPTIVE;
    flat_mark(a, j, 0, gt == 0);
    const uint8_t* base = i < kGroupPrefetch ? fs.gin[i] : a.c[j].in;
    uint32_t* out = i < kGroupPrefetch ? fs.gout[i] : a.c[j].out;
    const Split sp = split_bytes(base, n);
    group_count(adaptive, reinterpret_cast<const uint4*>(base + sp.head), sp.nvec, table, gt);
    const int L = (int)kLineBytes;
    if (gt < (int)sp.head) atomicAdd(&res[base[gt]], 1u);
    else if (gt >= L && gt < L + (int)sp.tail) atomicAdd(&res[base[sp.head + sp.nvec * 16 + (gt - L)]], 1u);
    group_sync(g);
    // reduce the table into res and clear it as it is read
    if (adaptive) {
      if (gt < HIST_BINS) {
        // bin b is the 32 words of row b; thread b reads them starting at
        // word b mod 32, so the 32 threads of a warp read 32 banks, with
        // all its loads in flight (a row per warp with a warp-wide add is a
        // chain of dependent steps per row: 1.2 us per chunk)
        uint32_t* row = table + (gt << 5);
        uint32_t sum = 0;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
          const int c = (k + gt) & 31;
          sum += row[c];
          row[c] = 0;
        }
        res[gt] += sum;
      }
    } else if (gt < HIST_BINS) {
      uint32_t sum = 0;
#pragma unroll
      for (int w = 0; w < kGroupWarps; ++w) {
        uint32_t* q = table + (g * kGroupWarps + w) * HIST_BINS + gt;
        sum += *q;
        *q = 0;
      }
      res[gt] += sum;
    }
    group_sync(g);
    flat_mark(a, j, 5, gt == 0);
    if (!released) {
      // the previous launch writes the stream state and may write the
      // same outputs
      pdl_wait();
      released = true;
    }
    const uint32_t rs = (uint32_t)((a.first_chunk + j) % kChunkRing);
    uint32_t h = 0;
    if (gt < HIST_BINS) {
      h = res[gt];
      res[gt] = 0;
      if (out) out[gt] = h;
      if (h) atomicAdd(&st->totals[gt], (unsigned long long)h);
      if (a.window > 1) st->whist[rs][gt] = h;
    }
    if (check == kCheckPredicted) {
      const uint32_t m = __reduce_max_sync(0xffffffffu, h);
      if (lane == 0) fs.gmax[g][gw] = m;
      group_sync(g);
      if (gt == 0) {
        uint32_t mx = 0;
#pragma unroll
        for (int k = 0; k < HIST_BINS / 32; ++k) mx = fs.gmax[g][k] > mx ? fs.gmax[g][k] : mx;
        st->rflag[rs] = reaches_theta(mx, n, a.theta) ? HIST_FLAG_ADAPTIVE : HIST_FLAG_PLAIN;
      }
    }
    epis += 1;
    flat_mark(a, j, 7, gt == 0);
  }
  if (gt == 0 && epis) atomicAdd(&fs.epis, epis);
}

// One CTA of 1024 threads per SM, each thread with four 16-byte loads in
// flight (64 registers).  Two CTAs per SM with two loads each keep as many
// bytes in flight, but the SM's two CTAs do not progress alike (the
// scheduler favours the older one), so one of them finishes its range well
// before the other and the SM then runs a single CTA at half its loads in
// flight; one CTA per SM has no such pair.  Measured (64 chunks of 16 MiB,
// CUDA events): 176 -> 166 us per launch overlapping the previous one,
// 205 -> 177 us waiting for it.
template <class A>
__global__ void __launch_bounds__(kThreads, 1) batch_flat_kernel(const __grid_constant__ A a) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* table = smem;
  uint32_t* lut = smem + kTableWords;  // slot table while counting, then scratch of the reduction
  uint32_t* gtables = kGroupOwnTables ? smem + kTableWords + kLutWords : smem;
  unsigned long long* pre =
      reinterpret_cast<unsigned long long*>(smem + kTableWords + kLutWords + kGroupOwnTables * kTableWords);
  __shared__ FlatShared<A::kCap> fs;
  const int t = threadIdx.x;

  pdl_launch_dependents();
  if (t < HIST_BINS) fs.eh[t] = 0;
  if (t == 0) {
    fs.cur = -1;
    fs.released = 0;
    fs.ring_ok = 0;
    fs.epis = 0;
    fs.take = 0;
  }
  zero_table(table);
  // in AUTO mode the work just before this launch is the prediction, whose
  // switches the cost split and the range read; otherwise the chunks may
  // come from the work just before this launch
  const bool wait_first = a.mode == HIST_MODE_AUTO || !a.early;
  if (wait_first) pdl_wait();
  if (a.planned) __syncthreads();
  else flat_prefix(a, pre, fs.wt, fs.sz);
  if (wait_first && t == 0) fs.released = 1;
  unsigned long long lo, hi, range;
  if (a.planned) {
    lo = a.plan_lo[blockIdx.x];
    hi = a.plan_lo[blockIdx.x + 1];
    range = a.range;
  } else {
    const unsigned long long W = pre[a.count];
    lo = W * blockIdx.x / gridDim.x;
    hi = W * (blockIdx.x + 1) / gridDim.x;
    range = W / gridDim.x;
  }
  uint32_t nwl = 0;
  if (a.planned && (a.plan_groups[blockIdx.x >> 5] >> (blockIdx.x & 31) & 1u)) {
    // the range holds whole chunks for the groups only
    const uint32_t s0 = a.plan_s[blockIdx.x], s1 = a.plan_s[blockIdx.x + 1];
    nwl = s1 - s0;
    for (uint32_t i = (uint32_t)t; i < nwl; i += kThreads) fs.wl[i] = (uint16_t)(s0 + i);
    for (uint32_t j = s0; j < s1; j += kWarps) flat_sizes(a, j, fs.sz);
  } else if (lo < hi) {
    nwl = flat_range(a, pre, fs.wt, lo, hi, range, table, lut, fs);
  }
  flat_flush(a, table, lut, fs, true);
  __syncthreads();
  if (nwl) {
    // the pointers of the groups' first chunks, warp w reading entries w,
    // w + 32 with warp-uniform indices (their misses overlap)
    for (uint32_t i = (uint32_t)(t >> 5); i < nwl && i < kGroupPrefetch; i += kWarps) {
      const ChunkDesc& d = a.c[fs.wl[i]];
      const uint8_t* in = d.in;
      uint32_t* out = d.out;
      if ((t & 31) == 0) {
        fs.gin[i] = in;
        fs.gout[i] = out;
      }
    }
    __syncthreads();
    flat_groups(a, nwl, gtables, fs);
    __syncthreads();
  }
  if (fs.epis) flat_finish(a, fs.epis, flat_check(a), flat_last_kernel(a), fs.cs);
}

// AUTO mode.  Chunk j's kernel is chunk j-1's switch (at the full budget
// the adaptive kernel's layout is then fixed: the full table after a
// non-empty chunk, since R3 saturates there; an empty chunk always switches
// to the plain kernel).  Since a chunk's histogram does not depend on the
// kernel that counts it, the one-bit dependency is broken by prediction:
//   1. predict_kernel takes each chunk's switch from a 4096-pixel sample
//      (every pixel of a smaller chunk), and below the full budget the
//      layout too;
//   2. batch_flat_kernel counts every chunk, all at once, with the kernel the
//      predictions give it (chunk 0: the stream's switch, exact); each
//      chunk's epilogue records its exact switch, and the last one lists the
//      chunks whose kernel was not the one their predecessor's exact switch
//      chose;
//   3. auto_redo_kernel counts each listed chunk again with that kernel and
//      rewrites its output, so every chunk's counts come from the kernel the
//      method chooses.  The list is empty unless a sample misjudged a chunk.

constexpr uint32_t kSampleVecs = HIST_BINS;  // 16-byte vectors per sample: 4096 pixels

// Before a flat launch of an AUTO stream, or of any adaptive stream below the
// full budget: CTA j samples chunk j (256 evenly spaced 16-byte vectors,
// 4096 pixels; a smaller chunk whole) and predicts from the sample what the
// chunk's own histogram gives -- its switch (AUTO) and, below the full
// budget, the binning pattern the rule derives from it, which becomes the
// layout chunk j+1 is counted with.  Chunk 0 is counted with the stream's
// pattern and kernel (exact).  A chunk's counts do not depend on its
// layout, so a prediction that differs from the exact pattern only costs
// speed; the epilogues still record the exact patterns and switches.
template <class A>
__global__ void __launch_bounds__(HIST_BINS) predict_kernel(const __grid_constant__ A a) {
  __shared__ uint32_t h[HIST_BINS];
  __shared__ uint32_t wm[HIST_BINS / 32];
  __shared__ EpiShared es;
  const int t = threadIdx.x;
  // An AUTO stream chains its launches (prediction, count, recount, the next
  // push's prediction) with programmatic dependent launch: this launch may
  // start while the work before it ends.  It reads the chunks only after
  // that work completes, unless the caller declared them complete, and it
  // waits before it reads or writes the stream's state.
  pdl_launch_dependents();
  if (!a.early) pdl_wait();
  const ChunkDesc d = a.c[blockIdx.x];
  h[t] = 0;
  __syncthreads();
  // the sample's vectors are counted from the chunk's first 16-byte
  // boundary (a sample of 256 vectors gains nothing from whole lines)
  const Split sp = split_bytes_at(d.in, d.n, 16);
  const uint4* body = reinterpret_cast<const uint4*>(d.in + sp.head);
  uint32_t sampled;
  if (sp.nvec >= kSampleVecs) {
    const uint4 q = ldg_stream(body + (size_t)t * sp.nvec / kSampleVecs);
    const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 16; ++k) atomicAdd(&h[(w4[k >> 2] >> (8 * (k & 3))) & 0xffu], 1u);
    sampled = 16 * kSampleVecs;
  } else {
    for (size_t i = t; i < sp.nvec; i += HIST_BINS) {
      const uint4 q = ldg_stream(body + i);
      const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int k = 0; k < 16; ++k) atomicAdd(&h[(w4[k >> 2] >> (8 * (k & 3))) & 0xffu], 1u);
    }
    count_edges_into(d.in, sp, h);
    sampled = d.n;
  }
  __syncthreads();
  pdl_wait();  // the stream's state is the work before's to write
  if (a.window > 1 && a.mode == HIST_MODE_AUTO) {
    // the window's prediction needs every sample (window_predict_kernel)
    const uint32_t slot = (uint32_t)((a.first_chunk + blockIdx.x) % kChunkRing);
    a.st->wsamp[slot][t] = h[t];
    if (t == 0) {
      a.st->wsn[slot] = sampled;
      a.st->wn[slot] = d.n;
    }
  }
  if (a.mode == HIST_MODE_AUTO) {
    const uint32_t m = __reduce_max_sync(0xffffffffu, h[t]);
    if ((t & 31) == 0) wm[t >> 5] = m;
    __syncthreads();
    if (t == 0) {
      uint32_t mx = 0;
#pragma unroll
      for (int i = 0; i < HIST_BINS / 32; ++i) mx = wm[i] > mx ? wm[i] : mx;
      a.st->rpred[(a.first_chunk + blockIdx.x) % kChunkRing] =
          reaches_theta(mx, sampled, a.theta) ? HIST_FLAG_ADAPTIVE : HIST_FLAG_PLAIN;
      if (blockIdx.x == 0) a.st->lk0[a.launch % kLaunchRing] = a.st->flag;  // chunk 0's kernel
    }
  }
  if (a.budget < HIST_BUDGET_MAX) {
    StreamDev* st = a.st;
    if (blockIdx.x == 0) copy_pattern(&st->ppat[a.first_chunk % kChunkRing], &st->pattern);
    if (blockIdx.x + 1 < a.count) {
      // the rule on the sample (proportions: its total is the sampled pixels;
      // an empty chunk gives the default pattern)
      hist_pattern& next = st->ppat[(a.first_chunk + blockIdx.x + 1) % kChunkRing];
      block_epilogue(h, sampled, a.budget, a.theta, next, es);
    }
  }
}

// A window of W > 1 chunks on the flat path.  The window histogram after
// chunk g is the sum of the histograms of chunks g-W+1 .. g (chunks before
// number 0 count as empty; chunks are numbered from the stream's first flat
// chunk, and a resumed stream restarts at 0).  The histograms of the last
// kChunkRing chunks stay in rings, so each chunk's window is summed on its
// own: one CTA per chunk of the batch, bin b in thread b, W loads per thread
// with eight in flight, then the window's largest bin and total.  (One CTA
// running through the chunks in order, adding chunk g and subtracting chunk
// g-W, took 90 us for the predictions and 27 us for the exact switches of a
// launch of 64 chunks at W = 32.)

// Largest bin and total of a 256-bin window held one bin per thread (all
// threads call; two barriers); returned to every thread.
template <class T>
__device__ __forceinline__ void window_max_sum(T v, T* smax, T* ssum, T& mx, T& sm) {
  const int b = threadIdx.x, w = b >> 5;
  T m = v, s = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T m2 = __shfl_xor_sync(0xffffffffu, m, o);
    m = m2 > m ? m2 : m;
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  if ((b & 31) == 0) {
    smax[w] = m;
    ssum[w] = s;
  }
  __syncthreads();
  mx = smax[0];
  sm = ssum[0];
#pragma unroll
  for (int i = 1; i < HIST_BINS / 32; ++i) {
    mx = smax[i] > mx ? smax[i] : mx;
    sm += ssum[i];
  }
  __syncthreads();
}

// Predicted window switches (AUTO): the same window over the chunks'
// samples, each scaled by its chunk's bytes over its sample's pixels, in
// FP32 (a prediction: FP64 is slow on this part, and a wrong guess costs a
// recount, never a wrong result).  CTA j: chunk g0 + j.
template <class A>
__global__ void __launch_bounds__(HIST_BINS) window_predict_kernel(const __grid_constant__ A a) {
  __shared__ float scale[HIST_WINDOW_MAX];
  __shared__ float smax[HIST_BINS / 32], ssum[HIST_BINS / 32];
  const StreamDev* st = a.st;
  const int b = threadIdx.x;
  // chained after the prediction (see predict_kernel): its samples first
  pdl_launch_dependents();
  pdl_wait();
  const unsigned long long W = a.window, g = a.first_chunk + blockIdx.x;
  const unsigned long long first = g >= W - 1 ? g - (W - 1) : 0ull;
  const uint32_t len = (uint32_t)(g - first + 1);
  // each window chunk's scale, one thread per chunk
  for (uint32_t k = (uint32_t)b; k < len; k += HIST_BINS) {
    const uint32_t slot = (uint32_t)((first + k) % kChunkRing);
    const uint32_t sn = __ldcg(&st->wsn[slot]);
    scale[k] = sn ? (float)__ldcg(&st->wn[slot]) / (float)sn : 0.0f;
  }
  __syncthreads();
  float v = 0.0f;
  for (uint32_t k0 = 0; k0 < len; k0 += 8) {
    uint32_t h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      h[k] = k0 + k < len ? __ldcg(&st->wsamp[(first + k0 + k) % kChunkRing][b]) : 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k0 + k < len) v += (float)h[k] * scale[k0 + k];
  }
  float mx, sm;
  window_max_sum(v, smax, ssum, mx, sm);
  if (b == 0)
    a.st->rpred[g % kChunkRing] = (sm > 0.0f && mx * 1000.0f >= sm * (float)a.theta) ? HIST_FLAG_ADAPTIVE : HIST_FLAG_PLAIN;
}

// Exact window switches after the flat launch, one CTA per chunk; the CTA
// of the last chunk writes the window after it.  The CTA that completes the
// launch's count then writes the stream's switch and last kernel and, in
// AUTO mode, lists the chunks whose predicted kernel was not the one their
// predecessor's window switch chose.
template <class A>
__global__ void __launch_bounds__(HIST_BINS) window_flat_kernel(const __grid_constant__ A a) {
  __shared__ unsigned long long smax[HIST_BINS / 32], ssum[HIST_BINS / 32];
  __shared__ int last;
  StreamDev* st = a.st;
  const int b = threadIdx.x;
  // chained after the counting launch (AUTO): its chunk histograms first
  pdl_launch_dependents();
  pdl_wait();
  const unsigned long long W = a.window, g0 = a.first_chunk, g = g0 + blockIdx.x;
  const unsigned long long first = g >= W - 1 ? g - (W - 1) : 0ull;
  const uint32_t len = (uint32_t)(g - first + 1);
  unsigned long long v = 0;
  for (uint32_t k0 = 0; k0 < len; k0 += 8) {
    uint32_t h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      h[k] = k0 + k < len ? __ldcg(&st->whist[(first + k0 + k) % kChunkRing][b]) : 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) v += h[k];
  }
  unsigned long long mx, sm;
  window_max_sum(v, smax, ssum, mx, sm);
  if (b == 0) st->rflag[g % kChunkRing] = reaches_theta(mx, sm, a.theta) ? HIST_FLAG_ADAPTIVE : HIST_FLAG_PLAIN;
  if (blockIdx.x + 1 == a.count) st->wmw[b] = v;
  const uint32_t ls = (uint32_t)(a.launch % kLaunchRing);
  __syncthreads();
  if (b == 0) {
    // the barrier orders the CTA's writes before this fence
    __threadfence();
    last = atomicAdd(&st->lwin[ls], 1u) + 1u == a.count;
  }
  __syncthreads();
  if (!last) return;
  // every chunk's switch is written (and fenced)
  __threadfence();
  uint32_t kern = a.mode == HIST_MODE_ADAPTIVE ? HIST_FLAG_ADAPTIVE : HIST_FLAG_PLAIN;
  if (a.mode == HIST_MODE_AUTO) {
    // chunk j's kernel had to be chunk j-1's window switch (chunk 0: the stream's)
    const uint32_t nr = redo_list(st, g0, a.count, ls, kern);
    if (b == 0) {
      st->lredo_n[ls] = nr;
      st->recounted += nr;
    }
  }
  if (b == 0) {
    st->flag = __ldcg(&st->rflag[(g0 + a.count - 1) % kChunkRing]);
    st->last_kernel = kern;
    st->lwin[ls] = 0;
  }
}

template <class A>
__global__ void __launch_bounds__(kThreads, 1) auto_redo_kernel(const __grid_constant__ A a) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* table = smem;
  uint32_t* lut = smem + kTableWords;  // slot table of a default-pattern layout, then scratch of the reduction
  __shared__ CtaShared cs;
  __shared__ EpiShared es;
  __shared__ int last;
  StreamDev* st = a.st;
  const uint32_t ls = (uint32_t)(a.launch % kLaunchRing);
  // chained after the counting launch (see predict_kernel)
  pdl_launch_dependents();
  pdl_wait();
  const uint32_t nr = st->lredo_n[ls];
  if (nr == 0) return;
  zero_table(table);
  __syncthreads();
  for (uint32_t r = 0; r < nr; ++r) {
    const uint32_t j = st->lredo[ls][r];  // never chunk 0: its kernel is known exactly
    const ChunkDesc d = a.c[j];
    const uint32_t slot = (uint32_t)((a.first_chunk + j) % kChunkRing);
    const uint32_t kern = st->rflag[(a.first_chunk + j - 1) % kChunkRing];
    // the adaptive kernel: at the full budget the full table after a
    // non-empty chunk, the default pattern after an empty one (with a window
    // of more than one chunk the switch can choose it there); below it, the
    // layout predict_kernel derived for the chunk
    int path = kern == HIST_FLAG_ADAPTIVE ? PATH_SHIFT : PATH_PLAIN;
    int lk = kern == HIST_FLAG_ADAPTIVE ? 5 : 0;
    if (kern == HIST_FLAG_ADAPTIVE && (a.budget < HIST_BUDGET_MAX || a.c[j - 1].n == 0)) {
      __syncthreads();
      if (a.budget < HIST_BUDGET_MAX) {
        copy_pattern_cg(&cs.pat, &st->ppat[slot]);
        __syncthreads();
      } else {
        saturated_pattern(0, a.budget, cs, es);
      }
      classify_pattern(cs.pat, lut, cs);
      path = cs.path;
      lk = cs.lk;
    }
    const Geo g = chunk_geo(d);
    count_call4(path, lk, g.body, g.begin, g.end, table, lut);
    const bool cleared = flush_table(path, lk, table, cs.pat, lut, cs, true);
    const Split sp = split_bytes(d.in, d.n);
    if (blockIdx.x == 0) {
      count_edges(d.in, sp, cs);
      __syncthreads();
    }
    if (!cleared) zero_table(table);
    const uint32_t mine = (g.end - g.begin) * 16u + (blockIdx.x == 0 ? (uint32_t)(sp.head + sp.tail) : 0u);
    if (threadIdx.x < HIST_BINS && cs.res[threadIdx.x]) atomicAdd(&st->racc[slot][threadIdx.x], cs.res[threadIdx.x]);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // after the barrier: publishes the CTA's adds before the byte count
      last = mine && atomicAdd(&st->rdone[slot], (unsigned long long)mine) + mine == d.n;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      if (threadIdx.x < HIST_BINS) {
        const uint32_t v = __ldcg(&st->racc[slot][threadIdx.x]);
        if (d.out) d.out[threadIdx.x] = v;
        st->racc[slot][threadIdx.x] = 0;
      }
      if (threadIdx.x == 0) st->rdone[slot] = 0;
    }
    __syncthreads();
  }
}

// Epilogue of the last pushed chunk (one CTA of 1024 threads).
// The moving-window histogram after the last chunk (none: zeros): the last
// chunk's histogram for a window of one, else the window kept by the flat
// launches.
__device__ __forceinline__ unsigned long long window_bin(const StreamDev* st, uint32_t window, bool any, int b) {
  if (!any) return 0ull;
  return window == 1 ? (unsigned long long)st->last_hist[b] : st->wmw[b];
}

__global__ void window_copy_kernel(const StreamDev* st, uint32_t window, bool any, unsigned long long* out) {
  const int b = threadIdx.x;
  if (b >= HIST_BINS) return;
  out[b] = window_bin(st, window, any, b);
}

// Change detection between the stream's totals and its moving-window
// histogram after the last chunk (256 threads).
__global__ void __launch_bounds__(HIST_BINS) stream_change_kernel(const StreamDev* st, uint32_t window, bool any,
                                                                  uint32_t tau_milli, hist_change_result* res) {
  __shared__ ChangeShared sh;
  const int b = threadIdx.x;
  const unsigned long long m = window_bin(st, window, any, b);
  const hist_change_result r = change_eval(st->totals[b], m, tau_milli, sh);
  if (b == 0) *res = r;
}

// The stream state of hist_stream_run_noalloc: one fixed array of the
// library (file scope, 256-byte aligned, sizeof(StreamDev) bytes), so that
// the call allocates no device memory.  Host code reaches it only through
// the address cudaGetSymbolAddress returns (noalloc_setup).
static __device__ __align__(256) StreamDev g_noalloc_state;

// The totals and status of a no-alloc run, to the caller's buffers.
__global__ void noalloc_out_kernel(const StreamDev* st, unsigned long long* totals, uint32_t* status) {
  const int b = threadIdx.x;
  if (b < HIST_BINS) totals[b] = st->totals[b];
  if (b == 0 && status) *status = st->status;
}

__global__ void init_kernel(StreamDev* st, uint32_t budget) {
  __shared__ CtaShared cs;
  __shared__ uint32_t zero[HIST_BINS];
  for (int i = threadIdx.x; i < HIST_BINS; i += blockDim.x) zero[i] = 0;
  __syncthreads();
  if (threadIdx.x < 32) warp_epilogue(zero, budget, HIST_THETA_MILLI_DEFAULT, cs.pat);
  __syncthreads();
  copy_pattern(&st->pattern, &cs.pat);
  copy_pattern(&st->last_pattern, &cs.pat);
}

}  // namespace

constexpr uint32_t kMaxStaging = 4;

struct hist_stream {
  hist_config cfg;
  StreamDev* d;
  int sms;
  int grid;
  unsigned long long chunks_launched;  // chunks pushed
  bool flat;   // batches run batch_flat_kernel
  bool autok;  // AUTO: predict, flat launch, recount
  bool predict;  // the layouts come from predict_kernel (adaptive kernel below the full budget)
  bool flat_full;  // the stream's pattern is the full table (known on the host)
  unsigned long long flat_launches;  // flat launches so far (scratch ring positions)
  unsigned long long flat_chunks;    // chunks of those launches
  unsigned long long resume_chunk;   // first chunk after the last set_state
  // tracing (optional)
  unsigned long long* trace;
  uint32_t trace_cap;
  uint32_t trace_next;
  // host-fed staging (optional)
  uint32_t depth;
  size_t max_chunk;
  uint8_t* staging[kMaxStaging];
  cudaEvent_t copied[kMaxStaging];
  cudaEvent_t consumed[kMaxStaging];
  cudaStream_t copy_stream;
  unsigned long long host_pushes;
  // the caller's device allocator (alloc null: cudaMalloc / cudaFree)
  hist_allocator alloc;
  // host buffer of a launch's parameters (null: one is allocated per launch)
  void* args;
};

namespace {

// Device memory of a stream: from the caller's allocator if it gave one.
int dev_alloc(hist_stream* st, void** p, size_t bytes) {
  *p = nullptr;
  if (!st->alloc.alloc) {
    const cudaError_t e = cudaMalloc(p, bytes);
    return e == cudaSuccess ? HIST_OK : (e == cudaErrorMemoryAllocation ? HIST_ENOMEM : cuda_fail(e));
  }
  void* q = st->alloc.alloc(bytes, st->alloc.ctx);
  if (!q) return HIST_ENOMEM;
  if ((uintptr_t)q % 256u) {
    st->alloc.free(q, bytes, st->alloc.ctx);
    return HIST_EINVAL;
  }
  *p = q;
  return HIST_OK;
}

void dev_free(hist_stream* st, void* p, size_t bytes) {
  if (!p) return;
  if (st->alloc.alloc) st->alloc.free(p, bytes, st->alloc.ctx);
  else cudaFree(p);
}

// A launch that may start while the work before it on `s` ends
// (programmatic dependent launch); the kernel waits (griddepcontrol.wait)
// before it reads what that work writes.
cudaError_t launch_chained(const void* fn, dim3 grid, dim3 block, void** params, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = grid;
  lc.blockDim = block;
  lc.dynamicSmemBytes = smem;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return cudaLaunchKernelExC(&lc, fn, params);
}

// Whether every chunk is at most kGroupChunkMax bytes: an AUTO launch of
// such chunks is split by the host, every chunk of weight 1 (the fixed
// costs dominate); with larger chunks the device's split, which weighs a
// chunk predicted to run the plain kernel twice, keeps the CTAs even
// (the degenerate workload in 16 MiB chunks, AUTO: 313 us per push with the
// weights, 399 us with every chunk of weight 1).
bool all_small(const size_t* ns, uint32_t count) {
  for (uint32_t i = 0; i < count; ++i)
    if (ns[i] > kGroupChunkMax) return false;
  return true;
}

// The host's copy of the CTAs' ranges of a flat launch, every chunk of cost
// weight 1: the batch's chunks placed end to end at their costs
// (flat_cost), total W; CTA b takes [W b / grid, W (b + 1) / grid)
// and starts at the last chunk whose cost position is at most the range's
// start -- what batch_flat_kernel's prefix and search compute otherwise
// (they read every chunk's size from the parameters: about 8 us per launch
// of 1024 chunks).
template <class A>
void flat_plan(A* a, uint32_t count, const size_t* ns, uint32_t grid) {
  unsigned long long W = 0;
  for (uint32_t i = 0; i < count; ++i) W += flat_cost(ns[i], 1, i, count);
  a->planned = 1;
  a->W = W;
  a->range = W / grid;
  uint32_t j = 0;
  unsigned long long pj = 0;  // cost position of chunk j
  for (uint32_t b = 0; b <= grid; ++b) {
    const unsigned long long lo = W * b / grid;
    a->plan_lo[b] = lo;
    if (b == grid) break;
    while (j + 1 < count && pj + flat_cost(ns[j], 1, j, count) <= lo) {
      pj += flat_cost(ns[j], 1, j, count);
      ++j;
    }
    a->plan_j[b] = (uint16_t)j;
    a->plan_pre[b] = pj;
  }
  // the chunks the groups take (group_chunk, on the host's copy of the sizes)
  const unsigned long long range = W / grid;
  auto whole = [&](uint32_t i) { return (unsigned long long)ns[i] * 4 <= range; };
  auto grouped = [&](uint32_t i) {
    if (ns[i] == 0 || ns[i] > kGroupChunkMax || i + 2 >= count || !whole(i)) return false;
    if (a->mode == HIST_MODE_PLAIN) return true;
    return a->budget == HIST_BUDGET_MAX && (i > 0 ? ns[i - 1] > 0 : a->chunk0_full != 0);
  };
  uint32_t i = 0;  // first chunk whose cost position is at least the range's start
  unsigned long long pi = 0;
  for (uint32_t b = 0; b <= grid; ++b) {
    const unsigned long long lo = a->plan_lo[b];
    while (i < count && pi < lo) {
      pi += flat_cost(ns[i], 1, i, count);
      ++i;
    }
    a->plan_s[b] = (uint16_t)i;
  }
  for (uint32_t b = 0; b < grid; ++b) {
    bool only = true;
    const uint32_t j0 = a->plan_j[b], s0 = a->plan_s[b], s1 = a->plan_s[b + 1];
    // a chunk that starts before the range and reaches into it
    for (uint32_t k = j0; k < s0 && only; ++k) only = whole(k);
    for (uint32_t k = s0; k < s1 && only; ++k) only = grouped(k);
    if (only) a->plan_groups[b >> 5] |= 1u << (b & 31);
  }
}

template <class A>
int launch_batch(hist_stream* st, uint32_t count, const uint8_t* const* ins, const size_t* ns, uint32_t* const* outs,
                 cudaStream_t s) {
  // the stream's parameter buffer: the header and the plan are cleared, the
  // chunk entries written (the launch copies the parameters)
  static_assert(sizeof(A) <= sizeof(LargeArgs), "one buffer for both parameter blocks");
  const bool own = st->args == nullptr;
  A* a = own ? (A*)calloc(1, sizeof(A)) : (A*)st->args;
  if (!a) return HIST_ENOMEM;
  if (!own) memset((void*)a, 0, offsetof(A, c));
  a->st = st->d;
  a->count = count;
  a->chunk0_full = st->flat_full ? 1u : 0u;
  a->first_chunk = st->flat_chunks;
  a->window = st->cfg.window;
  a->launch = st->flat_launches + 1;
  a->budget = st->cfg.budget;
  a->theta = st->cfg.theta_milli;
  a->mode = st->cfg.mode;
  a->trace = st->trace;
  a->trace_cap = st->trace_cap;
  a->trace_first = st->trace_next;
  a->early = (st->cfg.flags & HIST_OVERLAP_PUSHES) ? 1u : 0u;
  for (uint32_t i = 0; i < count; ++i) {
    a->c[i].in = ins[i];
    a->c[i].n = (uint32_t)ns[i];
    a->c[i].out = outs ? outs[i] : nullptr;
  }
  if (st->grid <= (int)kPlanCtas && (st->cfg.mode != HIST_MODE_AUTO || (st->cfg.window == 1 && all_small(ns, count))))
    flat_plan(a, count, ns, (uint32_t)st->grid);
  void* params[] = {a};
  cudaError_t e;
  const bool windowed = st->cfg.window > 1;
  if (st->autok && !windowed) {
    // predictions, the flat launch with the predicted kernels, the recount:
    // each may start while the one before ends (each waits for it before
    // it reads what that one writes)
    e = launch_chained((const void*)predict_kernel<A>, dim3(count), dim3(HIST_BINS), params, 0, s);
    if (e == cudaSuccess)
      e = launch_chained((const void*)batch_flat_kernel<A>, dim3((unsigned)st->grid), dim3(kThreads), params,
                         flat_smem_bytes<A>(), s);
    if (e == cudaSuccess)
      e = launch_chained((const void*)auto_redo_kernel<A>, dim3((unsigned)st->grid), dim3(kThreads), params,
                         kSmemBytes, s);
  } else if (st->autok) {
    // predictions, the window's prediction, the flat launch with the
    // predicted kernels, the window, the recount, chained the same way
    e = launch_chained((const void*)predict_kernel<A>, dim3(count), dim3(HIST_BINS), params, 0, s);
    if (e == cudaSuccess)
      e = launch_chained((const void*)window_predict_kernel<A>, dim3(count), dim3(HIST_BINS), params, 0, s);
    if (e == cudaSuccess)
      e = launch_chained((const void*)batch_flat_kernel<A>, dim3((unsigned)st->grid), dim3(kThreads), params,
                         flat_smem_bytes<A>(), s);
    if (e == cudaSuccess)
      e = launch_chained((const void*)window_flat_kernel<A>, dim3(count), dim3(HIST_BINS), params, 0, s);
    if (e == cudaSuccess)
      e = launch_chained((const void*)auto_redo_kernel<A>, dim3((unsigned)st->grid), dim3(kThreads), params,
                         kSmemBytes, s);
  } else if (st->flat && (windowed || st->predict)) {
    e = cudaSuccess;
    if (st->predict) e = cudaLaunchKernel((const void*)predict_kernel<A>, dim3(count), dim3(HIST_BINS), params, 0, s);
    if (e == cudaSuccess)
      e = cudaLaunchKernel((const void*)batch_flat_kernel<A>, dim3((unsigned)st->grid), dim3(kThreads), params,
                           flat_smem_bytes<A>(), s);
    if (e == cudaSuccess && windowed)
      e = cudaLaunchKernel((const void*)window_flat_kernel<A>, dim3(count), dim3(HIST_BINS), params, 0, s);
  } else {
    // PLAIN or ADAPTIVE at the full budget, window 1: one launch, which may
    // start while the previous launch on `s` finishes (see batch_flat_kernel)
    e = launch_chained((const void*)batch_flat_kernel<A>, dim3((unsigned)st->grid), dim3(kThreads), params,
                       flat_smem_bytes<A>(), s);
  }
  if (own) free(a);
  if (e != cudaSuccess) return cuda_fail(e);
  st->flat_launches += 1;
  st->flat_chunks += count;
  // at the full budget the pattern after a non-empty chunk is the full table
  // (the adaptive and AUTO modes; the plain mode never reads it)
  st->flat_full = st->cfg.mode != HIST_MODE_PLAIN && st->cfg.budget == HIST_BUDGET_MAX && ns[count - 1] > 0;
  st->chunks_launched += count;
  if (st->trace) st->trace_next += count;
  return HIST_OK;
}

int push_chunks(hist_stream* st, uint32_t count, const uint8_t* const* ins, const size_t* ns, uint32_t* const* outs,
                cudaStream_t s) {
  for (uint32_t i = 0; i < count; i += kMaxBatch) {
    const uint32_t c = count - i < kMaxBatch ? count - i : kMaxBatch;
    int rc = c <= kSmallBatch ? launch_batch<SmallArgs>(st, c, ins + i, ns + i, outs ? outs + i : nullptr, s)
                              : launch_batch<LargeArgs>(st, c, ins + i, ns + i, outs ? outs + i : nullptr, s);
    if (rc) return rc;
  }
  return HIST_OK;
}

bool config_ok(const hist_config* c) {
  return c && c->budget >= HIST_BUDGET_MIN && c->budget <= HIST_BUDGET_MAX && c->theta_milli <= 1000 &&
         c->mode <= HIST_MODE_ADAPTIVE && c->window >= 1 && c->window <= HIST_WINDOW_MAX &&
         (c->flags & ~HIST_OVERLAP_PUSHES) == 0;
}

int grid_for(const hist_config* cfg, int sms, const void* fn, size_t smem) {
  // every CTA that can be resident at once, or fewer if the caller asks
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int cap = per_sm * sms;
  const int g = cfg->grid ? (int)cfg->grid : cap;
  return g > cap ? cap : g;
}

// The counting kernels' shared-memory opt-in, once per (kernel, device).
int flat_kernels_setup() {
  static std::mutex mu;
  static int attr[4][kMaxDevices];
  std::lock_guard<std::mutex> lock(mu);
  int rc = ensure_smem_attr_bytes((const void*)batch_flat_kernel<SmallArgs>, attr[0], flat_smem_bytes<SmallArgs>());
  if (rc == HIST_OK)
    rc = ensure_smem_attr_bytes((const void*)batch_flat_kernel<LargeArgs>, attr[1], flat_smem_bytes<LargeArgs>());
  if (rc == HIST_OK) rc = ensure_smem_attr_bytes((const void*)auto_redo_kernel<SmallArgs>, attr[2], kSmemBytes);
  if (rc == HIST_OK) rc = ensure_smem_attr_bytes((const void*)auto_redo_kernel<LargeArgs>, attr[3], kSmemBytes);
  return rc;
}

// The grid of the counting launches (the larger variant's occupancy: the
// smaller one needs less shared memory).
int flat_grid(const hist_config* cfg, int sms) {
  return grid_for(cfg, sms, (const void*)batch_flat_kernel<LargeArgs>, flat_smem_bytes<LargeArgs>());
}

// Once per device, with that device current: the no-alloc state's device
// address and the counting kernels' shared-memory opt-in (none of it
// allocates).
int noalloc_setup(void** state) {
  static std::mutex mu;
  static void* ptr[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev < 0 || dev >= kMaxDevices) return HIST_EINVAL;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_state);
    if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    const int rc = flat_kernels_setup();
    if (rc) return rc;
    ptr[dev] = p;
  }
  *state = ptr[dev];
  return HIST_OK;
}

void release_staging(hist_stream* st) {
  for (uint32_t i = 0; i < kMaxStaging; ++i) {
    dev_free(st, st->staging[i], st->max_chunk);
    if (st->copied[i]) cudaEventDestroy(st->copied[i]);
    if (st->consumed[i]) cudaEventDestroy(st->consumed[i]);
    st->staging[i] = nullptr;
    st->copied[i] = st->consumed[i] = nullptr;
  }
  if (st->copy_stream) cudaStreamDestroy(st->copy_stream);
  st->copy_stream = nullptr;
  st->depth = 0;
  st->max_chunk = 0;
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
  c->window = 1;
}

int hist_stream_create(const hist_config* cfg, hist_stream** out) {
  return hist_stream_create_with_allocator(cfg, nullptr, out);
}

int hist_stream_create_with_allocator(const hist_config* cfg, const hist_allocator* alloc, hist_stream** out) {
  if (!out || !config_ok(cfg)) return HIST_EINVAL;
  *out = nullptr;
  if (alloc && (!alloc->alloc) != (!alloc->free)) return HIST_EINVAL;
  hist_stream* st = (hist_stream*)calloc(1, sizeof(hist_stream));
  if (!st) return HIST_ENOMEM;
  st->cfg = *cfg;
  if (alloc) st->alloc = *alloc;
  st->sms = sm_count();
  // AUTO adds the predicted switches and a recount; below the full budget
  // the adaptive kernel's layouts are predicted too; a window of more than
  // one chunk adds the window kernels
  st->flat = cfg->mode != HIST_MODE_AUTO;
  st->autok = cfg->mode == HIST_MODE_AUTO;
  st->predict = cfg->budget < HIST_BUDGET_MAX && cfg->mode != HIST_MODE_PLAIN;
  int rc = flat_kernels_setup();
  if (rc) {
    free(st);
    return rc;
  }
  st->grid = flat_grid(cfg, st->sms);
  rc = dev_alloc(st, (void**)&st->d, sizeof(StreamDev));
  if (rc) {
    free(st);
    return rc;
  }
  cudaError_t e = cudaMemset(st->d, 0, sizeof(StreamDev));
  if (e == cudaSuccess) {
    init_kernel<<<1, 256>>>(st->d, cfg->budget);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    dev_free(st, st->d, sizeof(StreamDev));
    free(st);
    return cuda_fail(e);
  }
  st->args = malloc(sizeof(LargeArgs));  // null: launches allocate their own
  *out = st;
  return HIST_OK;
}

int hist_stream_destroy(hist_stream* st) {
  if (!st) return HIST_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  release_staging(st);
  dev_free(st, st->d, sizeof(StreamDev));
  free(st->args);
  free(st);
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int hist_stream_push(hist_stream* st, const uint8_t* d_chunk, size_t n, uint32_t* d_chunk_out,
                     hist_cuda_stream s) {
  if (!st || (!d_chunk && n) || n >= ((size_t)1 << 32)) return HIST_EINVAL;
  return push_chunks(st, 1, &d_chunk, &n, d_chunk_out ? &d_chunk_out : nullptr, (cudaStream_t)s);
}

int hist_stream_push_many(hist_stream* st, uint32_t count, const uint8_t* const* d_chunks, const size_t* sizes,
                          uint32_t* const* d_chunk_outs, hist_cuda_stream s) {
  if (!st || (count && (!d_chunks || !sizes))) return HIST_EINVAL;
  for (uint32_t i = 0; i < count; ++i)
    if ((!d_chunks[i] && sizes[i]) || sizes[i] >= ((size_t)1 << 32)) return HIST_EINVAL;
  if (count == 0) return HIST_OK;
  return push_chunks(st, count, d_chunks, sizes, d_chunk_outs, (cudaStream_t)s);
}

int hist_stream_attach_staging(hist_stream* st, size_t max_chunk, uint32_t depth) {
  if (!st || max_chunk == 0 || max_chunk >= ((size_t)1 << 32) || depth < 2 || depth > kMaxStaging)
    return HIST_EINVAL;
  if (st->depth) return HIST_ESTATE;
  st->max_chunk = max_chunk;  // the staging buffers' size, also when they are freed
  int rc = HIST_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&st->copy_stream, cudaStreamNonBlocking);
  for (uint32_t i = 0; e == cudaSuccess && rc == HIST_OK && i < depth; ++i) {
    rc = dev_alloc(st, (void**)&st->staging[i], max_chunk);
    if (rc == HIST_OK) e = cudaEventCreateWithFlags(&st->copied[i], cudaEventDisableTiming);
    if (e == cudaSuccess && rc == HIST_OK) e = cudaEventCreateWithFlags(&st->consumed[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess || rc != HIST_OK) {
    release_staging(st);
    return rc != HIST_OK ? rc : (e == cudaErrorMemoryAllocation ? HIST_ENOMEM : cuda_fail(e));
  }
  st->depth = depth;
  st->host_pushes = 0;
  return HIST_OK;
}

int hist_stream_push_host(hist_stream* st, const uint8_t* h_chunk, size_t n, uint32_t* d_chunk_out,
                          hist_cuda_stream s) {
  if (!st || (!h_chunk && n)) return HIST_EINVAL;
  if (!st->depth) return HIST_ESTATE;
  if (n > st->max_chunk) return HIST_EINVAL;
  const uint32_t b = (uint32_t)(st->host_pushes % st->depth);
  cudaStream_t cs = st->copy_stream;
  // the buffer's previous chunk kernel must be done before it is overwritten
  cudaError_t e = cudaStreamWaitEvent(cs, st->consumed[b], 0);
  if (e == cudaSuccess && n) e = cudaMemcpyAsync(st->staging[b], h_chunk, n, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaEventRecord(st->copied[b], cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)s, st->copied[b], 0);
  if (e != cudaSuccess) return cuda_fail(e);
  const uint8_t* in = st->staging[b];
  int rc = push_chunks(st, 1, &in, &n, d_chunk_out ? &d_chunk_out : nullptr, (cudaStream_t)s);
  if (rc) return rc;
  e = cudaEventRecord(st->consumed[b], (cudaStream_t)s);
  if (e != cudaSuccess) return cuda_fail(e);
  st->host_pushes += 1;
  return HIST_OK;
}

int hist_stream_test_hold_ring(hist_stream* st, uint32_t launches) {
  if (!st || launches == 0 || launches > 1024) return HIST_EINVAL;
  // the next launch's number runs ahead of the launches the device has seen
  // complete, so its ring check waits for launches that never ran
  st->flat_launches += launches;
  return HIST_OK;
}

int hist_stream_trace(hist_stream* st, uint64_t* d_trace, uint32_t capacity_chunks) {
  if (!st || (d_trace && capacity_chunks == 0)) return HIST_EINVAL;
  st->trace = reinterpret_cast<unsigned long long*>(d_trace);
  st->trace_cap = d_trace ? capacity_chunks : 0;
  st->trace_next = 0;
  return HIST_OK;
}

int hist_stream_flush(hist_stream* st, hist_cuda_stream s) {
  (void)s;  // every push completes its chunks' epilogues in its own launches
  return st ? HIST_OK : HIST_EINVAL;
}

int hist_stream_totals(hist_stream* st, uint64_t* d_totals, hist_cuda_stream s) {
  if (!st || !d_totals) return HIST_EINVAL;
  const void* src = reinterpret_cast<const char*>(st->d) + offsetof(StreamDev, totals);
  cudaError_t e = cudaMemcpyAsync(d_totals, src, HIST_BINS * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)s);
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int hist_stream_window(hist_stream* st, uint64_t* d_window, hist_cuda_stream s) {
  if (!st || !d_window) return HIST_EINVAL;
  const bool any = st->chunks_launched > st->resume_chunk;
  window_copy_kernel<<<1, HIST_BINS, 0, (cudaStream_t)s>>>(st->d, st->cfg.window, any,
                                                            reinterpret_cast<unsigned long long*>(d_window));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int hist_stream_change(hist_stream* st, uint32_t tau_milli, hist_change_result* d_res, hist_cuda_stream s) {
  if (!st || !d_res || tau_milli > 1000) return HIST_EINVAL;
  const bool any = st->chunks_launched > st->resume_chunk;
  stream_change_kernel<<<1, HIST_BINS, 0, (cudaStream_t)s>>>(st->d, st->cfg.window, any, tau_milli, d_res);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int hist_stream_get_state(hist_stream* st, hist_stream_state* h, hist_cuda_stream s) {
  if (!st || !h) return HIST_EINVAL;
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
  h->recounted = tmp->recounted;
  free(tmp);
  return HIST_OK;
}

int hist_stream_set_state(hist_stream* st, const hist_stream_state* h, hist_cuda_stream s) {
  if (!st || !h) return HIST_EINVAL;
  if (hist_pattern_check(&h->pattern) != HIST_OK || hist_pattern_check(&h->last_pattern) != HIST_OK ||
      h->pattern.budget != st->cfg.budget || h->flag > HIST_FLAG_ADAPTIVE)
    return HIST_EINVAL;
  StreamDev* tmp = (StreamDev*)calloc(1, sizeof(StreamDev));
  if (!tmp) return HIST_ENOMEM;
  memcpy(tmp->totals, h->totals, sizeof(tmp->totals));
  memcpy(tmp->last_hist, h->last_hist, sizeof(tmp->last_hist));
  tmp->pattern = h->pattern;
  tmp->last_pattern = h->last_pattern;
  tmp->chunks = h->chunks;
  tmp->flag = h->flag;
  tmp->last_kernel = h->last_kernel;
  cudaError_t e = cudaMemcpyAsync(st->d, tmp, sizeof(StreamDev), cudaMemcpyHostToDevice, (cudaStream_t)s);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)s);
  free(tmp);
  st->flat_full = false;  // the next flat launch reads the restored pattern
  st->flat_launches = 0;   // the rings restart with the zeroed scratch
  st->flat_chunks = 0;
  st->resume_chunk = st->chunks_launched;  // and so does the moving window
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

int hist_stream_run_noalloc(const uint8_t* const* d_chunks, const size_t* sizes, uint32_t count,
                            const hist_config* cfg, uint32_t* d_chunk_outs, uint64_t* d_totals, uint32_t* d_status,
                            hist_cuda_stream s) {
  if (!cfg || !d_totals || count == 0 || count > HIST_NOALLOC_MAX_CHUNKS || !d_chunks || !sizes) return HIST_EINVAL;
  hist_config c = *cfg;
  c.grid = 0;  // ignored: the counting launch takes every resident CTA
  if (!config_ok(&c)) return HIST_EINVAL;
  for (uint32_t i = 0; i < count; ++i)
    if ((!d_chunks[i] && sizes[i]) || sizes[i] >= ((size_t)1 << 32)) return HIST_EINVAL;
  void* state = nullptr;
  int rc = noalloc_setup(&state);
  if (rc) return rc;
  // a fresh stream on the fixed state: the same launches as hist_stream_push_many
  hist_stream st;
  memset(&st, 0, sizeof(st));
  st.cfg = c;
  st.d = static_cast<StreamDev*>(state);
  st.sms = sm_count();
  st.flat = c.mode != HIST_MODE_AUTO;
  st.autok = c.mode == HIST_MODE_AUTO;
  st.predict = c.budget < HIST_BUDGET_MAX && c.mode != HIST_MODE_PLAIN;
  st.grid = flat_grid(&c, st.sms);
  uint32_t* outs[HIST_NOALLOC_MAX_CHUNKS];
  for (uint32_t i = 0; i < count; ++i) outs[i] = d_chunk_outs ? d_chunk_outs + (size_t)i * HIST_BINS : nullptr;
  cudaError_t e = cudaMemsetAsync(state, 0, sizeof(StreamDev), (cudaStream_t)s);
  if (e != cudaSuccess) return cuda_fail(e);
  init_kernel<<<1, 256, 0, (cudaStream_t)s>>>(st.d, c.budget);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e);
  rc = push_chunks(&st, count, d_chunks, sizes, outs, (cudaStream_t)s);
  if (rc) return rc;
  noalloc_out_kernel<<<1, HIST_BINS, 0, (cudaStream_t)s>>>(st.d, reinterpret_cast<unsigned long long*>(d_totals),
                                                           d_status);
  e = cudaGetLastError();
  return e == cudaSuccess ? HIST_OK : cuda_fail(e);
}

}  // extern "C"
