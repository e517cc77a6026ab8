/*
 * hist.h -- C ABI of the GB300 (sm_103a) library for exact 256-bin histograms
 * of 8-bit pixel streams, after "Fast Histograms using Adaptive CUDA Streams"
 * (Koppaka, Mudigere, Narasimhan, Narayanan; arXiv 1011.0235).
 *
 * The paper has three parts (Sec. III, Sec. IV):
 *   - a plain per-warp kernel (the NVIDIA SDK kernel it compares against,
 *     "NVHist") and an adaptive kernel ("AHist") that splits bins into
 *     sub-bins following a binning pattern (Sec. III.A);
 *   - a chunked stream that refreshes the binning pattern from the stream's
 *     own past histograms (Sec. III.B);
 *   - switching between the two kernels by the degeneracy of the last
 *     histogram (Sec. III.C).
 * Here all three run on the device: the pattern and the switch for chunk i+1
 * are computed by the kernels from chunk i's histogram, with no host round
 * trip.
 *
 * Conventions for every call below.
 *   - Pointers named d_* are device pointers (cudaMalloc, or any memory the
 *     device can address); h_* are host pointers.  The caller owns every
 *     buffer it passes; the library keeps no pointer past the call except
 *     where a call says so (stream and server objects).
 *   - `s` is a cudaStream_t.  Calls are asynchronous on `s` unless their name
 *     or comment says they synchronize.  Results are valid once `s` has
 *     reached the point of the call.
 *   - Return value: HIST_OK (0) or a negative HIST_E* code.  On an error
 *     nothing has been enqueued and no output has been written, except
 *     HIST_ECUDA, which reports a CUDA error raised while enqueuing
 *     (hist_last_cuda_error() returns it).
 *   - Histograms are uint32_t[256] (one chunk: n < 2^32 pixels) or
 *     uint64_t[256] (stream totals).  Bin b counts the pixels equal to b.
 *   - Input pointers may have any alignment and n may be any size (0
 *     included).
 */
#ifndef HIST_H
#define HIST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* hist_cuda_stream; /* the same type as cudaStream_t */

/* ---------------------------------------------------------------- codes -- */
#define HIST_OK 0
#define HIST_EINVAL (-1)    /* bad argument (null pointer, size, budget, mode ...) */
#define HIST_ENOMEM (-2)    /* a device or host allocation failed */
#define HIST_EBUDGET (-3)   /* admission: a request exceeds the server's byte budget */
#define HIST_ETIMEDOUT (-4) /* a bounded device or host wait ran out */
#define HIST_ECUDA (-5)     /* a CUDA call failed; see hist_last_cuda_error() */
#define HIST_EBUSY (-6)     /* no free slot right now; retry after a poll */
#define HIST_ESTATE (-7)    /* object in the wrong state for this call */

#define HIST_BINS 256
#define HIST_KMAX 32          /* sub-bins per bin: at most one per warp lane */
#define HIST_BUDGET_MIN 256   /* sub-bin table slots: one per bin ... */
#define HIST_BUDGET_MAX 8192  /* ... up to 32 per bin (a 32 KiB table) */
#define HIST_THETA_MILLI_DEFAULT 450 /* Sec. III.C: critical degeneracy 40-50 % */

#define HIST_FLAG_PLAIN 0u    /* the per-warp kernel (NVHist) */
#define HIST_FLAG_ADAPTIVE 1u /* the sub-binned kernel (AHist) */

const char* hist_strerror(int code);
/* The cudaError_t behind the last HIST_ECUDA returned on this thread. */
int hist_last_cuda_error(void);
/* Number of SMs the library sizes its grids for on the current device. */
int hist_device_sms(void);

/* ------------------------------------------------------ binning pattern -- */
/* Binning pattern (Sec. III.A, Figure 1): the sub-histogram table of the
 * adaptive kernel holds `used` slots; bin b owns the k_b = 2^log2k[b] slots
 * off[b] .. off[b]+k_b-1, and a pixel of value b read by warp lane l is
 * counted in slot off[b] + (l mod k_b) (sub-bins allotted to the lanes of a
 * warp cyclically, Sec. III.A).  The histogram is the per-bin sum of its
 * slots, so any valid pattern gives the exact histogram; the pattern only
 * changes speed.  Valid: log2k[b] <= 5, off[b] a multiple of k_b, the ranges
 * disjoint, used = sum k_b <= budget <= HIST_BUDGET_MAX.  776 bytes. */
typedef struct hist_pattern {
  uint16_t off[HIST_BINS];
  uint8_t log2k[HIST_BINS];
  uint32_t budget;
  uint32_t used;
} hist_pattern;

/* Host check of a host-resident pattern: HIST_OK or HIST_EINVAL. */
int hist_pattern_check(const hist_pattern* h_pat);

/* Device-side binning pattern from the previous histogram (Sec. III.B: the
 * sub-histogram indices are recomputed from the stream's past histograms; the
 * paper gives no formula, so the rule is this library's reading):
 *   T = sum h.  T = 0 gives default_pattern(budget).
 *   want_b = 1 + floor((budget - 256) * h_b / T)
 *   k0_b   = min(32, largest power of two <= want_b)
 *   f      = largest power of two <= 32 with sum_b max(f, k0_b) <= budget
 *   k_b    = max(f, k0_b)
 *   offsets: bins in order of decreasing k_b, ties by increasing b, packed
 *   from slot 0 (so off[b] is a multiple of k_b).
 * d_prev_hist: uint32_t[256] on the device.  d_pat: written.
 * budget outside [HIST_BUDGET_MIN, HIST_BUDGET_MAX] -> HIST_EINVAL. */
int binning_pattern(const uint32_t* d_prev_hist, uint32_t budget, hist_pattern* d_pat,
                    hist_cuda_stream s);

/* Default pattern for a stream's first chunk: the reading of Figure 1 as
 * eight regions of 32 bins with 1,2,4,8,8,4,2,1 sub-bins (960 slots, Sec.
 * III.A: 960 entries, 8 sub-bins at 127, 1 at the first bins), scaled by the
 * largest power of two s with 960 s <= budget (at most 32 per bin), or one
 * sub-bin per bin when budget < 960.  Written to d_pat on the device. */
int default_pattern(uint32_t budget, hist_pattern* d_pat, hist_cuda_stream s);

/* ------------------------------------------------------------ degeneracy -- */
/* Sec. III.C: degeneracy of a histogram = its largest bin over its total.
 * flag = HIST_FLAG_ADAPTIVE iff total > 0 and max * 1000 >= theta_milli *
 * total (exact integer compare), else HIST_FLAG_PLAIN.  maxbin is the lowest
 * bin holding the maximum (0 for an empty histogram). */
typedef struct hist_degeneracy_result {
  uint64_t max;
  uint64_t total;
  uint32_t maxbin;
  uint32_t flag;
} hist_degeneracy_result;

/* d_hist: uint32_t[256] / uint64_t[256] on the device; d_res written on the
 * device.  theta_milli > 1000 -> HIST_EINVAL. */
int degeneracy(const uint32_t* d_hist, uint32_t theta_milli, hist_degeneracy_result* d_res,
               hist_cuda_stream s);
int degeneracy_u64(const uint64_t* d_hist, uint32_t theta_milli, hist_degeneracy_result* d_res,
                   hist_cuda_stream s);

/* --------------------------------------------------------- one-shot kernels -- */
/* Plain per-warp kernel (NVHist, Sec. I and Table 2: one sub-histogram of 256
 * bins per warp in shared memory, merged per bin).  d_out: uint32_t[256],
 * overwritten.  n >= 2^32 -> HIST_EINVAL.  d_in may be null only if n == 0. */
int hist_plain(const uint8_t* d_in, size_t n, uint32_t* d_out, hist_cuda_stream s);

/* Adaptive kernel (AHist, Sec. III.A) with the device-resident pattern d_pat.
 * Same contract as hist_plain.  The pattern must be valid (as written by
 * binning_pattern / default_pattern, or checked with hist_pattern_check);
 * the kernel never addresses memory outside its own table whatever d_pat
 * holds, but an invalid pattern gives an unspecified histogram. */
int hist_adaptive(const uint8_t* d_in, size_t n, const hist_pattern* d_pat, uint32_t* d_out,
                  hist_cuda_stream s);

/* ------------------------------------------------------------- stream -- */
/* Chunked stream (Sec. III.B) with kernel switching (Sec. III.C).  The
 * stream keeps its state on the device: the running totals (the paper's
 * "Accumulator"), the last chunk's histogram, the pattern and the kernel the
 * next chunk will use.  Chunk i+1 uses the pattern and the switch computed
 * from chunk i's histogram (a moving window of one chunk).  The first chunk
 * runs the plain kernel with default_pattern(budget).
 *
 * The chunks of a push are counted back to back by one launch (one per
 * 1024 chunks), and each
 * chunk's exact switch and pattern are computed from its histogram in its
 * epilogue.  A chunk's counts do not depend on the kernel or the layout that
 * count it.  Where those depend on the previous chunk's histogram -- the
 * switch in AUTO mode, the pattern of the adaptive kernel below
 * HIST_BUDGET_MAX -- a launch before the count predicts them from a
 * 4096-pixel sample of the previous chunk; in AUTO mode a chunk whose
 * predicted kernel is not the one the switch chose is counted again with
 * that kernel (hist_stream_state.recounted), while a predicted layout that
 * differs from the exact pattern only costs speed.  At HIST_BUDGET_MAX the
 * layouts are known in advance (the rule gives the full table after every
 * non-empty chunk and the default pattern after an empty one) and are
 * checked against the exact patterns (status bit 8 otherwise). */
#define HIST_MODE_AUTO 0u     /* kernel chosen by the degeneracy switch */
#define HIST_MODE_PLAIN 1u    /* always the plain kernel (pattern still refreshed) */
#define HIST_MODE_ADAPTIVE 2u /* always the adaptive kernel */

/* Moving window (Sec. III.B: the accumulated histogram -- the stream
 * totals -- and the moving-window histogram; Sec. III.C: the switch follows
 * the last computed moving-window histogram).  The moving-window histogram
 * after chunk c is the sum of the histograms of chunks c-W+1 .. c (those that
 * exist), exact in uint64; the kernel of chunk c+1 in AUTO mode is its switch
 * (max bin * 1000 >= theta * total).  The binning pattern still comes from
 * chunk c alone.  W = 1 is the previous chunk. */
#define HIST_WINDOW_MAX 256u

/* hist_config.flags.
 * HIST_OVERLAP_PUSHES: the caller promises that the bytes of every chunk it
 * pushes are complete when the push is called -- written by work the host
 * has synchronised with (resident data, a synchronised copy or kernel).  A
 * push's counting launch may then begin reading its chunks while the work
 * before it on `s` (normally the stream's previous push) is still running,
 * so consecutive pushes overlap on the device.  Without the flag (default)
 * the counting launch still starts early and clears its tables, but reads
 * no chunk byte before the work before it on `s` has completed, so a chunk
 * written by the kernel just before the push -- even one that lets its
 * dependents start early -- is read whole.  The one-launch paths (PLAIN,
 * or ADAPTIVE at HIST_BUDGET_MAX, with a window of one chunk) overlap the
 * counting itself; an AUTO push (prediction, count, recount, chained the
 * same way) overlaps only its prediction's sampling with the work before
 * it, since the count needs the prediction; the other paths run after the
 * work before them. */
#define HIST_OVERLAP_PUSHES 1u

typedef struct hist_config {
  uint32_t budget;      /* sub-bin table slots, HIST_BUDGET_MIN..MAX (default MAX) */
  uint32_t theta_milli; /* critical degeneracy per mille, 0..1000 (default 450) */
  uint32_t mode;        /* HIST_MODE_* (default AUTO) */
  uint32_t grid;        /* CTAs of a push's counting launch; 0 = every CTA that can be resident */
  uint32_t window;      /* chunks in the moving window, 1..HIST_WINDOW_MAX (default 1) */
  uint32_t flags;       /* HIST_OVERLAP_PUSHES or 0 (default 0) */
  uint32_t reserved[2]; /* zero */
} hist_config;

void hist_config_init(hist_config* cfg);

typedef struct hist_stream hist_stream;

/* Allocates the stream's device state (about 15 MiB, cudaMalloc on the
 * current device: the state, the scratch rings of the one-launch paths and
 * the moving window's chunk histograms) and initialises it; synchronous (the
 * device is synchronized), so call it outside stream capture. */
int hist_stream_create(const hist_config* cfg, hist_stream** out);

/* A device-memory allocator of the caller's (a framework's caching
 * allocator, a pool).  alloc returns at least `bytes` bytes of device memory
 * on the current device, 256-byte aligned, or null when it has none; free
 * takes back a block with the size it was asked for.  Both are called only
 * from the host calls of the stream that uses them (create, attach_staging,
 * destroy), on the caller's thread. */
typedef struct hist_allocator {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* ctx);
  void* ctx; /* passed to both */
} hist_allocator;

/* hist_stream_create with the stream's device memory -- its state and any
 * staging buffers -- taken from `alloc` instead of cudaMalloc (alloc null:
 * hist_stream_create).  The allocator must stay valid until the stream is
 * destroyed.  HIST_ENOMEM when alloc returns null, HIST_EINVAL when it
 * returns a block that is not 256-byte aligned (the block is given back) or
 * when only one of alloc and free is set. */
int hist_stream_create_with_allocator(const hist_config* cfg, const hist_allocator* alloc, hist_stream** out);
/* Waits for the stream's work, frees its device state. */
int hist_stream_destroy(hist_stream* st);

/* Push one chunk (d_chunk, n pixels, n < 2^32).  d_chunk_out: optional
 * uint32_t[256] that receives the chunk's histogram, or null.  The chunk's
 * results (d_chunk_out, the totals, the next pattern and switch) are
 * complete once the push's own work on `s` is; the caller keeps d_chunk and
 * d_chunk_out alive until then.
 * Consecutive calls on one stream object must use the same `s`. */
int hist_stream_push(hist_stream* st, const uint8_t* d_chunk, size_t n, uint32_t* d_chunk_out,
                     hist_cuda_stream s);
/* Push `count` chunks in order; d_chunk_outs may be null (no per-chunk
 * outputs) or hold null entries. */
int hist_stream_push_many(hist_stream* st, uint32_t count, const uint8_t* const* d_chunks,
                          const size_t* sizes, uint32_t* const* d_chunk_outs, hist_cuda_stream s);
/* Kept for callers written against a deferred last epilogue: every push now
 * completes its own chunks, so this only checks its argument. */
int hist_stream_flush(hist_stream* st, hist_cuda_stream s);
/* Flush, then copy the running totals (uint64_t[256]) to d_totals. */
int hist_stream_totals(hist_stream* st, uint64_t* d_totals, hist_cuda_stream s);
/* Flush, then copy the moving-window histogram after the last pushed chunk
 * (uint64_t[256]; all zero before the first chunk) to d_window.  A stream
 * resumed with hist_stream_set_state restarts its window at that point. */
int hist_stream_window(hist_stream* st, uint64_t* d_window, hist_cuda_stream s);

/* Host-fed chunks (Sec. III.B: double-buffered transfers to the GPU overlapped
 * with the kernels).  attach_staging allocates `depth` (2..4) device staging
 * buffers of max_chunk bytes, an internal copy stream and events; call it
 * once, outside stream capture.  push_host copies h_chunk (n <= max_chunk; pin
 * it with cudaHostAlloc for the copy to overlap) into the next staging buffer
 * on the copy stream once the kernel that last read that buffer has finished,
 * makes `s` wait for the copy and pushes the staged chunk.  The caller may
 * reuse h_chunk once `s` has passed this call.  HIST_ESTATE without staging. */
int hist_stream_attach_staging(hist_stream* st, size_t max_chunk, uint32_t depth);
int hist_stream_push_host(hist_stream* st, const uint8_t* h_chunk, size_t n, uint32_t* d_chunk_out,
                          hist_cuda_stream s);

/* Tracing: the counting launch records %globaltimer (ns) for three CTAs
 * (the first, middle and last) into d_trace, a uint64_t array laid out
 * [chunk][3][8] for capacity_chunks chunks counted from this call; later
 * chunks are not recorded.  Each CTA counts a contiguous range of the
 * push's chunks placed end to end; a traced CTA records, for the chunks its
 * range touches, phase 0 (start of its piece of the chunk), 5 (its table
 * reduced) and 7 (end: its piece published, or the chunk's epilogue done),
 * and leaves the other entries unchanged.  d_trace null turns tracing off.
 * The caller keeps d_trace alive while tracing is on. */
int hist_stream_trace(hist_stream* st, uint64_t* d_trace, uint32_t capacity_chunks);

/* Test hook for the failure path of the one device wait: before a counting
 * launch adds into its scratch rings, its CTAs wait (bounded) until the
 * launch that last used those ring slots has finished.  This call makes the
 * stream's next launch wait for `launches` (1..1024) launches that never
 * run, so that wait runs out -- after a few seconds -- and the launch
 * completes with status bit 4 set in the stream state (its counts stay
 * exact: no other launch uses the rings).  Later launches do not wait.
 * HIST_EINVAL for a null stream or a count out of range. */
int hist_stream_test_hold_ring(hist_stream* st, uint32_t launches);

/* Stream state, for inspection and for checkpoint / resume. */
typedef struct hist_stream_state {
  uint64_t totals[HIST_BINS];   /* sum of all chunk histograms */
  uint32_t last_hist[HIST_BINS];/* histogram of the last chunk */
  hist_pattern pattern;         /* pattern the next chunk will be given */
  hist_pattern last_pattern;    /* pattern the last chunk was given */
  uint64_t chunks;              /* chunks completed */
  uint32_t flag;                /* switch from the last chunk (next kernel in AUTO) */
  uint32_t last_kernel;         /* kernel the last chunk ran */
  uint32_t status;              /* 0, or device-side error bits: 4 = a bounded wait
                                   ran out, 8 = a chunk's layout differed from the
                                   pattern rule (never expected) */
  uint32_t recounted;           /* AUTO streams: chunks counted a second time
                                   because their kernel was predicted from a
                                   sample that misjudged the chunk before */
  uint32_t reserved[6];
} hist_stream_state;

/* Copy the state to the host (after the stream's work on `s`) and
 * synchronize `s`. */
int hist_stream_get_state(hist_stream* st, hist_stream_state* h_state, hist_cuda_stream s);
/* Replace the stream's state (resume from a checkpoint); synchronizes `s`.
 * HIST_EINVAL if the state's patterns are invalid for this stream's budget. */
int hist_stream_set_state(hist_stream* st, const hist_stream_state* h_state, hist_cuda_stream s);

/* ---------------------------------------------------------------- batch -- */
/* Many histograms in one call (Sec. III.B: slices or packets too small for a
 * launch each are batched into one call that returns many histograms).
 * d_ptrs / d_sizes are DEVICE arrays of `count` image pointers and sizes
 * (each image below 2^32 bytes, any alignment); d_out is count x uint32_t[256]
 * on the device, overwritten: histogram i is d_out[256 i .. 256 i + 255].
 * Work: a memset of d_out and one kernel per HIST_BATCH_MAX_IMAGES images.
 * Each CTA takes an equal share of the images' concatenated bytes and counts
 * it in a lane-private sub-bin table (k = 32 sub-bins per bin), or with
 * 2^small_log2k sub-bins for images below small_bytes; a CTA adds into an
 * image's output where its share leaves the image.  No scratch memory. */
#define HIST_BATCH_MAX_IMAGES 4096u

typedef struct hist_batch_tuning {
  uint32_t ctas_per_sm; /* 1 or 2 (default 2) */
  uint32_t unroll;      /* 16-byte loads in flight per thread: 2 or 4 (4 needs ctas_per_sm 1; default 2) */
  uint32_t small_bytes; /* images below this size use small_log2k (default 0: none) */
  uint32_t small_log2k; /* 0..5 (default 5) */
  uint32_t reserved[4];
} hist_batch_tuning;

void hist_batch_tuning_init(hist_batch_tuning* t);
/* Enqueue the batch on `s`; tuning null = defaults.  HIST_EINVAL for a bad
 * tuning or null arrays with count > 0. */
int hist_batch(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t* d_out,
               const hist_batch_tuning* tuning, hist_cuda_stream s);

/* The same batch as an instantiated CUDA graph (memset + kernels), for
 * replaying over new contents of the same device arrays and buffers.  The
 * caller owns the graph (hist_batch_graph_destroy). */
typedef struct hist_batch_graph hist_batch_graph;
int hist_batch_capture(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t* d_out,
                       const hist_batch_tuning* tuning, hist_batch_graph** graph);
int hist_batch_graph_launch(hist_batch_graph* graph, hist_cuda_stream s);
int hist_batch_graph_destroy(hist_batch_graph* graph);

/* Autotuner: times every candidate setting (CTAs per SM, loads in flight,
 * sub-bins of small images) `repeats` times on this batch, synchronously, and
 * writes the fastest to *best (and its time in ms to *best_ms if not null).
 * d_out receives the batch's histograms. */
int hist_batch_autotune(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t* d_out,
                        uint32_t repeats, hist_batch_tuning* best, float* best_ms);

/* Batches tuned per distribution regime.  The autotuner keeps one setting
 * per regime of image (the paper has no autotuner: Sec. III.B batches small
 * slices into one call, and Sec. III.C chooses a kernel by degeneracy; the
 * regimes extend that choice to the batched call).  An image's regime comes
 * from a fixed sample of it:
 *   every pixel of an image of at most HIST_REGIME_SAMPLE (4096) pixels,
 *   else 256 runs of 16 consecutive pixels, run t starting at pixel
 *   floor(t n / 256); m = min(n, 4096) is the sample's size and h its 256-bin
 *   histogram.
 *   HIST_REGIME_DEGENERATE  max h * 1000 >= theta_milli * m (Sec. III.C's test)
 *   HIST_REGIME_PEAKED      otherwise, 64 * sum h^2 >= m^2: two sampled pixels
 *                           are equal with a chance of at least 1/64
 *   HIST_REGIME_WIDE        otherwise, and an empty image.
 * A setting names the layout an image of the regime is counted with: a
 * shift layout with 2^layout sub-bins per bin (0..5; 5 = the lane-private
 * table) or HIST_LAYOUT_PER_WARP (one 256-bin table per warp, the NVHist
 * layout), with a second layout for the regime's images below small_bytes
 * (whose table is cleared and reduced for few pixels).  Every layout gives
 * the exact histogram; the setting changes speed only. */
#define HIST_REGIMES 3u
#define HIST_REGIME_DEGENERATE 0u
#define HIST_REGIME_PEAKED 1u
#define HIST_REGIME_WIDE 2u
#define HIST_REGIME_SAMPLE 4096u
#define HIST_LAYOUT_PER_WARP 6u

typedef struct hist_regime_setting {
  uint32_t layout;       /* 0..5 or HIST_LAYOUT_PER_WARP */
  uint32_t small_bytes;  /* images of the regime below this size use small_layout (0: none) */
  uint32_t small_layout; /* 0..5 or HIST_LAYOUT_PER_WARP */
  uint32_t reserved;
} hist_regime_setting;

typedef struct hist_batch_table {
  uint32_t ctas_per_sm; /* 1 or 2, for the whole launch (default 2) */
  uint32_t unroll;      /* 2 or 4 loads in flight per thread (4 needs ctas_per_sm 1; default 2) */
  uint32_t theta_milli; /* the classifier's degeneracy threshold, 0..1000 (default 450) */
  uint32_t reserved;
  hist_regime_setting regime[HIST_REGIMES]; /* default: layout 5 for every regime, no small cut */
} hist_batch_table;

void hist_batch_table_init(hist_batch_table* t);

/* The regime of each image (rule above): d_regime is a device array of
 * `count` bytes, overwritten.  One kernel (a CTA per image, 4096 sampled
 * bytes at most).  theta_milli > 1000 or null arrays with count > 0 ->
 * HIST_EINVAL. */
int hist_batch_classify(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t theta_milli,
                        uint8_t* d_regime, hist_cuda_stream s);

/* hist_batch with a per-regime table: a memset of d_out, hist_batch_classify
 * into d_regime (count bytes on the device, the caller's; the regimes stay
 * there), then one counting kernel per HIST_BATCH_MAX_IMAGES images in which
 * each image is counted with its regime's setting.  No other device memory.
 * table null = hist_batch_table_init.  HIST_EINVAL for a bad table. */
int hist_batch_regimes(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count, uint32_t* d_out,
                       uint8_t* d_regime, const hist_batch_table* table, hist_cuda_stream s);

/* The same as an instantiated CUDA graph (memset, classification, counting),
 * destroyed with hist_batch_graph_destroy. */
int hist_batch_regimes_capture(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count,
                               uint32_t* d_out, uint8_t* d_regime, const hist_batch_table* table,
                               hist_batch_graph** graph);

/* What hist_batch_autotune_regimes measured (milliseconds, CUDA events,
 * mean of the repeats). */
typedef struct hist_regime_report {
  uint32_t images[HIST_REGIMES];      /* images of each regime */
  uint32_t candidates;                /* settings timed per regime */
  uint64_t bytes[HIST_REGIMES];       /* their bytes */
  float ms[HIST_REGIMES];             /* the regime's images alone, chosen setting */
  float ms_default[HIST_REGIMES];     /* the same images, the default setting (layout 5) */
  float batch_ms;                     /* the whole batch, chosen table */
  float batch_default_ms;             /* the whole batch, hist_batch_table_init */
  uint32_t reserved[4];
} hist_regime_report;

/* Autotuner, one setting per regime: classifies the batch (into d_regime),
 * then for each regime times every candidate setting (layouts per-warp and
 * 0..5, each with no small cut or a small cut at 64 KiB / 1 MiB with a
 * smaller layout) on that regime's images alone, `repeats` times each, and
 * keeps the fastest; then times the whole batch with the chosen settings
 * for each launch shape (CTAs per SM, loads in flight) and keeps the
 * fastest.  Synchronous; allocates temporary device arrays for the
 * sub-batches (freed before it returns).  Writes the table to *best and the
 * times to *report (may be null); d_out receives the batch's histograms
 * under the chosen table.  repeats 0 = 3. */
int hist_batch_autotune_regimes(const uint8_t* const* d_ptrs, const size_t* d_sizes, uint32_t count,
                                uint32_t* d_out, uint8_t* d_regime, uint32_t repeats, hist_batch_table* best,
                                hist_regime_report* report);

/* ------------------------------------------------ stream without allocation -- */
/* The paper has no counterpart of this call: it serves callers that cannot
 * allocate device memory where they need histograms -- code running while a
 * CUDA graph is being captured, real-time loops in which a cudaMalloc would
 * stall on a device-wide synchronisation, and hosts whose device memory
 * belongs to another allocator that must see every allocation.
 *
 * Runs a fresh stream (first chunk plain with default_pattern(cfg->budget),
 * then the switch and pattern of every chunk from the previous one, as
 * hist_stream_push does) over `count` chunks and writes, in order on `s`:
 *   d_chunk_outs  optional, count x uint32_t[256]: each chunk's histogram;
 *   d_totals      uint64_t[256]: the sum of the chunk histograms (overwritten);
 *   d_status      optional uint32_t: 0, or 4 if a bounded device wait ran out.
 * d_chunks / sizes are host arrays of `count` device pointers and sizes; each
 * size is below 2^32, and count is 1..HIST_NOALLOC_MAX_CHUNKS (more ->
 * HIST_EINVAL).  cfg->grid is ignored; cfg->window is honoured as by
 * hist_stream_create.
 *
 * It allocates no device memory (no cudaMalloc, cudaFree or other device
 * allocator): it runs the same launches as hist_stream_push_many on a stream
 * state -- about 15 MiB -- that is one fixed device array in the library,
 * held by every GPU that loads the library until the process exits, and
 * cleared and initialised on `s` at the start of every call.  The first call
 * on a device looks up that array's device address and sets the kernels up;
 * make that first call before any stream capture.  All calls share the
 * array: calls whose work overlaps on the GPU (on different streams, or from
 * several threads) race and give wrong results; run them in order on one
 * stream. */
#define HIST_NOALLOC_MAX_CHUNKS 128u
int hist_stream_run_noalloc(const uint8_t* const* d_chunks, const size_t* sizes, uint32_t count,
                            const hist_config* cfg, uint32_t* d_chunk_outs, uint64_t* d_totals,
                            uint32_t* d_status, hist_cuda_stream s);

/* ------------------------------------------------------ change detection -- */
/* Sec. III.B keeps an accumulated histogram and a moving-window histogram and
 * compares them to detect a change in the stream; it gives no rule.  The rule
 * here: the total-variation distance between the two histograms normalised
 * to sum 1, 1/2 sum_b |acc_b / sum(acc) - win_b / sum(win)|, against a
 * threshold tau (per mille; change iff distance >= tau / 1000), evaluated
 * exactly in 128-bit integers while sum(acc) < 2^56 and sum(win) < 2^40
 * (in_range says so; beyond it the result is unspecified).  Either histogram
 * empty: distance 0. */
#define HIST_CHANGE_TAU_MILLI_DEFAULT 250u

typedef struct hist_change_result {
  uint64_t dist_ppm; /* floor(10^6 x distance) */
  uint32_t flag;     /* 1: distance >= tau */
  uint32_t in_range; /* 1: the sums were within the exact range */
} hist_change_result;

/* d_acc, d_win: uint64_t[256] on the device; d_res: one result on the device. */
int hist_change(const uint64_t* d_acc, const uint64_t* d_win, uint32_t tau_milli, hist_change_result* d_res,
                hist_cuda_stream s);
/* Flush, then compare the stream's totals with its moving-window histogram. */
int hist_stream_change(hist_stream* st, uint32_t tau_milli, hist_change_result* d_res, hist_cuda_stream s);

/* ------------------------------------------------------------- ablation -- */
/* The adaptive kernel built up in Table 1's five cumulative steps, for
 * measuring what each step costs (with d_pat null: the per-warp kernel):
 *   1  read every packed pixel, write a 256-word result per CTA;
 *   2  + clear the shared sub-histogram;
 *   3  + read the binning pattern and compute every pixel's sub-bin address;
 *   4  + the shared-memory increments;
 *   5  + sum the sub-bins per bin and write the histogram (= hist_adaptive,
 *        or hist_plain without a pattern);
 *   6  stage 5 with warp-aggregated increments (the lanes holding one value
 *        elect a leader, which adds the group's size);
 *   7  stage 5 with the input staged through shared memory by 1-D bulk
 *        copies (cp.async.bulk into two 16 KiB buffers per CTA, completion
 *        on mbarriers) instead of each thread's own 16-byte loads.
 * Stages 5-7 overwrite d_out (uint32_t[256]); stages 1-4 write
 * hist_ablation_grid(n) x 256 words of scratch to d_sink, contents
 * unspecified.  Stage 7 takes d_sink as an optional status word: 0, or 1 if
 * an mbarrier wait ran out (bounded; the histogram is then incomplete).
 * n < 2^32; HIST_EINVAL for a bad stage or a missing buffer. */
int hist_ablation_grid(size_t n);
int hist_ablation(const uint8_t* d_in, size_t n, const hist_pattern* d_pat, uint32_t stage, uint32_t* d_out,
                  uint32_t* d_sink, hist_cuda_stream s);

/* --------------------------------------------------------------- server -- */
/* A serving loop (Sec. III.B's stream, for many independent streams whose
 * chunks arrive as requests).  Each of `streams` streams keeps its adaptive
 * state on the device -- totals, last histogram, the switch flag, the next
 * binning pattern and its layout -- so request j of stream s runs the kernel
 * and pattern chosen from request j-1 of s, exactly as hist_stream_push would
 * on a stream of its own (first request: plain kernel, default pattern).
 *
 * Continuous batching on the host (no device-side waits):
 *   submit  queues a request (FIFO); nothing is enqueued on the GPU.
 *   poll    writes one hist_completion per request that has finished since
 *           the last poll -- a request's epilogue on the GPU writes its
 *           completion word in pinned host memory once the request's output
 *           is written, so a request completes without waiting for the rest
 *           of its batch; it then updates the stream's state and writes the
 *           request's state word, and poll gives a returned request's stream
 *           back to admission once that word is seen -- and releases the
 *           batch slots whose completion event has fired (with them, their
 *           bytes of the budget); then it admits the next batch if one of
 *           max_inflight batch slots is free: in FIFO order, every queued
 *           request whose stream has no request on the GPU and whose bytes
 *           fit the HBM budget (bytes of all requests on the GPU <=
 *           hbm_budget), up to max_batch requests.  The batch is one kernel
 *           on the slot's own CUDA stream, so batches overlap on the device:
 *           a stream's next request may run in a batch that starts while its
 *           previous request's batch is still counting.
 *   drain   polls until nothing is queued or in flight (bounded by
 *           timeout_ms; HIST_ETIMEDOUT when it runs out).
 * A request's bytes (d_in, n < 2^32, any alignment) must stay valid and
 * unchanged, and d_out (uint32_t[256], or null) untouched, until its
 * completion has been returned by poll.  d_in is device memory, or pinned
 * host memory mapped into the device's address space: the batch kernels
 * then read the bytes over the host link (the host-fed variant).  The server owns its device state;
 * one host thread at a time may call it.  Results are exact: a request's
 * histogram and the stream's state do not depend on what else shares its
 * batch.  Any CUDA error is returned by the poll or drain that sees it. */
#define HIST_SERVER_MAX_STREAMS 4096u
#define HIST_SERVER_MAX_BATCH 1024u
#define HIST_SERVER_MAX_INFLIGHT 8u

typedef struct hist_server_config {
  uint32_t streams;        /* independent streams, 1..HIST_SERVER_MAX_STREAMS (default 256) */
  uint32_t max_batch;      /* requests per batch, 1..HIST_SERVER_MAX_BATCH (default 256) */
  uint32_t max_inflight;   /* batches on the GPU at once, 1..HIST_SERVER_MAX_INFLIGHT (default 4) */
  uint32_t theta_milli;    /* degeneracy threshold (default 450) */
  uint32_t pattern_budget; /* sub-bin table slots of every stream's patterns (default 8192) */
  uint32_t mode;           /* HIST_MODE_* for every stream (default AUTO) */
  uint64_t hbm_budget;     /* admission budget: request bytes on the GPU (default 32 GiB) */
  uint32_t reserved[4];
} hist_server_config;

typedef struct hist_server_stats {
  uint64_t submitted;      /* requests submitted */
  uint64_t completed;      /* requests returned by poll */
  uint64_t bytes;          /* bytes of the completed requests */
  uint64_t batches;        /* batches launched */
  uint64_t queued;         /* requests waiting now */
  uint64_t inflight_bytes; /* request bytes on the GPU now */
  uint64_t deferred;       /* admissions that skipped a request for the byte budget */
  uint64_t reserved[5];
} hist_server_stats;

/* One finished request.  Times are CLOCK_MONOTONIC nanoseconds (in
 * hist_server_replay: from the start of the replay). */
typedef struct hist_completion {
  uint64_t tag;       /* the caller's tag */
  uint32_t stream;
  uint32_t status;    /* 0 */
  uint64_t bytes;
  uint64_t submit_ns; /* submitted (replay: scheduled arrival) */
  uint64_t admit_ns;  /* its batch was launched */
  uint64_t done_ns;   /* poll saw the request complete */
} hist_completion;

typedef struct hist_server hist_server;

void hist_server_config_init(hist_server_config* c);
/* Allocates the per-stream state, max_inflight batch slots (about 1.1 MiB of
 * device memory each) and their CUDA streams, and 64 KiB of pinned, mapped
 * host memory for the requests' completion and state words; synchronizes
 * the device.  HIST_EINVAL for a bad config. */
int hist_server_create(const hist_server_config* cfg, hist_server** out);
/* Waits for the GPU, then frees everything. */
int hist_server_destroy(hist_server* srv);
/* Queue a request: the next chunk of stream `stream`.  HIST_EBUDGET if n
 * alone exceeds the HBM budget (it could never be admitted). */
int hist_server_submit(hist_server* srv, uint32_t stream, const uint8_t* d_in, size_t n, uint32_t* d_out,
                       uint64_t tag);
/* Return finished requests (at most `cap` completions are written; the rest
 * stay for the next poll), release finished batches and admit one batch.
 * *n_done = completions written. */
int hist_server_poll(hist_server* srv, hist_completion* h_done, uint32_t cap, uint32_t* n_done);
/* Poll until idle; timeout_ms 0 = no limit.  Completions are discarded. */
int hist_server_drain(hist_server* srv, uint32_t timeout_ms);
/* Drain, then copy stream `stream`'s state to the host (status is 0). */
int hist_server_stream_state(hist_server* srv, uint32_t stream, hist_stream_state* h_state);
int hist_server_get_stats(hist_server* srv, hist_server_stats* h_stats);

/* Replay a schedule in real time on the calling thread: request i is
 * submitted once arrival_ns (ns after the start of the call, non-decreasing)
 * has passed, and the loop polls until every request has completed and
 * every batch has retired (the server is idle again when it returns);
 * h_done[i] receives request i's completion (tag = the request's tag).
 * Latency of request i = h_done[i].done_ns - h_done[i].submit_ns.
 * timeout_ms bounds the whole replay (0 = no limit). */
typedef struct hist_request {
  uint64_t arrival_ns;
  uint32_t stream;
  uint32_t reserved;
  const uint8_t* d_in;
  uint64_t n;
  uint32_t* d_out;
  uint64_t tag;
} hist_request;

int hist_server_replay(hist_server* srv, const hist_request* h_reqs, uint32_t count, hist_completion* h_done,
                       uint32_t timeout_ms);

#ifdef __cplusplus
}
#endif
#endif
