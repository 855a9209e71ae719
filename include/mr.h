/*
 * mr.h — C ABI of the GB300 fused map-and-reduce library (libmrgb.so).
 *
 * The library runs MapReduce jobs whose map and reduce functions are built
 * in ("functor pairs"), following the programming model of arXiv:1309.0215
 * Sec. II-A: map is applied to every element of an input array and emits
 * intermediate key/value pairs; reduce folds all values that share a key; the
 * result pairs may be ordered.  Every emitted pair is combined at once into a
 * container (Sec. III-A "Efficient combiners"): an array for integer keys in
 * a fixed range, a hash table for open-ended keys (Sec. III-A "Hash table and
 * array containers").  Whether per-worker (here: per-CTA shared-memory) local
 * arrays are kept or eliminated in favour of atomics on the global array is
 * decided automatically from the container's footprint (Sec. III-E, last
 * paragraph), unless the caller pins a container.
 *
 * Conventions
 *  - All pointers are plain host or device addresses; no framework types.
 *  - Every call returns an mr_status; no exception or longjmp crosses the ABI.
 *  - A context is single-threaded: calls on one mr_ctx must not overlap.
 *    Different contexts may be used from different threads.
 *  - Work is enqueued on the context's CUDA stream; mr_run returns before the
 *    GPU finishes.  mr_fetch / mr_poll / mr_sync observe completion.
 *  - Status MR_ECUDA means a CUDA call failed; mr_last_error() gives the text.
 */
#ifndef MR_H_
#define MR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MR_OK = 0,
  MR_EINVAL = 1,      /* bad argument (null pointer, bad size, bad enum) */
  MR_ENOMEM = 2,      /* device or host allocation failed */
  MR_ECUDA = 3,       /* a CUDA runtime/driver call failed */
  MR_EOVERFLOW = 4,   /* a caller-pinned hash container was too small */
  MR_ETIMEOUT = 5,    /* a bounded device wait gave up */
  MR_EBUDGET = 6,     /* the job does not fit the context's HBM budget */
  MR_ENOTREADY = 7,   /* the job has not finished yet (mr_poll) */
  MR_ENOJOB = 8       /* unknown or released job id */
} mr_status;

/* Built-in map/reduce functor pairs. */
typedef enum {
  /* Word Count (paper Table I, hash-table container).  Input: bytes.  map:
   * a token is a maximal run of bytes that are not ASCII whitespace
   * (' ', \t, \n, \v, \f, \r); each emits (token, 1).  reduce: sum.
   * Output ordered by count descending, then key bytes ascending (unsigned,
   * a proper prefix first). */
  MR_WORDCOUNT = 0,
  /* Histogram (paper Table I, array container) over interleaved R,G,B bytes:
   * byte 3p+c emits (c*256 + value, 1).  Input length must be a multiple of
   * 3.  Output: 768 uint64 bins, bins[c*256 + v]. */
  MR_HIST_RGB8 = 1,
  /* Linear-regression sums over int8 pairs (x = b[2i], y = b[2i+1]); five
   * fixed keys.  Input length must be even.  Output: int64 {Σx, Σy, Σx²,
   * Σy², Σxy}. */
  MR_LINREG_I8 = 2,
  /* k-means (Lloyd) over FP32 points [n][km_dims]: km_iters rounds of
   * assign-to-nearest-centroid (squared Euclidean, the lowest index wins an
   * exact tie) then centroid = mean of assigned points (an empty cluster keeps
   * its centroid).  The key is the cluster id (array container of K*D sums +
   * K counts).  Assignments equal FP64 argmin; centroids are FP64 means
   * rounded to FP32; points must be finite (other values give unspecified
   * results).  Output layout (packed): float centroids[K][D], int32
   * assign[n], zero padding to an 8-byte boundary, uint64 stats[4] =
   * {points whose fast-pass result was re-checked (FP32 direct differences),
   * points of those that needed the FP64 definition, iterations, device
   * waits that timed out (0 unless mr_fetch returned MR_ETIMEOUT)}, summed
   * over the iterations. */
  MR_KMEANS_F32 = 3,
  /* Large-key histogram (the paper's Histogram application with 16M unique
   * keys, Sec. IV data sets; array container without local arrays,
   * Sec. III-E).  Input: uint32 keys (input_bytes a multiple of 4, a device
   * input 4-byte aligned); key k < hist_bins emits (k, 1), any other key
   * (hist_bins, 1).  Output: uint64 bins[hist_bins + 1]. */
  MR_HIST_U32 = 4,
  /* Bloom-filter build (the paper's Bloom Filter application: k-mers of a
   * chromosome, 30M elements into 300M entries, Sec. IV data sets; array
   * container without local arrays, Sec. III-E).  Input: ASCII bases.  Each
   * window of bloom_kmer bytes that are all 'A','C','G','T' is one element
   * with code = base-4 number of the window (A=0 .. T=3, first base most
   * significant).  With mix = the SplitMix64 output function, a = mix(code)
   * mod m and b = 1 + mix(code ^ 0x9E3779B97F4A7C15) mod (m - 1), the element
   * sets bits (a + i*b) mod m for i < bloom_hashes (m = bloom_bits).  Output:
   * ceil(m / 8) bytes, bit j = bit (j mod 8) of byte j / 8. */
  MR_BLOOM_DNA = 5
} mr_kind;

typedef enum {
  MR_C_AUTO = 0,          /* let the library choose (paper Sec. III-E rule) */
  MR_C_SMEM_ARRAY = 1,    /* local arrays in shared memory, flushed to the global array */
  MR_C_GLOBAL_ARRAY = 2,  /* no local arrays: atomics straight on the global array */
  MR_C_HASH = 3,          /* global open-addressing hash table */
  MR_C_CLUSTER_ARRAY = 4  /* large-key histogram only, never chosen by
                             MR_C_AUTO: local arrays spread over the shared
                             memory of a thread-block cluster of 8 CTAs
                             (distributed shared memory), one slice of the
                             bins per CTA; up to 8 x (opt-in shared memory /
                             4) - 1 bins */
} mr_container;

typedef enum {
  MR_RUN_PLAIN = 0,       /* one launch sequence per job, in submission order */
  MR_RUN_BATCHED = 1,     /* all pending array/hash jobs in one persistent launch */
  MR_RUN_CONCURRENT = 2   /* the jobs of the run (independent by construction)
                           * run concurrently: 2 to 8 shared-memory RGB
                           * histograms and int8 regressions as one fused
                           * launch on the context stream (each job's kernel
                           * time is that launch's); otherwise one launch
                           * sequence per job on internal streams forked from
                           * and joined back into the context stream */
} mr_mode;

typedef enum {
  MR_KM_FP32 = 0,         /* FP32 SIMT distances, exact re-check of near ties */
  MR_KM_BF16_TC = 1,      /* BF16 tensor-core distance GEMM (tcgen05, FP32
                             accumulate) on split operands x = hi + lo (three
                             BF16 products), FP32 then FP64 re-check of near
                             ties; D <= 64, K <= 256 */
  MR_KM_BF16X1_TC = 2     /* as MR_KM_BF16_TC with a single BF16 product (more
                             points fall back to the FP32 re-check) */
} mr_km_precision;

typedef struct mr_ctx mr_ctx;

typedef struct {
  uint32_t struct_size;   /* sizeof(mr_config) */
  int device;             /* CUDA device ordinal */
  void* cuda_stream;      /* cudaStream_t to enqueue on; NULL = library-owned stream */
  uint64_t hbm_budget;    /* max device bytes held by this context; 0 = unlimited */
  /* Optional device allocator (e.g. a framework's caching allocator).  When
   * alloc is NULL the library allocates stream-ordered (cudaMallocFromPoolAsync
   * on its stream) from a memory pool of its own, which keeps freed memory
   * for reuse until mr_destroy (so a job's containers cost no new mapping
   * after the first use).  alloc returns NULL on failure; free must accept
   * any pointer alloc returned. */
  void* (*alloc)(void* user, size_t bytes);
  void (*free)(void* user, void* ptr);
  void* alloc_user;
  uint32_t flags;         /* MR_FLAG_* bits */
} mr_config;

/* mr_config.flags: record CUDA timing events around each job's kernels so
 * that mr_job_elapsed_ms can report the job's device time. */
#define MR_FLAG_TIMING 1u
/* mr_config.flags: on the first batched mr_run of a context, time candidate
 * tile sizes and histogram container thresholds on the pending batch itself
 * and keep the fastest (see mr_get_tuning). */
#define MR_FLAG_AUTOTUNE 2u

/* Batched-launch parameters chosen by the autotuner (or the defaults). */
typedef struct {
  uint64_t arr_tile;           /* bytes per tile of histogram / regression jobs (multiple of 1536) */
  uint64_t wc_tile;            /* bytes per tile of word-count jobs (multiple of 512) */
  uint64_t hist_global_below;  /* histogram jobs smaller than this use global atomics (no local arrays) */
  float best_ms;               /* device time of the batch with these values (0 if not tuned) */
  uint32_t tuned;              /* 1 once the autotuner has run */
} mr_tuning;

typedef struct {
  uint32_t struct_size;   /* sizeof(mr_job_desc) */
  mr_kind kind;
  const void* input;      /* job input (host or device address) */
  uint64_t input_bytes;
  int input_on_device;    /* 1: device pointer, borrowed until the job completes;
                             0: host pointer, copied before mr_add_job returns */
  mr_container container; /* MR_C_AUTO unless the caller pins one */
  /* k-means only */
  uint32_t km_dims;       /* D */
  uint32_t km_k;          /* K */
  uint32_t km_iters;      /* number of Lloyd rounds (no early stop) */
  const float* km_init;   /* K*D initial centroids; same memory space as input */
  uint32_t km_precision;  /* mr_km_precision */
  /* word count only: initial hash-table slots (power of two, 0 = automatic) */
  uint64_t wc_slots;
  /* large-key histogram only: number of bins, >= 1 */
  uint32_t hist_bins;
  /* Bloom filter only: bases per element (1..32), bits set per element
   * (1..32) and filter size in bits (2..2^32) */
  uint32_t bloom_kmer;
  uint32_t bloom_hashes;
  uint64_t bloom_bits;
  /* word count only, plain runs: 1 = pipelined map and reduce (mapper warps
   * hand the keys their local cache cannot hold to reducer warps through
   * shared-memory rings, paper Sec. III-D); 0 = each warp inserts its own
   * misses.  Results are identical. */
  uint32_t wc_pipelined;
} mr_job_desc;

/* Create a context on cfg->device.  *out receives the handle.  A context is
 * the runtime that carries jobs through the basic workflow of Sec. II-A
 * (Fig. 1: split, map, partition, reduce, merge) on one GPU; it owns the
 * stream, the containers of its jobs and their results.
 * Errors: MR_EINVAL (null, bad struct_size, bad device), MR_ECUDA. */
mr_status mr_create(const mr_config* cfg, mr_ctx** out);

/* Destroy a context: waits for its work, frees every job and container. */
void mr_destroy(mr_ctx* ctx);

/* Validate a job, choose its container, reserve its device memory (and copy a
 * host input to the device) and queue it for the next mr_run.  A job is the
 * paper's MapReduce job (Sec. II-A "Programming model": an input array and a
 * map/reduce function pair, here a built-in mr_kind); the container choice
 * is the automatic detection of Sec. III-E unless desc->container pins one.
 * *job_id receives an id > 0.  Errors: MR_EINVAL, MR_ENOMEM, MR_EBUDGET,
 * MR_ECUDA. */
mr_status mr_add_job(mr_ctx* ctx, const mr_job_desc* desc, uint64_t* job_id);

/* Enqueue every pending job on the context stream: the map phase (split of
 * the input over CTAs and warps, map with its combiner into local
 * containers), the reduce into the global container, and the merge and
 * optional ordering of the result (Sec. II-A workflow, Fig. 1; Sec. III-A
 * combiners and containers).  PLAIN launches each job's kernels in order; BATCHED runs all pending word-count / RGB-histogram /
 * regression jobs in one persistent kernel, followed by one merge + sort for
 * all word-count jobs, captured as one CUDA graph (k-means, large-key
 * histogram and Bloom-filter jobs always run plain, after the batch).
 * Returns when the work is enqueued (an autotuning run waits).  Jobs that
 * could not be launched (MR_ENOMEM, MR_EBUDGET, MR_ECUDA on the way) stay
 * pending for the next mr_run. */
mr_status mr_run(mr_ctx* ctx, mr_mode mode);

/* Copy a finished job's result into host memory buf (buf_bytes long): the
 * output of the workflow's last step (Sec. II-A: the merged result pairs,
 * ordered where the kind orders them; layouts under mr_kind).
 * Blocks until the job is done.  With buf == NULL only *needed is set (the
 * result size in bytes).  A word-count job whose automatic hash table
 * overflowed is re-run with a larger table inside this call.
 * Errors: MR_ENOJOB, MR_EINVAL (buf too small), MR_EOVERFLOW, MR_ECUDA. */
mr_status mr_fetch(mr_ctx* ctx, uint64_t job_id, void* buf, uint64_t buf_bytes, uint64_t* needed);

/* Device address and size of a finished job's result (valid until
 * mr_release).  Blocks until the job is done (same rules as mr_fetch). */
mr_status mr_result_device(mr_ctx* ctx, uint64_t job_id, const void** dptr, uint64_t* bytes);

/* Re-run, in place, the jobs of the last batched mr_run (same inputs;
 * results are recomputed and overwritten) by relaunching the CUDA graph
 * captured for that batch (captured again first if a job's hash table was
 * regrown since).  Errors: MR_ENOJOB if one of those jobs was released,
 * MR_EINVAL if there was no batched run. */
mr_status mr_rerun(mr_ctx* ctx);

/* Current batched-launch parameters of the context. */
mr_status mr_get_tuning(const mr_ctx* ctx, mr_tuning* out);

/* Free a job's containers and result (the global container of Sec. III-A
 * and the merged output).  Waits for the job if it is running. */
mr_status mr_release(mr_ctx* ctx, uint64_t job_id);

/* Serving (not in the paper, whose runtime runs one job at a time; it is the
 * continuous-batching request loop this library adds around the Sec. II-A
 * workflow): admit a request if the context's HBM budget allows (MR_EBUDGET
 * otherwise; nothing is queued and the caller retries once results have been
 * released).  Admitted k-means, large-key histogram and Bloom requests are
 * launched at once, round robin on three internal streams.  The others are
 * batched continuously: whenever one of four further internal streams (at
 * the higher stream priority) has finished its previous micro-batch, every
 * admitted word-count, histogram and regression request that is not running
 * yet is launched on it as one persistent batch (plus one merge + sort for
 * its word-count requests).  Requests that arrive while others run are
 * therefore picked up as soon as a stream frees, and micro-batches overlap
 * on the device.  mr_poll and mr_fetch also drive this launching.
 * Containers stay resident until mr_release. */
mr_status mr_submit(mr_ctx* ctx, const mr_job_desc* desc, uint64_t* job_id);

/* Serving companion of mr_submit (no counterpart in the paper): MR_OK when
 * the job has finished, MR_ENOTREADY while it runs; also launches admitted
 * requests as streams free up. */
mr_status mr_poll(mr_ctx* ctx, uint64_t job_id);

/* Wait for all work enqueued on the context. */
mr_status mr_sync(mr_ctx* ctx);

/* Device bytes currently held by the context's jobs. */
uint64_t mr_bytes_in_use(const mr_ctx* ctx);

/* Diagnostic options of a context (none is part of the paper's method).
 * They reach code paths that ordinary runs reach only at full size or on a
 * failure, so that tests can check them on small inputs.  An option applies
 * to the jobs launched after it is set. */
typedef enum {
  /* Polls a bounded device wait makes before it gives up: the mbarrier
   * waits of the k-means bulk-copy and tensor-core pipelines (default 2^20
   * polls of at most 1 us each) and the ring waits of the pipelined word
   * count (default 2^22 polls of ~128 ns).  value = UINT64_MAX restores the
   * default; 0 gives up at the first wait, so the job's mr_fetch returns
   * MR_ETIMEOUT.  At most 2^40. */
  MR_OPT_WAIT_POLLS = 0,
  /* Upper bound on the CTAs of the k-means persistent kernels (0 = none: one
   * CTA, or two, per SM), so that a small input runs many tiles per CTA and
   * reaches the pipelines' steady state. */
  MR_OPT_KM_GRID_CAP = 1,
  /* k-means tensor-core pass: tiles each CTA's bulk-copy thread stages before
   * it stops (0 = no limit).  The waits for the tiles it never stages run
   * out (after MR_OPT_WAIT_POLLS polls) while earlier tiles are still in the
   * pipeline, so the kernel's timeout path runs with copies and MMAs in
   * flight; mr_fetch returns MR_ETIMEOUT. */
  MR_OPT_KM_STOP_COPIES = 2
} mr_option;

/* Set a diagnostic option.  Errors: MR_EINVAL (null context, unknown
 * option, value out of range). */
mr_status mr_set_option(mr_ctx* ctx, mr_option opt, uint64_t value);

/* Device time in milliseconds between the start and the end of a finished
 * job's kernel sequence on the context stream (the context must have been
 * created with MR_FLAG_TIMING).  Blocks until the job is done.
 * Errors: MR_ENOJOB, MR_ENOTREADY (not run yet), MR_EINVAL (no timing). */
mr_status mr_job_elapsed_ms(mr_ctx* ctx, uint64_t job_id, float* ms);

/* Device time of a finished job's main kernel: *ms = the summed duration of
 * its launches, *launches = how many were timed.  The main kernel is the
 * distance (assignment) pass of each k-means iteration, the map pass of a
 * word count, and the one counting kernel of the other kinds; each launch is
 * bracketed by CUDA events on the stream it runs on (up to 64 launches per
 * job are timed).  Needs MR_FLAG_TIMING; blocks until the job is done.
 * Errors: MR_ENOJOB, MR_ENOTREADY (not run yet), MR_EINVAL (no timing, or a
 * job of the batched launch, whose kernels are shared by all its jobs). */
mr_status mr_job_kernel_ms(mr_ctx* ctx, uint64_t job_id, float* ms, uint32_t* launches);

/* Number of CUDA kernels this context has launched so far (all jobs). */
uint64_t mr_kernel_launches(const mr_ctx* ctx);

/* SIMD hashing of variable-length strings (the paper's SIMDH-Padding and
 * SIMDH-Stream, Sec. III-C, with warp lanes as the SIMD lanes): the 64-bit
 * FNV-1a hash (offset basis 0xcbf29ce484222325, prime 0x100000001b3, one
 * byte at a time) of each of ntok tokens.  Token i is the tok_len[i] bytes
 * at text + tok_off[i]; every token must lie inside the text, and
 * text_bytes < 2^32.  All pointers are device addresses (text needs no
 * alignment); hashes[i] receives token i's hash.  method: */
#define MR_SIMDH_PADDING 0  /* 32 consecutive tokens per warp round, one per lane; rounds = longest, shorter lanes masked */
#define MR_SIMDH_STREAM 1   /* a lane that finishes takes the next token at once (ballot + prefix count refill) */
#define MR_SIMDH_WIDE 2     /* Padding's grouping, four bytes per load through a funnel shift */
/* Enqueued on cuda_stream (NULL = the legacy default stream); returns once
 * launched.  Errors: MR_EINVAL (bad method or size, null pointer),
 * MR_ECUDA. */
mr_status mr_simdh_hash(const uint8_t* text, uint64_t text_bytes, const uint32_t* tok_off, const uint32_t* tok_len,
                        uint64_t ntok, int method, uint64_t* hashes, void* cuda_stream);

/* Word count that allocates no device memory (the paper has no counterpart;
 * this is a deployment convenience).
 *
 * Who needs it: callers that cannot call cudaMalloc — for example a host
 * program that reserves the GPU's memory up front for its own pool and does
 * not let other components allocate, or a latency-critical loop that cannot
 * accept the implicit synchronisation and unpredictable cost of cudaMalloc
 * and cudaFree.  The job's hash table and sort scratch live in a fixed
 * device array inside the library (about 19 MiB, sized for
 * MR_NOALLOC_WC_SLOTS table slots) that every GPU loading the library holds
 * until the process exits.
 *
 * Arguments: d_input / input_bytes = the text in device memory (borrowed);
 * d_out = caller-owned device buffer of out_cap bytes, which must be at
 * least 16 + 24 * MR_NOALLOC_WC_SLOTS + input_bytes; on success *out_bytes
 * is the size of the result written to d_out, in the MR_WORDCOUNT layout;
 * cuda_stream = cudaStream_t to run on (NULL = the legacy default stream).
 * The call blocks until the job has finished on that stream.
 *
 * The first call on a device looks up the device address of the scratch
 * array (with that device current); make that first call before any stream
 * capture.  Every call on a device shares the same array, and each call
 * clears it before use: calls whose work overlaps on the GPU (other threads
 * or streams) race and give wrong results.
 *
 * Errors: MR_EINVAL (null pointer, out_cap too small, input_bytes >=
 * 2^40 - 1), MR_EOVERFLOW (more distinct words than the fixed table holds;
 * the result is then invalid), MR_ECUDA. */
#define MR_NOALLOC_WC_SLOTS 131072u
mr_status mr_wordcount_noalloc(const void* d_input, uint64_t input_bytes, void* d_out, uint64_t out_cap,
                               uint64_t* out_bytes, void* cuda_stream);

const char* mr_status_str(mr_status s);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char* mr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MR_H_ */
