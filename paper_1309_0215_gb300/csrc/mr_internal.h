// Internal declarations shared by the CUDA translation units of libmrgb.so.
#pragma once
#include <utility>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "../../include/mr.h"
#include "dev_wordcount.cuh"

namespace mrgb {

// ---------------------------------------------------------------- helpers
void set_last_error(const char* where, cudaError_t e);

#define MR_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) {                                \
      ::mrgb::set_last_error(#expr, e_);                    \
      return MR_ECUDA;                                      \
    }                                                       \
  } while (0)

struct DevInfo {
  int sms = 0;
  int smem_optin = 0;   // max dynamic shared memory per block (opt-in)
  int l2_bytes = 0;
};

// ------------------------------------------------------------ array jobs
// RGB8 histogram, local arrays in shared memory ("lane-column" layout:
// bins x 32 u32 columns, one column per lane, shared by all warps of a CTA).
// bins must be zeroed before the launch.
cudaError_t launch_hist_smem(const uint8_t* in, uint64_t n, uint64_t* bins, int grid, cudaStream_t s);
// RGB8 histogram without local arrays: atomics straight on the global bins.
cudaError_t launch_hist_global(const uint8_t* in, uint64_t n, uint64_t* bins, int grid, cudaStream_t s);
// int8 regression sums; sums must be zeroed before the launch.
cudaError_t launch_linreg(const int8_t* in, uint64_t n, int64_t* sums, int grid, cudaStream_t s);
// Independent array jobs run as one launch (shared-memory histograms and
// regressions; at most ARRAY_FUSE_MAX).
constexpr int ARRAY_FUSE_MAX = 8;
struct ArrayJobs {
  uint32_t n;
  uint32_t kind[ARRAY_FUSE_MAX];
  const uint8_t* in[ARRAY_FUSE_MAX];
  uint64_t bytes[ARRAY_FUSE_MAX];
  void* out[ARRAY_FUSE_MAX];
};
cudaError_t launch_array_fused(const ArrayJobs& jobs, int grid, cudaStream_t s);

int hist_smem_bytes();         // dynamic shared memory the smem histogram needs
int hist_block_threads();

// ------------------------------------------------------ kernel timing
// Event pairs around each launch of a job's main kernel (the distance pass of
// every k-means iteration, the word-count map pass, the one counting kernel of
// the other kinds), recorded when the context times its jobs.  Events are
// created on first use; launches past MAX are not timed.
struct KTimer {
  static constexpr uint32_t MAX = 64;
  cudaEvent_t ev[2 * MAX] = {};
  uint32_t n = 0;  // launches timed in the current run
};
cudaError_t kt_begin(KTimer* t, cudaStream_t s);  // no-op for t == nullptr
cudaError_t kt_end(KTimer* t, cudaStream_t s);
void kt_destroy(KTimer* t);

// ------------------------------------------- large-key histogram, Bloom
// Largest bin count whose local arrays (nbins + 1 u32) fit one CTA, and a
// thread-block cluster of CTAs.
int hk_smem_max_bins(const DevInfo& di);
int hk_cluster_max_bins(const DevInfo& di);
// Histogram of n u32 keys into out[nbins + 1] (zeroed here).  container:
// MR_C_SMEM_ARRAY local arrays per CTA, MR_C_CLUSTER_ARRAY local arrays
// spread over a cluster's shared memory, else atomics on the global array.
// wide: count straight into the u64 output (needed from 2^32 keys on); else
// into the u32 counters (nbins + 1 words) and widen at the end.
cudaError_t launch_hist_keys(const uint32_t* keys, uint64_t n, uint32_t nbins, int container, void* counters,
                             bool wide, unsigned long long* out, const DevInfo& di, cudaStream_t s, uint64_t* nk,
                             KTimer* kt = nullptr);
// Bloom-filter build over n bases into ceil(m / 32) u32 words (zeroed here).
cudaError_t launch_bloom(const uint8_t* seq, uint64_t n, uint32_t L, uint64_t m, uint32_t h, uint32_t* bits,
                         const DevInfo& di, cudaStream_t s, uint64_t* nk, KTimer* kt = nullptr);

// --------------------------------------------------------- word count job
struct WcBuffers {
  uint64_t cap = 0;            // global hash-table slots (power of two)
  uint64_t* key = nullptr;     // [cap][2] 128-bit keys, {0, 0} = empty
  uint64_t* cnt = nullptr;     // [cap] combined counts (contiguous after key)
  uint32_t* state = nullptr;   // 64 bytes: word 0 overflow flag, 64-bit fields 1..4 post-phase bounds
  uint8_t* sortbuf = nullptr;  // post-phase scratch for cap records
  uint8_t* out = nullptr;      // result: header + records + key bytes
  uint64_t out_cap = 0;
};
uint64_t wc_table_bytes(uint64_t cap);
uint64_t wc_state_bytes();
size_t wc_sortbuf_bytes(uint64_t records);
uint64_t wc_out_bytes(uint64_t cap, uint64_t n);
int wc_map_smem_bytes();
uint64_t wc_compact_blocks(uint64_t cap);
wc::JobDev wc_job_dev(const uint8_t* in, uint64_t n, const WcBuffers& b, uint64_t blk0);
// Compaction, sort (by job, count desc, key asc), bounds and gather for
// njobs jobs (jobs: device array, or nullptr for one job; hjobs: the same
// descriptors in host memory, njobs of them).  sms sizes persistent grids.
cudaError_t launch_wordcount_post_multi(const wc::JobDev* jobs, const wc::JobDev* hjobs, uint32_t njobs,
                                        uint64_t nblocks, uint64_t records, uint8_t* sortbuf, int sms,
                                        cudaStream_t s, uint64_t* nk);
// Zero the table and state, run map+combine, compaction, sort and gather.
// *nk is incremented by the number of kernels launched.
// pipelined: the map pass runs as mapper warps handing cache misses to
// reducer warps through shared-memory rings (wc_pipe_kernel).
// pipe_polls: polls of the pipelined pass's bounded ring waits (< 0: default).
cudaError_t launch_wordcount(const uint8_t* in, uint64_t n, const WcBuffers& b, const DevInfo& di, cudaStream_t s,
                             uint64_t* nk, bool pipelined = false, KTimer* kt = nullptr, long long pipe_polls = -1);

// ---------------------------------------------------------------- k-means
// Programmatic dependent launch: the kernel may be scheduled while the
// kernel before it on the stream is still finishing (its launch and ramp
// overlap that kernel's tail); it must call pdl_wait() before touching any
// memory, which returns once the earlier kernel has completed and its writes
// are visible.  Used only for kernels that start with pdl_wait() and follow
// another kernel on the stream.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

struct KmBuffers {
  uint32_t n = 0, d = 0, k = 0;
  float* cent = nullptr;        // [k][d] current centroids (FP32 state)
  float* cent_bf16_norm = nullptr;
  int32_t* assign = nullptr;    // [n]
  long long* sums = nullptr;    // [k][d] fixed-point sums
  unsigned long long* counts = nullptr;  // [k]
  unsigned long long* stats = nullptr;   // [4]
  uint32_t* flagged = nullptr;  // [n] indices of points to re-check
  uint32_t* nflag = nullptr;    // [8] counters: [0] FP64 list, [1] FP32 list, [2] max|x| bits, [3] max||c|| bits, [4] pairs,
                                //     [5] points deferred to the FP64 stage
  uint32_t* deferred = nullptr; // [n] points whose choice needs the FP64 definition
  uint2* pairs = nullptr;       // [n] {point, k1 | k2 << 16}: exact choice between two centroids
  float* xnorm = nullptr;       // [n] ||x||
  float* cnorm = nullptr;       // [k] ||c|| and ||c||^2
  uint16_t* xb = nullptr;       // BF16 copy of the points [n][d]
  uint16_t* cb = nullptr;       // BF16 centroids [k][d]
  unsigned int* maxabs = nullptr;  // [1] bits of max |x|
  uint32_t* kcursor = nullptr;  // [k] counting-sort write cursors
  long long* part = nullptr;    // [CTAs][k][d] partial sums of the local-array update (nullptr: sort path)
  KTimer* kt = nullptr;         // times the distance pass of each iteration
  int fx_shift = 32;            // fixed-point scale exponent
  int precision = 0;
  // diagnostics (mr_set_option): polls of a bounded device wait (< 0: the
  // default), cap on the CTAs of the persistent kernels (0: none), tiles the
  // tensor-core kernel's bulk-copy thread stages per CTA (0: all)
  long long polls = -1;
  uint32_t grid_cap = 0;
  uint32_t stop_copies = 0;
};
size_t km_scratch_bytes(uint32_t n, uint32_t d, uint32_t k, int precision);
cudaError_t km_carve(KmBuffers& b, uint8_t* base, size_t bytes);
cudaError_t launch_kmeans(const float* x, const float* init, uint32_t iters, KmBuffers& b, const DevInfo& di,
                          cudaStream_t s, float* out_cent, int32_t* out_assign, unsigned long long* out_stats,
                          uint64_t* nk);
bool km_tc_supported(uint32_t d, uint32_t k);

// --------------------------------------------------------- batched launch
struct BatchJob {
  uint32_t kind;       // mr_kind
  uint32_t container;  // mr_container chosen
  const uint8_t* in;
  uint64_t n;
  void* out;           // histogram bins / regression sums
  wc::JobDev wc;       // word count
  uint64_t tile_begin; // first tile index of this job in the batch's tile space
  uint64_t ntiles;
  uint64_t zchunk0;    // first clearing chunk of this job's container (batch_zero_chunks)
};
cudaError_t batch_prepare();
// Zero the jobs' containers (total_zchunks chunks, see batch_zero_chunks),
// then run every tile in one persistent launch.
cudaError_t launch_batch(const BatchJob* jobs_dev, uint32_t njobs, uint64_t total_tiles, unsigned long long* cursor,
                         uint64_t arr_tile, uint64_t wc_tile, uint64_t total_zchunks, const DevInfo& di,
                         cudaStream_t s, uint64_t* nk);
uint64_t batch_tiles_for(uint32_t kind, uint64_t n, uint64_t arr_tile, uint64_t wc_tile);
// Chunks of BATCH_ZCHUNK bytes that clearing the job's container takes.
constexpr uint64_t BATCH_ZCHUNK = 64 * 1024;
uint64_t batch_zero_chunks(uint32_t kind, uint64_t wc_cap);

}  // namespace mrgb
