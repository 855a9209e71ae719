// Host runtime behind the C ABI in include/mr.h: contexts, jobs, the
// container planner (paper Sec. III-E automatic detection), plain and batched
// launch sequencing, result fetch, and HBM-budget admission for serving.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "mr_internal.h"

namespace mrgb {

static thread_local std::string g_last_error;

void set_last_error(const char* where, cudaError_t e) {
  g_last_error = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

cudaError_t kt_begin(KTimer* t, cudaStream_t s) {
  if (!t || t->n >= KTimer::MAX) return cudaSuccess;
  cudaEvent_t* ev = t->ev + 2 * t->n;
  cudaError_t e = cudaSuccess;
  if (!ev[0]) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess && !ev[1]) e = cudaEventCreate(&ev[1]);
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
  return e;
}

cudaError_t kt_end(KTimer* t, cudaStream_t s) {
  if (!t || t->n >= KTimer::MAX) return cudaSuccess;
  const cudaError_t e = cudaEventRecord(t->ev[2 * t->n + 1], s);
  if (e == cudaSuccess) ++t->n;
  return e;
}

void kt_destroy(KTimer* t) {
  if (!t) return;
  for (cudaEvent_t& e : t->ev)
    if (e) cudaEventDestroy(e);
  delete t;
}

}  // namespace mrgb

using namespace mrgb;

namespace {

enum JobState { JOB_PENDING = 0, JOB_ENQUEUED = 1, JOB_SERVE_QUEUED = 2 };

struct Job {
  uint64_t id = 0;
  mr_job_desc desc{};
  mr_container container = MR_C_AUTO;
  JobState state = JOB_PENDING;
  const uint8_t* in = nullptr;   // device input
  void* in_owned = nullptr;      // device copy of a host input
  uint64_t in_owned_bytes = 0;
  void* slab = nullptr;          // containers + scratch + result
  uint64_t slab_bytes = 0;
  void* result = nullptr;
  uint64_t result_bytes = 0;     // fixed-size kinds
  cudaEvent_t done = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;  // timing events (MR_FLAG_TIMING)
  KTimer* kt = nullptr;                     // main-kernel launches (MR_FLAG_TIMING)
  // word count
  WcBuffers wc;
  bool wc_auto = true;
  // large-key histogram: u32 counters (null: count straight into the u64 result)
  void* hk_counters = nullptr;
  // k-means
  KmBuffers km;
  float* km_init_dev = nullptr;
  void* km_init_owned = nullptr;
};

}  // namespace

struct mr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  DevInfo di;
  void* (*alloc)(void*, size_t) = nullptr;
  void (*free_fn)(void*, void*) = nullptr;
  void* alloc_user = nullptr;
  // without a caller allocator: the context's own stream-ordered pool, whose
  // release threshold keeps freed memory mapped for reuse (the default pool
  // returns it to the system at every synchronisation)
  cudaMemPool_t pool = nullptr;
  uint64_t budget = 0;
  uint64_t in_use = 0;
  uint32_t flags = 0;
  uint64_t launches = 0;
  uint64_t next_id = 1;
  std::map<uint64_t, Job*> jobs;
  std::vector<uint64_t> pending;
  // batched launch scratch and the last batch's graph
  void* batch_desc = nullptr;
  uint64_t batch_desc_bytes = 0;
  void* batch_wc = nullptr;
  uint64_t batch_wc_bytes = 0;
  void* batch_sort = nullptr;
  uint64_t batch_sort_bytes = 0;
  void* batch_cursor = nullptr;
  cudaGraphExec_t batch_exec = nullptr;
  std::vector<uint64_t> batch_ids;
  uint64_t batch_launches = 0;  // kernels per replay of the graph
  mr_tuning tune{1536ull * 2048, 512ull * 2048, 0, 0.f, 0};  // the autotuner's usual choice on GB300
  // serving: continuous batching over a few internal streams ("slots")
  struct Slot {
    cudaStream_t s = nullptr;
    cudaEvent_t busy = nullptr;
    bool used = false;
    void* desc = nullptr;
    uint64_t desc_bytes = 0;
    void* wcd = nullptr;
    uint64_t wcd_bytes = 0;
    void* sort = nullptr;
    uint64_t sort_bytes = 0;
    void* cursor = nullptr;
  };
  static constexpr int SERVE_SLOTS = 4;
  Slot slots[SERVE_SLOTS];
  // plain-only requests (k-means, large-key histogram, Bloom) need no slot:
  // they run on these streams, round robin, beside the micro-batches (three:
  // more k-means jobs interleaved only stretch each one's latency)
  static constexpr int SERVE_AUX = 3;
  cudaStream_t serve_aux[SERVE_AUX] = {};
  uint32_t serve_aux_next = 0;
  std::vector<Job*> serve_pending;  // admitted, waiting for a free slot
  cudaEvent_t serve_ready = nullptr;
  // concurrent runs: jobs after the first run on these streams,
  // forked from and joined back into the context stream
  static constexpr int PLAIN_AUX = 3;
  cudaStream_t plain_aux[PLAIN_AUX] = {};
  cudaEvent_t plain_fork = nullptr;
  cudaEvent_t plain_join[PLAIN_AUX] = {};
  // CUDA events and kernel timers of released (finished) jobs, reused by
  // later jobs so that adding a job creates none in the steady state
  std::vector<cudaEvent_t> ev_done, ev_timing;
  std::vector<KTimer*> kt_pool;
  // diagnostics (mr_set_option), applied to jobs when they are launched
  long long opt_polls = -1;       // bounded device waits: polls (< 0: default)
  uint32_t opt_km_grid_cap = 0;   // k-means persistent kernels: CTA cap (0: none)
  uint32_t opt_km_stop_copies = 0;  // k-means tensor-core kernel: tiles staged per CTA (0: all)
};

namespace {

cudaError_t pooled_event(mr_ctx* c, bool timing, cudaEvent_t* e) {
  std::vector<cudaEvent_t>& pool = timing ? c->ev_timing : c->ev_done;
  if (!pool.empty()) {
    *e = pool.back();
    pool.pop_back();
    return cudaSuccess;
  }
  return timing ? cudaEventCreate(e) : cudaEventCreateWithFlags(e, cudaEventDisableTiming);
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

mr_status dev_alloc(mr_ctx* c, uint64_t bytes, void** out) {
  *out = nullptr;
  if (bytes == 0) bytes = 256;
  if (c->budget && c->in_use + bytes > c->budget) return MR_EBUDGET;
  void* p = nullptr;
  if (c->alloc) {
    p = c->alloc(c->alloc_user, (size_t)bytes);
    if (!p) return MR_ENOMEM;
  } else {
    cudaError_t e = cudaMallocFromPoolAsync(&p, (size_t)bytes, c->pool, c->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_last_error("cudaMallocFromPoolAsync", e);
      return e == cudaErrorMemoryAllocation ? MR_ENOMEM : MR_ECUDA;
    }
  }
  c->in_use += bytes;
  *out = p;
  return MR_OK;
}

void dev_free(mr_ctx* c, void* p, uint64_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 256;
  if (c->free_fn) c->free_fn(c->alloc_user, p);
  else cudaFreeAsync(p, c->stream);
  c->in_use -= bytes < c->in_use ? bytes : c->in_use;
}

inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

inline uint64_t km_stats_offset(uint64_t K, uint64_t D, uint64_t N) { return (K * D * 4 + N * 4 + 7) & ~7ull; }

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Planner: the paper keeps per-worker local arrays while each one fits the
// per-core cache and eliminates them otherwise (Sec. III-E).  The GB300 local
// store of a worker (CTA) is its shared memory, so an array job keeps local
// arrays when its lane-column copy fits the opt-in shared memory of one CTA.
mr_container plan_container(const mr_ctx* c, const mr_job_desc* d) {
  switch (d->kind) {
    case MR_WORDCOUNT:
      return MR_C_HASH;
    case MR_HIST_RGB8:
      if (d->container == MR_C_SMEM_ARRAY || d->container == MR_C_GLOBAL_ARRAY) return d->container;
      // small jobs cannot amortise zeroing and merging a CTA's local arrays
      if (d->input_bytes < c->tune.hist_global_below) return MR_C_GLOBAL_ARRAY;
      return hist_smem_bytes() <= c->di.smem_optin ? MR_C_SMEM_ARRAY : MR_C_GLOBAL_ARRAY;
    case MR_HIST_U32:
      // local arrays while every bin of the job fits one CTA's shared
      // memory; beyond that the global array (L2-resident up to ~100 MB of
      // counters) replaces them, as the paper does for large arrays.
      // Measured on 256M uniform keys: one CTA's local arrays beat the global
      // array 10-118x wherever they fit; local arrays spread over a
      // thread-block cluster (MR_C_CLUSTER_ARRAY, chosen only on request)
      // ran at ~90G keys/s, below the global array at every size they hold.
      if (d->container != MR_C_AUTO) return d->container;
      return d->hist_bins <= (uint32_t)hk_smem_max_bins(c->di) ? MR_C_SMEM_ARRAY : MR_C_GLOBAL_ARRAY;
    case MR_BLOOM_DNA:
      return MR_C_GLOBAL_ARRAY;
    case MR_LINREG_I8:
    case MR_KMEANS_F32:
    default:
      return MR_C_SMEM_ARRAY;
  }
}

// Kinds that the batched kernel does not cover: they run plain, after the batch.
bool plain_only(mr_kind k) { return k == MR_KMEANS_F32 || k == MR_HIST_U32 || k == MR_BLOOM_DNA; }

mr_status validate(const mr_ctx* c, const mr_job_desc* d) {
  if (!d || d->struct_size < sizeof(mr_job_desc)) return MR_EINVAL;
  if ((unsigned)d->kind > (unsigned)MR_BLOOM_DNA) return MR_EINVAL;
  if ((unsigned)d->container > (unsigned)MR_C_CLUSTER_ARRAY) return MR_EINVAL;
  if (d->container == MR_C_CLUSTER_ARRAY && d->kind != MR_HIST_U32) return MR_EINVAL;
  if (d->input_bytes && !d->input) return MR_EINVAL;
  switch (d->kind) {
    case MR_WORDCOUNT:
      if (d->container != MR_C_AUTO && d->container != MR_C_HASH) return MR_EINVAL;
      if (d->input_bytes >= (1ull << 40) - 1) return MR_EINVAL;
      if (d->wc_slots && (d->wc_slots & (d->wc_slots - 1))) return MR_EINVAL;
      if (d->wc_slots && (d->wc_slots < 1024 || d->wc_slots > (1ull << 32))) return MR_EINVAL;
      if (d->wc_pipelined > 1) return MR_EINVAL;
      break;
    case MR_HIST_RGB8:
      if (d->input_bytes % 3) return MR_EINVAL;
      if (d->container == MR_C_HASH) return MR_EINVAL;
      break;
    case MR_LINREG_I8:
      if (d->input_bytes % 2) return MR_EINVAL;
      if (d->container == MR_C_HASH) return MR_EINVAL;
      break;
    case MR_KMEANS_F32: {
      if (d->container == MR_C_HASH || d->container == MR_C_GLOBAL_ARRAY) return MR_EINVAL;
      if (d->km_dims == 0 || d->km_k == 0 || !d->km_init || d->km_iters == 0) return MR_EINVAL;
      if (d->km_dims > 1024 || d->km_k > 4096) return MR_EINVAL;
      const uint64_t row = (uint64_t)d->km_dims * 4;
      if (d->input_bytes % row) return MR_EINVAL;
      const uint64_t n = d->input_bytes / row;
      if (n == 0 || n > 0x7fffffffull) return MR_EINVAL;
      if (d->km_precision > MR_KM_BF16X1_TC) return MR_EINVAL;
      if (d->km_precision != MR_KM_FP32 && !km_tc_supported(d->km_dims, d->km_k)) return MR_EINVAL;
      break;
    }
    case MR_HIST_U32:
      if (d->input_bytes % 4 || d->hist_bins == 0 || d->hist_bins == 0xFFFFFFFFu) return MR_EINVAL;
      if (d->container == MR_C_HASH) return MR_EINVAL;
      if (d->container == MR_C_SMEM_ARRAY && d->hist_bins > (uint32_t)hk_smem_max_bins(c->di)) return MR_EINVAL;
      if (d->container == MR_C_CLUSTER_ARRAY && d->hist_bins > (uint32_t)hk_cluster_max_bins(c->di)) return MR_EINVAL;
      if (d->input_on_device && (reinterpret_cast<uintptr_t>(d->input) & 3)) return MR_EINVAL;
      break;
    case MR_BLOOM_DNA:
      if (d->container != MR_C_AUTO && d->container != MR_C_GLOBAL_ARRAY) return MR_EINVAL;
      if (d->bloom_kmer == 0 || d->bloom_kmer > 32 || d->bloom_hashes == 0 || d->bloom_hashes > 32) return MR_EINVAL;
      if (d->bloom_bits < 2 || d->bloom_bits > (1ull << 32)) return MR_EINVAL;
      break;
  }
  (void)c;
  return MR_OK;
}

mr_status alloc_wc(mr_ctx* c, Job* j, uint64_t cap) {
  const uint64_t n = j->desc.input_bytes;
  WcBuffers& b = j->wc;
  const uint64_t t_bytes = align256(wc_table_bytes(cap));
  const uint64_t s_bytes = align256(wc_state_bytes());
  const uint64_t sb_bytes = align256(wc_sortbuf_bytes(cap));
  const uint64_t o_bytes = align256(wc_out_bytes(cap, n));
  const uint64_t total = t_bytes + s_bytes + sb_bytes + o_bytes;
  void* slab = nullptr;
  mr_status st = dev_alloc(c, total, &slab);
  if (st) return st;
  uint8_t* p = static_cast<uint8_t*>(slab);
  b.cap = cap;
  b.key = reinterpret_cast<uint64_t*>(p);
  b.cnt = b.key + 2 * cap;
  b.state = reinterpret_cast<uint32_t*>(p + t_bytes);
  b.sortbuf = p + t_bytes + s_bytes;
  b.out = p + t_bytes + s_bytes + sb_bytes;
  b.out_cap = wc_out_bytes(cap, n);
  j->slab = slab;
  j->slab_bytes = total;
  j->result = b.out;
  return MR_OK;
}

mr_status alloc_job_memory(mr_ctx* c, Job* j) {
  const mr_job_desc& d = j->desc;
  switch (d.kind) {
    case MR_WORDCOUNT: {
      uint64_t cap = d.wc_slots;
      j->wc_auto = cap == 0;
      if (!cap) {
        // estimate: at most one distinct key per 16 input bytes, capped at
        // 2^17 slots; a table that overflows is regrown 4x and the job re-run
        cap = next_pow2(d.input_bytes / 16 + 1);
        if (cap < 4096) cap = 4096;
        if (cap > (1ull << 17)) cap = 1ull << 17;
      }
      return alloc_wc(c, j, cap);
    }
    case MR_HIST_RGB8: {
      j->result_bytes = 768 * 8;
      mr_status st = dev_alloc(c, 768 * 8, &j->slab);
      if (st) return st;
      j->slab_bytes = 768 * 8;
      j->result = j->slab;
      return MR_OK;
    }
    case MR_LINREG_I8: {
      j->result_bytes = 5 * 8;
      mr_status st = dev_alloc(c, 64, &j->slab);
      if (st) return st;
      j->slab_bytes = 64;
      j->result = j->slab;
      return MR_OK;
    }
    case MR_HIST_U32: {
      const uint64_t nb = (uint64_t)d.hist_bins + 1;
      const uint64_t res = align256(nb * 8);
      // u32 counters while no bin can reach 2^32
      const bool wide = d.input_bytes / 4 >= (1ull << 32);
      const uint64_t cnt = wide ? 0 : align256(nb * 4);
      mr_status st = dev_alloc(c, res + cnt, &j->slab);
      if (st) return st;
      j->slab_bytes = res + cnt;
      j->result = j->slab;
      j->result_bytes = nb * 8;
      j->hk_counters = wide ? nullptr : static_cast<uint8_t*>(j->slab) + res;
      return MR_OK;
    }
    case MR_BLOOM_DNA: {
      const uint64_t bytes = align256((d.bloom_bits + 31) / 32 * 4);
      mr_status st = dev_alloc(c, bytes, &j->slab);
      if (st) return st;
      j->slab_bytes = bytes;
      j->result = j->slab;
      j->result_bytes = (d.bloom_bits + 7) / 8;
      return MR_OK;
    }
    case MR_KMEANS_F32: {
      const uint32_t D = d.km_dims, K = d.km_k;
      const uint32_t N = (uint32_t)(d.input_bytes / ((uint64_t)D * 4));
      // result: centroids [K*D] f32 | assignments [N] i32 | pad to 8 | stats [4] u64
      const uint64_t res_bytes = km_stats_offset(K, D, N) + 32;
      const uint64_t res = align256(res_bytes);
      const uint64_t scr = align256(km_scratch_bytes(N, D, K, (int)d.km_precision));
      const uint64_t init_bytes = d.input_on_device ? 0 : align256((uint64_t)K * D * 4);
      mr_status st = dev_alloc(c, res + scr + init_bytes, &j->slab);
      if (st) return st;
      j->slab_bytes = res + scr + init_bytes;
      uint8_t* p = static_cast<uint8_t*>(j->slab);
      j->result = p;
      j->result_bytes = res_bytes;
      j->km.n = N;
      j->km.d = D;
      j->km.k = K;
      j->km.precision = (int)d.km_precision;
      cudaError_t e = km_carve(j->km, p + res, scr);
      if (e != cudaSuccess) {
        set_last_error("km_carve", e);
        return MR_EINVAL;
      }
      if (!d.input_on_device) {
        j->km_init_dev = reinterpret_cast<float*>(p + res + scr);
        MR_CUDA_TRY(cudaMemcpyAsync(j->km_init_dev, d.km_init, (size_t)K * D * 4, cudaMemcpyHostToDevice, c->stream));
      } else {
        j->km_init_dev = const_cast<float*>(d.km_init);
      }
      return MR_OK;
    }
  }
  return MR_EINVAL;
}

// A job is freed only once it has finished (mr_release waits for it), so its
// events can go back to the context's pools.
void free_job(mr_ctx* c, Job* j) {
  if (j->done) c->ev_done.push_back(j->done);
  if (j->t0) c->ev_timing.push_back(j->t0);
  if (j->t1) c->ev_timing.push_back(j->t1);
  if (j->kt) c->kt_pool.push_back(j->kt);
  dev_free(c, j->slab, j->slab_bytes);
  dev_free(c, j->in_owned, j->in_owned_bytes);
  delete j;
}

// The captured graph names the jobs' containers; it is dropped (and captured
// again by mr_rerun) when one of them moves.
void drop_batch_graph(mr_ctx* c) {
  if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
  c->batch_exec = nullptr;
}

int grid_for(const mr_ctx* c, uint64_t bytes, uint64_t bytes_per_block, int max_per_sm) {
  uint64_t g = (bytes + bytes_per_block - 1) / bytes_per_block;
  const uint64_t gmax = (uint64_t)c->di.sms * max_per_sm;
  if (g > gmax) g = gmax;
  if (g < 1) g = 1;
  return (int)g;
}

mr_status enqueue_plain_on(mr_ctx* c, Job* j, cudaStream_t st) {
  const uint64_t n = j->desc.input_bytes;
  if (j->t0) MR_CUDA_TRY(cudaEventRecord(j->t0, st));
  if (j->kt) j->kt->n = 0;
  switch (j->desc.kind) {
    case MR_HIST_RGB8: {
      MR_CUDA_TRY(cudaMemsetAsync(j->result, 0, 768 * 8, st));
      MR_CUDA_TRY(kt_begin(j->kt, st));
      if (j->container == MR_C_GLOBAL_ARRAY) {
        MR_CUDA_TRY(launch_hist_global(j->in, n, static_cast<uint64_t*>(j->result), grid_for(c, n, 512 * 64, 4),
                                       st));
        ++c->launches;
      } else {
        // a CTA is worth launching once each of its 32 warps gets a few 1536-byte steps
        MR_CUDA_TRY(launch_hist_smem(j->in, n, static_cast<uint64_t*>(j->result),
                                     grid_for(c, n, 1536ull * 32 * 4, 1), st));
        ++c->launches;
      }
      MR_CUDA_TRY(kt_end(j->kt, st));
      break;
    }
    case MR_LINREG_I8:
      MR_CUDA_TRY(cudaMemsetAsync(j->result, 0, 5 * 8, st));
      MR_CUDA_TRY(kt_begin(j->kt, st));
      MR_CUDA_TRY(launch_linreg(reinterpret_cast<const int8_t*>(j->in), n, static_cast<int64_t*>(j->result),
                                grid_for(c, n, 512ull * 16 * 8, 2), st));
      MR_CUDA_TRY(kt_end(j->kt, st));
      ++c->launches;
      break;
    case MR_WORDCOUNT:
      MR_CUDA_TRY(launch_wordcount(j->in, n, j->wc, c->di, st, &c->launches, j->desc.wc_pipelined != 0, j->kt,
                                   c->opt_polls));
      break;
    case MR_HIST_U32:
      MR_CUDA_TRY(launch_hist_keys(reinterpret_cast<const uint32_t*>(j->in), n / 4, j->desc.hist_bins,
                                   (int)j->container, j->hk_counters, j->hk_counters == nullptr,
                                   static_cast<unsigned long long*>(j->result), c->di, st, &c->launches, j->kt));
      break;
    case MR_BLOOM_DNA:
      MR_CUDA_TRY(launch_bloom(j->in, n, j->desc.bloom_kmer, j->desc.bloom_bits, j->desc.bloom_hashes,
                               static_cast<uint32_t*>(j->result), c->di, st, &c->launches, j->kt));
      break;
    case MR_KMEANS_F32: {
      uint8_t* p = static_cast<uint8_t*>(j->result);
      const uint32_t K = j->km.k, D = j->km.d, N = j->km.n;
      float* oc = reinterpret_cast<float*>(p);
      int32_t* oa = reinterpret_cast<int32_t*>(p + (uint64_t)K * D * 4);
      unsigned long long* os = reinterpret_cast<unsigned long long*>(p + km_stats_offset(K, D, N));
      j->km.kt = j->kt;
      j->km.polls = c->opt_polls;
      j->km.grid_cap = c->opt_km_grid_cap;
      j->km.stop_copies = c->opt_km_stop_copies;
      MR_CUDA_TRY(launch_kmeans(reinterpret_cast<const float*>(j->in), j->km_init_dev, j->desc.km_iters, j->km,
                                c->di, st, oc, oa, os, &c->launches));
      break;
    }
  }
  if (j->t1) MR_CUDA_TRY(cudaEventRecord(j->t1, st));
  MR_CUDA_TRY(cudaEventRecord(j->done, st));
  j->state = JOB_ENQUEUED;
  return MR_OK;
}

mr_status enqueue_plain(mr_ctx* c, Job* j) { return enqueue_plain_on(c, j, c->stream); }

// MR_RUN_CONCURRENT: the jobs of a run are independent (each has its own
// input, containers and result), so they run concurrently.  Two to
// ARRAY_FUSE_MAX shared-memory histograms and regressions run as one fused
// launch on the context stream (each CTA takes its share of every job in
// turn).  Otherwise the first job goes on the context stream and the others
// round robin on PLAIN_AUX internal streams that wait for the work already
// on the context stream; the context stream then waits for them, so later
// work on it (and the next run) sees every job done.  Either way two
// bandwidth-bound jobs overlap their ramp-up and tail.
// Array jobs that fit one fused launch: shared-memory histograms and regressions.
bool array_fusable(const Job* j) {
  return (j->desc.kind == MR_HIST_RGB8 && j->container != MR_C_GLOBAL_ARRAY) || j->desc.kind == MR_LINREG_I8;
}

mr_status enqueue_array_fused(mr_ctx* c, const std::vector<Job*>& jobs) {
  cudaStream_t st = c->stream;
  ArrayJobs A{};
  A.n = (uint32_t)jobs.size();
  uint64_t total = 0;
  for (size_t i = 0; i < jobs.size(); ++i) {
    Job* j = jobs[i];
    if (j->t0) MR_CUDA_TRY(cudaEventRecord(j->t0, st));
    if (j->kt) j->kt->n = 0;
    A.kind[i] = (uint32_t)j->desc.kind;
    A.in[i] = j->in;
    A.bytes[i] = j->desc.input_bytes;
    A.out[i] = j->result;
    total += j->desc.input_bytes;
  }
  // every job's kernel time is the fused launch's
  for (Job* j : jobs) MR_CUDA_TRY(kt_begin(j->kt, st));
  MR_CUDA_TRY(launch_array_fused(A, grid_for(c, total, 1536ull * 32 * 4, 1), st));
  c->launches += 2;  // clearing the results, then the fused pass
  for (Job* j : jobs) {
    MR_CUDA_TRY(kt_end(j->kt, st));
    if (j->t1) MR_CUDA_TRY(cudaEventRecord(j->t1, st));
    MR_CUDA_TRY(cudaEventRecord(j->done, st));
    j->state = JOB_ENQUEUED;
  }
  return MR_OK;
}

mr_status enqueue_concurrent(mr_ctx* c, const std::vector<Job*>& jobs) {
  bool fuse = jobs.size() >= 2 && jobs.size() <= (size_t)ARRAY_FUSE_MAX;
  for (const Job* j : jobs) fuse = fuse && array_fusable(j);
  if (fuse) return enqueue_array_fused(c, jobs);
  if (jobs.size() <= 1) {
    for (Job* j : jobs) {
      mr_status st = enqueue_plain(c, j);
      if (st) return st;
    }
    return MR_OK;
  }
  if (!c->plain_fork) {
    MR_CUDA_TRY(cudaEventCreateWithFlags(&c->plain_fork, cudaEventDisableTiming));
    for (int a = 0; a < mr_ctx::PLAIN_AUX; ++a) {
      MR_CUDA_TRY(cudaStreamCreateWithFlags(&c->plain_aux[a], cudaStreamNonBlocking));
      MR_CUDA_TRY(cudaEventCreateWithFlags(&c->plain_join[a], cudaEventDisableTiming));
    }
  }
  MR_CUDA_TRY(cudaEventRecord(c->plain_fork, c->stream));
  const int used = (int)(jobs.size() - 1 < (size_t)mr_ctx::PLAIN_AUX ? jobs.size() - 1 : mr_ctx::PLAIN_AUX);
  for (int a = 0; a < used; ++a) MR_CUDA_TRY(cudaStreamWaitEvent(c->plain_aux[a], c->plain_fork, 0));
  for (size_t i = 0; i < jobs.size(); ++i) {
    mr_status st = enqueue_plain_on(c, jobs[i], i == 0 ? c->stream : c->plain_aux[(i - 1) % mr_ctx::PLAIN_AUX]);
    if (st) return st;
  }
  for (int a = 0; a < used; ++a) {
    MR_CUDA_TRY(cudaEventRecord(c->plain_join[a], c->plain_aux[a]));
    MR_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->plain_join[a], 0));
  }
  return MR_OK;
}

mr_status ensure_scratch(mr_ctx* c, void** p, uint64_t* have, uint64_t need) {
  need = align256(need ? need : 256);
  if (need <= *have) return MR_OK;
  dev_free(c, *p, *have);
  *p = nullptr;
  *have = 0;
  mr_status st = dev_alloc(c, need, p);
  if (st) return st;
  *have = need;
  return MR_OK;
}

struct BatchPlan {
  std::vector<BatchJob> bj;
  std::vector<wc::JobDev> wj;
  uint64_t tiles = 0, wc_blocks = 0, wc_records = 0, zchunks = 0;
};

void plan_batch(const std::vector<Job*>& jobs, const mr_tuning& tp, BatchPlan& P) {
  for (Job* j : jobs) {
    BatchJob b{};
    b.kind = (uint32_t)j->desc.kind;
    b.container = (uint32_t)j->container;
    if (j->desc.kind == MR_HIST_RGB8 && j->desc.container == MR_C_AUTO)
      b.container = j->desc.input_bytes < tp.hist_global_below ? MR_C_GLOBAL_ARRAY : MR_C_SMEM_ARRAY;
    b.in = j->in;
    b.n = j->desc.input_bytes;
    b.out = j->result;
    if (j->desc.kind == MR_WORDCOUNT) {
      b.wc = wc_job_dev(j->in, b.n, j->wc, P.wc_blocks);
      P.wc_blocks += wc_compact_blocks(j->wc.cap);
      P.wc_records += j->wc.cap;
      P.wj.push_back(b.wc);
    }
    b.tile_begin = P.tiles;
    b.ntiles = batch_tiles_for(b.kind, b.n, tp.arr_tile, tp.wc_tile);
    P.tiles += b.ntiles;
    b.zchunk0 = P.zchunks;
    P.zchunks += batch_zero_chunks(b.kind, j->desc.kind == MR_WORDCOUNT ? j->wc.cap : 0);
    P.bj.push_back(b);
  }
}

// Build the batch's descriptors for the given parameters, capture the launch
// sequence into a CUDA graph and instantiate it (not launched).
mr_status build_batch_graph(mr_ctx* c, const std::vector<Job*>& jobs, const mr_tuning& tp, cudaGraphExec_t* out) {
  *out = nullptr;
  BatchPlan P;
  plan_batch(jobs, tp, P);
  std::vector<BatchJob>& bj = P.bj;
  std::vector<wc::JobDev>& wj = P.wj;
  const uint64_t tiles = P.tiles, wc_blocks = P.wc_blocks, wc_records = P.wc_records;
  mr_status st = ensure_scratch(c, &c->batch_desc, &c->batch_desc_bytes, bj.size() * sizeof(BatchJob));
  if (!st) st = ensure_scratch(c, &c->batch_wc, &c->batch_wc_bytes, wj.size() * sizeof(wc::JobDev));
  if (!st && !wj.empty()) st = ensure_scratch(c, &c->batch_sort, &c->batch_sort_bytes, wc_sortbuf_bytes(wc_records));
  if (!st && !c->batch_cursor) st = dev_alloc(c, 256, &c->batch_cursor);
  if (st) return st;
  MR_CUDA_TRY(cudaMemcpyAsync(c->batch_desc, bj.data(), bj.size() * sizeof(BatchJob), cudaMemcpyHostToDevice,
                              c->stream));
  if (!wj.empty())
    MR_CUDA_TRY(cudaMemcpyAsync(c->batch_wc, wj.data(), wj.size() * sizeof(wc::JobDev), cudaMemcpyHostToDevice,
                                c->stream));
  MR_CUDA_TRY(batch_prepare());
  uint64_t nk = 0;
  cudaGraph_t g = nullptr;
  MR_CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = launch_batch(static_cast<const BatchJob*>(c->batch_desc), (uint32_t)bj.size(), tiles,
                               static_cast<unsigned long long*>(c->batch_cursor), tp.arr_tile, tp.wc_tile,
                               P.zchunks, c->di, c->stream, &nk);
  if (e == cudaSuccess && !wj.empty())
    e = launch_wordcount_post_multi(static_cast<const wc::JobDev*>(c->batch_wc), wj.data(), (uint32_t)wj.size(),
                                    wc_blocks, wc_records, static_cast<uint8_t*>(c->batch_sort), c->di.sms,
                                    c->stream, &nk);
  cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    set_last_error("batch graph capture", e != cudaSuccess ? e : e2);
    return MR_ECUDA;
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    set_last_error("cudaGraphInstantiate", e);
    return MR_ECUDA;
  }
  c->batch_launches = nk;
  return MR_OK;
}

// Time one candidate parameter set on the batch (device time of one run).
mr_status time_candidate(mr_ctx* c, const std::vector<Job*>& jobs, const mr_tuning& tp, float* ms) {
  cudaGraphExec_t ex = nullptr;
  mr_status st = build_batch_graph(c, jobs, tp, &ex);
  if (st) return st;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaGraphLaunch(ex, c->stream);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(a, c->stream);
  if (e == cudaSuccess) e = cudaGraphLaunch(ex, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(b, c->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaGraphExecDestroy(ex);
  if (e != cudaSuccess) {
    set_last_error("autotune timing", e);
    return MR_ECUDA;
  }
  return MR_OK;
}

// Coordinate search over the batch parameters on the pending batch itself.
mr_status autotune_batch(mr_ctx* c, const std::vector<Job*>& jobs) {
  mr_tuning best = c->tune;
  float best_ms = 0.f;
  mr_status st = time_candidate(c, jobs, best, &best_ms);
  if (st) return st;
  // Larger word-count tiles mean fewer job switches per CTA (each switch
  // flushes and clears the warps' hot-key caches); smaller ones balance
  // better at the end of a batch.
  const uint64_t arr_c[] = {1536ull * 32, 1536ull * 128, 1536ull * 512, 1536ull * 2048};
  const uint64_t wc_c[] = {512ull * 32, 512ull * 128, 512ull * 512, 512ull * 2048, 512ull * 8192};
  const uint64_t hg_c[] = {0, 1ull << 14, 1ull << 17};
  const int ncand[3] = {4, 5, 3};
  for (int dim = 0; dim < 3; ++dim) {
    for (int k = 0; k < ncand[dim]; ++k) {
      mr_tuning t = best;
      if (dim == 0) t.arr_tile = arr_c[k];
      else if (dim == 1) t.wc_tile = wc_c[k];
      else t.hist_global_below = hg_c[k];
      if (t.arr_tile == best.arr_tile && t.wc_tile == best.wc_tile && t.hist_global_below == best.hist_global_below)
        continue;
      float ms = 0.f;
      st = time_candidate(c, jobs, t, &ms);
      if (st) return st;
      if (ms < best_ms) {
        best = t;
        best_ms = ms;
      }
    }
  }
  best.best_ms = best_ms;
  best.tuned = 1;
  c->tune = best;
  if (const char* path = getenv("MR_TUNE_CACHE")) {
    if (FILE* f = fopen(path, "a")) {
      fprintf(f, "sms=%d jobs=%zu arr_tile=%llu wc_tile=%llu hist_global_below=%llu ms=%.4f\n", c->di.sms, jobs.size(),
              (unsigned long long)best.arr_tile, (unsigned long long)best.wc_tile,
              (unsigned long long)best.hist_global_below, best.best_ms);
      fclose(f);
    }
  }
  return MR_OK;
}

mr_status enqueue_batched(mr_ctx* c, std::vector<Job*>& jobs) {
  std::vector<Job*> batched;
  for (Job* j : jobs)
    if (!plain_only(j->desc.kind)) batched.push_back(j);
  if (!batched.empty()) {
    drop_batch_graph(c);
    c->batch_ids.clear();
    if ((c->flags & MR_FLAG_AUTOTUNE) && !c->tune.tuned) {
      mr_status st = autotune_batch(c, batched);
      if (st) return st;
    }
    for (Job* j : batched)
      if (j->t0) MR_CUDA_TRY(cudaEventRecord(j->t0, c->stream));
    mr_status st = build_batch_graph(c, batched, c->tune, &c->batch_exec);
    if (st) return st;
    MR_CUDA_TRY(cudaGraphLaunch(c->batch_exec, c->stream));
    c->launches += c->batch_launches;
    for (Job* j : batched) {
      c->batch_ids.push_back(j->id);
      if (j->t1) MR_CUDA_TRY(cudaEventRecord(j->t1, c->stream));
      MR_CUDA_TRY(cudaEventRecord(j->done, c->stream));
      j->state = JOB_ENQUEUED;
    }
  }
  for (Job* j : jobs)
    if (plain_only(j->desc.kind)) {
      mr_status st = enqueue_plain(c, j);
      if (st) return st;
    }
  return MR_OK;
}

// Serving: plain-only requests (k-means, large-key histogram, Bloom) are
// launched at once on the auxiliary streams, round robin; the other admitted
// requests that are not running yet go as one micro-batch on a slot whose
// previous micro-batch has finished.  Requests that arrive while the GPU is
// busy are picked up as soon as a slot frees, so successive micro-batches
// overlap on the device.  Slot streams have the higher stream priority, so
// when SMs free up the block scheduler serves the micro-batches (most
// requests, each short) before the next blocks of a long k-means.  Returns
// MR_OK also when no slot is free (the requests stay queued).
mr_status serve_pump(mr_ctx* c) {
  if (c->serve_pending.empty()) return MR_OK;
  if (!c->serve_aux[0]) {
    int least = 0, greatest = 0;
    MR_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    for (auto& sl : c->slots) {
      MR_CUDA_TRY(cudaStreamCreateWithPriority(&sl.s, cudaStreamNonBlocking, greatest));
      MR_CUDA_TRY(cudaEventCreateWithFlags(&sl.busy, cudaEventDisableTiming));
    }
    for (auto& a : c->serve_aux) MR_CUDA_TRY(cudaStreamCreateWithPriority(&a, cudaStreamNonBlocking, least));
  }
  // every stream used here must see the submit-time copies and clears on the context stream
  if (!c->serve_ready) MR_CUDA_TRY(cudaEventCreateWithFlags(&c->serve_ready, cudaEventDisableTiming));
  MR_CUDA_TRY(cudaEventRecord(c->serve_ready, c->stream));
  std::vector<Job*> arr;
  for (size_t i = 0; i < c->serve_pending.size(); ++i) {
    Job* j = c->serve_pending[i];
    if (!plain_only(j->desc.kind)) {
      arr.push_back(j);
      continue;
    }
    cudaStream_t as = c->serve_aux[c->serve_aux_next++ % mr_ctx::SERVE_AUX];
    cudaError_t e = cudaStreamWaitEvent(as, c->serve_ready, 0);
    mr_status st = e == cudaSuccess ? enqueue_plain_on(c, j, as) : MR_ECUDA;
    if (e != cudaSuccess) set_last_error("cudaStreamWaitEvent", e);
    if (st) {
      // the requests not launched yet stay queued
      std::vector<Job*> left(arr);
      left.insert(left.end(), c->serve_pending.begin() + (ptrdiff_t)i, c->serve_pending.end());
      c->serve_pending.swap(left);
      return st;
    }
  }
  c->serve_pending.swap(arr);
  if (c->serve_pending.empty()) return MR_OK;
  mr_ctx::Slot* slot = nullptr;
  for (auto& sl : c->slots) {
    if (!sl.used) {
      slot = &sl;
      break;
    }
    const cudaError_t q = cudaEventQuery(sl.busy);
    if (q == cudaSuccess) {
      slot = &sl;
      break;
    }
    if (q != cudaErrorNotReady) {
      set_last_error("cudaEventQuery(slot)", q);
      return MR_ECUDA;
    }
  }
  if (!slot) return MR_OK;
  std::vector<Job*> jobs;
  jobs.swap(c->serve_pending);
  MR_CUDA_TRY(cudaStreamWaitEvent(slot->s, c->serve_ready, 0));
  for (Job* j : jobs)
    if (j->t0) MR_CUDA_TRY(cudaEventRecord(j->t0, slot->s));
  BatchPlan P;
  plan_batch(jobs, c->tune, P);
  mr_status st = ensure_scratch(c, &slot->desc, &slot->desc_bytes, P.bj.size() * sizeof(BatchJob));
  if (!st) st = ensure_scratch(c, &slot->wcd, &slot->wcd_bytes, P.wj.size() * sizeof(wc::JobDev));
  if (!st && !P.wj.empty()) st = ensure_scratch(c, &slot->sort, &slot->sort_bytes, wc_sortbuf_bytes(P.wc_records));
  if (!st && !slot->cursor) st = dev_alloc(c, 256, &slot->cursor);
  if (st) {
    c->serve_pending.insert(c->serve_pending.begin(), jobs.begin(), jobs.end());
    return st;
  }
  MR_CUDA_TRY(
      cudaMemcpyAsync(slot->desc, P.bj.data(), P.bj.size() * sizeof(BatchJob), cudaMemcpyHostToDevice, slot->s));
  if (!P.wj.empty())
    MR_CUDA_TRY(cudaMemcpyAsync(slot->wcd, P.wj.data(), P.wj.size() * sizeof(wc::JobDev), cudaMemcpyHostToDevice,
                                slot->s));
  MR_CUDA_TRY(batch_prepare());
  MR_CUDA_TRY(launch_batch(static_cast<const BatchJob*>(slot->desc), (uint32_t)P.bj.size(), P.tiles,
                           static_cast<unsigned long long*>(slot->cursor), c->tune.arr_tile, c->tune.wc_tile,
                           P.zchunks, c->di, slot->s, &c->launches));
  if (!P.wj.empty())
    MR_CUDA_TRY(launch_wordcount_post_multi(static_cast<const wc::JobDev*>(slot->wcd), P.wj.data(),
                                            (uint32_t)P.wj.size(), P.wc_blocks, P.wc_records,
                                            static_cast<uint8_t*>(slot->sort), c->di.sms, slot->s, &c->launches));
  for (Job* j : jobs) {
    if (j->t1) MR_CUDA_TRY(cudaEventRecord(j->t1, slot->s));
    MR_CUDA_TRY(cudaEventRecord(j->done, slot->s));
    j->state = JOB_ENQUEUED;
  }
  // the slot is free again once its micro-batch is done
  MR_CUDA_TRY(cudaEventRecord(slot->busy, slot->s));
  slot->used = true;
  return MR_OK;
}

// Block until the queued request j has been launched.
mr_status serve_launch_now(mr_ctx* c, Job* j) {
  while (j->state == JOB_SERVE_QUEUED) {
    mr_status st = serve_pump(c);
    if (st) return st;
    if (j->state != JOB_SERVE_QUEUED) break;
    // every slot is busy: wait for the one that was launched first to drain
    for (auto& sl : c->slots)
      if (sl.used) {
        MR_CUDA_TRY(cudaEventSynchronize(sl.busy));
        break;
      }
  }
  return MR_OK;
}

Job* find_job(mr_ctx* c, uint64_t id) {
  auto it = c->jobs.find(id);
  return it == c->jobs.end() ? nullptr : it->second;
}

// Wait for a job; for an automatic word-count table that overflowed, regrow
// it (4x) and re-run until it fits.
mr_status serve_launch_now(mr_ctx* c, Job* j);

mr_status wait_job(mr_ctx* c, Job* j, uint64_t* wc_result_bytes = nullptr) {
  if (j->state == JOB_SERVE_QUEUED) {
    mr_status st = serve_launch_now(c, j);
    if (st) return st;
  }
  if (j->state == JOB_PENDING) return MR_ENOTREADY;
  MR_CUDA_TRY(cudaEventSynchronize(j->done));
  if (j->desc.kind == MR_KMEANS_F32) {
    // stats[3] counts device waits that gave up (bounded mbarrier waits)
    unsigned long long to = 0;
    const uint64_t so = km_stats_offset(j->km.k, j->km.d, j->km.n) + 24;
    MR_CUDA_TRY(cudaMemcpyAsync(&to, static_cast<uint8_t*>(j->result) + so, 8, cudaMemcpyDeviceToHost, c->stream));
    MR_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return to ? MR_ETIMEOUT : MR_OK;
  }
  if (j->desc.kind != MR_WORDCOUNT) return MR_OK;
  for (;;) {
    // the flag words and the result header, read with one synchronisation
    uint32_t st[4];
    uint64_t hdr[2];
    MR_CUDA_TRY(cudaMemcpyAsync(st, j->wc.state, 16, cudaMemcpyDeviceToHost, c->stream));
    MR_CUDA_TRY(cudaMemcpyAsync(hdr, j->wc.out, 16, cudaMemcpyDeviceToHost, c->stream));
    MR_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (st[0] & 2u) return MR_ETIMEOUT;  // a pipelined map pass whose reducer stalled
    if (!(st[0] & 1u)) {
      if (wc_result_bytes) *wc_result_bytes = 16 + 24 * hdr[0] + hdr[1];
      return MR_OK;
    }
    if (!j->wc_auto) return MR_EOVERFLOW;
    // the job's containers move: a captured batch graph that names them is stale
    for (uint64_t id : c->batch_ids)
      if (id == j->id) {
        drop_batch_graph(c);
        break;
      }
    const uint64_t cap = j->wc.cap * 4;
    if (cap > (1ull << 32)) return MR_EOVERFLOW;
    dev_free(c, j->slab, j->slab_bytes);
    j->slab = nullptr;
    mr_status s = alloc_wc(c, j, cap);
    if (s) return s;
    MR_CUDA_TRY(launch_wordcount(j->in, j->desc.input_bytes, j->wc, c->di, c->stream, &c->launches,
                                 j->desc.wc_pipelined != 0, nullptr, c->opt_polls));
    MR_CUDA_TRY(cudaEventRecord(j->done, c->stream));
    MR_CUDA_TRY(cudaEventSynchronize(j->done));
  }
}

mr_status result_size(mr_ctx* c, Job* j, uint64_t* bytes) {
  if (j->desc.kind == MR_WORDCOUNT) {
    uint64_t hdr[2];
    MR_CUDA_TRY(cudaMemcpyAsync(hdr, j->wc.out, 16, cudaMemcpyDeviceToHost, c->stream));
    MR_CUDA_TRY(cudaStreamSynchronize(c->stream));
    *bytes = 16 + 24 * hdr[0] + hdr[1];
  } else {
    *bytes = j->result_bytes;
  }
  return MR_OK;
}

mr_status add_job_impl(mr_ctx* c, const mr_job_desc* desc, uint64_t* job_id) {
  if (!c || !job_id) return MR_EINVAL;
  mr_status st = validate(c, desc);
  if (st) return st;
  Job* j = new (std::nothrow) Job();
  if (!j) return MR_ENOMEM;
  j->desc = *desc;
  j->container = plan_container(c, desc);
  cudaError_t e = pooled_event(c, false, &j->done);
  if (e == cudaSuccess && (c->flags & MR_FLAG_TIMING)) {
    e = pooled_event(c, true, &j->t0);
    if (e == cudaSuccess) e = pooled_event(c, true, &j->t1);
    if (e == cudaSuccess && !c->kt_pool.empty()) {
      j->kt = c->kt_pool.back();
      c->kt_pool.pop_back();
    } else if (e == cudaSuccess && !(j->kt = new (std::nothrow) KTimer())) {
      e = cudaErrorMemoryAllocation;
    }
  }
  if (e != cudaSuccess) {
    set_last_error("cudaEventCreate", e);
    free_job(c, j);
    return MR_ECUDA;
  }
  if (desc->input_on_device || desc->input_bytes == 0) {
    j->in = static_cast<const uint8_t*>(desc->input);
  } else {
    st = dev_alloc(c, desc->input_bytes, &j->in_owned);
    if (st) {
      free_job(c, j);
      return st;
    }
    j->in_owned_bytes = desc->input_bytes;
    e = cudaMemcpyAsync(j->in_owned, desc->input, desc->input_bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) {
      set_last_error("cudaMemcpyAsync(H2D)", e);
      free_job(c, j);
      return MR_ECUDA;
    }
    j->in = static_cast<const uint8_t*>(j->in_owned);
  }
  st = alloc_job_memory(c, j);
  if (st) {
    free_job(c, j);
    return st;
  }
  if (!desc->input_on_device) {
    // host buffers (input, k-means init) may be reused once this call returns
    e = cudaEventRecord(j->done, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(j->done);
    if (e != cudaSuccess) {
      set_last_error("host input copy", e);
      free_job(c, j);
      return MR_ECUDA;
    }
  }
  j->id = c->next_id++;
  c->jobs[j->id] = j;
  *job_id = j->id;
  return MR_OK;
}

}  // namespace

extern "C" {

const char* mr_status_str(mr_status s) {
  switch (s) {
    case MR_OK: return "MR_OK";
    case MR_EINVAL: return "MR_EINVAL: invalid argument";
    case MR_ENOMEM: return "MR_ENOMEM: out of memory";
    case MR_ECUDA: return "MR_ECUDA: CUDA error";
    case MR_EOVERFLOW: return "MR_EOVERFLOW: hash container too small";
    case MR_ETIMEOUT: return "MR_ETIMEOUT: device wait timed out";
    case MR_EBUDGET: return "MR_EBUDGET: HBM budget exceeded";
    case MR_ENOTREADY: return "MR_ENOTREADY: job not finished";
    case MR_ENOJOB: return "MR_ENOJOB: no such job";
  }
  return "unknown mr_status";
}

const char* mr_last_error(void) { return g_last_error.c_str(); }

mr_status mr_create(const mr_config* cfg, mr_ctx** out) {
  if (!cfg || !out || cfg->struct_size < sizeof(mr_config)) return MR_EINVAL;
  if ((cfg->alloc == nullptr) != (cfg->free == nullptr)) return MR_EINVAL;
  *out = nullptr;
  int ndev = 0;
  MR_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (cfg->device < 0 || cfg->device >= ndev) return MR_EINVAL;
  DeviceGuard g(cfg->device);
  mr_ctx* c = new (std::nothrow) mr_ctx();
  if (!c) return MR_ENOMEM;
  c->device = cfg->device;
  c->alloc = cfg->alloc;
  c->free_fn = cfg->free;
  c->alloc_user = cfg->alloc_user;
  c->budget = cfg->hbm_budget;
  c->flags = cfg->flags;
  cudaError_t e = cudaDeviceGetAttribute(&c->di.sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->di.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->di.l2_bytes, cudaDevAttrL2CacheSize, c->device);
  if (e == cudaSuccess) {
    if (cfg->cuda_stream) {
      c->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    } else {
      e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
      c->own_stream = e == cudaSuccess;
    }
  }
  if (e == cudaSuccess && !c->alloc) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c->device;
    e = cudaMemPoolCreate(&c->pool, &props);
    if (e == cudaSuccess) {
      uint64_t keep = ~0ull;  // never trim at synchronisation; the pool goes with the context
      e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
  }
  if (e != cudaSuccess) {
    set_last_error("mr_create", e);
    if (c->pool) cudaMemPoolDestroy(c->pool);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return MR_ECUDA;
  }
  *out = c;
  return MR_OK;
}

void mr_destroy(mr_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto& kv : c->jobs) free_job(c, kv.second);
  c->jobs.clear();
  for (auto& sl : c->slots)
    if (sl.s) cudaStreamSynchronize(sl.s);
  for (auto a : c->serve_aux)
    if (a) cudaStreamSynchronize(a);
  drop_batch_graph(c);
  for (auto& sl : c->slots) {
    dev_free(c, sl.desc, sl.desc_bytes);
    dev_free(c, sl.wcd, sl.wcd_bytes);
    dev_free(c, sl.sort, sl.sort_bytes);
    dev_free(c, sl.cursor, 256);
  }
  dev_free(c, c->batch_desc, c->batch_desc_bytes);
  dev_free(c, c->batch_wc, c->batch_wc_bytes);
  dev_free(c, c->batch_sort, c->batch_sort_bytes);
  dev_free(c, c->batch_cursor, 256);
  cudaStreamSynchronize(c->stream);
  for (auto& sl : c->slots) {
    if (sl.busy) cudaEventDestroy(sl.busy);
    if (sl.s) cudaStreamDestroy(sl.s);
  }
  for (auto a : c->serve_aux)
    if (a) cudaStreamDestroy(a);
  if (c->serve_ready) cudaEventDestroy(c->serve_ready);
  for (int a = 0; a < mr_ctx::PLAIN_AUX; ++a) {
    if (c->plain_aux[a]) {
      cudaStreamSynchronize(c->plain_aux[a]);
      cudaStreamDestroy(c->plain_aux[a]);
    }
    if (c->plain_join[a]) cudaEventDestroy(c->plain_join[a]);
  }
  if (c->plain_fork) cudaEventDestroy(c->plain_fork);
  for (cudaEvent_t e : c->ev_done) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_timing) cudaEventDestroy(e);
  for (KTimer* t : c->kt_pool) kt_destroy(t);
  cudaStreamSynchronize(c->stream);
  // memory still held (none, normally) is released once it is freed
  if (c->pool) cudaMemPoolDestroy(c->pool);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

mr_status mr_add_job(mr_ctx* c, const mr_job_desc* desc, uint64_t* job_id) {
  if (!c) return MR_EINVAL;
  DeviceGuard g(c->device);
  mr_status st = add_job_impl(c, desc, job_id);
  if (st == MR_OK) c->pending.push_back(*job_id);
  return st;
}

mr_status mr_run(mr_ctx* c, mr_mode mode) {
  if (!c || (mode != MR_RUN_PLAIN && mode != MR_RUN_BATCHED && mode != MR_RUN_CONCURRENT)) return MR_EINVAL;
  DeviceGuard g(c->device);
  std::vector<Job*> jobs;
  for (uint64_t id : c->pending) {
    Job* j = find_job(c, id);
    if (j && j->state == JOB_PENDING) jobs.push_back(j);
  }
  c->pending.clear();
  mr_status st = MR_OK;
  if (mode == MR_RUN_BATCHED) {
    st = enqueue_batched(c, jobs);
  } else if (mode == MR_RUN_CONCURRENT) {
    st = enqueue_concurrent(c, jobs);
  } else {
    for (Job* j : jobs)
      if ((st = enqueue_plain(c, j)) != MR_OK) break;
  }
  // jobs that were not launched (an allocation or launch failed on the way)
  // stay pending, so that a later mr_run can launch them
  if (st)
    for (Job* j : jobs)
      if (j->state == JOB_PENDING) c->pending.push_back(j->id);
  return st;
}

mr_status mr_fetch(mr_ctx* c, uint64_t job_id, void* buf, uint64_t buf_bytes, uint64_t* needed) {
  if (!c) return MR_EINVAL;
  DeviceGuard g(c->device);
  Job* j = find_job(c, job_id);
  if (!j) return MR_ENOJOB;
  uint64_t bytes = 0;
  mr_status st = wait_job(c, j, &bytes);
  if (st) return st;
  if (j->desc.kind != MR_WORDCOUNT && (st = result_size(c, j, &bytes)) != MR_OK) return st;
  if (needed) *needed = bytes;
  if (!buf) return MR_OK;
  if (buf_bytes < bytes) return MR_EINVAL;
  MR_CUDA_TRY(cudaMemcpyAsync(buf, j->result, bytes, cudaMemcpyDeviceToHost, c->stream));
  MR_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MR_OK;
}

mr_status mr_result_device(mr_ctx* c, uint64_t job_id, const void** dptr, uint64_t* bytes) {
  if (!c || !dptr || !bytes) return MR_EINVAL;
  DeviceGuard g(c->device);
  Job* j = find_job(c, job_id);
  if (!j) return MR_ENOJOB;
  mr_status st = wait_job(c, j);
  if (st) return st;
  st = result_size(c, j, bytes);
  if (st) return st;
  *dptr = j->result;
  return MR_OK;
}

mr_status mr_release(mr_ctx* c, uint64_t job_id) {
  if (!c) return MR_EINVAL;
  DeviceGuard g(c->device);
  Job* j = find_job(c, job_id);
  if (!j) return MR_ENOJOB;
  if (j->state == JOB_ENQUEUED) MR_CUDA_TRY(cudaEventSynchronize(j->done));
  for (size_t i = 0; i < c->serve_pending.size(); ++i)
    if (c->serve_pending[i] == j) {
      c->serve_pending.erase(c->serve_pending.begin() + i);
      break;
    }
  for (uint64_t id : c->batch_ids)
    if (id == job_id) {
      drop_batch_graph(c);
      c->batch_ids.clear();
      break;
    }
  c->jobs.erase(job_id);
  for (size_t i = 0; i < c->pending.size(); ++i)
    if (c->pending[i] == job_id) {
      c->pending.erase(c->pending.begin() + i);
      break;
    }
  free_job(c, j);
  return MR_OK;
}

mr_status mr_submit(mr_ctx* c, const mr_job_desc* desc, uint64_t* job_id) {
  if (!c) return MR_EINVAL;
  DeviceGuard g(c->device);
  mr_status st = add_job_impl(c, desc, job_id);
  if (st) return st;
  Job* j = find_job(c, *job_id);
  j->state = JOB_SERVE_QUEUED;
  c->serve_pending.push_back(j);
  return serve_pump(c);
}

mr_status mr_poll(mr_ctx* c, uint64_t job_id) {
  if (!c) return MR_EINVAL;
  DeviceGuard g(c->device);
  mr_status ps = serve_pump(c);
  if (ps) return ps;
  Job* j = find_job(c, job_id);
  if (!j) return MR_ENOJOB;
  if (j->state == JOB_PENDING || j->state == JOB_SERVE_QUEUED) return MR_ENOTREADY;
  cudaError_t e = cudaEventQuery(j->done);
  if (e == cudaSuccess) return MR_OK;
  if (e == cudaErrorNotReady) return MR_ENOTREADY;
  set_last_error("cudaEventQuery", e);
  return MR_ECUDA;
}

mr_status mr_sync(mr_ctx* c) {
  if (!c) return MR_EINVAL;
  DeviceGuard g(c->device);
  while (!c->serve_pending.empty()) {
    Job* j = c->serve_pending.front();
    mr_status st = serve_launch_now(c, j);
    if (st) return st;
  }
  for (auto& sl : c->slots)
    if (sl.s) MR_CUDA_TRY(cudaStreamSynchronize(sl.s));
  for (auto a : c->serve_aux)
    if (a) MR_CUDA_TRY(cudaStreamSynchronize(a));
  MR_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MR_OK;
}

uint64_t mr_bytes_in_use(const mr_ctx* c) { return c ? c->in_use : 0; }

mr_status mr_set_option(mr_ctx* c, mr_option opt, uint64_t value) {
  if (!c) return MR_EINVAL;
  switch (opt) {
    case MR_OPT_WAIT_POLLS:
      if (value != UINT64_MAX && value > (1ull << 40)) return MR_EINVAL;
      c->opt_polls = value == UINT64_MAX ? -1 : (long long)value;
      return MR_OK;
    case MR_OPT_KM_GRID_CAP:
      if (value > 0xFFFFFFFFull) return MR_EINVAL;
      c->opt_km_grid_cap = (uint32_t)value;
      return MR_OK;
    case MR_OPT_KM_STOP_COPIES:
      if (value > 0xFFFFFFFFull) return MR_EINVAL;
      c->opt_km_stop_copies = (uint32_t)value;
      return MR_OK;
  }
  return MR_EINVAL;
}

uint64_t mr_kernel_launches(const mr_ctx* c) { return c ? c->launches : 0; }

mr_status mr_rerun(mr_ctx* c) {
  if (!c) return MR_EINVAL;
  DeviceGuard g(c->device);
  if (c->batch_ids.empty()) return MR_EINVAL;
  std::vector<Job*> jobs;
  for (uint64_t id : c->batch_ids) {
    Job* j = find_job(c, id);
    if (!j) return MR_ENOJOB;
    jobs.push_back(j);
  }
  if (!c->batch_exec) {  // a job's containers moved since the capture
    mr_status st = build_batch_graph(c, jobs, c->tune, &c->batch_exec);
    if (st) return st;
  }
  for (Job* j : jobs)
    if (j->t0) MR_CUDA_TRY(cudaEventRecord(j->t0, c->stream));
  MR_CUDA_TRY(cudaGraphLaunch(c->batch_exec, c->stream));
  c->launches += c->batch_launches;
  for (Job* j : jobs) {
    if (j->t1) MR_CUDA_TRY(cudaEventRecord(j->t1, c->stream));
    MR_CUDA_TRY(cudaEventRecord(j->done, c->stream));
    j->state = JOB_ENQUEUED;
  }
  return MR_OK;
}

mr_status mr_get_tuning(const mr_ctx* c, mr_tuning* out) {
  if (!c || !out) return MR_EINVAL;
  *out = c->tune;
  return MR_OK;
}

mr_status mr_job_kernel_ms(mr_ctx* c, uint64_t job_id, float* ms, uint32_t* launches) {
  if (!c || !ms || !launches) return MR_EINVAL;
  DeviceGuard g(c->device);
  Job* j = find_job(c, job_id);
  if (!j) return MR_ENOJOB;
  if (j->state == JOB_PENDING) return MR_ENOTREADY;
  if (!j->kt || j->kt->n == 0) return MR_EINVAL;
  MR_CUDA_TRY(cudaEventSynchronize(j->kt->ev[2 * j->kt->n - 1]));
  float sum = 0.f;
  for (uint32_t i = 0; i < j->kt->n; ++i) {
    float t = 0.f;
    MR_CUDA_TRY(cudaEventElapsedTime(&t, j->kt->ev[2 * i], j->kt->ev[2 * i + 1]));
    sum += t;
  }
  *ms = sum;
  *launches = j->kt->n;
  return MR_OK;
}

mr_status mr_job_elapsed_ms(mr_ctx* c, uint64_t job_id, float* ms) {
  if (!c || !ms) return MR_EINVAL;
  DeviceGuard g(c->device);
  Job* j = find_job(c, job_id);
  if (!j) return MR_ENOJOB;
  if (j->state == JOB_PENDING) return MR_ENOTREADY;
  if (!j->t0 || !j->t1) return MR_EINVAL;
  MR_CUDA_TRY(cudaEventSynchronize(j->t1));
  MR_CUDA_TRY(cudaEventElapsedTime(ms, j->t0, j->t1));
  return MR_OK;
}

}  // extern "C"
