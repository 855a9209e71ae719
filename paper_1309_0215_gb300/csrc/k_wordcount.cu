// Word count: hash-table container (arXiv:1309.0215 Table I, Sec. III-A).
//
// Map (Sec. II-A): a token is a maximal run of bytes that are not ASCII
// whitespace; each emits (token, 1).  Reduce: sum.  Output ordered by count
// descending, then key bytes ascending (Sec. II-A "ordered (optional)").
//
// GB300 design
//  * Split (Sec. II-A, Fig. 1): 512-byte segments; a warp owns the tokens
//    whose FIRST byte lies in its segment and reads past the segment end to
//    finish them.  The segment (+64-byte halo) is staged in shared memory
//    with coalesced 128-bit loads.
//  * Token boundaries: each lane classifies its 16 bytes with SIMD-within-a-
//    register byte compares; a warp prefix sum over the per-lane start masks
//    lists every token start of the segment, and lanes take tokens from the
//    list 32 at a time — the GPU form of the paper's SIMD hashing (Sec.
//    III-C): lanes are the SIMD units and a lane that finishes a token takes
//    the next one from the list (as SIMDH-Stream refills a lane), the warp
//    prefix sum replacing the paper's prefix-sum lookup table.  A short token
//    is read as 16 bytes at once and becomes its own 128-bit key.
//  * Combiner / local container (Sec. III-A, Sec. III-D): a 2-way cache of
//    hot keys per warp in shared memory, merged into the global container
//    every few dozen segments (the paper's bounded local table handed to the
//    reduce side; see dev_wordcount.cuh).
//  * Global container: open addressing with a 128-bit CAS per new key and an
//    atomicAdd per combine (see dev_wordcount.cuh).
//  * Merge + sort: occupied slots of every job are compacted into one record
//    array and sorted by (job, count desc, key asc), so a batch of jobs is
//    ordered by a single launch sequence.  The sort path follows the record
//    capacity: up to 2^17 records a sample sort of compact (job/count word,
//    first 8 key bytes, index) keys, whose buckets are placed by rank in
//    shared memory; a batch of jobs whose tables each hold at most 2^17 slots
//    the same sample sort per job, all jobs side by side (segmented: one
//    sample, splitter set and bucket range per job); up to 2^20 a bitonic
//    block sort and merge passes; beyond, a stable LSD radix sort (8-bit
//    digits) whose digit positions equal in every key are skipped, decided on
//    the device so the sequence can be captured in a CUDA graph.  Records
//    that tie on both words (keys sharing their first 8 bytes and their
//    count) are then ordered by the full comparison (one thread per short
//    run, one CTA per longer run: bitonic sort up to 2048, merge sort
//    beyond).  Per-job boundaries and a scan of key lengths then place each
//    job's records and key bytes in its result: {u64 n, u64 key bytes;
//    n x {u64 count, u64 key_off, u64 key_len}; key bytes}.
#include "mr_internal.h"
#include "dev_wordcount.cuh"

namespace mrgb {
namespace {

using wc::JobDev;
using wc::WarpLocal;

constexpr int MAP_WARPS = 8;                 // per-warp-cache map kernel: 5 CTAs per SM
constexpr int MAP_THREADS = MAP_WARPS * 32;
constexpr int CTA_WARPS = 32;               // CTA-table map kernel: 1 CTA per SM
constexpr int CTA_THREADS = CTA_WARPS * 32;
// From this input size on the plain map pass uses the CTA-table kernel for a
// 16-byte-aligned input (whose next segment each warp loads ahead): each CTA
// then sees enough tokens (tens of thousands) that its table pays for its
// final merge of up to 4,096 keys into the global container (at 16 MiB the
// two kernels take the same time, at 48 MiB this one 6% less).
constexpr uint64_t CTA_MAP_MIN_BYTES = 32ull << 20;
constexpr int CB = 1024;            // records per compaction / sort / scan block
constexpr uint64_t CNT_MAX = (1ull << 40) - 1;

__device__ __forceinline__ JobDev job_at(const JobDev* jobs, const JobDev& single, uint32_t j) {
  return jobs ? jobs[j] : single;
}

// Plain map + combine pass for small inputs: each warp combines into its own
// hot-key cache (wc::WarpLocal) and inserts its misses at once (one slot per
// probe step: the misses of a round are few and mostly found at their first
// slot, where the second load costs more than it saves).
__global__ void __launch_bounds__(MAP_THREADS, 5) wc_map_kernel(JobDev J) {
  extern __shared__ __align__(16) unsigned char wc_smem[];
  WarpLocal& L = reinterpret_cast<WarpLocal*>(wc_smem)[threadIdx.x >> 5];
  wc::local_clear(L);
  int occ = 0;
  const uint64_t nseg = (J.n + wc::SEG - 1) / wc::SEG;
  const uint64_t gw = (uint64_t)blockIdx.x * MAP_WARPS + (threadIdx.x >> 5);
  const uint64_t nw = (uint64_t)gridDim.x * MAP_WARPS;
  for (uint64_t seg = gw; seg < nseg; seg += nw) wc::warp_segment<1>(J, seg, L, occ);
  wc::local_flush<1>(L, occ, J);
}

// Plain map + combine pass for large inputs: one CTA of CTA_WARPS warps per
// SM, sharing one local table (wc::CtaTableBig, 4,096 slots); a warp's
// misses are queued and sent to the global container 32 at a time; at the
// end every warp empties its queue and the CTA merges its table into the
// global container.
__global__ void __launch_bounds__(CTA_THREADS, 1) wc_map_cta_kernel(JobDev J) {
  extern __shared__ __align__(16) unsigned char wc_smem[];
  wc::CtaTableBig& T = *reinterpret_cast<wc::CtaTableBig*>(wc_smem);
  wc::MapWarp& W = reinterpret_cast<wc::MapWarp*>(wc_smem + sizeof(wc::CtaTableBig))[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < wc::CtaTableBig::SLOTS; i += CTA_THREADS) T.key[i] = make_ulonglong2(0ull, 0ull);
  __syncthreads();
  const uint64_t nseg = (J.n + wc::SEG - 1) / wc::SEG;
  const uint64_t gw = (uint64_t)blockIdx.x * CTA_WARPS + (threadIdx.x >> 5);
  const uint64_t nw = (uint64_t)gridDim.x * CTA_WARPS;
  uint32_t qn = 0, qhd = 0;
  // the warp's next segment is loaded while it works on the current one
  uint4 pre[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
  bool have = gw < nseg && wc::seg_prefetchable(J, gw);
  if (have) wc::seg_prefetch(J, gw, pre);
  for (uint64_t seg = gw; seg < nseg; seg += nw) {
    const uint64_t base = seg * wc::SEG;
    uint4 cur[2] = {pre[0], pre[1]};
    const bool cur_ok = have;
    have = seg + nw < nseg && wc::seg_prefetchable(J, seg + nw);
    if (have) wc::seg_prefetch(J, seg + nw, pre);
    const int total = wc::stage_tokens(J, seg, W, cur_ok ? cur : nullptr);
    for (int r0 = 0; r0 < total; r0 += 32) {
      const int i = r0 + lane;
      bool m = false;
      wc::Tok t{0, 0, 0};
      if (i < total) {
        t = wc::read_token(J.in, J.n, base, W, W.starts[i]);
        m = !wc::cta_add(T, t);
      }
      wc::mq_push(J, W, m, t, qn, qhd);
      __syncwarp();
    }
  }
  __syncwarp();
  if ((uint32_t)lane < qn) {
    const uint32_t q = (qhd + (uint32_t)lane) & (wc::MQ - 1);
    wc::global_insert(J, W.qw0[q], W.qw1[q], W.qh[q], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < wc::CtaTableBig::SLOTS; i += CTA_THREADS) {
    const ulonglong2 k = T.key[i];
    if (k.y != 0) wc::global_insert(J, k.x, k.y, T.h[i], T.cnt[i]);
  }
}


// ------------------------------------------------- pipelined map / reduce
// Sec. III-D pipelines the map and reduce phases on the hyper-threads of a
// core: map threads combine into a bounded local table and hand what it
// cannot hold to reduce threads, which insert into the global container.
// Here a CTA pairs PIPE_PAIRS mapper warps with as many reducer warps.  A
// mapper tokenizes, hashes and combines into its hot-key cache, and pushes
// the tokens the cache did not take into its own ring in shared memory
// (single producer, single consumer); its reducer warp inserts them into the
// global container, so the global-memory latency is spent by the reducers
// while the mappers go on tokenizing.  A mapper never waits for room: a
// round whose misses do not fit the ring sends them straight to the global
// container.  A reducer polls with __nanosleep and a bounded count; one that
// gives up marks its ring dead and its mapper drains the rest itself.
constexpr int PIPE_PAIRS = 4;
constexpr int PIPE_THREADS = 2 * PIPE_PAIRS * 32;
constexpr int RING = 256;
constexpr long long PIPE_SPIN_LIMIT = 1ll << 22;  // default polls of ~128 ns: about half a second

struct RingRec {
  unsigned long long w0, w1;
  uint32_t h, pad;
};
struct Ring {
  RingRec rec[RING];
  unsigned int head;  // records consumed (written by the reducer)
  unsigned int tail;  // records published (written by the mapper)
  unsigned int done;  // the mapper has published its last record
  unsigned int dead;  // the reducer gave up and no longer touches the ring
};
struct PipeSmem {
  WarpLocal local[PIPE_PAIRS];
  Ring ring[PIPE_PAIRS];
};

__device__ __forceinline__ unsigned vload(const unsigned int* p) { return *reinterpret_cast<const volatile unsigned int*>(p); }
__device__ __forceinline__ void vstore(unsigned int* p, unsigned v) { *reinterpret_cast<volatile unsigned int*>(p) = v; }

// polls: how many times a ring wait polls before it gives up (0: at once).
__global__ void __launch_bounds__(PIPE_THREADS, 4) wc_pipe_kernel(JobDev J, long long polls) {
  extern __shared__ __align__(16) unsigned char pipe_smem[];
  PipeSmem& S = *reinterpret_cast<PipeSmem*>(pipe_smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x < PIPE_PAIRS) {
    Ring& R = S.ring[threadIdx.x];
    R.head = R.tail = R.done = R.dead = 0;
  }
  __syncthreads();
  if (warp < PIPE_PAIRS) {
    // ------------------------------------------------------------ mapper
    WarpLocal& L = S.local[warp];
    Ring& R = S.ring[warp];
    wc::local_clear(L);
    int occ = 0;
    const unsigned below = (1u << lane) - 1u;
    auto push = [&](bool m, const wc::Tok& t) {
      const unsigned mm = __ballot_sync(0xffffffffu, m);
      if (!mm) return;
      const unsigned cnt = (unsigned)__popc(mm);
      const unsigned tail = vload(&R.tail);  // this warp is the only writer
      const unsigned head = vload(&R.head);
      if (!vload(&R.dead) && tail - head + cnt <= (unsigned)RING) {
        if (m) {
          RingRec& rr = R.rec[(tail + (unsigned)__popc(mm & below)) % RING];
          rr.w0 = t.w0;
          rr.w1 = t.w1;
          rr.h = t.h;
        }
        __syncwarp();
        if (lane == 0) {
          __threadfence_block();
          vstore(&R.tail, tail + cnt);
        }
      } else if (m) {
        wc::global_insert(J, t.w0, t.w1, t.h, 1);
      }
    };
    const uint64_t nseg = (J.n + wc::SEG - 1) / wc::SEG;
    const uint64_t stride = (uint64_t)gridDim.x * PIPE_PAIRS;
    for (uint64_t seg = (uint64_t)blockIdx.x * PIPE_PAIRS + warp; seg < nseg; seg += stride)
      wc::warp_segment_t(J, seg, L, occ, push);
    wc::local_flush(L, occ, J);
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      vstore(&R.done, 1u);
    }
    // wait for the reducer to drain the ring (or to give up)
    bool drained = false, dead = false;
    for (long long it = 0; it < polls; ++it) {
      dead = vload(&R.dead) != 0;
      drained = vload(&R.head) == vload(&R.tail);
      if (dead || drained) break;
      __nanosleep(128);
    }
    dead = __shfl_sync(0xffffffffu, dead, 0);
    drained = __shfl_sync(0xffffffffu, drained, 0);
    if (dead && !drained) {
      __threadfence_block();
      for (unsigned q = vload(&R.head) + lane; q < vload(&R.tail); q += 32) {
        const RingRec r = R.rec[q % RING];
        wc::global_insert(J, r.w0, r.w1, r.h, 1);
      }
    } else if (!dead && !drained && lane == 0) {
      atomicOr(J.state, 2u);  // the reducer neither finished nor gave up in time
    }
  } else {
    // ----------------------------------------------------------- reducer
    Ring& R = S.ring[warp - PIPE_PAIRS];
    unsigned head = 0;
    long long idle = 0;
    for (;;) {
      unsigned tail = 0, dn = 0;
      if (lane == 0) {
        dn = vload(&R.done);  // read before tail: with done set, the tail read is final
        __threadfence_block();
        tail = vload(&R.tail);
      }
      tail = __shfl_sync(0xffffffffu, tail, 0);
      dn = __shfl_sync(0xffffffffu, dn, 0);
      if (tail != head) {
        __threadfence_block();
        const unsigned n = (tail - head) < 32u ? (tail - head) : 32u;
        if ((unsigned)lane < n) {
          const RingRec r = R.rec[(head + (unsigned)lane) % RING];
          wc::global_insert(J, r.w0, r.w1, r.h, 1);
        }
        __syncwarp();
        head += n;
        if (lane == 0) {
          __threadfence_block();
          vstore(&R.head, head);
        }
        idle = 0;
        continue;
      }
      if (dn) break;
      if (++idle > polls) {
        if (lane == 0) {
          __threadfence_block();
          vstore(&R.dead, 1u);
        }
        break;
      }
      __nanosleep(128);
    }
  }
}

// ------------------------------------------------------------------ sort
struct SortRec {
  unsigned long long key1;  // job << 40 | (2^40 - 1 - count): ascending = job, then count descending
  unsigned long long s0;    // key bytes 0..7, big-endian, zero padded
  unsigned long long s1;    // key bytes 8..15
  uint32_t len;             // key length (saturated at 2^32 - 1)
  uint32_t idx;             // index of the record's source offset (long keys)
};
static_assert(sizeof(SortRec) == 32, "SortRec layout");

// Radix sort geometry: one 256-thread CTA per tile of 2048 records, 8 items
// per thread; tile histograms are scanned in chunks of 32 tiles.
constexpr int RT = 256;
constexpr int RIPT = 8;
constexpr int RTILE = RT * RIPT;
constexpr int RCHUNK = 32;
constexpr int NPASS = 16;       // 8 digits of s0, then 8 digits of key1
constexpr int FIX_THREAD = 32;  // tie runs up to this long: one thread's insertion sort
// The radix sort runs ~70 short launches whatever the record count; below
// this capacity the comparison sort (fewer, fuller launches) is faster.
constexpr uint64_t RADIX_MIN_RECORDS = 1ull << 20;

struct Post {
  SortRec* r0;
  SortRec* r1;
  unsigned long long* src;   // [R] input offset of a long key
  unsigned long long* excl;  // [R] exclusive scan of key lengths in sorted order
  unsigned long long* bsum;  // [ceil(R / CB)]
  // [0] number of records; [2] tie runs of up to SB records listed; [3] tie
  // runs longer than SB listed; [4..7] OR of ~key1, key1, ~s0, s0 (digits
  // equal in every key)
  unsigned long long* glob;
  unsigned long long* kh[2];  // radix ping-pong: key1
  unsigned long long* kl[2];  // s0
  uint32_t* kv[2];            // record index
  uint32_t* hist;             // [tiles][256] digit counts, per pass
  uint32_t* csum;             // [chunks][256] chunk sums, then chunk offsets
  uint32_t* plan;             // [NPASS] bit 0 active, bit 1 source buffer; [NPASS] final buffer
  uint2* runs;                // tie runs longer than FIX_THREAD: {first, length}
  struct KeyRec* kr[2];       // compact keys for the comparison sort of small record sets
  uint32_t* ss;               // sample sort: [0] buckets, [8..) group tickets; counts, offsets (+ end), cursors
  uint32_t* ss_rank;          // sample sort: [S] ranks of the sample
  struct KeyRec* spl;         // sample sort: the nb - 1 splitters
  uint16_t* bkt;              // sample sort: [R] bucket of each compacted record
  // segmented sample sort (several jobs sorted side by side, one bucket set
  // per job); jcur == nullptr outside it
  struct SegJob* seg;         // [jobs] where each job's records and buckets start
  uint32_t* jcur;             // [jobs] records compacted per job (cleared with bcnt)
  uint32_t* bcnt;             // [buckets] records per bucket
  uint32_t* boff;             // [buckets + 1] first record of each bucket (dense)
  uint2* bpos;                // [records] bucket and place in the bucket of each record (dense)
  uint32_t* kidx;             // [records] record indices in bucket order (dense)
  struct KeyRec* kra;         // [records] keys of a bucket too large to rank (dense)
  uint32_t* big;              // [buckets] buckets over one warp's share (count in glob[13])
};

__device__ __forceinline__ uint64_t bswap64(uint64_t v) {
  const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
  return ((uint64_t)__byte_perm(lo, 0, 0x0123) << 32) | __byte_perm(hi, 0, 0x0123);
}

__device__ bool rec_less(const SortRec& a, const SortRec& b, const JobDev* jobs, const JobDev& single,
                         const unsigned long long* src) {
  if (a.key1 != b.key1) return a.key1 < b.key1;
  if (a.s0 != b.s0) return a.s0 < b.s0;
  if (a.s1 != b.s1) return a.s1 < b.s1;
  if (a.len <= 16 || b.len <= 16) return a.len < b.len;
  // both longer than 16 bytes with the same first 16 (same job): compare on
  const uint8_t* in = job_at(jobs, single, (uint32_t)(a.key1 >> 40)).in;
  const uint64_t oa = src[a.idx], ob = src[b.idx];
  const uint32_t m = a.len < b.len ? a.len : b.len;
  for (uint32_t i = 16; i < m; ++i) {
    const uint8_t ca = in[oa + i], cb = in[ob + i];
    if (ca != cb) return ca < cb;
  }
  return a.len < b.len;
}

__device__ __forceinline__ uint32_t find_job_by_block(const JobDev* jobs, uint32_t njobs, uint64_t b) {
  uint32_t lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (jobs[mid].blk0 <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}


// One occupied slot (key words w0, w1; count cnt) -> its sort record at index i.
__device__ __forceinline__ void compact_record(const JobDev& J, uint32_t j, uint64_t cnt, uint64_t w0, uint64_t w1,
                                               uint64_t i, const Post& P) {
  SortRec rec;
  rec.key1 = ((uint64_t)j << 40) | (CNT_MAX - (cnt < CNT_MAX ? cnt : CNT_MAX));
  rec.idx = (uint32_t)i;
  if ((w1 >> 56) != 0xFF) {
    rec.len = (uint32_t)(w1 >> 56);
    rec.s0 = bswap64(w0);
    rec.s1 = bswap64(w1 & wc::LEN_MASK);
    P.src[i] = 0;
  } else {
    const uint64_t len = w1 & wc::LEN_MASK;
    const uint64_t off = w0 - 1;
    rec.len = len < 0xffffffffull ? (uint32_t)len : 0xffffffffu;
    uint64_t s0 = 0, s1 = 0;
    for (int q = 0; q < 16; ++q) {
      const uint64_t b = J.in[off + q];
      if (q < 8) s0 |= b << (56 - 8 * q);
      else s1 |= b << (56 - 8 * (q - 8));
    }
    rec.s0 = s0;
    rec.s1 = s1;
    P.src[i] = off;
  }
  P.r0[i] = rec;
}

// Occupied slots of every job -> records.  The slots are cut into blocks of
// CB (job j's blocks start at blk0); a CTA of CT threads takes a contiguous
// range of blocks, finding its first block's job once and following the job
// boundaries from there, and loads CPT slots per thread at a time.  The first
// block of a job also zeroes the job's result header (a job with no records
// keeps {0, 0}).  Records are packed from index 0 for the whole batch, or,
// for the segmented sort, from the start of each job's own slot range
// (P.jcur counts them per job).
constexpr int CT = 256;
constexpr int CPT = CB / CT;
__global__ void __launch_bounds__(CT) wc_compact_kernel(const JobDev* jobs, JobDev single, uint32_t njobs,
                                                        uint64_t nblocks, Post P) {
  __shared__ uint32_t wsum[CT / 32];
  __shared__ unsigned long long blk_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t per = (nblocks + gridDim.x - 1) / gridDim.x;
  const uint64_t b0 = (uint64_t)blockIdx.x * per;
  const uint64_t b1 = b0 + per < nblocks ? b0 + per : nblocks;
  if (b0 >= b1) return;
  uint32_t j = jobs ? find_job_by_block(jobs, njobs, b0) : 0;
  JobDev J = job_at(jobs, single, j);
  uint64_t next = jobs && j + 1 < njobs ? jobs[j + 1].blk0 : ~0ull;
  for (uint64_t b = b0; b < b1; ++b) {
    while (b >= next) {  // uniform across the CTA
      J = jobs[++j];
      next = j + 1 < njobs ? jobs[j + 1].blk0 : ~0ull;
    }
    if (b == J.blk0 && threadIdx.x < 2) reinterpret_cast<unsigned long long*>(J.out)[threadIdx.x] = 0;
    const uint64_t s0 = (b - J.blk0) * CB + threadIdx.x;
    uint64_t w0[CPT], w1[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const uint64_t slot = s0 + (uint64_t)q * CT;
      w0[q] = w1[q] = 0;
      if (slot < J.cap) {
        const ulonglong2 k = *reinterpret_cast<const ulonglong2*>(J.key + 2 * slot);
        w0[q] = k.x;
        w1[q] = k.y;
      }
    }
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < CPT; ++q) c += w1[q] != 0;
    // counts loaded before the scan and the reservation, so their latency
    // overlaps them (and before any record store, which could alias them)
    uint64_t cnt[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) cnt[q] = w1[q] != 0 ? J.cnt[s0 + (uint64_t)q * CT] : 0ull;
    uint32_t incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t ex = incl - c, total = 0;
#pragma unroll
    for (int w = 0; w < CT / 32; ++w) {
      const uint32_t v = wsum[w];
      if (w < warp) ex += v;
      total += v;
    }
    if (threadIdx.x == 0) {
      if (P.jcur)  // segmented sort: the job's records fill the start of its own slot range
        blk_base = total ? J.blk0 * CB + atomicAdd(P.jcur + j, total) : 0ull;
      else
        blk_base = total ? atomicAdd(P.glob, (unsigned long long)total) : 0ull;
    }
    __syncthreads();
    uint64_t i = blk_base + ex;
#pragma unroll
    for (int q = 0; q < CPT; ++q)
      if (w1[q] != 0) compact_record(J, j, cnt[q], w0[q], w1[q], i++, P);
  }
}

// Tie runs of up to SB records are ordered by one CTA's bitonic sort in
// shared memory (SB_THREADS threads); longer ones by one CTA's merge sort.
constexpr int SB = 2048;
constexpr int SB_THREADS = 1024;

// Compact-key sort of small record sets: KSB records per CTA in the block
// sort, then merge passes of KMT threads x KMI outputs per CTA (KMT * KMI
// divides 2 * KSB, so a merge tile never spans two pairs of runs).
constexpr int KSB = 512;
constexpr int KSB_THREADS = 256;
constexpr int KMT = 128;
constexpr int KMI = 4;
static_assert((2 * KSB) % (KMT * KMI) == 0, "merge tile must divide a pair of block-sorted runs");

// Compact key: (key1, s0, index).  The index only makes the order total;
// records that tie on (key1, s0) are put in the output order afterwards by
// the tie fix-up.
struct KeyRec {
  unsigned long long k1, k0;  // key1, s0 of the record
  uint32_t idx, pad;          // record index
};
struct KeyCmp {
  __device__ bool less(const KeyRec& a, const KeyRec& b) const {
    if (a.k1 != b.k1) return a.k1 < b.k1;
    if (a.k0 != b.k0) return a.k0 < b.k0;
    return a.idx < b.idx;
  }
  __device__ static KeyRec pad() { return KeyRec{~0ull, ~0ull, 0xffffffffu, 0u}; }
};

// Splitter s (key words s.x = key1, s.y = s0, index si) below key k (k.x,
// k.y, index ki): the borrow of the 160-bit subtraction s - k, no branches.
__device__ __forceinline__ bool key_below(ulonglong2 s, uint32_t si, ulonglong2 k, uint32_t ki) {
  uint32_t borrow;
  asm("{\n\t.reg .u32 t;\n\t"
      "sub.cc.u32 t, %1, %6;\n\t"
      "subc.cc.u32 t, %2, %7;\n\t"
      "subc.cc.u32 t, %3, %8;\n\t"
      "subc.cc.u32 t, %4, %9;\n\t"
      "subc.cc.u32 t, %5, %10;\n\t"
      "subc.u32 %0, 0, 0;\n\t}"
      : "=r"(borrow)
      : "r"(si), "r"((uint32_t)s.y), "r"((uint32_t)(s.y >> 32)), "r"((uint32_t)s.x), "r"((uint32_t)(s.x >> 32)),
        "r"(ki), "r"((uint32_t)k.y), "r"((uint32_t)(k.y >> 32)), "r"((uint32_t)k.x), "r"((uint32_t)(k.x >> 32)));
  return borrow != 0;
}

// Block sort: NB items per CTA (NT threads), bitonic network in shared memory.
template <class R, class C, int NB, int NT>
__global__ void __launch_bounds__(NT) blocksort_kernel(R* data, const unsigned long long* glob, C cmp) {
  extern __shared__ __align__(16) unsigned char bs_raw[];
  R* sh = reinterpret_cast<R*>(bs_raw);
  const uint64_t m = glob[0];
  const uint64_t b0 = (uint64_t)blockIdx.x * NB;
  if (b0 >= m) return;
  for (int i = threadIdx.x; i < NB; i += NT) sh[i] = b0 + i < m ? data[b0 + i] : C::pad();
  __syncthreads();
  for (int k = 2; k <= NB; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int t = threadIdx.x; t < NB / 2; t += NT) {
        const int lo = 2 * jj * (t / jj) + (t % jj);
        const int hi = lo + jj;
        const bool up = (lo & k) == 0;
        const R a = sh[lo], b = sh[hi];
        if (cmp.less(b, a) == up) {
          sh[lo] = b;
          sh[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < NB; i += NT)
    if (b0 + i < m) data[b0 + i] = sh[i];
}

// Number of A records among the first kk outputs of merge(A[0..la), B[0..lb)),
// found by the whole warp: each step probes 32 evenly spaced positions at once
// (the "A[i] < B[kk-1-i]" predicate is true on a prefix), shrinking the range
// about 33-fold, so a search over L records costs ~log_33(L) dependent loads.
template <class R, class C>
__device__ uint64_t corank_warp(const R* A, uint64_t la, const R* B, uint64_t lb, uint64_t kk, const C& cmp) {
  const int lane = threadIdx.x & 31;
  uint64_t lo = kk > lb ? kk - lb : 0;
  uint64_t hi = kk < la ? kk : la;
  while (lo < hi) {
    const uint64_t span = hi - lo;
    const uint64_t m = lo + (span * (uint64_t)(lane + 1)) / 33;
    const bool pr = cmp.less(A[m], B[kk - 1 - m]);
    const unsigned bal = __ballot_sync(0xffffffffu, pr);
    const int nt = __popc(bal);
    const uint64_t mt = __shfl_sync(0xffffffffu, m, nt > 0 ? nt - 1 : 0);
    const uint64_t mf = __shfl_sync(0xffffffffu, m, nt < 32 ? nt : 31);
    const uint64_t nlo = nt > 0 ? mt + 1 : lo;
    const uint64_t nhi = nt < 32 ? mf : hi;
    lo = nlo;
    hi = nhi;
  }
  return lo;
}

// One merge pass: runs of L sorted items are merged pairwise.  A CTA owns
// T * I consecutive outputs: two warps find where its range starts and ends
// in the two runs, the CTA stages both input windows in shared memory, and
// each thread merges I outputs from there.
template <class R, class C, int T, int I>
__global__ void __launch_bounds__(T) merge_kernel(const R* __restrict__ src, R* __restrict__ dst, uint64_t L,
                                                  const unsigned long long* glob, C cmp) {
  constexpr int TILE = T * I;
  extern __shared__ __align__(16) unsigned char mg_raw[];
  R* ms = reinterpret_cast<R*>(mg_raw);
  __shared__ uint64_t cr[2];
  const uint64_t m = glob[0];
  const uint64_t o0 = (uint64_t)blockIdx.x * TILE;
  if (o0 >= m) return;
  const uint64_t a0 = (o0 / (2 * L)) * (2 * L);  // TILE divides 2L: a tile never spans two pairs
  const uint64_t la = (m - a0) < L ? (m - a0) : L;
  const uint64_t b0 = a0 + L;
  const uint64_t lb = b0 < m ? ((m - b0) < L ? (m - b0) : L) : 0;
  const R* A = src + a0;
  const R* B = src + b0;
  const uint64_t kk0 = o0 - a0;
  const uint64_t kk1 = (kk0 + TILE) < la + lb ? kk0 + TILE : la + lb;
  if (lb == 0) {  // a lone run: copy
    for (uint64_t t = kk0 + threadIdx.x; t < kk1; t += T) dst[a0 + t] = A[t];
    return;
  }
  const int warp = threadIdx.x >> 5;
  if (warp < 2) {
    const uint64_t kk = warp == 0 ? kk0 : kk1;
    const uint64_t c = corank_warp(A, la, B, lb, kk, cmp);
    if ((threadIdx.x & 31) == 0) cr[warp] = c;
  }
  __syncthreads();
  const uint64_t i0 = cr[0], i1 = cr[1];
  const uint32_t na = (uint32_t)(i1 - i0);
  const uint32_t nb = (uint32_t)((kk1 - i1) - (kk0 - i0));
  for (uint32_t t = threadIdx.x; t < na; t += T) ms[t] = A[i0 + t];
  for (uint32_t t = threadIdx.x; t < nb; t += T) ms[na + t] = B[kk0 - i0 + t];
  __syncthreads();
  const R* sa = ms;
  const R* sb = ms + na;
  const uint32_t r0 = threadIdx.x * I;
  const uint32_t tot = na + nb;
  if (r0 >= tot) return;
  uint32_t lo = r0 > nb ? r0 - nb : 0, hi = r0 < na ? r0 : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (cmp.less(sa[mid], sb[r0 - 1 - mid])) lo = mid + 1;
    else hi = mid;
  }
  uint32_t i = lo, j = r0 - lo;
  for (int t = 0; t < I && r0 + t < tot; ++t) {
    bool takeA;
    if (j >= nb) takeA = true;
    else if (i >= na) takeA = false;
    else takeA = cmp.less(sa[i], sb[j]);
    dst[o0 + r0 + t] = takeA ? sa[i++] : sb[j++];
  }
}

// Exclusive scan of the block sums P.bsum[0..nb) in place, by one CTA.
__device__ void bsum_scan(Post& P, uint64_t nb) {
  __shared__ unsigned long long carry;
  __shared__ unsigned long long wsum[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t b = 0; b < nb; b += CB) {
    const uint64_t i = b + threadIdx.x;
    const unsigned long long v = i < nb ? __ldcg(P.bsum + i) : 0;
    unsigned long long incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const unsigned long long w = wsum[lane];
      unsigned long long wi = w;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      wsum[lane] = wi - w;
    }
    __syncthreads();
    const unsigned long long ex = carry + wsum[warp] + incl - v;
    if (i < nb) P.bsum[i] = ex;
    __syncthreads();
    if (threadIdx.x == CB - 1) carry = ex + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) P.glob[9] = carry;  // all key bytes
}


// Per-block sums of the key lengths.  With fuse (few blocks) the block that
// finishes last (a ticket in P.glob[8]) then scans them in place; with many
// blocks the tickets would serialise on one address, so wc_bscan_kernel does
// the scan instead.
__global__ void __launch_bounds__(CB) wc_lensum_kernel(Post P, bool fuse) {
  pdl_wait();
  __shared__ unsigned long long ws[32];
  __shared__ bool last;
  const SortRec* recs = P.r1;
  const uint64_t m = *P.glob;
  // fused: one block per CB records (all of them, for the ticket count);
  // otherwise a persistent grid over the live blocks
  for (uint64_t blk = blockIdx.x; fuse ? blk == blockIdx.x : blk * CB < m; blk += gridDim.x) {
    const uint64_t i = blk * CB + threadIdx.x;
    unsigned long long v = i < m ? recs[i].len : 0;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long s = 0;
      for (int w = 0; w < 32; ++w) s += ws[w];
      P.bsum[blk] = s;
    }
    __syncthreads();
  }
  if (!fuse) return;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(P.glob + 8, 1ull) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  bsum_scan(P, gridDim.x);
}

// Blocks past the last record hold no lengths: only the live ones are scanned.
__global__ void __launch_bounds__(CB) wc_bscan_kernel(Post P, uint64_t nb) {
  pdl_wait();
  const uint64_t live = (P.glob[0] + CB - 1) / CB;
  bsum_scan(P, live < nb ? live : nb);
}
constexpr uint64_t LENSUM_FUSE_BLOCKS = 4096;

// Exclusive length scan per record; each job's first / end record and the
// scan at both are stored in the job's state as 64-bit fields 1..4.
__global__ void __launch_bounds__(CB) wc_bounds_kernel(const JobDev* jobs, JobDev single, Post P) {
  pdl_wait();
  __shared__ unsigned long long wsum[32];
  const SortRec* recs = P.r1;
  const uint64_t m = *P.glob;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t blk = blockIdx.x; blk * CB < m; blk += gridDim.x) {
    const uint64_t i = blk * CB + threadIdx.x;
    const uint32_t len = i < m ? recs[i].len : 0;
    unsigned long long incl = len;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const unsigned long long w = wsum[lane];
      unsigned long long wi = w;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      wsum[lane] = wi - w;
    }
    __syncthreads();
    if (i < m) {
      const unsigned long long ex = P.bsum[blk] + wsum[warp] + incl - len;
      P.excl[i] = ex;
      const uint32_t j = (uint32_t)(recs[i].key1 >> 40);
      const bool first = i == 0 || (uint32_t)(recs[i - 1].key1 >> 40) != j;
      const bool last = i + 1 == m || (uint32_t)(recs[i + 1].key1 >> 40) != j;
      unsigned long long* st = reinterpret_cast<unsigned long long*>(job_at(jobs, single, j).state);
      if (first) {
        st[1] = i;
        st[2] = ex;
      }
      if (last) {
        st[3] = i + 1;
        st[4] = ex + len;
      }
    }
    __syncthreads();
  }
}

// Records and key bytes into each job's result.
// Record li of a job's nrec (key bytes at koff of kbytes) into its result.
__device__ __forceinline__ void emit_record(const JobDev& J, const Post& P, const SortRec& r, uint64_t li,
                                            uint64_t nrec, uint64_t koff, uint64_t kbytes) {
  unsigned long long* out = reinterpret_cast<unsigned long long*>(J.out);
  if (li == 0) {
    out[0] = nrec;
    out[1] = kbytes;
  }
  unsigned long long* rec = out + 2 + 3 * li;
  rec[0] = CNT_MAX - (r.key1 & CNT_MAX);
  rec[1] = koff;
  rec[2] = r.len;
  uint8_t* keys = J.out + 16 + 24 * nrec + koff;
  if (r.len <= 15) {
    for (uint32_t q = 0; q < r.len; ++q)
      keys[q] = (uint8_t)(q < 8 ? r.s0 >> (56 - 8 * q) : r.s1 >> (56 - 8 * (q - 8)));
  } else {
    const uint8_t* s = J.in + P.src[r.idx];
    for (uint32_t q = 0; q < r.len; ++q) keys[q] = s[q];
  }
}
__device__ __forceinline__ void gather_one(const JobDev* jobs, const JobDev& single, const Post& P,
                                           const SortRec* recs, uint64_t i) {
  const SortRec r = recs[i];
  const uint32_t j = (uint32_t)(r.key1 >> 40);
  const JobDev J = job_at(jobs, single, j);
  const unsigned long long* st = reinterpret_cast<const unsigned long long*>(J.state);
  const uint64_t first = st[1], scan0 = st[2], end = st[3], scan1 = st[4];
  emit_record(J, P, r, i - first, end - first, P.excl[i] - scan0, scan1 - scan0);
}
__global__ void __launch_bounds__(256) wc_gather_kernel(const JobDev* jobs, JobDev single, Post P) {
  pdl_wait();
  const SortRec* recs = P.r1;
  const uint64_t m = *P.glob;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    gather_one(jobs, single, P, recs, i);
}

// One job: its records are all records (first 0, end m, key bytes in
// P.glob[9]), so the bounds pass is not needed: each block scans its key
// lengths from the block sums and writes its records straight away.
__global__ void __launch_bounds__(CB) wc_gather1_kernel(JobDev J, Post P) {
  pdl_wait();
  __shared__ unsigned long long wsum[32];
  const SortRec* recs = P.r1;
  const uint64_t m = P.glob[0], kbytes = P.glob[9];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t blk = blockIdx.x; blk * CB < m; blk += gridDim.x) {
    const uint64_t i = blk * CB + threadIdx.x;
    SortRec r{};
    if (i < m) r = recs[i];
    unsigned long long incl = i < m ? r.len : 0;
    const unsigned long long len = incl;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const unsigned long long w = wsum[lane];
      unsigned long long wi = w;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      wsum[lane] = wi - w;
    }
    __syncthreads();
    if (i < m) emit_record(J, P, r, i, m, P.bsum[blk] + wsum[warp] + incl - len, kbytes);
    __syncthreads();
  }
}


// ------------------------------------------------------------ radix sort
// Keys and record indices of the compacted records, and which of the 16
// digit positions differ between keys (bitwise OR of ~key and of key: a
// digit position is constant iff both ORs agree there as complements).
__global__ void __launch_bounds__(CB) wc_rkeys_kernel(Post P) {
  __shared__ unsigned long long red[4][32];
  const uint64_t m = *P.glob;
  const uint64_t i = (uint64_t)blockIdx.x * CB + threadIdx.x;
  if ((uint64_t)blockIdx.x * CB >= m) return;
  unsigned long long v[4] = {0, 0, 0, 0};
  if (i < m) {
    const SortRec r = P.r0[i];
    P.kh[0][i] = r.key1;
    P.kl[0][i] = r.s0;
    P.kv[0][i] = (uint32_t)i;
    v[0] = ~r.key1;
    v[1] = r.key1;
    v[2] = ~r.s0;
    v[3] = r.s0;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    for (int o = 16; o; o >>= 1) v[q] |= __shfl_xor_sync(0xffffffffu, v[q], o);
    if (lane == 0) red[q][warp] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      unsigned long long w = red[q][lane];
      for (int o = 16; o; o >>= 1) w |= __shfl_xor_sync(0xffffffffu, w, o);
      if (lane == 0 && w) atomicOr(P.glob + 4 + q, w);
    }
  }
}

// Pass plan: a pass is run only if its digit differs between keys; its
// source is the buffer the previous run pass wrote.
__global__ void wc_rplan_kernel(Post P) {
  const uint64_t m = P.glob[0];
  const unsigned long long and_hi = ~P.glob[4], or_hi = P.glob[5];
  const unsigned long long and_lo = ~P.glob[6], or_lo = P.glob[7];
  uint32_t cur = 0;
  for (int p = 0; p < NPASS; ++p) {
    const unsigned long long diff = p < 8 ? (and_lo ^ or_lo) : (and_hi ^ or_hi);
    const bool active = m > 1 && ((diff >> (8 * (p & 7))) & 0xFFull) != 0;
    P.plan[p] = active ? (1u | (cur << 1)) : 0u;
    if (active) cur ^= 1u;
  }
  P.plan[NPASS] = cur;
}

__device__ __forceinline__ uint32_t rdigit(const Post& P, int p, uint32_t buf, uint64_t i) {
  const unsigned long long w = p < 8 ? P.kl[buf][i] : P.kh[buf][i];
  return (uint32_t)(w >> (8 * (p & 7))) & 0xFFu;
}

// Digit counts of each tile.
__global__ void __launch_bounds__(RT) wc_rhist_kernel(Post P, int p) {
  __shared__ uint32_t h[256];
  const uint32_t plan = P.plan[p];
  if (!(plan & 1u)) return;
  const uint64_t m = *P.glob;
  const uint64_t t0 = (uint64_t)blockIdx.x * RTILE;
  if (t0 >= m) return;
  const uint32_t src = (plan >> 1) & 1u;
  h[threadIdx.x] = 0;
  __syncthreads();
  for (int k = 0; k < RIPT; ++k) {
    const uint64_t i = t0 + (uint64_t)k * RT + threadIdx.x;
    if (i < m) atomicAdd(&h[rdigit(P, p, src, i)], 1u);
  }
  __syncthreads();
  P.hist[(uint64_t)blockIdx.x * 256 + threadIdx.x] = h[threadIdx.x];
}

// Per digit and chunk of RCHUNK tiles: the tiles' counts become exclusive
// prefixes within the chunk (in place), the chunk's sum goes to P.csum.
__global__ void __launch_bounds__(RT) wc_rscan1_kernel(Post P, int p) {
  if (!(P.plan[p] & 1u)) return;
  const uint64_t m = *P.glob;
  const uint64_t ntiles = (m + RTILE - 1) / RTILE;
  const uint64_t b0 = (uint64_t)blockIdx.x * RCHUNK;
  if (b0 >= ntiles) return;
  const uint64_t b1 = (b0 + RCHUNK) < ntiles ? b0 + RCHUNK : ntiles;
  uint32_t cnt[RCHUNK];
#pragma unroll
  for (int q = 0; q < RCHUNK; ++q) cnt[q] = b0 + q < b1 ? P.hist[(b0 + q) * 256 + threadIdx.x] : 0u;
  uint32_t sum = 0;
#pragma unroll
  for (int q = 0; q < RCHUNK; ++q) {
    if (b0 + q < b1) P.hist[(b0 + q) * 256 + threadIdx.x] = sum;
    sum += cnt[q];
  }
  P.csum[(uint64_t)blockIdx.x * 256 + threadIdx.x] = sum;
}

// One CTA: chunk offsets = digit base (exclusive scan of the digit totals)
// + exclusive scan over the chunks of that digit.
__global__ void __launch_bounds__(RT) wc_rscan2_kernel(Post P, int p) {
  __shared__ uint32_t tot[RT];
  if (!(P.plan[p] & 1u)) return;
  const uint64_t m = *P.glob;
  const uint64_t nchunks = ((m + RTILE - 1) / RTILE + RCHUNK - 1) / RCHUNK;
  const int d = threadIdx.x;
  uint32_t run = 0;
  for (uint64_t c = 0; c < nchunks; ++c) {
    const uint32_t t = P.csum[c * 256 + d];
    P.csum[c * 256 + d] = run;
    run += t;
  }
  tot[d] = run;
  __syncthreads();
  if (d == 0) {
    uint32_t acc = 0;
    for (int q = 0; q < RT; ++q) {
      const uint32_t t = tot[q];
      tot[q] = acc;
      acc += t;
    }
  }
  __syncthreads();
  const uint32_t base = tot[d];
  for (uint64_t c = 0; c < nchunks; ++c) P.csum[c * 256 + d] += base;
}

// Stable scatter of one tile.  Items are taken in 8 rounds of 256 (round k,
// warp w, lane l = tile position 256k + 32w + l), so tile order is (round,
// warp, lane).  Per round: lanes with the same digit are found with 8
// ballots (one per digit bit); each warp's digit counts are prefix-summed
// over the warps in order, on top of the counts of earlier rounds and of
// earlier tiles (chunk offset + the tile's prefix within its chunk).
__global__ void __launch_bounds__(RT) wc_rscatter_kernel(Post P, int p) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t wh[RT / 32][256];
  const uint32_t plan = P.plan[p];
  if (!(plan & 1u)) return;
  const uint64_t m = *P.glob;
  const uint64_t b = blockIdx.x;
  const uint64_t t0 = b * RTILE;
  if (t0 >= m) return;
  const uint32_t src = (plan >> 1) & 1u, dst = src ^ 1u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // chunk offset + this tile's prefix within the chunk
  run[threadIdx.x] = P.csum[(b / RCHUNK) * 256 + threadIdx.x] + P.hist[b * 256 + threadIdx.x];
  const unsigned below = (1u << lane) - 1u;
  for (int k = 0; k < RIPT; ++k) {
    const uint64_t i = t0 + (uint64_t)k * RT + threadIdx.x;
    const bool valid = i < m;
    unsigned long long hi = 0, lo = 0;
    uint32_t val = 0, d = 0;
    if (valid) {
      hi = P.kh[src][i];
      lo = P.kl[src][i];
      val = P.kv[src][i];
      d = (uint32_t)((p < 8 ? lo : hi) >> (8 * (p & 7))) & 0xFFu;
    }
    unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int bit = 0; bit < 8; ++bit) {
      const unsigned bb = __ballot_sync(0xffffffffu, valid && ((d >> bit) & 1u));
      peers &= ((d >> bit) & 1u) ? bb : ~bb;
    }
#pragma unroll
    for (int q = 0; q < RT / 32; ++q) wh[q][threadIdx.x] = 0;
    __syncthreads();
    const uint32_t wrank = (uint32_t)__popc(peers & below);
    if (valid && wrank == 0) wh[warp][d] = (uint32_t)__popc(peers);
    __syncthreads();
    {
      uint32_t r = run[threadIdx.x];
#pragma unroll
      for (int q = 0; q < RT / 32; ++q) {
        const uint32_t x = wh[q][threadIdx.x];
        wh[q][threadIdx.x] = r;
        r += x;
      }
      run[threadIdx.x] = r;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = wh[warp][d] + wrank;
      P.kh[dst][pos] = hi;
      P.kl[dst][pos] = lo;
      P.kv[dst][pos] = val;
    }
    __syncthreads();
  }
}

// Compact keys of the compacted records (small record sets).
__global__ void __launch_bounds__(256) wc_kkeys_kernel(Post P) {
  const uint64_t m = *P.glob;
  const uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x;
  if (i >= m) return;
  const SortRec r = P.r0[i];
  P.kr[0][i] = KeyRec{r.key1, r.s0, (uint32_t)i, 0u};
}

// Records in key order.
__global__ void __launch_bounds__(256) wc_kgather_kernel(Post P, const KeyRec* sorted) {
  const uint64_t m = *P.glob;
  const uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x;
  if (i >= m) return;
  P.r1[i] = P.r0[sorted[i].idx];
}

// Records in radix order.
__global__ void __launch_bounds__(256) wc_rgather_kernel(Post P) {
  const uint64_t m = *P.glob;
  const uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x;
  if (i >= m) return;
  const uint32_t fin = m > 1 ? P.plan[NPASS] : 0u;
  P.r1[i] = P.r0[m > 1 ? P.kv[fin][i] : i];
}

__device__ __forceinline__ bool rtie(const SortRec& a, const SortRec& b) { return a.key1 == b.key1 && a.s0 == b.s0; }

// Records that tie on (key1, s0) are ordered by the full comparison: a run
// of up to FIX_THREAD by its first thread; longer ones are listed for
// wc_rfix_cta_kernel: up to SB records in P.runs from the front (count in
// P.glob[2]), longer ones from the back (count in P.glob[3]).  Every listed run is longer than FIX_THREAD, so both lists
// together hold fewer than max_runs entries.
__device__ __forceinline__ void rfix_one(const Post& P, const JobDev* jobs, const JobDev& single, uint64_t max_runs,
                                         uint64_t i, uint64_t m) {
  if (i + 1 >= m) return;
  SortRec* r = P.r1;
  if (!rtie(r[i], r[i + 1])) return;
  if (i > 0 && rtie(r[i - 1], r[i])) return;  // not the first of its run
  uint64_t L = 2;
  while (i + L < m && L <= (uint64_t)SB && rtie(r[i], r[i + L])) ++L;
  if (L > (uint64_t)SB) {
    // longer than SB: the run is contiguous, so gallop then bisect for its end
    uint64_t lo = i + SB, hi = m, step = SB;
    for (;;) {
      const uint64_t q = lo + step;
      if (q >= m) break;
      if (!rtie(r[i], r[q])) {
        hi = q;
        break;
      }
      lo = q;
      step *= 2;
    }
    while (hi - lo > 1) {
      const uint64_t mid = lo + (hi - lo) / 2;
      if (rtie(r[i], r[mid])) lo = mid;
      else hi = mid;
    }
    L = hi - i;
  }
  if (L <= (uint64_t)FIX_THREAD) {
    for (uint64_t a = i + 1; a < i + L; ++a) {
      const SortRec x = r[a];
      uint64_t q = a;
      while (q > i && rec_less(x, r[q - 1], jobs, single, P.src)) {
        r[q] = r[q - 1];
        --q;
      }
      r[q] = x;
    }
  } else if (L <= (uint64_t)SB) {
    const unsigned long long k = atomicAdd(P.glob + 2, 1ull);
    if (k < max_runs) P.runs[k] = make_uint2((uint32_t)i, (uint32_t)L);
  } else {
    const unsigned long long k = atomicAdd(P.glob + 3, 1ull);
    if (k < max_runs) P.runs[max_runs - 1 - k] = make_uint2((uint32_t)i, (uint32_t)L);
  }
}

__global__ void __launch_bounds__(256) wc_rfix_kernel(Post P, const JobDev* jobs, JobDev single, uint64_t max_runs) {
  pdl_wait();
  const uint64_t m = *P.glob;
  for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i + 1 < m; i += (uint64_t)gridDim.x * 256)
    rfix_one(P, jobs, single, max_runs, i, m);
}

// Full record order (a pad, idx == ~0, sorts last).
struct RecCmp {
  const JobDev* jobs;
  JobDev single;
  const unsigned long long* src;
  __device__ bool less(const SortRec& a, const SortRec& b) const {
    const bool a_pad = a.idx == 0xffffffffu, b_pad = b.idx == 0xffffffffu;
    if (a_pad || b_pad) return b_pad && !a_pad;
    return rec_less(a, b, jobs, single, src);
  }
  __device__ static SortRec pad() { return SortRec{~0ull, ~0ull, ~0ull, 0xffffffffu, 0xffffffffu}; }
};

// CTA-wide bitonic sort of sh[0..n2) (n2 a power of two).
template <class R, class C>
__device__ void cta_bitonic(R* sh, int n2, const C& cmp) {
  for (int kk = 2; kk <= n2; kk <<= 1) {
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      for (int t = threadIdx.x; t < n2 / 2; t += blockDim.x) {
        const int lo = 2 * jj * (t / jj) + (t % jj);
        const int hi = lo + jj;
        const bool up = (lo & kk) == 0;
        const R a = sh[lo], b = sh[hi];
        if (cmp.less(b, a) == up) {
          sh[lo] = b;
          sh[hi] = a;
        }
      }
      __syncthreads();
    }
  }
}

// r[0..L) into sh (padded to a power of two) and sorted there; L <= capacity.
template <class R, class C>
__device__ void cta_sort_smem(const R* r, int L, R* sh, const C& cmp) {
  int n2 = 1;
  while (n2 < L) n2 <<= 1;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) sh[i] = i < L ? r[i] : C::pad();
  __syncthreads();
  cta_bitonic(sh, n2, cmp);
}

// Sort r[0..L) by one CTA: tiles of up to cap records (a power of two)
// sorted in shared memory, then merge passes of doubling width between r and
// tmp; in a pass each thread finds where its share of a pair's outputs starts
// in the two inputs (binary search on the merge path) and merges
// sequentially.  Returns the buffer that holds the result (r or tmp).
template <class R, class C>
__device__ R* cta_sort(R* r, R* tmp, uint64_t L, R* sh, int cap, const C& cmp) {
  for (uint64_t t0 = 0; t0 < L; t0 += cap) {
    const int n = (int)(L - t0 < (uint64_t)cap ? L - t0 : (uint64_t)cap);
    cta_sort_smem(r + t0, n, sh, cmp);
    for (int i = threadIdx.x; i < n; i += blockDim.x) r[t0 + i] = sh[i];
    __syncthreads();
  }
  R* in = r;
  R* out = tmp;
  for (uint64_t W = cap; W < L; W *= 2) {
    for (uint64_t a0 = 0; a0 < L; a0 += 2 * W) {
      const uint64_t la = L - a0 < W ? L - a0 : W;
      const uint64_t lb = L - a0 > W ? (L - a0 - W < W ? L - a0 - W : W) : 0;
      const R* A = in + a0;
      const R* B = A + la;
      const uint64_t tot = la + lb;
      const uint64_t per = (tot + blockDim.x - 1) / blockDim.x;
      const uint64_t kk = (uint64_t)threadIdx.x * per;
      if (kk >= tot) continue;
      uint64_t lo = kk > lb ? kk - lb : 0, hi = kk < la ? kk : la;
      while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (cmp.less(A[mid], B[kk - 1 - mid])) lo = mid + 1;
        else hi = mid;
      }
      uint64_t i = lo, j = kk - lo;
      const uint64_t e = kk + per < tot ? kk + per : tot;
      for (uint64_t o = kk; o < e; ++o) {
        const bool takeA = j >= lb || (i < la && !cmp.less(B[j], A[i]));
        out[a0 + o] = takeA ? A[i++] : B[j++];
      }
    }
    __syncthreads();
    R* t = in;
    in = out;
    out = t;
  }
  return in;
}

// One CTA per listed tie run: runs of up to SB records (P.runs from the
// front) by a bitonic sort in shared memory, longer ones (P.runs from the
// back) by a merge sort with the same place in P.r0 (free once the records
// are in key order) as scratch.
__global__ void __launch_bounds__(SB_THREADS) wc_rfix_cta_kernel(Post P, const JobDev* jobs, JobDev single,
                                                                 uint64_t max_runs) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char rf_raw[];
  SortRec* sh = reinterpret_cast<SortRec*>(rf_raw);
  const RecCmp cmp{jobs, single, P.src};
  uint64_t nl = P.glob[2], nh = P.glob[3];
  if (nl > max_runs) nl = max_runs;
  if (nh > max_runs - nl) nh = max_runs - nl;
  for (uint64_t k = blockIdx.x; k < nl + nh; k += gridDim.x) {
    const uint2 run = k < nl ? P.runs[k] : P.runs[max_runs - 1 - (k - nl)];
    SortRec* const home = P.r1 + run.x;
    if (k < nl) {
      cta_sort_smem(home, (int)run.y, sh, cmp);
      for (int i = threadIdx.x; i < (int)run.y; i += blockDim.x) home[i] = sh[i];
    } else {
      const SortRec* res = cta_sort(home, P.r0 + run.x, run.y, sh, SB, cmp);
      if (res != home)
        for (uint64_t i = threadIdx.x; i < run.y; i += blockDim.x) home[i] = res[i];
    }
    __syncthreads();
  }
}

// Sample sort of compact keys, for record capacities up to SS_MAX_RECORDS:
// five launches instead of a block sort and one launch per merge pass.
// Splitters drawn from evenly spaced records of the compacted array (hash
// order, so effectively a random sample) cut the keys into buckets of about
// SS_B records; one CTA per bucket then places each key by its rank, the
// number of smaller keys in the bucket (keys are distinct: the index breaks
// ties), counted against the bucket held in shared memory; every thread
// reads the same key at a time, so the reads are broadcasts.  The sample is
// ranked the same way, in parts.  A bucket over SS_RANK_MAX records (rare
// with SS_OVER samples per bucket) is sorted by its CTA with bitonic tiles
// and merge passes (the bucket code is shared with the segmented sort,
// further down).
constexpr uint64_t SS_MAX_RECORDS = 1ull << 17;
constexpr int SS_B = 128;
constexpr int SS_MAXB = (int)(SS_MAX_RECORDS / SS_B);
constexpr int SS_OVER = 4;
constexpr int SS_SMAX = SS_MAXB * SS_OVER;
constexpr int SS_RANK_MAX = 1024;
constexpr int SS_HDR = 32;  // [0] buckets, [8, 8 + SS_SMAX / 256) sample-group tickets
constexpr int SS_WORDS = SS_HDR + 3 * SS_MAXB + 1;
constexpr int SS_BPT = (SS_MAXB + 255) / 256;  // buckets per thread in the offset scan (256 threads)
static_assert(SS_MAXB <= 65535 && SS_BPT <= 8, "bucket ids are 16-bit; the offset scan holds SS_BPT counts a thread");
static_assert(SS_SMAX * 20 <= 227 * 1024, "the ranked sample must fit one CTA's shared memory");
static_assert(8 + SS_SMAX / 256 <= SS_HDR, "one ticket per group of 256 samples");
__device__ __forceinline__ uint32_t* ss_cnt(const Post& P) { return P.ss + SS_HDR; }
__device__ __forceinline__ uint32_t* ss_off(const Post& P) { return P.ss + SS_HDR + SS_MAXB; }  // nb + 1 entries
__device__ __forceinline__ uint32_t* ss_cur(const Post& P) { return P.ss + SS_HDR + 1 + 2 * SS_MAXB; }

__device__ __forceinline__ KeyRec key_of(const SortRec& r, uint64_t i) { return KeyRec{r.key1, r.s0, (uint32_t)i, 0u}; }

// Keys in shared memory as (key1, s0) pairs plus indices.  rank() counts the
// keys below a given one; one comparison is the borrow of the 160-bit
// difference b - a (five chained 32-bit subtractions, no branches).
struct KeySoA {
  ulonglong2* k;
  uint32_t* idx;
  __device__ KeySoA(unsigned char* raw, int cap)
      : k(reinterpret_cast<ulonglong2*>(raw)), idx(reinterpret_cast<uint32_t*>(reinterpret_cast<ulonglong2*>(raw) + cap)) {}
  __device__ void put(int i, const KeyRec& r) {
    k[i] = make_ulonglong2(r.k1, r.k0);
    idx[i] = r.idx;
  }
  __device__ uint32_t rank(int j0, int j1, unsigned long long a1, unsigned long long a0, uint32_t ai) const {
    const uint32_t a1h = (uint32_t)(a1 >> 32), a1l = (uint32_t)a1, a0h = (uint32_t)(a0 >> 32), a0l = (uint32_t)a0;
    uint32_t r = 0;
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
      const ulonglong2 b = k[j];
      const uint32_t bi = idx[j];
      uint32_t borrow;
      asm("{\n\t.reg .u32 t;\n\t"
          "sub.cc.u32 t, %1, %6;\n\t"
          "subc.cc.u32 t, %2, %7;\n\t"
          "subc.cc.u32 t, %3, %8;\n\t"
          "subc.cc.u32 t, %4, %9;\n\t"
          "subc.cc.u32 t, %5, %10;\n\t"
          "subc.u32 %0, 0, 0;\n\t}"
          : "=r"(borrow)
          : "r"(bi), "r"((uint32_t)b.y), "r"((uint32_t)(b.y >> 32)), "r"((uint32_t)b.x), "r"((uint32_t)(b.x >> 32)),
            "r"(ai), "r"(a0l), "r"(a0h), "r"(a1l), "r"(a1h));
      r -= borrow;  // borrow is 0 or 0xffffffff
    }
    return r;
  }
};
constexpr int SS_PARTS = 16;  // the sample's ranks are counted in this many parts
static_assert(SS_SMAX / SS_PARTS <= 256, "a part's slice of the sample fits one slot per thread");

__device__ __forceinline__ void ss_geometry(uint64_t m, uint64_t& nb, uint64_t& S) {
  nb = (m + SS_B - 1) / SS_B;
  nb = nb < 1 ? 1 : (nb > (uint64_t)SS_MAXB ? (uint64_t)SS_MAXB : nb);
  S = m < nb * SS_OVER ? m : nb * SS_OVER;
}

// Ranks of the sample (evenly spaced records), counted in SS_PARTS parts:
// CTA (c, part) ranks samples 256c.. (one per thread, held in registers)
// against the part-th slice of the sample (in shared memory) and adds to
// P.ss_rank; the last of a group's SS_PARTS CTAs (a ticket) then holds the
// group's final ranks and writes the splitters among them: splitter b is the
// sample of rank ((b + 1) * S) / nb (distinct ranks, as S >= nb).  CTA 0
// also records the number of buckets.  Tickets, bucket counters and rank
// counters start at zero (cleared with P.glob).
__global__ void __launch_bounds__(256, 4) wc_ss_sample_kernel(Post P) {
  pdl_wait();
  __shared__ __align__(16) unsigned char sp_raw[256 * 20];  // KeySoA of 256 keys
  const uint64_t m = P.glob[0];
  uint64_t nb, S;
  ss_geometry(m, nb, S);
  const uint32_t c = blockIdx.x / SS_PARTS, part = blockIdx.x % SS_PARTS;
  if (blockIdx.x == 0 && threadIdx.x == 0) P.ss[0] = (uint32_t)nb;
  if ((uint64_t)c * 256 >= S) return;
  const uint64_t q0 = (S * part) / SS_PARTS, q1 = (S * (part + 1)) / SS_PARTS;
  KeySoA K(sp_raw, 256);
  for (uint64_t j = q0 + threadIdx.x; j < q1; j += 256) {
    const uint64_t q = ((2 * j + 1) * m) / (2 * S);
    K.put((int)(j - q0), key_of(P.r0[q], q));
  }
  const uint64_t j = (uint64_t)c * 256 + threadIdx.x;
  KeyRec own{0ull, 0ull, 0u, 0u};
  if (j < S) {
    const uint64_t q = ((2 * j + 1) * m) / (2 * S);
    own = key_of(P.r0[q], q);
  }
  __syncthreads();
  if (j < S) {
    const uint32_t r = K.rank(0, (int)(q1 - q0), own.k1, own.k0, own.idx);
    if (r) atomicAdd(&P.ss_rank[j], r);
  }
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&P.ss[8 + c], 1u) == SS_PARTS - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (j < S) {
    const uint64_t r = __ldcg(P.ss_rank + j);
    const uint64_t u = (r * nb + S - 1) / S;  // the only candidate b + 1
    if (u >= 1 && u < nb && (u * S) / nb == r) P.spl[u - 1] = own;
  }
}

// Bucket of each record (number of splitters below its key) and bucket sizes.
__global__ void __launch_bounds__(256) wc_ss_count_kernel(Post P) {
  pdl_wait();
  __shared__ KeyRec spl[SS_MAXB];
  __shared__ uint32_t cnt[SS_MAXB];
  const uint64_t m = P.glob[0];
  if ((uint64_t)blockIdx.x * 256 >= m) return;
  uint64_t nb, S;
  ss_geometry(m, nb, S);
  for (uint64_t t = threadIdx.x; t + 1 < nb; t += 256) spl[t] = P.spl[t];
  for (uint64_t t = threadIdx.x; t < nb; t += 256) cnt[t] = 0u;
  __syncthreads();
  const uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x;
  if (i < m) {
    const ulonglong2 kk = *reinterpret_cast<const ulonglong2*>(P.r0 + i);
    uint32_t lo = 0, hi = (uint32_t)nb - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (key_below(make_ulonglong2(spl[mid].k1, spl[mid].k0), spl[mid].idx, kk, (uint32_t)i)) lo = mid + 1;
      else hi = mid;
    }
    P.bkt[i] = (uint16_t)lo;
    atomicAdd(&cnt[lo], 1u);
  }
  __syncthreads();
  for (uint64_t t = threadIdx.x; t < nb; t += 256)
    if (cnt[t]) atomicAdd(&ss_cnt(P)[t], cnt[t]);
}

// Bucket offsets (each CTA scans the counts; CTA 0 stores them), then each
// CTA reserves one range per bucket it holds and places its keys there.
__global__ void __launch_bounds__(256) wc_ss_scatter_kernel(Post P) {
  pdl_wait();
  __shared__ uint32_t off[SS_MAXB + 1];
  __shared__ uint32_t cnt[SS_MAXB];
  __shared__ uint32_t wsum[8];
  const uint64_t m = P.glob[0];
  const uint32_t nb = P.ss[0];
  if (blockIdx.x > 0 && (uint64_t)blockIdx.x * 256 >= m) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // exclusive scan of the counts, SS_BPT consecutive buckets per thread
  const uint32_t b0 = SS_BPT * threadIdx.x;
  uint32_t c[SS_BPT], tot = 0;
#pragma unroll
  for (int q = 0; q < SS_BPT; ++q) {
    c[q] = b0 + q < nb ? ss_cnt(P)[b0 + q] : 0u;
    tot += c[q];
  }
  uint32_t incl = tot;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint32_t ex = incl - tot;
  for (int w = 0; w < warp; ++w) ex += wsum[w];
#pragma unroll
  for (int q = 0; q < SS_BPT; ++q) {
    if (b0 + q < nb) off[b0 + q] = ex;
    ex += c[q];
  }
  if (threadIdx.x == 0) off[nb] = (uint32_t)m;
  for (uint32_t t = threadIdx.x; t < nb; t += 256) cnt[t] = 0u;
  __syncthreads();
  if (blockIdx.x == 0)
    for (uint32_t t = threadIdx.x; t <= nb; t += 256) ss_off(P)[t] = off[t];
  if ((uint64_t)blockIdx.x * 256 >= m) return;
  const uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x;
  uint32_t b = 0, r = 0;
  if (i < m) {
    b = P.bkt[i];
    r = atomicAdd(&cnt[b], 1u);
  }
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < nb; t += 256)
    if (cnt[t]) cnt[t] = off[t] + atomicAdd(&ss_cur(P)[t], cnt[t]);
  __syncthreads();
  if (i < m) P.kr[0][cnt[b] + r] = key_of(P.r0[i], i);
}

// ------------------------------------------- segmented sample sort (batches)
// A batch of word-count jobs whose tables hold at most SS_MAX_RECORDS slots
// each is sorted job by job, all jobs side by side: every job gets its own
// sample, splitters and buckets of about SEG_B records, a bucket never mixes
// jobs, and the work per record stays that of a sort of at most 2^17
// records however many records the batch holds (a radix sort of the whole
// batch runs a dozen digit passes over all of them).  Compaction puts job
// j's records at the start of the job's own slot range; the plan then gives
// each job a dense range (jobs in order) and a range of buckets.  Buckets are
// placed by rank, one warp per bucket, from the bucket's keys in the warp's
// shared memory; the few over SEG_WCAP records are listed and placed by a
// CTA each.
struct SegJob {
  uint32_t cbase;  // first record of the job in slot order (compacted records)
  uint32_t d;      // first record of the job in the dense sorted order
  uint32_t m;      // records of the job
  uint32_t nb;     // buckets of the job
  uint32_t bbase;  // first bucket of the job
  uint32_t pad[3];
};
static_assert(sizeof(SegJob) == 32, "SegJob layout");
constexpr int SEG_B = 64;                                // records per bucket, on average
constexpr int SEG_OVER = 2;                              // samples per bucket
constexpr int SEG_MAXB = (int)(SS_MAX_RECORDS / SEG_B);  // buckets of one job, at most
constexpr int SEG_SMAX = SEG_MAXB * SEG_OVER;            // sample of one job, at most
constexpr int SEG_T = 256;
constexpr int SEG_I = 8;
constexpr int SEG_TILE = SEG_T * SEG_I;   // dense records per tile of the count and scatter passes
constexpr int SEG_SAMPLE_T = 512;         // threads of the sample sort
constexpr int SEG_BPT = SEG_MAXB / 256;   // bucket counts per thread in the offset scan
constexpr int SEG_COUNT_SMEM = SEG_MAXB * (16 + 4 + 4);  // splitters (keys, indices), bucket counts
constexpr int SEG_WCAP = 256;             // largest bucket one warp places
constexpr int SEG_WARPS = 8;              // warps per CTA of the warp pass
constexpr int SEG_WARP_SMEM = SEG_WARPS * SEG_WCAP * 20;
constexpr int SEG_BT = 128;               // threads of the large-bucket pass
constexpr int SEG_FB_CAP = 1024;          // bitonic tile of its merge sort
// shared memory of a CTA that places one bucket (ranked keys, or the merge sort's tile)
constexpr int BUCKET_CTA_SMEM = SEG_FB_CAP * (int)sizeof(KeyRec) > SS_RANK_MAX * 20 ? SEG_FB_CAP * (int)sizeof(KeyRec)
                                                                                  : SS_RANK_MAX * 20;
static_assert(SEG_MAXB % 256 == 0 && SEG_SMAX * (int)sizeof(KeyRec) <= 227 * 1024, "segmented sort geometry");

// Buckets and sample size of a job of m records (m <= SS_MAX_RECORDS).
__host__ __device__ __forceinline__ void seg_geom(uint64_t m, uint64_t& nb, uint64_t& S) {
  nb = (m + SEG_B - 1) / SEG_B;
  nb = nb < 1 ? 1 : (nb > (uint64_t)SEG_MAXB ? (uint64_t)SEG_MAXB : nb);
  S = m < nb * SEG_OVER ? m : nb * SEG_OVER;
}

// Per-job record counts (P.jcur, from the compaction) -> dense and bucket
// ranges; one CTA scans the jobs in chunks of CB.  P.glob[0] = records,
// P.glob[12] = buckets.  Both sums stay below 2^32 (the record indices are
// 32-bit), so they are scanned as the two halves of one 64-bit word.
__global__ void __launch_bounds__(CB) wc_seg_plan_kernel(const JobDev* jobs, uint32_t njobs, Post P) {
  __shared__ unsigned long long ws[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long carry = 0;
  for (uint32_t j0 = 0; j0 < njobs; j0 += CB) {
    const uint32_t j = j0 + threadIdx.x;
    uint64_t m = 0, nb = 0, S = 0;
    if (j < njobs) {
      m = P.jcur[j];
      seg_geom(m, nb, S);
    }
    const unsigned long long v = (nb << 32) | m;
    unsigned long long incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const unsigned long long w = ws[lane];
      unsigned long long wi = w;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      ws[lane] = wi - w;
      if (lane == 31) ws[32] = wi;
    }
    __syncthreads();
    const unsigned long long ex = carry + ws[warp] + incl - v;
    if (j < njobs)
      P.seg[j] = SegJob{(uint32_t)(jobs[j].blk0 * CB), (uint32_t)ex, (uint32_t)m, (uint32_t)nb, (uint32_t)(ex >> 32),
                        {0u, 0u, 0u}};
    carry += ws[32];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.glob[0] = carry & 0xffffffffull;
    P.glob[12] = carry >> 32;
  }
}

// Splitters of each job: its sample (S evenly spaced records of the job in
// slot order, i.e. hash order) sorted by one CTA with a bitonic network in
// shared memory; splitter u - 1 is the sample of rank (u * S) / nb.
__global__ void __launch_bounds__(SEG_SAMPLE_T) wc_seg_sample_kernel(Post P, uint32_t njobs) {
  extern __shared__ __align__(16) unsigned char sg_raw[];
  KeyRec* sh = reinterpret_cast<KeyRec*>(sg_raw);
  for (uint32_t j = blockIdx.x; j < njobs; j += gridDim.x) {
    const SegJob g = P.seg[j];
    uint64_t nb, S;
    seg_geom(g.m, nb, S);
    if (nb < 2) continue;
    int n2 = 1;
    while (n2 < (int)S) n2 <<= 1;
    for (int t = threadIdx.x; t < n2; t += SEG_SAMPLE_T) {
      if (t < (int)S) {
        const uint64_t q = g.cbase + ((2 * (uint64_t)t + 1) * g.m) / (2 * S);
        const ulonglong2 kk = *reinterpret_cast<const ulonglong2*>(P.r0 + q);
        sh[t] = KeyRec{kk.x, kk.y, (uint32_t)q, 0u};
      } else {
        sh[t] = KeyCmp::pad();
      }
    }
    __syncthreads();
    cta_bitonic(sh, n2, KeyCmp{});
    for (uint64_t u = 1 + threadIdx.x; u < nb; u += SEG_SAMPLE_T) P.spl[g.bbase + u - 1] = sh[(u * S) / nb];
    __syncthreads();
  }
}

// The job that holds dense record k < records: the last job that starts at
// or before k (a job without records starts where the next one does, so the
// last one starting there has records).
__device__ __forceinline__ uint32_t seg_job_of(const SegJob* seg, uint32_t njobs, uint64_t k) {
  uint32_t lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (seg[mid].d <= k) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Bucket of each record (its job's splitters in shared memory) and its place
// in the bucket: a CTA counts its records per bucket in shared memory, then
// reserves each bucket's share with one global atomic whose old value is
// where the share starts.  A tile of SEG_TILE dense records usually lies in
// one job; one that spans several takes them one job at a time.
__global__ void __launch_bounds__(SEG_T) wc_seg_count_kernel(Post P, uint32_t njobs) {
  extern __shared__ __align__(16) unsigned char sc_raw[];
  ulonglong2* sk = reinterpret_cast<ulonglong2*>(sc_raw);                  // splitter (key1, s0)
  uint32_t* si = reinterpret_cast<uint32_t*>(sc_raw + SEG_MAXB * 16);    // splitter index
  uint32_t* cnt = si + SEG_MAXB;
  const uint64_t M = P.glob[0];
  // a contiguous range of tiles per CTA: the job of its first record is
  // found once, later tiles follow the job boundaries
  const uint64_t ntiles = (M + SEG_TILE - 1) / SEG_TILE, per = (ntiles + gridDim.x - 1) / gridDim.x;
  const uint64_t tb = (uint64_t)blockIdx.x * per, te = tb + per < ntiles ? tb + per : ntiles;
  uint32_t jt = tb < te ? seg_job_of(P.seg, njobs, tb * SEG_TILE) : 0u;
  for (uint64_t tile = tb; tile < te; ++tile) {
    const uint64_t k0 = tile * SEG_TILE;
    const uint64_t k1 = k0 + SEG_TILE < M ? k0 + SEG_TILE : M;
    while (k0 >= (uint64_t)P.seg[jt].d + P.seg[jt].m) ++jt;  // uniform: a job that ends by k0
    uint32_t bk[SEG_I], lr[SEG_I];
    for (uint32_t j = jt; j < njobs; ++j) {
      const SegJob g = P.seg[j];
      if (g.d >= k1) break;
      if (g.m == 0) continue;
      for (uint32_t t = threadIdx.x; t + 1 < g.nb; t += SEG_T) {
        const KeyRec r = P.spl[g.bbase + t];
        sk[t] = make_ulonglong2(r.k1, r.k0);
        si[t] = r.idx;
      }
      for (uint32_t t = threadIdx.x; t < g.nb; t += SEG_T) cnt[t] = 0u;
      __syncthreads();
      const uint64_t a = k0 > g.d ? k0 : g.d;
      const uint64_t b = k1 < (uint64_t)g.d + g.m ? k1 : (uint64_t)g.d + g.m;
#pragma unroll
      for (int q = 0; q < SEG_I; ++q) {
        const uint64_t k = k0 + q * SEG_T + threadIdx.x;
        if (k >= a && k < b) {
          const uint32_t i = g.cbase + (uint32_t)(k - g.d);
          const ulonglong2 kk = *reinterpret_cast<const ulonglong2*>(P.r0 + i);
          uint32_t lo = 0, hi = g.nb - 1;
          while (lo < hi) {  // first splitter not below the key
            const uint32_t mid = (lo + hi) >> 1;
            if (key_below(sk[mid], si[mid], kk, i)) lo = mid + 1;
            else hi = mid;
          }
          bk[q] = lo;
          lr[q] = atomicAdd(&cnt[lo], 1u);
        }
      }
      __syncthreads();
      for (uint32_t t = threadIdx.x; t < g.nb; t += SEG_T)
        if (cnt[t]) cnt[t] = atomicAdd(P.bcnt + g.bbase + t, cnt[t]);
      __syncthreads();
#pragma unroll
      for (int q = 0; q < SEG_I; ++q) {
        const uint64_t k = k0 + q * SEG_T + threadIdx.x;
        if (k >= a && k < b) P.bpos[k] = make_uint2(g.bbase + bk[q], cnt[bk[q]] + lr[q]);
      }
      __syncthreads();
    }
  }
}

// Bucket offsets, one CTA per job: the job's dense start plus the exclusive
// scan of its bucket counts; boff[bbase + nb] is the job's end (the next
// job's start, written by both with the same value).
__global__ void __launch_bounds__(256) wc_seg_offsets_kernel(Post P, uint32_t njobs) {
  __shared__ uint32_t wsum[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t j = blockIdx.x; j < njobs; j += gridDim.x) {
    const SegJob g = P.seg[j];
    const uint32_t b0 = SEG_BPT * threadIdx.x;
    uint32_t c[SEG_BPT], tot = 0;
#pragma unroll
    for (int q = 0; q < SEG_BPT; ++q) {
      c[q] = b0 + q < g.nb ? P.bcnt[g.bbase + b0 + q] : 0u;
      tot += c[q];
    }
    uint32_t incl = tot;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t ex = g.d + incl - tot;
    for (int w = 0; w < warp; ++w) ex += wsum[w];
#pragma unroll
    for (int q = 0; q < SEG_BPT; ++q) {
      if (b0 + q < g.nb) P.boff[g.bbase + b0 + q] = ex;
      ex += c[q];
    }
    if (threadIdx.x == 0) P.boff[g.bbase + g.nb] = g.d + g.m;
    __syncthreads();
  }
}

// Record indices (slot order) to their places in bucket order.
__global__ void __launch_bounds__(SEG_T) wc_seg_scatter_kernel(Post P, uint32_t njobs) {
  // tiles interleaved across CTAs: the CTAs running at a time write into a
  // few jobs' ranges, where the L2 merges the partial-sector stores
  __shared__ uint32_t jfirst;
  const uint64_t M = P.glob[0];
  for (uint64_t k0 = (uint64_t)blockIdx.x * SEG_TILE; k0 < M; k0 += (uint64_t)gridDim.x * SEG_TILE) {
    if (threadIdx.x == 0) jfirst = seg_job_of(P.seg, njobs, k0);
    __syncthreads();
    uint32_t j = jfirst;
    SegJob g = P.seg[j];
#pragma unroll
    for (int q = 0; q < SEG_I; ++q) {
      const uint64_t k = k0 + q * SEG_T + threadIdx.x;
      if (k < M) {
        while (k >= (uint64_t)g.d + g.m) g = P.seg[++j];
        const uint2 bp = P.bpos[k];
        P.kidx[P.boff[bp.x] + bp.y] = g.cbase + (uint32_t)(k - g.d);
      }
    }
    __syncthreads();
  }
}

// Rank of key a among k[0..n): the number of keys below it.  rank128
// compares {index, s0, key1 low word} (one shared-memory load each, one
// comparison = the borrow of a 4-word subtraction), for keys whose key1 high
// word (the job, and the count's bits from 2^32 up) is the same; rank160
// adds key1's high word.
__device__ __forceinline__ uint32_t rank128(const uint4* k, int n, uint4 a) {
  uint32_t r = 0;
#pragma unroll 4
  for (int j = 0; j < n; ++j) {
    const uint4 b = k[j];
    uint32_t borrow;
    asm("{\n\t.reg .u32 t;\n\t"
        "sub.cc.u32 t, %1, %5;\n\t"
        "subc.cc.u32 t, %2, %6;\n\t"
        "subc.cc.u32 t, %3, %7;\n\t"
        "subc.cc.u32 t, %4, %8;\n\t"
        "subc.u32 %0, 0, 0;\n\t}"
        : "=r"(borrow)
        : "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w), "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w));
    r -= borrow;  // borrow is 0 or 0xffffffff: b < a
  }
  return r;
}
__device__ __forceinline__ uint32_t rank160(const uint4* k, const uint32_t* hi, int n, uint4 a, uint32_t ah) {
  uint32_t r = 0;
#pragma unroll 4
  for (int j = 0; j < n; ++j) {
    const uint4 b = k[j];
    const uint32_t bh = hi[j];
    uint32_t borrow;
    asm("{\n\t.reg .u32 t;\n\t"
        "sub.cc.u32 t, %1, %6;\n\t"
        "subc.cc.u32 t, %2, %7;\n\t"
        "subc.cc.u32 t, %3, %8;\n\t"
        "subc.cc.u32 t, %4, %9;\n\t"
        "subc.cc.u32 t, %5, %10;\n\t"
        "subc.u32 %0, 0, 0;\n\t}"
        : "=r"(borrow)
        : "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w), "r"(bh), "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(ah));
    r -= borrow;
  }
  return r;
}

// Bucket placement, shared by the one-job sample sort (keys of bucket b in
// P.kr[0][off[b]..off[b + 1]), offsets in ss_off, bucket count in ss[0])
// and the segmented sort (record indices in P.kidx, keys read from P.r0,
// offsets in P.boff, bucket count in glob[12]).  A bucket's keys go to
// shared memory as {index, s0 lo, s0 hi, key1 lo} plus key1 hi; each record
// is then written to the place its rank in the bucket gives (keys are
// distinct: the index breaks ties).  When key1's high word is the same in
// every key of the bucket (one job, every count below 2^32: always so in the
// segmented sort's buckets) the rank compares 128 bits, else 160.
template <bool SEG>
__device__ __forceinline__ void bucket_key(const Post& P, uint32_t o, uint32_t t, uint4* k4, uint32_t* kh) {
  unsigned long long k1, k0;
  uint32_t i;
  if (SEG) {
    i = P.kidx[o + t];
    const ulonglong2 kk = *reinterpret_cast<const ulonglong2*>(P.r0 + i);
    k1 = kk.x;
    k0 = kk.y;
  } else {
    const KeyRec r = P.kr[0][o + t];
    k1 = r.k1;
    k0 = r.k0;
    i = r.idx;
  }
  k4[t] = make_uint4(i, (uint32_t)k0, (uint32_t)(k0 >> 32), (uint32_t)k1);
  kh[t] = (uint32_t)(k1 >> 32);
}
template <bool SEG>
__device__ __forceinline__ uint64_t bucket_count(const Post& P) {
  return SEG ? P.glob[12] : (uint64_t)P.ss[0];
}
template <bool SEG>
__device__ __forceinline__ const uint32_t* bucket_off(const Post& P) {
  return SEG ? P.boff : ss_off(P);
}
__device__ __forceinline__ void place_by_rank(const Post& P, uint32_t o, uint32_t L, const uint4* k4,
                                              const uint32_t* kh, bool same_hi, uint32_t t0, uint32_t stride) {
  if (same_hi) {
    for (uint32_t t = t0; t < L; t += stride) {
      const uint4 a = k4[t];
      P.r1[o + rank128(k4, (int)L, a)] = P.r0[a.x];
    }
  } else {
    for (uint32_t t = t0; t < L; t += stride) {
      const uint4 a = k4[t];
      P.r1[o + rank160(k4, kh, (int)L, a, kh[t])] = P.r0[a.x];
    }
  }
}

// Segmented sort: one warp per bucket of up to WCAP records, from the
// warp's slice of shared memory (many buckets per SM, each warp its own
// chain of loads); larger buckets are listed for wc_seg_bucket_cta_kernel.
template <int WCAP>
__global__ void __launch_bounds__(SEG_WARPS * 32) wc_seg_bucket_warp_kernel(Post P) {
  constexpr bool SEG = true;
  extern __shared__ __align__(16) unsigned char sw_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint4* k4 = reinterpret_cast<uint4*>(sw_raw) + warp * WCAP;
  uint32_t* kh = reinterpret_cast<uint32_t*>(sw_raw + SEG_WARPS * WCAP * 16) + warp * WCAP;
  const uint64_t nbk = bucket_count<SEG>(P);
  const uint32_t* off = bucket_off<SEG>(P);
  const uint64_t nw = (uint64_t)gridDim.x * SEG_WARPS;
  for (uint64_t b = (uint64_t)blockIdx.x * SEG_WARPS + warp; b < nbk; b += nw) {
    const uint32_t o = off[b], L = off[b + 1] - o;
    if (L > (uint32_t)WCAP) {
      if (lane == 0) P.big[atomicAdd(P.glob + 13, 1ull)] = (uint32_t)b;
      continue;
    }
#pragma unroll
    for (int q = 0; q < WCAP / 32; ++q) {
      const uint32_t t = lane + 32 * q;
      if (t < L) bucket_key<SEG>(P, o, t, k4, kh);
    }
    __syncwarp();
    bool same = true;
    for (uint32_t t = lane; t < L; t += 32) same &= kh[t] == kh[0];
    place_by_rank(P, o, L, k4, kh, __all_sync(0xffffffffu, same), lane, 32);
    __syncwarp();
  }
}

// A bucket by one CTA: up to SS_RANK_MAX records placed by rank as above,
// larger ones (many times the mean size: rare) sorted by the CTA's bitonic
// tiles and merge passes on compact keys, then gathered.  The segmented sort
// builds those keys in P.kra and uses the bucket's place in P.r1 as scratch;
// the one-job sort has them in P.kr[0] and P.kr[1].
template <bool SEG, int T>
__device__ __forceinline__ void bucket_by_cta(const Post& P, uint32_t o, uint32_t L, unsigned char* raw) {
  uint4* k4 = reinterpret_cast<uint4*>(raw);
  uint32_t* kh = reinterpret_cast<uint32_t*>(raw + SS_RANK_MAX * 16);
  if (L <= (uint32_t)SS_RANK_MAX) {
#pragma unroll
    for (int q = 0; q < SS_RANK_MAX / T; ++q) {
      const uint32_t t = threadIdx.x + q * T;
      if (t < L) bucket_key<SEG>(P, o, t, k4, kh);
    }
    __syncthreads();
    int same = 1;
    for (uint32_t t = threadIdx.x; t < L; t += T) same &= kh[t] == kh[0];
    place_by_rank(P, o, L, k4, kh, __syncthreads_and(same), threadIdx.x, T);
    __syncthreads();
    return;
  }
  KeyRec* a;
  KeyRec* tmp;
  if (SEG) {
    a = P.kra + o;
    tmp = reinterpret_cast<KeyRec*>(P.r1 + o);
    for (uint32_t t = threadIdx.x; t < L; t += T) {
      const uint32_t i = P.kidx[o + t];
      const ulonglong2 kk = *reinterpret_cast<const ulonglong2*>(P.r0 + i);
      a[t] = KeyRec{kk.x, kk.y, i, 0u};
    }
    __syncthreads();
  } else {
    a = P.kr[0] + o;
    tmp = P.kr[1] + o;
  }
  KeyRec* sh = reinterpret_cast<KeyRec*>(raw);
  const KeyRec* res = cta_sort(a, tmp, L, sh, SEG_FB_CAP, KeyCmp{});
  if (SEG && res != a) {  // the result sits in the bucket's output place: move it out first
    for (uint32_t t = threadIdx.x; t < L; t += T) a[t] = res[t];
    __syncthreads();
    res = a;
  }
  for (uint32_t t = threadIdx.x; t < L; t += T) P.r1[o + t] = P.r0[res[t].idx];
  __syncthreads();
}

// Segmented sort: the listed large buckets, one CTA each.
__global__ void __launch_bounds__(SEG_BT) wc_seg_bucket_cta_kernel(Post P) {
  extern __shared__ __align__(16) unsigned char sb_raw[];
  const uint64_t nbig = P.glob[13];
  for (uint64_t q0 = blockIdx.x; q0 < nbig; q0 += gridDim.x) {
    const uint32_t b = P.big[q0];
    bucket_by_cta<true, SEG_BT>(P, P.boff[b], P.boff[b + 1] - P.boff[b], sb_raw);
  }
}

// One-job sample sort: one CTA of SS_BUCKET_T threads per bucket (a few
// hundred buckets of up to a few hundred keys: the largest bucket's ranking
// sets the pass's length, so all of a CTA's threads share each bucket).
constexpr int SS_BUCKET_T = 512;
__global__ void __launch_bounds__(SS_BUCKET_T, 2) wc_ss_bucket_kernel(Post P) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char sb_raw[];
  const uint32_t b = blockIdx.x;
  if (b >= P.ss[0]) return;
  const uint32_t o = ss_off(P)[b];
  bucket_by_cta<false, SS_BUCKET_T>(P, o, ss_off(P)[b + 1] - o, sb_raw);
}

inline uint64_t a256(uint64_t x) { return (x + 255) & ~255ull; }

constexpr uint64_t ca256(uint64_t x) { return (x + 255) & ~255ull; }
constexpr uint64_t rtiles(uint64_t R) { return (R + RTILE - 1) / RTILE; }
constexpr uint64_t rchunks(uint64_t R) { return (rtiles(R) + RCHUNK - 1) / RCHUNK; }
constexpr uint64_t max_runs(uint64_t R) { return R / (FIX_THREAD + 1) + 1; }
// glob, and for sample-sorted capacities the sample-sort words, cleared by one memset
constexpr uint64_t head_bytes(uint64_t R) { return 256 + (R <= SS_MAX_RECORDS ? ca256((SS_WORDS + SS_SMAX) * 4) : 0); }
constexpr uint64_t sortbuf_bytes(uint64_t R) {
  return head_bytes(R) + 2 * ca256(R * sizeof(SortRec)) + 2 * ca256(R * 8) + ca256(((R + CB - 1) / CB) * 8) +
         ca256(max_runs(R) * 8) +
         (R >= RADIX_MIN_RECORDS ? 4 * ca256(R * 8) + 2 * ca256(R * 4) + ca256(rtiles(R) * 256 * 4) +
                                       ca256(rchunks(R) * 256 * 4) + 256
                                 : 2 * ca256(R * sizeof(KeyRec)) + ca256(R * 2) + ca256(SS_MAXB * sizeof(KeyRec)));
}

// Bytes of the parts every sort path shares (head, record arrays, scans,
// run list); the path's own arrays follow.
constexpr uint64_t post_common_bytes(uint64_t R) {
  return head_bytes(R) + 2 * ca256(R * sizeof(SortRec)) + 2 * ca256(R * 8) + ca256(((R + CB - 1) / CB) * 8) +
         ca256(max_runs(R) * 8);
}

// Segmented sample sort of a batch (see SegJob): the decision, made on the
// host from the jobs' table sizes, and the bucket and sample bounds.
struct SegGeom {
  bool on = false;
  uint64_t nbmax = 0;  // buckets, at most
  uint64_t smax = 0;   // largest sample of one job
  uint64_t bytes = 0;  // scratch past post_common_bytes
};

uint64_t seg_bytes(uint64_t R, uint64_t njobs, uint64_t nbmax) {
  return ca256(njobs * sizeof(SegJob)) + ca256((njobs + nbmax) * 4) + ca256((nbmax + 1) * 4) +
         ca256(nbmax * sizeof(KeyRec)) + ca256(nbmax * 4) + ca256(R * 8) + ca256(R * 4) + ca256(R * sizeof(KeyRec));
}

// Several jobs, more records than the one-job sample sort takes, and every
// table a whole number of compaction blocks of at most SS_MAX_RECORDS slots
// laid end to end (job j's slots start at blk0 * CB), so that each job's
// records have a range of their own and a job's sort is the one-job sort's.
SegGeom seg_geometry(const JobDev* hjobs, uint32_t njobs, uint64_t R) {
  SegGeom G;
  if (njobs < 2 || R <= SS_MAX_RECORDS || R >= (1ull << 32)) return G;
  uint64_t base = 0;
  for (uint32_t j = 0; j < njobs; ++j) {
    const uint64_t cap = hjobs[j].cap;
    if (cap < (uint64_t)CB || cap > SS_MAX_RECORDS || cap % CB || hjobs[j].blk0 * CB != base) return G;
    base += cap;
    uint64_t nb, S;
    seg_geom(cap, nb, S);
    G.nbmax += nb;
    if (S > G.smax) G.smax = S;
  }
  if (base != R) return G;
  G.bytes = seg_bytes(R, njobs, G.nbmax);
  G.on = post_common_bytes(R) + G.bytes <= sortbuf_bytes(R);
  return G;
}

void carve_seg(Post& P, uint8_t* base, uint64_t R, uint32_t njobs, const SegGeom& G) {
  uint8_t* p = base + post_common_bytes(R);
  P.seg = reinterpret_cast<SegJob*>(p);
  p += a256(njobs * sizeof(SegJob));
  P.jcur = reinterpret_cast<uint32_t*>(p);
  P.bcnt = P.jcur + njobs;
  p += a256((njobs + G.nbmax) * 4);
  P.boff = reinterpret_cast<uint32_t*>(p);
  p += a256((G.nbmax + 1) * 4);
  P.spl = reinterpret_cast<KeyRec*>(p);
  p += a256(G.nbmax * sizeof(KeyRec));
  P.big = reinterpret_cast<uint32_t*>(p);
  p += a256(G.nbmax * 4);
  P.bpos = reinterpret_cast<uint2*>(p);
  p += a256(R * 8);
  P.kidx = reinterpret_cast<uint32_t*>(p);
  p += a256(R * 4);
  P.kra = reinterpret_cast<KeyRec*>(p);
}

Post carve_post(uint8_t* p, uint64_t R) {
  Post P{};
  P.glob = reinterpret_cast<unsigned long long*>(p);
  if (R <= SS_MAX_RECORDS) {
    P.ss = reinterpret_cast<uint32_t*>(p + 256);
    P.ss_rank = P.ss + SS_WORDS;
  }
  p += head_bytes(R);
  P.r0 = reinterpret_cast<SortRec*>(p);
  p += a256(R * sizeof(SortRec));
  P.r1 = reinterpret_cast<SortRec*>(p);
  p += a256(R * sizeof(SortRec));
  P.src = reinterpret_cast<unsigned long long*>(p);
  p += a256(R * 8);
  P.excl = reinterpret_cast<unsigned long long*>(p);
  p += a256(R * 8);
  P.bsum = reinterpret_cast<unsigned long long*>(p);
  p += a256(((R + CB - 1) / CB) * 8);
  P.runs = reinterpret_cast<uint2*>(p);
  p += a256(max_runs(R) * 8);
  if (R < RADIX_MIN_RECORDS) {  // comparison sort of compact keys
    for (int q = 0; q < 2; ++q) {
      P.kr[q] = reinterpret_cast<KeyRec*>(p);
      p += a256(R * sizeof(KeyRec));
    }
    P.bkt = reinterpret_cast<uint16_t*>(p);
    p += a256(R * 2);
    P.spl = reinterpret_cast<KeyRec*>(p);
    return P;
  }
  for (int q = 0; q < 2; ++q) {
    P.kh[q] = reinterpret_cast<unsigned long long*>(p);
    p += a256(R * 8);
    P.kl[q] = reinterpret_cast<unsigned long long*>(p);
    p += a256(R * 8);
  }
  for (int q = 0; q < 2; ++q) {
    P.kv[q] = reinterpret_cast<uint32_t*>(p);
    p += a256(R * 4);
  }
  P.hist = reinterpret_cast<uint32_t*>(p);
  p += a256(rtiles(R) * 256 * 4);
  P.csum = reinterpret_cast<uint32_t*>(p);
  p += a256(rchunks(R) * 256 * 4);
  P.plan = reinterpret_cast<uint32_t*>(p);
  return P;
}

uint32_t ilog2(uint64_t x) {
  uint32_t l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

}  // namespace

uint64_t wc_table_bytes(uint64_t cap) { return cap * 24; }
uint64_t wc_state_bytes() { return 64; }

size_t wc_sortbuf_bytes(uint64_t R) { return sortbuf_bytes(R); }

uint64_t wc_out_bytes(uint64_t cap, uint64_t n) {
  // at most cap records; key bytes never exceed the input
  return 16 + 24 * cap + n;
}

int wc_map_smem_bytes() { return MAP_WARPS * (int)sizeof(WarpLocal); }
static int wc_map_cta_smem_bytes() { return (int)(sizeof(wc::CtaTableBig) + CTA_WARPS * sizeof(wc::MapWarp)); }

wc::JobDev wc_job_dev(const uint8_t* in, uint64_t n, const WcBuffers& b, uint64_t blk0) {
  JobDev J;
  J.in = in;
  J.n = n;
  J.key = reinterpret_cast<unsigned long long*>(b.key);
  J.cnt = reinterpret_cast<unsigned long long*>(b.cnt);
  J.cap = b.cap;
  J.log2cap = ilog2(b.cap);
  J.state = b.state;
  J.out = b.out;
  J.blk0 = blk0;
  return J;
}

uint64_t wc_compact_blocks(uint64_t cap) { return (cap + CB - 1) / CB; }

cudaError_t launch_wordcount_post_multi(const wc::JobDev* jobs, const wc::JobDev* hjobs, uint32_t njobs,
                                        uint64_t nblocks, uint64_t R, uint8_t* sortbuf, int sms, cudaStream_t s,
                                        uint64_t* nk) {
  cudaError_t e;
  const JobDev& single = hjobs[0];
  Post P = carve_post(sortbuf, R);
  const SegGeom G = jobs ? seg_geometry(hjobs, njobs, R) : SegGeom{};
  if (G.on) carve_seg(P, sortbuf, R, njobs, G);
  if ((e = cudaMemsetAsync(P.glob, 0, head_bytes(R), s)) != cudaSuccess) return e;
  if (G.on && (e = cudaMemsetAsync(P.jcur, 0, (njobs + G.nbmax) * 4, s)) != cudaSuccess) return e;
  {
    const uint64_t cmax = 4ull * (uint64_t)(sms > 0 ? sms : 1);  // 4 CTAs of CT threads per SM (registers)
    wc_compact_kernel<<<(unsigned)(nblocks < cmax ? nblocks : cmax), CT, 0, s>>>(jobs, single, njobs, nblocks, P);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ++*nk;
  const uint64_t nb = (R + CB - 1) / CB;
  const unsigned g256 = (unsigned)((R + 255) / 256);
  if (G.on) {
    // segmented sample sort: per-job splitters and buckets, all jobs side by side
    int n2 = 1;
    while ((uint64_t)n2 < G.smax) n2 <<= 1;
    const int sg_smem = n2 * (int)sizeof(KeyRec);
    if ((e = cudaFuncSetAttribute(wc_seg_sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sg_smem)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(wc_seg_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  SEG_COUNT_SMEM)) != cudaSuccess)
      return e;
    const uint64_t sm = (uint64_t)(sms > 0 ? sms : 1);
    const uint64_t tiles = (R + SEG_TILE - 1) / SEG_TILE;
    const unsigned gt = (unsigned)(tiles < 8 * sm ? tiles : 8 * sm);
    const unsigned gc = (unsigned)(tiles < 4 * sm ? tiles : 4 * sm);  // count: 4 CTAs per SM (shared memory)
    const uint64_t wcta = (G.nbmax + SEG_WARPS - 1) / SEG_WARPS;
    const unsigned gw = (unsigned)(wcta < 4 * sm ? wcta : 4 * sm);  // 4 CTAs per SM (registers)
    wc_seg_plan_kernel<<<1, CB, 0, s>>>(jobs, njobs, P);
    wc_seg_sample_kernel<<<njobs, SEG_SAMPLE_T, sg_smem, s>>>(P, njobs);
    wc_seg_count_kernel<<<gc, SEG_T, SEG_COUNT_SMEM, s>>>(P, njobs);
    wc_seg_offsets_kernel<<<njobs, 256, 0, s>>>(P, njobs);
    wc_seg_scatter_kernel<<<gt, SEG_T, 0, s>>>(P, njobs);
    wc_seg_bucket_warp_kernel<SEG_WCAP><<<gw, SEG_WARPS * 32, SEG_WARP_SMEM, s>>>(P);
    wc_seg_bucket_cta_kernel<<<(unsigned)sm, SEG_BT, BUCKET_CTA_SMEM, s>>>(P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *nk += 6;  // the last one is counted with the tie fix-up below
  } else if (R <= SS_MAX_RECORDS) {
    // sample sort of (key1, s0, index) keys; the bucket pass gathers the records
    const uint64_t nbmax = (R + SS_B - 1) / SS_B < (uint64_t)SS_MAXB ? (R + SS_B - 1) / SS_B : (uint64_t)SS_MAXB;
    const uint64_t smax = R < nbmax * SS_OVER ? R : nbmax * SS_OVER;
    const uint64_t sblocks = (smax + 255) / 256 < 1 ? 1 : (smax + 255) / 256;
    if ((e = launch_pdl(wc_ss_sample_kernel, dim3((unsigned)(sblocks * SS_PARTS)), dim3(256), 0, s, P)) !=
            cudaSuccess ||
        (e = launch_pdl(wc_ss_count_kernel, dim3(g256), dim3(256), 0, s, P)) != cudaSuccess ||
        (e = launch_pdl(wc_ss_scatter_kernel, dim3(g256), dim3(256), 0, s, P)) != cudaSuccess ||
        (e = launch_pdl(wc_ss_bucket_kernel, dim3((unsigned)(nbmax < 1 ? 1 : nbmax)), dim3(SS_BUCKET_T),
                        BUCKET_CTA_SMEM, s, P)) != cudaSuccess)
      return e;
    *nk += 3;  // the last one is counted with the tie fix-up below
  } else if (R < RADIX_MIN_RECORDS) {
    // small record sets: comparison sort of (key1, s0, index) keys
    constexpr int kbs = KSB * (int)sizeof(KeyRec), kmg = KMT * KMI * (int)sizeof(KeyRec);
    static_assert(kbs <= 40 * 1024 && kmg <= 40 * 1024, "sort tiles must fit the default shared-memory limit");
    wc_kkeys_kernel<<<g256, 256, 0, s>>>(P);
    blocksort_kernel<KeyRec, KeyCmp, KSB, KSB_THREADS><<<(unsigned)((R + KSB - 1) / KSB), KSB_THREADS, kbs, s>>>(
        P.kr[0], P.glob, KeyCmp{});
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *nk += 2;
    KeyRec* ks = P.kr[0];
    KeyRec* kd = P.kr[1];
    for (uint64_t L = KSB; L < R; L *= 2) {
      merge_kernel<KeyRec, KeyCmp, KMT, KMI><<<(unsigned)((R + KMT * KMI - 1) / (KMT * KMI)), KMT, kmg, s>>>(
          ks, kd, L, P.glob, KeyCmp{});
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      ++*nk;
      KeyRec* t = ks;
      ks = kd;
      kd = t;
    }
    wc_kgather_kernel<<<g256, 256, 0, s>>>(P, ks);
  } else {
    // large record sets: radix sort by (key1, s0)
    wc_rkeys_kernel<<<(unsigned)nb, CB, 0, s>>>(P);
    wc_rplan_kernel<<<1, 1, 0, s>>>(P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *nk += 2;
    for (int p = 0; p < NPASS; ++p) {
      wc_rhist_kernel<<<(unsigned)rtiles(R), RT, 0, s>>>(P, p);
      wc_rscan1_kernel<<<(unsigned)rchunks(R), RT, 0, s>>>(P, p);
      wc_rscan2_kernel<<<1, RT, 0, s>>>(P, p);
      wc_rscatter_kernel<<<(unsigned)rtiles(R), RT, 0, s>>>(P, p);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      *nk += 4;
    }
    wc_rgather_kernel<<<g256, 256, 0, s>>>(P);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // ties on (key1, s0): the full order (the count below also takes the
  // sort path's last launch)
  // the tail's grids cover the live records only (loops over them)
  const uint64_t smc = (uint64_t)(sms > 0 ? sms : 1);
  const unsigned gp256 = (unsigned)(g256 < 8 * smc ? g256 : 8 * smc);  // 8 CTAs per SM (gather: 32 registers)
  const unsigned gpfix = (unsigned)(g256 < 6 * smc ? g256 : 6 * smc);  // 6 (tie fix-up: 40 registers)
  const unsigned gpcb = (unsigned)(nb < 2 * smc ? nb : 2 * smc);
  const int fx_smem = SB * (int)sizeof(SortRec);
  if ((e = cudaFuncSetAttribute(wc_rfix_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, fx_smem)) !=
      cudaSuccess)
    return e;
  if ((e = launch_pdl(wc_rfix_kernel, dim3(gpfix), dim3(256), 0, s, P, jobs, single, max_runs(R))) != cudaSuccess ||
      (e = launch_pdl(wc_rfix_cta_kernel, dim3(64), dim3(SB_THREADS), (size_t)fx_smem, s, P, jobs, single,
                      max_runs(R))) != cudaSuccess)
    return e;
  *nk += 3;
  if ((e = launch_pdl(wc_lensum_kernel, dim3(nb <= LENSUM_FUSE_BLOCKS ? (unsigned)nb : gpcb), dim3(CB), 0, s, P,
                      nb <= LENSUM_FUSE_BLOCKS)) != cudaSuccess)
    return e;
  if (nb > LENSUM_FUSE_BLOCKS) {
    if ((e = launch_pdl(wc_bscan_kernel, dim3(1), dim3(CB), 0, s, P, nb)) != cudaSuccess) return e;
    ++*nk;
  }
  if (jobs) {
    if ((e = launch_pdl(wc_bounds_kernel, dim3(gpcb), dim3(CB), 0, s, jobs, single, P)) != cudaSuccess ||
        (e = launch_pdl(wc_gather_kernel, dim3(gp256), dim3(256), 0, s, jobs, single, P)) != cudaSuccess)
      return e;
  } else {  // one job: bounds known, scan and gather in one pass
    if ((e = launch_pdl(wc_gather1_kernel, dim3(gpcb), dim3(CB), 0, s, single, P)) != cudaSuccess) return e;
    --*nk;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *nk += 3;
  return cudaSuccess;
}

cudaError_t launch_wordcount(const uint8_t* in, uint64_t n, const WcBuffers& b, const DevInfo& di, cudaStream_t s,
                             uint64_t* nk, bool pipelined, KTimer* kt, long long pipe_polls) {
  cudaError_t e;
  // table (keys then counts) and state words start at zero
  if ((e = cudaMemsetAsync(b.key, 0, wc_table_bytes(b.cap), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b.state, 0, wc_state_bytes(), s)) != cudaSuccess) return e;
  const JobDev J = wc_job_dev(in, n, b, 0);
  if (n > 0 && pipelined) {
    const int smem = (int)sizeof(PipeSmem);
    if ((e = cudaFuncSetAttribute(wc_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
      return e;
    const uint64_t nseg = (n + wc::SEG - 1) / wc::SEG;
    uint64_t grid = (nseg + PIPE_PAIRS - 1) / PIPE_PAIRS;
    const uint64_t gmax = 4ull * di.sms;
    if (grid > gmax) grid = gmax;
    if ((e = kt_begin(kt, s)) != cudaSuccess) return e;
    wc_pipe_kernel<<<(unsigned)grid, PIPE_THREADS, smem, s>>>(J, pipe_polls < 0 ? PIPE_SPIN_LIMIT : pipe_polls);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = kt_end(kt, s)) != cudaSuccess) return e;
    ++*nk;
  } else if (n >= CTA_MAP_MIN_BYTES && (reinterpret_cast<uintptr_t>(in) & 15) == 0) {
    const int smem = wc_map_cta_smem_bytes();
    if ((e = cudaFuncSetAttribute(wc_map_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess)
      return e;
    const uint64_t nseg = (n + wc::SEG - 1) / wc::SEG;
    uint64_t grid = (nseg + CTA_WARPS - 1) / CTA_WARPS;
    const uint64_t gmax = (uint64_t)di.sms;
    if (grid > gmax) grid = gmax;
    if ((e = kt_begin(kt, s)) != cudaSuccess) return e;
    wc_map_cta_kernel<<<(unsigned)grid, CTA_THREADS, smem, s>>>(J);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = kt_end(kt, s)) != cudaSuccess) return e;
    ++*nk;
  } else if (n > 0) {
    const int smem = wc_map_smem_bytes();
    if ((e = cudaFuncSetAttribute(wc_map_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
      return e;
    const uint64_t nseg = (n + wc::SEG - 1) / wc::SEG;
    uint64_t grid = (nseg + MAP_WARPS - 1) / MAP_WARPS;
    const uint64_t gmax = 5ull * di.sms;
    if (grid > gmax) grid = gmax;
    if ((e = kt_begin(kt, s)) != cudaSuccess) return e;
    wc_map_kernel<<<(unsigned)grid, MAP_THREADS, smem, s>>>(J);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = kt_end(kt, s)) != cudaSuccess) return e;
    ++*nk;
  }
  return launch_wordcount_post_multi(nullptr, &J, 1, wc_compact_blocks(b.cap), b.cap, b.sortbuf, di.sms, s, nk);
}

}  // namespace mrgb

// ---------------------------------------------------------------------------
// Word count without device allocation.
//
// Some callers cannot call cudaMalloc: a host program that has reserved the
// GPU's memory up front for its own pool and does not allow other components
// to allocate, or a latency-critical loop where the implicit synchronisation
// and unpredictable cost of cudaMalloc / cudaFree are not acceptable.  For
// them the hash table and sort scratch of one word-count job live in the
// file-scope array below, sized for NOALLOC_SLOTS table slots.  Every GPU
// that loads this library keeps the array (about 19 MiB) until the process
// exits.
#include <mutex>

namespace mrgb {
namespace {
constexpr uint64_t NOALLOC_SLOTS = 1ull << 17;
constexpr uint64_t NOALLOC_TABLE_BYTES = NOALLOC_SLOTS * 24;
constexpr uint64_t NOALLOC_STATE_BYTES = 256;
constexpr uint64_t NOALLOC_SORT_BYTES = sortbuf_bytes(NOALLOC_SLOTS);
constexpr uint64_t NOALLOC_SCRATCH_BYTES = NOALLOC_TABLE_BYTES + NOALLOC_STATE_BYTES + NOALLOC_SORT_BYTES;
constexpr int NOALLOC_MAX_DEVICES = 64;
}  // namespace
}  // namespace mrgb

static __device__ __align__(256) unsigned char g_wc_noalloc_scratch[mrgb::NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_base[mrgb::NOALLOC_MAX_DEVICES] = {};
int g_noalloc_sms[mrgb::NOALLOC_MAX_DEVICES] = {};

// Once per device, with that device current: the device address of the
// scratch array (host code only sees a host-side stand-in for the symbol).
mr_status noalloc_setup(int dev, void** base, int* sms) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (dev < 0 || dev >= mrgb::NOALLOC_MAX_DEVICES) return MR_EINVAL;
  if (!g_noalloc_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_wc_noalloc_scratch);
    if (e != cudaSuccess) {
      mrgb::set_last_error("cudaGetSymbolAddress(g_wc_noalloc_scratch)", e);
      return MR_ECUDA;
    }
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
      mrgb::set_last_error("cudaDeviceGetAttribute", e);
      return MR_ECUDA;
    }
    g_noalloc_sms[dev] = n;
    g_noalloc_base[dev] = p;
  }
  *base = g_noalloc_base[dev];
  *sms = g_noalloc_sms[dev];
  return MR_OK;
}
}  // namespace

extern "C" mr_status mr_wordcount_noalloc(const void* d_input, uint64_t input_bytes, void* d_out, uint64_t out_cap,
                                          uint64_t* out_bytes, void* cuda_stream) {
  using namespace mrgb;
  if ((!d_input && input_bytes) || !d_out || !out_bytes) return MR_EINVAL;
  if (input_bytes >= (1ull << 40) - 1) return MR_EINVAL;
  if (out_cap < wc_out_bytes(NOALLOC_SLOTS, input_bytes)) return MR_EINVAL;
  int dev = 0;
  MR_CUDA_TRY(cudaGetDevice(&dev));
  void* base = nullptr;
  DevInfo di;
  mr_status st = noalloc_setup(dev, &base, &di.sms);
  if (st) return st;
  uint8_t* p = static_cast<uint8_t*>(base);
  WcBuffers b;
  b.cap = NOALLOC_SLOTS;
  b.key = reinterpret_cast<uint64_t*>(p);
  b.cnt = b.key + 2 * NOALLOC_SLOTS;
  b.state = reinterpret_cast<uint32_t*>(p + NOALLOC_TABLE_BYTES);
  b.sortbuf = p + NOALLOC_TABLE_BYTES + NOALLOC_STATE_BYTES;
  b.out = static_cast<uint8_t*>(d_out);
  b.out_cap = out_cap;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  uint64_t nk = 0;
  // launch_wordcount clears the table and the state words before the map pass
  MR_CUDA_TRY(launch_wordcount(static_cast<const uint8_t*>(d_input), input_bytes, b, di, s, &nk));
  uint32_t state[4] = {0, 0, 0, 0};
  uint64_t hdr[2] = {0, 0};
  MR_CUDA_TRY(cudaMemcpyAsync(state, b.state, sizeof(state), cudaMemcpyDeviceToHost, s));
  MR_CUDA_TRY(cudaMemcpyAsync(hdr, d_out, sizeof(hdr), cudaMemcpyDeviceToHost, s));
  MR_CUDA_TRY(cudaStreamSynchronize(s));
  if (state[0] & 1u) return MR_EOVERFLOW;
  *out_bytes = 16 + 24 * hdr[0] + hdr[1];
  return MR_OK;
}
