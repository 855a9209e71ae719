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
//  * Combiner / local container (Sec. III-A, Sec. III-D): a 256-slot table per
//    warp in shared memory, flushed into the global container when half full
//    (the paper's bounded local table handed to the reduce side).
//  * Global container: open addressing with a 128-bit CAS per new key and an
//    atomicAdd per combine (see dev_wordcount.cuh).
//  * Merge + sort: occupied slots of every job are compacted into one record
//    array and sorted once by (job, count desc, key asc) — a shared-memory
//    bitonic sort of 2048-record blocks, then merge passes whose split points
//    come from a warp-cooperative 33-way search and whose inputs are staged in
//    shared memory — so a batch
//    of jobs is ordered by a single launch sequence; per-job boundaries and a
//    scan of key lengths place each job's records and key bytes in its
//    result: {u64 n, u64 key bytes; n x {u64 count, u64 key_off, u64 key_len};
//    key bytes}.
#include "mr_internal.h"
#include "dev_wordcount.cuh"

namespace mrgb {
namespace {

using wc::JobDev;
using wc::WarpLocal;

constexpr int MAP_WARPS = 8;
constexpr int MAP_THREADS = MAP_WARPS * 32;
constexpr int CB = 1024;            // records per compaction / sort / scan block
constexpr uint64_t CNT_MAX = (1ull << 40) - 1;

__device__ __forceinline__ JobDev job_at(const JobDev* jobs, const JobDev& single, uint32_t j) {
  return jobs ? jobs[j] : single;
}

__global__ void __launch_bounds__(MAP_THREADS, 5) wc_map_kernel(JobDev J) {
  extern __shared__ __align__(16) unsigned char wc_smem[];
  WarpLocal& L = reinterpret_cast<WarpLocal*>(wc_smem)[threadIdx.x >> 5];
  wc::local_clear(L);
  int occ = 0;
  const uint64_t nseg = (J.n + wc::SEG - 1) / wc::SEG;
  const uint64_t gw = (uint64_t)blockIdx.x * MAP_WARPS + (threadIdx.x >> 5);
  const uint64_t nw = (uint64_t)gridDim.x * MAP_WARPS;
  for (uint64_t seg = gw; seg < nseg; seg += nw) wc::warp_segment(J, seg, L, occ);
  wc::local_flush(L, occ, J);
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

struct Post {
  SortRec* r0;
  SortRec* r1;
  unsigned long long* src;   // [R] input offset of a long key
  unsigned long long* excl;  // [R] exclusive scan of key lengths in sorted order
  unsigned long long* bsum;  // [ceil(R / CB)]
  unsigned long long* glob;  // [0] number of records
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

__device__ __forceinline__ int block_excl_scan(int v, int* tmp, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = tmp[lane];
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    tmp[lane] = wi - w;
    if (lane == 31) tmp[32] = wi;
  }
  __syncthreads();
  const int r = tmp[warp] + incl - v;
  total = tmp[32];
  __syncthreads();
  return r;
}

// Occupied slots of every job -> records.  Block b belongs to the job whose
// block range contains b.  The first block of a job also zeroes the job's
// result header (a job with no records keeps {0, 0}).
__global__ void __launch_bounds__(CB) wc_compact_kernel(const JobDev* jobs, JobDev single, uint32_t njobs, Post P) {
  __shared__ int tmp[33];
  __shared__ unsigned long long blk_base;
  const uint32_t j = jobs ? find_job_by_block(jobs, njobs, blockIdx.x) : 0;
  const JobDev J = job_at(jobs, single, j);
  const uint64_t slot = ((uint64_t)blockIdx.x - J.blk0) * CB + threadIdx.x;
  if (blockIdx.x == J.blk0 && threadIdx.x < 2) reinterpret_cast<unsigned long long*>(J.out)[threadIdx.x] = 0;
  uint64_t w0 = 0, w1 = 0;
  if (slot < J.cap) {
    w0 = J.key[2 * slot];
    w1 = J.key[2 * slot + 1];
  }
  const bool occ = w1 != 0;
  int total;
  const int r = block_excl_scan(occ ? 1 : 0, tmp, total);
  if (threadIdx.x == 0) blk_base = total ? atomicAdd(P.glob, (unsigned long long)total) : 0ull;
  __syncthreads();
  if (!occ) return;
  const uint64_t i = blk_base + (uint64_t)r;
  const uint64_t cnt = J.cnt[slot];
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

// Block sort: SB records per CTA, bitonic network in shared memory.
constexpr int SB = 2048;
constexpr int SB_THREADS = 1024;

__global__ void __launch_bounds__(SB_THREADS) wc_blocksort_kernel(const JobDev* jobs, JobDev single, Post P) {
  extern __shared__ __align__(16) unsigned char bs_raw[];
  SortRec* sh = reinterpret_cast<SortRec*>(bs_raw);
  const uint64_t m = *P.glob;
  const uint64_t b0 = (uint64_t)blockIdx.x * SB;
  if (b0 >= m) return;
  for (int i = threadIdx.x; i < SB; i += blockDim.x) {
    if (b0 + i < m) sh[i] = P.r0[b0 + i];
    else sh[i] = SortRec{~0ull, ~0ull, ~0ull, 0xffffffffu, 0xffffffffu};
  }
  __syncthreads();
  for (int k = 2; k <= SB; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int t = threadIdx.x; t < SB / 2; t += blockDim.x) {
        const int lo = 2 * jj * (t / jj) + (t % jj);
        const int hi = lo + jj;
        const bool up = (lo & k) == 0;
        const SortRec a = sh[lo], b = sh[hi];
        const bool a_pad = a.idx == 0xffffffffu, b_pad = b.idx == 0xffffffffu;
        bool b_lt_a;
        if (a_pad || b_pad) b_lt_a = a_pad && !b_pad;
        else b_lt_a = rec_less(b, a, jobs, single, P.src);
        if (b_lt_a == up) {
          sh[lo] = b;
          sh[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < SB; i += blockDim.x)
    if (b0 + i < m) P.r0[b0 + i] = sh[i];
}

// Number of A records among the first kk outputs of merge(A[0..la), B[0..lb)),
// found by the whole warp: each step probes 32 evenly spaced positions at once
// (the "A[i] < B[kk-1-i]" predicate is true on a prefix), shrinking the range
// about 33-fold, so a search over L records costs ~log_33(L) dependent loads.
__device__ uint64_t corank_warp(const SortRec* A, uint64_t la, const SortRec* B, uint64_t lb, uint64_t kk,
                                const JobDev* jobs, const JobDev& single, const unsigned long long* src) {
  const int lane = threadIdx.x & 31;
  uint64_t lo = kk > lb ? kk - lb : 0;
  uint64_t hi = kk < la ? kk : la;
  while (lo < hi) {
    const uint64_t span = hi - lo;
    const uint64_t m = lo + (span * (uint64_t)(lane + 1)) / 33;
    const bool pr = rec_less(A[m], B[kk - 1 - m], jobs, single, src);
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

// One merge pass: runs of L sorted records are merged pairwise.  A CTA owns
// MTILE consecutive outputs: two warps find where its range starts and ends
// in the two runs, the CTA stages both input windows in shared memory, and
// each thread merges MI outputs from there.
constexpr int MT = 256;
constexpr int MI = 8;
constexpr int MTILE = MT * MI;

__global__ void __launch_bounds__(MT) wc_merge_kernel(const SortRec* __restrict__ src, SortRec* __restrict__ dst,
                                                      uint64_t L, const JobDev* jobs, JobDev single, Post P) {
  extern __shared__ __align__(16) unsigned char mg_raw[];
  SortRec* ms = reinterpret_cast<SortRec*>(mg_raw);
  __shared__ uint64_t cr[2];
  const uint64_t m = *P.glob;
  const uint64_t o0 = (uint64_t)blockIdx.x * MTILE;
  if (o0 >= m) return;
  const uint64_t a0 = (o0 / (2 * L)) * (2 * L);  // MTILE divides 2L: a tile never spans two pairs
  const uint64_t la = (m - a0) < L ? (m - a0) : L;
  const uint64_t b0 = a0 + L;
  const uint64_t lb = b0 < m ? ((m - b0) < L ? (m - b0) : L) : 0;
  const SortRec* A = src + a0;
  const SortRec* B = src + b0;
  const uint64_t kk0 = o0 - a0;
  const uint64_t kk1 = (kk0 + MTILE) < la + lb ? kk0 + MTILE : la + lb;
  if (lb == 0) {  // a lone run: copy
    for (uint64_t t = kk0 + threadIdx.x; t < kk1; t += MT) dst[a0 + t] = A[t];
    return;
  }
  const int warp = threadIdx.x >> 5;
  if (warp < 2) {
    const uint64_t kk = warp == 0 ? kk0 : kk1;
    const uint64_t c = corank_warp(A, la, B, lb, kk, jobs, single, P.src);
    if ((threadIdx.x & 31) == 0) cr[warp] = c;
  }
  __syncthreads();
  const uint64_t i0 = cr[0], i1 = cr[1];
  const uint32_t na = (uint32_t)(i1 - i0);
  const uint32_t nb = (uint32_t)((kk1 - i1) - (kk0 - i0));
  for (uint32_t t = threadIdx.x; t < na; t += MT) ms[t] = A[i0 + t];
  for (uint32_t t = threadIdx.x; t < nb; t += MT) ms[na + t] = B[kk0 - i0 + t];
  __syncthreads();
  const SortRec* sa = ms;
  const SortRec* sb = ms + na;
  const uint32_t r0 = threadIdx.x * MI;
  const uint32_t tot = na + nb;
  if (r0 >= tot) return;
  uint32_t lo = r0 > nb ? r0 - nb : 0, hi = r0 < na ? r0 : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (rec_less(sa[mid], sb[r0 - 1 - mid], jobs, single, P.src)) lo = mid + 1;
    else hi = mid;
  }
  uint32_t i = lo, j = r0 - lo;
  for (int t = 0; t < MI && r0 + t < tot; ++t) {
    bool takeA;
    if (j >= nb) takeA = true;
    else if (i >= na) takeA = false;
    else takeA = rec_less(sa[i], sb[j], jobs, single, P.src);
    dst[o0 + r0 + t] = takeA ? sa[i++] : sb[j++];
  }
}

__global__ void __launch_bounds__(CB) wc_lensum_kernel(const SortRec* recs, Post P) {
  __shared__ unsigned long long ws[32];
  const uint64_t m = *P.glob;
  const uint64_t i = (uint64_t)blockIdx.x * CB + threadIdx.x;
  unsigned long long v = i < m ? recs[i].len : 0;
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < 32; ++w) s += ws[w];
    P.bsum[blockIdx.x] = s;
  }
}

// exclusive scan of the block sums (one CTA)
__global__ void __launch_bounds__(CB) wc_bscan_kernel(Post P, uint64_t nb) {
  __shared__ unsigned long long carry;
  __shared__ unsigned long long wsum[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t b = 0; b < nb; b += CB) {
    const uint64_t i = b + threadIdx.x;
    const unsigned long long v = i < nb ? P.bsum[i] : 0;
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
}

// Exclusive length scan per record; each job's first / end record and the
// scan at both are stored in the job's state as 64-bit fields 1..4.
__global__ void __launch_bounds__(CB) wc_bounds_kernel(const SortRec* recs, const JobDev* jobs, JobDev single, Post P) {
  __shared__ unsigned long long wsum[32];
  const uint64_t m = *P.glob;
  const uint64_t i = (uint64_t)blockIdx.x * CB + threadIdx.x;
  if ((uint64_t)blockIdx.x * CB >= m) return;
  const uint32_t len = i < m ? recs[i].len : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
  if (i >= m) return;
  const unsigned long long ex = P.bsum[blockIdx.x] + wsum[warp] + incl - len;
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

// Records and key bytes into each job's result.
__global__ void __launch_bounds__(256) wc_gather_kernel(const SortRec* recs, const JobDev* jobs, JobDev single, Post P) {
  const uint64_t m = *P.glob;
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const SortRec r = recs[i];
  const uint32_t j = (uint32_t)(r.key1 >> 40);
  const JobDev J = job_at(jobs, single, j);
  const unsigned long long* st = reinterpret_cast<const unsigned long long*>(J.state);
  const uint64_t first = st[1], scan0 = st[2], end = st[3], scan1 = st[4];
  const uint64_t nrec = end - first, li = i - first;
  unsigned long long* out = reinterpret_cast<unsigned long long*>(J.out);
  if (li == 0) {
    out[0] = nrec;
    out[1] = scan1 - scan0;
  }
  const uint64_t koff = P.excl[i] - scan0;
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

inline uint64_t a256(uint64_t x) { return (x + 255) & ~255ull; }

Post carve_post(uint8_t* p, uint64_t R) {
  Post P;
  P.glob = reinterpret_cast<unsigned long long*>(p);
  p += 256;
  P.r0 = reinterpret_cast<SortRec*>(p);
  p += a256(R * sizeof(SortRec));
  P.r1 = reinterpret_cast<SortRec*>(p);
  p += a256(R * sizeof(SortRec));
  P.src = reinterpret_cast<unsigned long long*>(p);
  p += a256(R * 8);
  P.excl = reinterpret_cast<unsigned long long*>(p);
  p += a256(R * 8);
  P.bsum = reinterpret_cast<unsigned long long*>(p);
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

size_t wc_sortbuf_bytes(uint64_t R) {
  const uint64_t nb = (R + CB - 1) / CB;
  return 256 + 2 * a256(R * sizeof(SortRec)) + 2 * a256(R * 8) + a256(nb * 8);
}

uint64_t wc_out_bytes(uint64_t cap, uint64_t n) {
  // at most cap records; key bytes never exceed the input
  return 16 + 24 * cap + n;
}

int wc_map_smem_bytes() { return MAP_WARPS * (int)sizeof(WarpLocal); }

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

cudaError_t launch_wordcount_post_multi(const wc::JobDev* jobs, const wc::JobDev& single, uint32_t njobs,
                                        uint64_t nblocks, uint64_t R, uint8_t* sortbuf, cudaStream_t s,
                                        uint64_t* nk) {
  cudaError_t e;
  Post P = carve_post(sortbuf, R);
  if ((e = cudaMemsetAsync(P.glob, 0, 8, s)) != cudaSuccess) return e;
  wc_compact_kernel<<<(unsigned)nblocks, CB, 0, s>>>(jobs, single, njobs, P);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const uint64_t nb = (R + CB - 1) / CB;
  const int bs_smem = SB * (int)sizeof(SortRec);
  const int mg_smem = MTILE * (int)sizeof(SortRec);
  if ((e = cudaFuncSetAttribute(wc_blocksort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bs_smem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(wc_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mg_smem)) !=
      cudaSuccess)
    return e;
  wc_blocksort_kernel<<<(unsigned)((R + SB - 1) / SB), SB_THREADS, bs_smem, s>>>(jobs, single, P);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *nk += 2;
  SortRec* src = P.r0;
  SortRec* dst = P.r1;
  for (uint64_t L = SB; L < R; L *= 2) {
    wc_merge_kernel<<<(unsigned)((R + MTILE - 1) / MTILE), MT, mg_smem, s>>>(src, dst, L, jobs, single, P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nk;
    SortRec* t = src;
    src = dst;
    dst = t;
  }
  wc_lensum_kernel<<<(unsigned)nb, CB, 0, s>>>(src, P);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  wc_bscan_kernel<<<1, CB, 0, s>>>(P, nb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  wc_bounds_kernel<<<(unsigned)nb, CB, 0, s>>>(src, jobs, single, P);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  wc_gather_kernel<<<(unsigned)((R + 255) / 256), 256, 0, s>>>(src, jobs, single, P);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *nk += 4;
  return cudaSuccess;
}

cudaError_t launch_wordcount(const uint8_t* in, uint64_t n, const WcBuffers& b, const DevInfo& di, cudaStream_t s,
                             uint64_t* nk) {
  cudaError_t e;
  // table (keys then counts) and state words start at zero
  if ((e = cudaMemsetAsync(b.key, 0, wc_table_bytes(b.cap), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b.state, 0, wc_state_bytes(), s)) != cudaSuccess) return e;
  const JobDev J = wc_job_dev(in, n, b, 0);
  if (n > 0) {
    const int smem = wc_map_smem_bytes();
    if ((e = cudaFuncSetAttribute(wc_map_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
      return e;
    const uint64_t nseg = (n + wc::SEG - 1) / wc::SEG;
    uint64_t grid = (nseg + MAP_WARPS - 1) / MAP_WARPS;
    const uint64_t gmax = 5ull * di.sms;
    if (grid > gmax) grid = gmax;
    wc_map_kernel<<<(unsigned)grid, MAP_THREADS, smem, s>>>(J);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nk;
  }
  return launch_wordcount_post_multi(nullptr, J, 1, wc_compact_blocks(b.cap), b.cap, b.sortbuf, s, nk);
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
// that loads this library keeps the array (about 14 MiB) until the process
// exits.
#include <mutex>

namespace mrgb {
namespace {
constexpr uint64_t NOALLOC_SLOTS = 1ull << 17;
constexpr uint64_t NOALLOC_TABLE_BYTES = NOALLOC_SLOTS * 24;
constexpr uint64_t NOALLOC_STATE_BYTES = 256;
constexpr uint64_t NOALLOC_SORT_BYTES = 256 + 2 * ((NOALLOC_SLOTS * sizeof(SortRec) + 255) & ~255ull) +
                                        2 * ((NOALLOC_SLOTS * 8 + 255) & ~255ull) +
                                        ((((NOALLOC_SLOTS + CB - 1) / CB) * 8 + 255) & ~255ull);
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
