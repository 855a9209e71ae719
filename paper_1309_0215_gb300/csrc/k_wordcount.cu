// Word count: hash-table container (arXiv:1309.0215 Table I, Sec. III-A).
//
// Map (Sec. II-A): a token is a maximal run of bytes that are not ASCII
// whitespace; each emits (token, 1).  Reduce: sum.  Output ordered by count
// descending, then key bytes ascending.
//
// GB300 design
//  * Split (Sec. II-A, Fig. 1): the input is cut into 512-byte segments; a warp
//    owns the tokens whose FIRST byte lies in its segment and reads past the
//    segment end to finish them.  A warp stages its segment (+64-byte halo)
//    in shared memory with coalesced 128-bit loads.
//  * Token boundaries: each lane classifies its 16 bytes and builds a 16-bit
//    token-start mask; a warp prefix sum of the mask popcounts compacts all
//    starts of the segment into a list, and lanes then take tokens from the
//    list 32 at a time.  This is the GPU form of the paper's SIMD hashing
//    (Sec. III-C): lanes are SIMD units, and a lane that finishes a token takes
//    the next one from the list instead of idling, as in SIMDH-Stream; the
//    prefix sum plays the role of the paper's prefix-sum lookup table.
//  * Hash: FNV-1a 64 (the paper's Listing 2 shape: a byte-at-a-time update
//    loop, with FNV as one of its two example functions), followed by a 64-bit
//    finaliser so low and high bits are both usable.
//  * Combiner / local container (Sec. III-A; bounded local table of Sec.
//    III-D): each warp owns a 256-slot hash table in shared memory; every
//    token is combined into it at once.  Keys of <= 16 bytes are held in the
//    slot as two packed words, so equality needs no memory reads.  When the
//    table is half full it is flushed (partitioned by the global table's hash)
//    into the global container, as the paper's map workers hand full local
//    tables to the reduce side.
//  * Global container: open addressing with linear probing.  A slot's key word
//    (length << 40 | offset + 1) is claimed with one 64-bit CAS and never
//    changes afterwards; the key bytes are the token's bytes in the resident,
//    immutable input, so a reader that sees a non-zero word can compare keys
//    at once (no BUSY state, no publish race).  Counts combine in place with
//    64-bit atomicAdd.  Probing is bounded; running out of probes raises an
//    overflow flag and the host re-runs the job with a larger table.
//  * Merge + sort (Sec. II-A "ordered (optional)"): occupied slots are
//    compacted, sorted by (count desc, key asc) with a shared-memory bitonic
//    block sort plus merge-path passes, and gathered into the result layout
//    {u64 n, u64 key bytes; n x {u64 count, u64 key_off, u64 key_len}; keys}.
#include "mr_internal.h"

namespace mrgb {
namespace {

constexpr int WC_WARPS = 8;
constexpr int WC_THREADS = WC_WARPS * 32;
constexpr int SEG = 512;
constexpr int HALO = 64;
constexpr int LT = 256;                 // local slots per warp
constexpr int LT_FLUSH_AT = LT / 2;     // flush before a round when occupancy >= this
constexpr uint64_t OFF_MASK = (1ull << 40) - 1;
constexpr uint32_t LEN_SAT = (1u << 24) - 1;
constexpr int MAX_PROBES = 4096;
constexpr uint64_t FNV_OFFSET = 0xcbf29ce484222325ull;
constexpr uint64_t FNV_PRIME = 0x100000001b3ull;

struct WarpSmem {
  unsigned long long h[LT];
  unsigned long long off[LT];
  unsigned long long k0[LT];
  unsigned long long k1[LT];
  uint32_t len[LT];
  uint32_t cnt[LT];
  uint8_t buf[SEG + HALO];
  uint16_t starts[SEG / 2];
};

__device__ __forceinline__ bool is_ws(uint32_t c) { return c == 32u || (c - 9u) < 5u; }

__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33; k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

struct Tok {
  uint64_t h, off, k0, k1;
  uint32_t len;
};

// Read the token that starts at segment-relative byte r.
__device__ __forceinline__ Tok read_token(const uint8_t* __restrict__ in, uint64_t n, uint64_t base,
                                          const uint8_t* buf, uint32_t bufn, uint32_t r) {
  Tok t;
  t.off = base + r;
  uint64_t h = FNV_OFFSET, k0 = 0, k1 = 0;
  uint32_t len = 0;
  for (;;) {
    uint32_t c;
    if (r < bufn) {
      c = buf[r];
    } else {
      uint64_t gi = base + r;
      if (gi >= n) break;
      c = in[gi];
    }
    if (is_ws(c)) break;
    h = (h ^ c) * FNV_PRIME;
    if (len < 8) k0 |= (uint64_t)c << (8 * len);
    else if (len < 16) k1 |= (uint64_t)c << (8 * (len - 8));
    ++len;
    ++r;
  }
  h = fmix64(h);
  t.h = h ? h : 1;
  t.k0 = k0;
  t.k1 = k1;
  t.len = len;
  return t;
}

// Do the tokens at offsets a and b (b's length len) have equal bytes?
__device__ bool tok_equal_global(const uint8_t* __restrict__ in, uint64_t n, uint64_t a, uint64_t b, uint32_t len) {
  if (a == b) return true;
  if (a + len > n) return false;
  for (uint32_t i = 0; i < len; ++i)
    if (in[a + i] != in[b + i]) return false;
  return a + len == n || is_ws(in[a + len]);
}

__device__ void global_insert(const uint8_t* __restrict__ in, uint64_t n, unsigned long long* gkey,
                              unsigned long long* gcnt, uint64_t cap, uint32_t* state, uint64_t h, uint64_t off,
                              uint32_t len, uint64_t cnt) {
  const uint32_t lsat = len < LEN_SAT ? len : LEN_SAT;
  const unsigned long long mine = ((unsigned long long)lsat << 40) | (off + 1);
  uint64_t slot = (h >> 20) & (cap - 1);
  for (int p = 0; p < MAX_PROBES; ++p) {
    unsigned long long w = *reinterpret_cast<volatile unsigned long long*>(gkey + slot);
    if (w == 0) {
      unsigned long long prev = atomicCAS(gkey + slot, 0ull, mine);
      if (prev == 0) {
        atomicAdd(gcnt + slot, (unsigned long long)cnt);
        return;
      }
      w = prev;
    }
    if ((uint32_t)(w >> 40) == lsat && tok_equal_global(in, n, (w & OFF_MASK) - 1, off, len)) {
      atomicAdd(gcnt + slot, (unsigned long long)cnt);
      return;
    }
    slot = (slot + 1) & (cap - 1);
  }
  atomicOr(state, 1u);  // overflow: the host re-runs with a larger table
}

__device__ __forceinline__ bool local_equal(const WarpSmem& S, int slot, const Tok& t, const uint8_t* __restrict__ in,
                                            uint64_t n) {
  if (S.h[slot] != t.h || S.len[slot] != t.len) return false;
  if (t.len <= 16) return S.k0[slot] == t.k0 && S.k1[slot] == t.k1;
  return tok_equal_global(in, n, S.off[slot], t.off, t.len);
}

// Warp-synchronous combine of one token per active lane into the warp's
// local table.  occ (warp-uniform) counts occupied slots.
__device__ __forceinline__ void local_insert(WarpSmem& S, bool active, const Tok& t, int& occ,
                                             const uint8_t* __restrict__ in, uint64_t n) {
  const int lane = threadIdx.x & 31;
  int slot = (int)(t.h & (LT - 1));
  bool pending = active;
  while (__any_sync(0xffffffffu, pending)) {
    bool empty = false, match = false;
    if (pending) {
      if (S.h[slot] == 0) empty = true;
      else match = local_equal(S, slot, t, in, n);
    }
    if (match) {
      atomicAdd(&S.cnt[slot], 1u);
      pending = false;
    }
    const unsigned em = __ballot_sync(0xffffffffu, empty);
    bool claimed = false;
    if (empty) {
      // lanes that found the same empty slot: the lowest one claims it
      const unsigned grp = __match_any_sync(em, slot);
      claimed = lane == __ffs(grp) - 1;
      if (claimed) {
        S.h[slot] = t.h;
        S.off[slot] = t.off;
        S.k0[slot] = t.k0;
        S.k1[slot] = t.k1;
        S.len[slot] = t.len;
        S.cnt[slot] = 0;
      }
    }
    occ += __popc(__ballot_sync(0xffffffffu, claimed));
    __syncwarp();
    if (pending && !empty && !match) slot = (slot + 1) & (LT - 1);
  }
}

__device__ void local_flush(WarpSmem& S, int& occ, const uint8_t* __restrict__ in, uint64_t n,
                            unsigned long long* gkey, unsigned long long* gcnt, uint64_t cap, uint32_t* state) {
  const int lane = threadIdx.x & 31;
  for (int s = lane; s < LT; s += 32) {
    if (S.h[s] != 0) {
      global_insert(in, n, gkey, gcnt, cap, state, S.h[s], S.off[s], S.len[s], S.cnt[s]);
      S.h[s] = 0;
    }
  }
  __syncwarp();
  occ = 0;
}

__global__ void __launch_bounds__(WC_THREADS, 2)
wc_map_kernel(const uint8_t* __restrict__ in, uint64_t n, unsigned long long* gkey, unsigned long long* gcnt,
              uint64_t cap, uint32_t* state) {
  extern __shared__ __align__(16) unsigned char wc_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpSmem& S = reinterpret_cast<WarpSmem*>(wc_smem)[warp];
  for (int i = lane; i < LT; i += 32) S.h[i] = 0;
  __syncwarp();
  int occ = 0;
  const uint64_t nseg = (n + SEG - 1) / SEG;
  const uint64_t gw = (uint64_t)blockIdx.x * WC_WARPS + warp;
  const uint64_t nw = (uint64_t)gridDim.x * WC_WARPS;
  const bool aligned = ((uintptr_t)in & 15) == 0;
  for (uint64_t seg = gw; seg < nseg; seg += nw) {
    const uint64_t base = seg * SEG;
    const uint64_t rem = n - base;
    const uint32_t bufn = rem < (uint64_t)(SEG + HALO) ? (uint32_t)rem : (uint32_t)(SEG + HALO);
    if (aligned && bufn == SEG + HALO) {
      const uint4* src = reinterpret_cast<const uint4*>(in + base);
      reinterpret_cast<uint4*>(S.buf)[lane] = src[lane];
      if (lane < HALO / 16) reinterpret_cast<uint4*>(S.buf)[32 + lane] = src[32 + lane];
    } else {
      for (uint32_t r = lane; r < bufn; r += 32) S.buf[r] = in[base + r];
    }
    __syncwarp();
    // token-start mask of this lane's 16 bytes
    uint32_t mask = 0;
    {
      const uint32_t r0 = lane * 16;
      bool pws;
      if (r0 == 0) pws = (base == 0) ? true : is_ws(in[base - 1]);
      else pws = (r0 - 1 < bufn) ? is_ws(S.buf[r0 - 1]) : true;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const uint32_t r = r0 + j;
        if (r < bufn) {
          const bool w = is_ws(S.buf[r]);
          if (!w && pws) mask |= 1u << j;
          pws = w;
        }
      }
    }
    const int c = __popc(mask);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    {
      int o = incl - c;
      uint32_t m = mask;
      while (m) {
        const int j = __ffs(m) - 1;
        S.starts[o++] = (uint16_t)(lane * 16 + j);
        m &= m - 1;
      }
    }
    __syncwarp();
    for (int r0 = 0; r0 < total; r0 += 32) {
      if (occ >= LT_FLUSH_AT) local_flush(S, occ, in, n, gkey, gcnt, cap, state);
      const int i = r0 + lane;
      const bool active = i < total;
      Tok t;
      if (active) t = read_token(in, n, base, S.buf, bufn, S.starts[i]);
      else t.h = 0, t.off = 0, t.k0 = 0, t.k1 = 0, t.len = 0;
      local_insert(S, active, t, occ, in, n);
    }
    __syncwarp();
  }
  local_flush(S, occ, in, n, gkey, gcnt, cap, state);
}

// ------------------------------------------------------------------ sort
struct SortRec {
  unsigned long long nc;   // ~count  (ascending nc = descending count)
  unsigned long long s0;   // key bytes 0..7, big-endian, zero padded
  unsigned long long s1;   // key bytes 8..15
  uint32_t len;
  uint32_t idx;            // index into the offsets array
};
static_assert(sizeof(SortRec) == 32, "SortRec layout");

__device__ __forceinline__ bool rec_less(const SortRec& a, const SortRec& b, const uint8_t* __restrict__ in,
                                         const unsigned long long* offs) {
  if (a.nc != b.nc) return a.nc < b.nc;
  if (a.s0 != b.s0) return a.s0 < b.s0;
  if (a.s1 != b.s1) return a.s1 < b.s1;
  if (a.len <= 16 || b.len <= 16) return a.len < b.len;
  // both longer than 16 bytes with the same first 16: compare the rest
  const uint64_t oa = offs[a.idx], ob = offs[b.idx];
  const uint32_t m = a.len < b.len ? a.len : b.len;
  for (uint32_t i = 16; i < m; ++i) {
    const uint8_t ca = in[oa + i], cb = in[ob + i];
    if (ca != cb) return ca < cb;
  }
  return a.len < b.len;
}

constexpr int CB = 1024;  // compaction / block-sort / scan block size (records)

__device__ __forceinline__ int block_excl_scan(int v, int* tmp, int& total) {
  // blockDim.x == 1024 assumed by callers
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
    int w = tmp[lane];
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

__global__ void __launch_bounds__(CB)
wc_compact_kernel(const uint8_t* __restrict__ in, uint64_t n, const unsigned long long* gkey,
                  const unsigned long long* gcnt, uint64_t cap, uint32_t* state, SortRec* recs,
                  unsigned long long* offs) {
  __shared__ int tmp[33];
  __shared__ uint32_t blk_base;
  const uint64_t s = (uint64_t)blockIdx.x * CB + threadIdx.x;
  const unsigned long long w = s < cap ? gkey[s] : 0ull;
  int total;
  const int r = block_excl_scan(w != 0, tmp, total);
  if (threadIdx.x == 0) blk_base = total ? atomicAdd(state + 1, (uint32_t)total) : 0u;
  __syncthreads();
  if (w == 0) return;
  const uint32_t i = blk_base + (uint32_t)r;
  const uint64_t off = (w & OFF_MASK) - 1;
  uint32_t len = (uint32_t)(w >> 40);
  if (len == LEN_SAT) {
    uint64_t e = off + len;
    while (e < n && !is_ws(in[e])) ++e;
    len = (uint32_t)(e - off);
  }
  unsigned long long s0 = 0, s1 = 0;
  const uint32_t l16 = len < 16 ? len : 16;
  for (uint32_t j = 0; j < l16; ++j) {
    const unsigned long long b = in[off + j];
    if (j < 8) s0 |= b << (56 - 8 * j);
    else s1 |= b << (56 - 8 * (j - 8));
  }
  SortRec rec;
  rec.nc = ~gcnt[s];
  rec.s0 = s0;
  rec.s1 = s1;
  rec.len = len;
  rec.idx = i;
  recs[i] = rec;
  offs[i] = off;
}

__global__ void __launch_bounds__(512)
wc_blocksort_kernel(SortRec* recs, const uint32_t* state, const uint8_t* __restrict__ in,
                    const unsigned long long* offs) {
  __shared__ SortRec sh[CB];
  const uint32_t m = state[1];
  const uint64_t b0 = (uint64_t)blockIdx.x * CB;
  if (b0 >= m) return;
  for (int i = threadIdx.x; i < CB; i += blockDim.x) {
    if (b0 + i < m) sh[i] = recs[b0 + i];
    else sh[i] = SortRec{~0ull, ~0ull, ~0ull, 0xffffffffu, 0xffffffffu};
  }
  __syncthreads();
  for (int k = 2; k <= CB; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int t = threadIdx.x;  // 512 threads, one pair each
      const int lo = 2 * j * (t / j) + (t % j);
      const int hi = lo + j;
      const bool up = (lo & k) == 0;
      SortRec a = sh[lo], b = sh[hi];
      const bool a_pad = a.idx == 0xffffffffu, b_pad = b.idx == 0xffffffffu;
      bool b_lt_a;
      if (a_pad || b_pad) b_lt_a = a_pad && !b_pad;
      else b_lt_a = rec_less(b, a, in, offs);
      if (b_lt_a == up) {
        sh[lo] = b;
        sh[hi] = a;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < CB; i += blockDim.x)
    if (b0 + i < m) recs[b0 + i] = sh[i];
}

constexpr int MERGE_ITEMS = 8;

__global__ void __launch_bounds__(256)
wc_merge_kernel(const SortRec* __restrict__ src, SortRec* __restrict__ dst, const uint32_t* state, uint64_t L,
                const uint8_t* __restrict__ in, const unsigned long long* offs) {
  const uint64_t m = state[1];
  const uint64_t k0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * MERGE_ITEMS;
  if (k0 >= m) return;
  const uint64_t a0 = (k0 / (2 * L)) * (2 * L);
  const uint64_t la = (m - a0) < L ? (m - a0) : L;
  const uint64_t b0 = a0 + L;
  const uint64_t lb = b0 < m ? ((m - b0) < L ? (m - b0) : L) : 0;
  const SortRec* A = src + a0;
  const SortRec* B = src + b0;
  const uint64_t kk = k0 - a0;
  uint64_t lo = kk > lb ? kk - lb : 0;
  uint64_t hi = kk < la ? kk : la;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (rec_less(A[mid], B[kk - 1 - mid], in, offs)) lo = mid + 1;
    else hi = mid;
  }
  uint64_t i = lo, j = kk - lo;
  const uint64_t end = a0 + la + lb;
  for (int t = 0; t < MERGE_ITEMS && k0 + t < end; ++t) {
    bool takeA;
    if (j >= lb) takeA = true;
    else if (i >= la) takeA = false;
    else takeA = rec_less(A[i], B[j], in, offs);
    dst[k0 + t] = takeA ? A[i++] : B[j++];
  }
}

// Sum of key lengths per block of CB sorted records.
__global__ void __launch_bounds__(CB)
wc_lensum_kernel(const SortRec* recs, const uint32_t* state, unsigned long long* bsum) {
  const uint32_t m = state[1];
  const uint64_t i = (uint64_t)blockIdx.x * CB + threadIdx.x;
  unsigned long long v = i < m ? recs[i].len : 0;
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ unsigned long long ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < 32; ++w) s += ws[w];
    bsum[blockIdx.x] = s;
  }
}

// Exclusive scan of the block sums (one CTA) and the result header.
__global__ void __launch_bounds__(CB)
wc_bscan_kernel(unsigned long long* bsum, uint64_t nb, const uint32_t* state, unsigned long long* out_hdr) {
  __shared__ unsigned long long carry;
  __shared__ unsigned long long wsum[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t b = 0; b < nb; b += CB) {
    const uint64_t i = b + threadIdx.x;
    const unsigned long long v = i < nb ? bsum[i] : 0;
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
    const unsigned long long excl = carry + wsum[warp] + incl - v;
    if (i < nb) bsum[i] = excl;
    __syncthreads();
    if (threadIdx.x == CB - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out_hdr[0] = state[1];
    out_hdr[1] = carry;
  }
}

// Write the records and copy the key bytes.
__global__ void __launch_bounds__(CB)
wc_gather_kernel(const SortRec* recs, const uint32_t* state, const unsigned long long* bsum,
                 const uint8_t* __restrict__ in, const unsigned long long* offs, uint8_t* out) {
  const uint32_t m = state[1];
  const uint64_t i = (uint64_t)blockIdx.x * CB + threadIdx.x;
  if ((uint64_t)blockIdx.x * CB >= m) return;
  const uint32_t len = i < m ? recs[i].len : 0;
  // block-exclusive scan of lengths in 64-bit
  __shared__ unsigned long long wsum[32];
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
  const SortRec r = recs[i];
  const unsigned long long koff = bsum[blockIdx.x] + wsum[warp] + incl - len;
  unsigned long long* rec = reinterpret_cast<unsigned long long*>(out + 16 + 24 * i);
  rec[0] = ~r.nc;
  rec[1] = koff;
  rec[2] = len;
  uint8_t* keys = out + 16 + 24 * (uint64_t)m + koff;
  const uint64_t src = offs[r.idx];
  for (uint32_t j = 0; j < len; ++j) keys[j] = in[src + j];
}

}  // namespace

size_t wc_sortbuf_bytes(uint64_t cap) {
  const uint64_t nb = (cap + CB - 1) / CB;
  return 2 * cap * sizeof(SortRec) + cap * sizeof(unsigned long long) + nb * sizeof(unsigned long long) + 256;
}

uint64_t wc_out_bytes(uint64_t cap, uint64_t n) {
  // at most min(cap, n/1 tokens) records; key bytes never exceed n
  return 16 + 24 * cap + n;
}

cudaError_t launch_wordcount(const uint8_t* in, uint64_t n, const WcBuffers& b, const DevInfo& di, cudaStream_t s,
                             uint64_t* nk) {
  cudaError_t e;
  // table: key and count arrays are contiguous (key then cnt)
  if ((e = cudaMemsetAsync(b.key, 0, 2 * b.cap * sizeof(uint64_t), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b.state, 0, 4 * sizeof(uint32_t), s)) != cudaSuccess) return e;
  unsigned long long* gkey = reinterpret_cast<unsigned long long*>(b.key);
  unsigned long long* gcnt = reinterpret_cast<unsigned long long*>(b.cnt);
  if (n > 0) {
    const int smem = WC_WARPS * (int)sizeof(WarpSmem);
    if ((e = cudaFuncSetAttribute(wc_map_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
      return e;
    const uint64_t nseg = (n + SEG - 1) / SEG;
    uint64_t grid = (nseg + WC_WARPS - 1) / WC_WARPS;
    const uint64_t gmax = 2ull * di.sms;
    if (grid > gmax) grid = gmax;
    wc_map_kernel<<<(unsigned)grid, WC_THREADS, smem, s>>>(in, n, gkey, gcnt, b.cap, b.state);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nk;
  }
  return launch_wordcount_post(in, n, b, s, nk);
}

cudaError_t launch_wordcount_post(const uint8_t* in, uint64_t n, const WcBuffers& b, cudaStream_t s, uint64_t* nk) {
  cudaError_t e;
  (void)n;
  unsigned long long* gkey = reinterpret_cast<unsigned long long*>(b.key);
  unsigned long long* gcnt = reinterpret_cast<unsigned long long*>(b.cnt);
  SortRec* r0 = reinterpret_cast<SortRec*>(b.sortbuf);
  SortRec* r1 = r0 + b.cap;
  unsigned long long* offs = reinterpret_cast<unsigned long long*>(r1 + b.cap);
  unsigned long long* bsum = offs + b.cap;
  const uint64_t nb = (b.cap + CB - 1) / CB;
  wc_compact_kernel<<<(unsigned)nb, CB, 0, s>>>(in, n, gkey, gcnt, b.cap, b.state, r0, offs);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  wc_blocksort_kernel<<<(unsigned)nb, 512, 0, s>>>(r0, b.state, in, offs);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *nk += 2;
  SortRec* src = r0;
  SortRec* dst = r1;
  for (uint64_t L = CB; L < b.cap; L *= 2) {
    const uint64_t threads = (b.cap + MERGE_ITEMS - 1) / MERGE_ITEMS;
    wc_merge_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(src, dst, b.state, L, in, offs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nk;
    SortRec* t = src;
    src = dst;
    dst = t;
  }
  wc_lensum_kernel<<<(unsigned)nb, CB, 0, s>>>(src, b.state, bsum);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  wc_bscan_kernel<<<1, CB, 0, s>>>(bsum, nb, b.state, reinterpret_cast<unsigned long long*>(b.out));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  wc_gather_kernel<<<(unsigned)nb, CB, 0, s>>>(src, b.state, bsum, in, offs, b.out);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *nk += 3;
  return cudaSuccess;
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
// that loads this library keeps the array (about 11 MiB) until the process
// exits.
#include <mutex>

namespace mrgb {
namespace {
constexpr uint64_t NOALLOC_SLOTS = 1ull << 17;
constexpr uint64_t NOALLOC_TABLE_BYTES = 2 * NOALLOC_SLOTS * 8;
constexpr uint64_t NOALLOC_STATE_BYTES = 256;
constexpr uint64_t NOALLOC_SORT_BYTES =
    ((2 * NOALLOC_SLOTS * sizeof(SortRec) + NOALLOC_SLOTS * 8 + ((NOALLOC_SLOTS + CB - 1) / CB) * 8 + 256) + 255) &
    ~255ull;
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
  b.cnt = b.key + NOALLOC_SLOTS;
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
