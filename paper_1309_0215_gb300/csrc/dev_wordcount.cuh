// Device code of the word-count map + combine pass, shared by the plain
// kernel (k_wordcount.cu) and the persistent batched kernel (k_batch.cu).
//
// Map (arXiv:1309.0215 Sec. II-A): a token is a maximal run of bytes that are
// not ASCII whitespace; each emits (token, 1); reduce is a sum.
//
// Key encoding (128 bits, the container's key):
//   short token, 1..15 bytes:  w0 = bytes 0..7 (little-endian, zero padded)
//                              w1 = bytes 8..14 | length << 56
//   long token, >= 16 bytes:   w0 = offset of an occurrence in the input + 1
//                              w1 = 0xFF << 56 | length
// A short key is its own identity (no memory read to compare); a long key
// is compared byte for byte against the resident, immutable input.  w1 is
// never zero, so {0, 0} marks an empty slot.
//
// Global container: open addressing, linear probing, a slot = 16-byte key
// claimed with one 128-bit atomic CAS (written once, never changed) plus a
// 64-bit count updated with atomicAdd.  Running out of probes raises the
// job's overflow flag (the host then re-runs with a larger table).
//
// Local container (the paper's combiner, Sec. III-A, with the bounded local
// table of Sec. III-D), shaped for Zipf-like key streams: a 2-way cache of
// hot keys per warp in shared memory (two candidate slots per key, one
// compare each, no probing) absorbs the frequent keys, and the rest go
// straight to the global container, where such rarer keys do not contend.
// No warp collective is used: lanes of one round that carry the same key
// simply add to the same slot count (shared-memory atomics), and an empty
// slot is claimed with a 64-bit shared-memory CAS.  The cache is merged into
// the global container every CACHE_EPOCH segments (so it can re-learn which
// keys are hot) and at the end.
#pragma once
#include <cstdint>

namespace mrgb {
namespace wc {

constexpr int SEG = 512;                // bytes per warp step (16 per lane)
constexpr int HALO = 64;                // staged bytes after the segment
constexpr int BUF = SEG + HALO;
constexpr int LT = 128;                 // hot-key cache entries per warp
constexpr int CACHE_EPOCH = 64;         // segments between cache merges
constexpr int MAX_PROBES = 4096;
constexpr uint64_t LONG_TAG = 0xFFull << 56;
constexpr uint64_t LEN_MASK = (1ull << 56) - 1;

struct WarpLocal {
  unsigned long long w0[LT];
  unsigned long long w1[LT];
  uint32_t h[LT];
  uint32_t cnt[LT];
  uint8_t buf[BUF];
  uint32_t wsb[BUF / 32 + 2];  // whitespace bitmap of buf: bit j of word q = byte 32q + j
  uint16_t starts[SEG / 2];
};
static_assert(sizeof(WarpLocal) % 16 == 0, "WarpLocal must keep 16-byte alignment");

// One word-count job as the kernels see it.
struct JobDev {
  const uint8_t* in;
  uint64_t n;
  unsigned long long* key;   // [cap][2]
  unsigned long long* cnt;   // [cap]
  uint64_t cap;              // power of two
  uint32_t log2cap;
  uint32_t* state;           // [0] overflow flag; [2..7] filled by the post phase
  uint8_t* out;
  uint64_t blk0;             // first compaction block of this job
};

__device__ __forceinline__ bool is_ws(uint32_t c) { return c == 32u || (c - 9u) < 5u; }

// 0x80 in every byte of u that is ASCII whitespace (0x20, or 0x09..0x0D),
// else 0: exact per byte, with no carry between bytes.  Space: the byte of
// u ^ 0x20202020 is zero iff ((b & 0x7F) + 0x7F) | b has its top bit clear.
// 9..13: with h = b & 0x7F, h + 0x77 reaches 0x80 iff h >= 9 and h + 0x72
// iff h >= 14; bytes >= 0x80 are excluded by their own top bit.
__device__ __forceinline__ uint32_t ws_bytes(uint32_t u) {
  const uint32_t x = u ^ 0x20202020u;
  const uint32_t sp = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x);
  const uint32_t h = u & 0x7F7F7F7Fu;
  const uint32_t rg = (h + 0x77777777u) & ~(h + 0x72727272u) & ~u;
  return (sp | rg) & 0x80808080u;
}
// compress a 0xFF-per-byte mask to 4 bits (byte i -> bit i)
__device__ __forceinline__ uint32_t byte_bits(uint32_t m) { return ((m & 0x80808080u) * 0x00204081u) >> 28; }

__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// 32-bit multiply-xorshift mix of the four 32-bit words of a short key
// (the key is compared exactly; the hash only spreads slots).
__device__ __forceinline__ uint32_t hash_short(uint64_t w0, uint64_t w1) {
  uint32_t h = (uint32_t)w0 * 0x9E3779B1u;
  h ^= __funnelshift_l((uint32_t)(w0 >> 32) * 0x85EBCA77u, (uint32_t)(w0 >> 32) * 0x85EBCA77u, 13);
  h ^= __funnelshift_l((uint32_t)w1 * 0xC2B2AE3Du, (uint32_t)w1 * 0xC2B2AE3Du, 7);
  h ^= (uint32_t)(w1 >> 32) * 0x27D4EB2Fu;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  return h;
}

struct Tok {
  uint64_t w0, w1;
  uint32_t h;
};

// Bytes of two long tokens of equal length len, at offsets a and b.
__device__ inline bool long_equal(const uint8_t* __restrict__ in, uint64_t a, uint64_t b, uint64_t len) {
  if (a == b) return true;
  for (uint64_t i = 0; i < len; ++i)
    if (in[a + i] != in[b + i]) return false;
  return true;
}

// The token starting at segment-relative byte r (its first 16 bytes are
// always inside the staged buffer; bytes past the input end were staged as
// spaces).  Its length comes from the segment's whitespace bitmap.
template <class B>
__device__ __forceinline__ Tok read_token(const uint8_t* __restrict__ in, uint64_t n, uint64_t base, const B& W,
                                          uint32_t r) {
  const uint32_t* wb = reinterpret_cast<const uint32_t*>(W.buf);
  // m bit i: byte r + 1 + i is whitespace
  const uint32_t p = r + 1, wi = p >> 5, bs = p & 31;
  const uint32_t m = __funnelshift_r(W.wsb[wi], W.wsb[wi + 1], bs);
  Tok t;
  if (m & 0x7FFFu) {
    const uint32_t a = r >> 2, sh = (r & 3) * 8;
    const uint32_t x0 = wb[a], x1 = wb[a + 1], x2 = wb[a + 2], x3 = wb[a + 3], x4 = wb[a + 4];
    const uint32_t u0 = __funnelshift_r(x0, x1, sh), u1 = __funnelshift_r(x1, x2, sh);
    const uint32_t u2 = __funnelshift_r(x2, x3, sh), u3 = __funnelshift_r(x3, x4, sh);
    const uint32_t L = __ffs(m);  // 1..15 (byte 0 is a token byte)
    uint64_t k0 = (uint64_t)u0 | ((uint64_t)u1 << 32);
    uint64_t k1 = (uint64_t)u2 | ((uint64_t)u3 << 32);
    if (L < 8) {
      k0 &= (1ull << (8 * L)) - 1;
      k1 = 0;
    } else {
      k1 &= (1ull << (8 * (L - 8))) - 1;
    }
    t.w0 = k0;
    t.w1 = k1 | ((uint64_t)L << 56);
    t.h = hash_short(t.w0, t.w1);
    return t;
  }
  // long token: FNV-1a 64 over its bytes, then the length is mixed in
  const uint64_t off = base + r;
  uint64_t h = 0xcbf29ce484222325ull, len = 0;
  for (uint64_t i = off; i < n; ++i) {
    const uint32_t rel = (uint32_t)(i - base);
    const uint32_t c = (i - base) < (uint64_t)BUF ? W.buf[rel] : in[i];
    if (is_ws(c)) break;
    h = (h ^ c) * 0x100000001b3ull;
    ++len;
  }
  t.w0 = off + 1;
  t.w1 = LONG_TAG | (len & LEN_MASK);
  t.h = (uint32_t)fmix64(h ^ len);
  return t;
}

__device__ __forceinline__ void ld_slot(const unsigned long long* p, uint64_t& a, uint64_t& b) {
  asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

__device__ __forceinline__ void cas_slot(unsigned long long* p, uint64_t n0, uint64_t n1, uint64_t& o0, uint64_t& o1) {
  asm volatile(
      "{\n\t.reg .b128 d, c, v;\n\t"
      "mov.b128 c, {%2, %2};\n\t"
      "mov.b128 v, {%3, %4};\n\t"
      "atom.relaxed.gpu.global.cas.b128 d, [%5], c, v;\n\t"
      "mov.b128 {%0, %1}, d;\n\t}\n"
      : "=l"(o0), "=l"(o1)
      : "l"(0ull), "l"(n0), "l"(n1), "l"(p)
      : "memory");
}

__device__ __forceinline__ uint64_t global_slot(uint32_t h, uint32_t log2cap) {
  return log2cap ? (uint64_t)((h * 0x9E3779B1u) >> (32 - log2cap)) : 0;
}

// Combine (key, c) into the job's global container.  Linear probing, two
// slots per step: both slots are loaded before either is examined, so a
// key that is not in its first slot costs no second round trip to L2, and
// the lanes of a warp, which probe different keys, finish in fewer steps.
// A slot loaded before a CAS on the slot before it may be stale, which is
// harmless: a slot only ever changes from empty to a key.
__device__ __forceinline__ bool slot_take(const JobDev& J, uint64_t s, uint64_t r0, uint64_t r1, uint64_t w0,
                                          uint64_t w1, bool is_long, uint64_t c) {
  unsigned long long* sp = J.key + 2 * s;
  if (r0 == 0 || r1 == 0) {  // empty, or a read that raced the CAS: ask the CAS
    cas_slot(sp, w0, w1, r0, r1);
    if (r0 == 0 && r1 == 0) {
      atomicAdd(J.cnt + s, (unsigned long long)c);
      return true;
    }
  }
  if (r1 == w1 && (r0 == w0 || (is_long && long_equal(J.in, r0 - 1, w0 - 1, w1 & LEN_MASK)))) {
    atomicAdd(J.cnt + s, (unsigned long long)c);
    return true;
  }
  return false;
}

// WIDTH = 2 loads two slots per step; WIDTH = 1 is plain linear probing,
// kept for the persistent batch kernel, whose registers are tight.
template <int WIDTH = 2>
__device__ inline void global_insert(const JobDev& J, uint64_t w0, uint64_t w1, uint32_t h, uint64_t c) {
  uint64_t slot = global_slot(h, J.log2cap);
  const bool is_long = (w1 >> 56) == 0xFF;
  const uint64_t mask = J.cap - 1;
  for (int p = 0; p < MAX_PROBES; p += WIDTH) {
    if (WIDTH == 2) {
      const uint64_t sb = (slot + 1) & mask;
      uint64_t a0, a1, b0, b1;
      ld_slot(J.key + 2 * slot, a0, a1);
      ld_slot(J.key + 2 * sb, b0, b1);
      if (slot_take(J, slot, a0, a1, w0, w1, is_long, c)) return;
      if (slot_take(J, sb, b0, b1, w0, w1, is_long, c)) return;
    } else {
      uint64_t a0, a1;
      ld_slot(J.key + 2 * slot, a0, a1);
      if (slot_take(J, slot, a0, a1, w0, w1, is_long, c)) return;
    }
    slot = (slot + WIDTH) & mask;
  }
  atomicOr(J.state, 1u);
}

// Combine one token per active lane into the warp's cache; all 32 lanes call
// this together (the warp syncs inside).  A short key that sits in one of its
// two cache slots adds 1 there.  Otherwise the first of its slots that is
// empty is claimed by a CAS on the slot's w1: the winner fills the slot with
// count 1; a loser whose key turns out to be the winner's (read after a warp
// sync) adds 1 to it.  Returns true for a token the cache did not take —
// long keys (>= 16 bytes), keys whose slots are held by other keys, lost
// claims for other keys — which the caller sends to the global container.
__device__ __forceinline__ bool combine_local(WarpLocal& L, bool active, const Tok& t) {
  const bool is_long = (t.w1 >> 56) == 0xFF;
  const int s0 = (int)(t.h & (LT - 1)), s1 = (int)((t.h >> 16) & (LT - 1));
  bool done = !active;
  int want = -1;
  if (active && !is_long) {
    const uint64_t a1 = L.w1[s0], b1 = L.w1[s1];
    if (a1 == t.w1 && L.w0[s0] == t.w0) {
      atomicAdd(&L.cnt[s0], 1u);
      done = true;
    } else if (b1 == t.w1 && L.w0[s1] == t.w0) {
      atomicAdd(&L.cnt[s1], 1u);
      done = true;
    } else if (a1 == 0) {
      want = s0;
    } else if (b1 == 0) {
      want = s1;
    }
  }
  __syncwarp();
  unsigned long long old = ~0ull;
  if (want >= 0) old = atomicCAS(&L.w1[want], 0ull, (unsigned long long)t.w1);
  const bool won = want >= 0 && old == 0;
  if (won) {
    L.w0[want] = t.w0;
    L.h[want] = t.h;
    L.cnt[want] = 1u;
    done = true;
  }
  __syncwarp();
  if (want >= 0 && !won && old == t.w1 && L.w0[want] == t.w0) {
    atomicAdd(&L.cnt[want], 1u);
    done = true;
  }
  return !done;
}

__device__ inline void local_clear(WarpLocal& L) {
  for (int s = threadIdx.x & 31; s < LT; s += 32) L.w1[s] = 0;
  __syncwarp();
}

// Merge the warp's cache into the global container and empty it.
template <int WIDTH = 2>
__device__ inline void local_flush(WarpLocal& L, int& occ, const JobDev& J) {
  __syncwarp();
  for (int s = threadIdx.x & 31; s < LT; s += 32) {
    if (L.w1[s] != 0) {
      global_insert<WIDTH>(J, L.w0[s], L.w1[s], L.h[s], L.cnt[s]);
      L.w1[s] = 0;
    }
  }
  __syncwarp();
  occ = 0;
}

__device__ __forceinline__ uint4 shfl_down_u4(const uint4& v, int d) {
  return make_uint4(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d),
                    __shfl_down_sync(0xffffffffu, v.z, d), __shfl_down_sync(0xffffffffu, v.w, d));
}
__device__ __forceinline__ uint4 shfl_u4(const uint4& v, int src) {
  return make_uint4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                    __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}
// Bytes [sh, sh + 16) of the 32-byte little-endian window a | b (sh < 16).
__device__ __forceinline__ uint4 shift_window(const uint4& a, const uint4& b, uint32_t sh) {
  const uint32_t q = sh >> 2, r = (sh & 3) * 8;
  // t_i = word i + q of the window, picked without indexing registers
  const uint32_t t0 = q == 0 ? a.x : q == 1 ? a.y : q == 2 ? a.z : a.w;
  const uint32_t t1 = q == 0 ? a.y : q == 1 ? a.z : q == 2 ? a.w : b.x;
  const uint32_t t2 = q == 0 ? a.z : q == 1 ? a.w : q == 2 ? b.x : b.y;
  const uint32_t t3 = q == 0 ? a.w : q == 1 ? b.x : q == 2 ? b.y : b.z;
  const uint32_t t4 = q == 0 ? b.x : q == 1 ? b.y : q == 2 ? b.z : b.w;
  return make_uint4(__funnelshift_r(t0, t1, r), __funnelshift_r(t1, t2, r), __funnelshift_r(t2, t3, r),
                    __funnelshift_r(t3, t4, r));
}

// Stage segment seg of the job (and its 64-byte halo) in the warp's buffer
// W (members buf, wsb, starts), build the whitespace bitmap and the list of
// token starts (segment-relative offsets of the tokens whose first byte lies
// in the segment) and return how many there are.  All 32 lanes call this.
// pre: when not null, the caller already loaded this lane's 16 bytes of the
// segment (pre[0]) and, for lanes 0..3, of the halo (pre[1]) from a
// 16-byte-aligned segment with at least BUF bytes left (seg_prefetchable).
template <class B>
__device__ inline int stage_tokens(const JobDev& J, uint64_t seg, B& L, const uint4* pre = nullptr) {
  const int lane = threadIdx.x & 31;
  const uint64_t base = seg * SEG;
  const uint8_t* __restrict__ in = J.in;
  const uint64_t n = J.n;
  const uint64_t rem = n - base;
  // stage the segment and its halo; bytes past the input end read as spaces
  const uintptr_t sa = reinterpret_cast<uintptr_t>(in + base);
  uint4 mine;
  if (pre) {
    mine = pre[0];
    reinterpret_cast<uint4*>(L.buf)[lane] = mine;
    if (lane < HALO / 16) reinterpret_cast<uint4*>(L.buf)[32 + lane] = pre[1];
  } else if (rem >= (uint64_t)BUF && (sa & 15) == 0) {
    const uint4* src = reinterpret_cast<const uint4*>(sa);
    mine = __ldg(src + lane);
    reinterpret_cast<uint4*>(L.buf)[lane] = mine;
    if (lane < HALO / 16) reinterpret_cast<uint4*>(L.buf)[32 + lane] = __ldg(src + 32 + lane);
  } else if (rem >= (uint64_t)BUF) {
    // unaligned input: the 37 aligned words covering the 576 staged bytes
    // (each holds at least one input byte, so no load leaves the input's
    // 16-byte blocks), shifted into place; lane l needs words l and l + 1,
    // lanes 0..3 also words 32 + l and 33 + l for the halo
    const uint32_t sh = (uint32_t)(sa & 15);
    const uint4* src = reinterpret_cast<const uint4*>(sa - sh);
    const uint4 a = __ldg(src + lane);
    const uint4 e = lane <= HALO / 16 ? __ldg(src + 32 + lane) : make_uint4(0u, 0u, 0u, 0u);
    uint4 b = shfl_down_u4(a, 1), en = shfl_down_u4(e, 1);
    const uint4 w32 = shfl_u4(e, 0);
    if (lane == 31) b = w32;
    mine = shift_window(a, b, sh);
    reinterpret_cast<uint4*>(L.buf)[lane] = mine;
    if (lane < HALO / 16) reinterpret_cast<uint4*>(L.buf)[32 + lane] = shift_window(e, en, sh);
  } else {
    for (uint32_t r = lane; r < (uint32_t)BUF; r += 32) L.buf[r] = r < rem ? in[base + r] : (uint8_t)' ';
    __syncwarp();
    mine = reinterpret_cast<const uint4*>(L.buf)[lane];
  }
  // token starts among this lane's 16 bytes (staged bytes past the input
  // end are spaces, so the input end needs no test of its own)
  const uint32_t wsm = byte_bits(ws_bytes(mine.x)) | (byte_bits(ws_bytes(mine.y)) << 4) |
                       (byte_bits(ws_bytes(mine.z)) << 8) | (byte_bits(ws_bytes(mine.w)) << 12);
  {
    // whitespace bitmap of the staged bytes: the segment from the lanes'
    // masks; the halo by lane l testing its bytes l and 32 + l, one ballot
    // per 32 bytes
    static_assert(HALO == 64, "the halo is two bitmap words");
    __syncwarp();  // lanes 0..3 staged the halo
    const uint32_t h0 = __ballot_sync(0xffffffffu, is_ws(L.buf[SEG + lane]));
    const uint32_t h1 = __ballot_sync(0xffffffffu, is_ws(L.buf[SEG + 32 + lane]));
    const uint32_t up = __shfl_down_sync(0xffffffffu, wsm, 1);
    if ((lane & 1) == 0) L.wsb[lane >> 1] = (wsm & 0xFFFFu) | (up << 16);
    if (lane == 0) {
      L.wsb[SEG / 32] = h0;
      L.wsb[SEG / 32 + 1] = h1;
      L.wsb[BUF / 32] = 0xFFFFFFFFu;  // past the halo
    }
  }
  uint32_t prev = __shfl_up_sync(0xffffffffu, wsm >> 15, 1) & 1u;
  if (lane == 0) prev = (base == 0) ? 1u : (uint32_t)is_ws(in[base - 1]);
  const uint32_t start = ~wsm & ((wsm << 1) | prev) & 0xFFFFu;
  const int c = __popc(start);
  int incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  {
    int o = incl - c;
    uint32_t m = start;
    while (m) {
      const int j = __ffs(m) - 1;
      L.starts[o++] = (uint16_t)(lane * 16 + j);
      m &= m - 1;
    }
  }
  __syncwarp();
  return total;
}

// Whether segment seg can be staged from registers loaded ahead of time
// (16-byte aligned, a full buffer of input left), and that load.
__device__ __forceinline__ bool seg_prefetchable(const JobDev& J, uint64_t seg) {
  return seg * SEG + BUF <= J.n && (reinterpret_cast<uintptr_t>(J.in + seg * SEG) & 15) == 0;
}
__device__ __forceinline__ void seg_prefetch(const JobDev& J, uint64_t seg, uint4 (&pre)[2]) {
  const int lane = threadIdx.x & 31;
  const uint4* src = reinterpret_cast<const uint4*>(J.in + seg * SEG);
  pre[0] = __ldg(src + lane);
  if (lane < HALO / 16) pre[1] = __ldg(src + 32 + lane);
}

// One warp maps and combines the tokens whose first byte lies in segment seg.
// miss(lane_has_miss, token) is called by all 32 lanes after each round of
// up to 32 tokens and disposes of the tokens the cache did not take.
template <int WIDTH = 2, class Miss>
__device__ inline void warp_segment_t(const JobDev& J, uint64_t seg, WarpLocal& L, int& occ, Miss&& miss) {
  const int lane = threadIdx.x & 31;
  const uint64_t base = seg * SEG;
  const int total = stage_tokens(J, seg, L);
  for (int r0 = 0; r0 < total; r0 += 32) {
    const int i = r0 + lane;
    const bool active = i < total;
    Tok t;
    if (active) t = read_token(J.in, J.n, base, L, L.starts[i]);
    else t.w0 = 0, t.w1 = 0, t.h = 0;
    const bool m = combine_local(L, active, t);
    miss(m, t);
    __syncwarp();
  }
  // occ counts segments since the last cache merge
  if (++occ >= CACHE_EPOCH) local_flush<WIDTH>(L, occ, J);
}

// ---------------------------------------------------------------------------
// Local container of the plain map kernel for large inputs: one table per CTA
// in shared memory, shared by its warps (the paper's bounded local table,
// Sec. III-D, here per thread block).  Open addressing with two candidate
// slots per key; a slot is claimed once and never changes key, so once a
// CTA has seen a couple of thousand distinct keys the table is read-only
// apart from its counts, and it holds the keys that were frequent early on
// (for a Zipf-like stream, the hot ones).  A slot is {w0, w1} read with one
// 128-bit load.  A claim CASes w1 from 0 to CT_BUSY, writes w0, hash and
// count, fences and then stores w1.  Both words start at zero and keys whose
// w0 is 0 (tokens of NUL bytes) never enter the table, so a read that meets
// a claim half done (w1 already stored, w0 not yet seen) does not match and
// the token goes on as a miss.  A key may end up in two slots (two lanes
// claiming it at once); both counts reach the global container, which
// merges them.
constexpr unsigned long long CT_BUSY = 1ull;  // no key has w1 == 1 (its length byte is >= 1)
template <int NS>
struct CtaTableT {
  static constexpr int SLOTS = NS;  // a power of two
  ulonglong2 key[NS];  // {w0, w1}
  uint32_t h[NS];
  uint32_t cnt[NS];
};
// the table of the large-input map kernel and the batch kernel (one CTA of
// 32 warps per SM)
using CtaTableBig = CtaTableT<4096>;

// Per-warp state of the plain map kernel: the staged segment, its
// whitespace bitmap and token list, and a queue of the tokens the table did
// not take, which go to the global container 32 at a time (full warps, so
// the global probing runs once per 32 misses instead of once per round).
constexpr int MQ = 64;
struct MapWarp {
  uint8_t buf[BUF];
  uint32_t wsb[BUF / 32 + 2];
  uint16_t starts[SEG / 2];
  unsigned long long qw0[MQ], qw1[MQ];
  uint32_t qh[MQ];
};
static_assert(sizeof(CtaTableBig) % 16 == 0 && sizeof(MapWarp) % 16 == 0, "staging buffers must stay 16-byte aligned");

// Count one short token in the CTA table; false if neither of its two
// slots holds it or could be claimed for it (and for every long token).
template <class TT>
__device__ __forceinline__ bool cta_add(TT& T, const Tok& t) {
  if ((t.w1 >> 56) == 0xFF || t.w0 == 0) return false;
  const uint32_t s0 = t.h & (TT::SLOTS - 1);
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const uint32_t s = (s0 + p) & (TT::SLOTS - 1);
    unsigned long long k0, k1;
    asm volatile("ld.volatile.shared::cta.v2.u64 {%0, %1}, [%2];"
                 : "=l"(k0), "=l"(k1)
                 : "r"((uint32_t)__cvta_generic_to_shared(&T.key[s]))
                 : "memory");
    if (k1 == t.w1 && k0 == t.w0) {
      atomicAdd(&T.cnt[s], 1u);
      return true;
    }
    if (k1 == 0 && atomicCAS(&T.key[s].y, 0ull, CT_BUSY) == 0ull) {
      T.key[s].x = t.w0;
      T.h[s] = t.h;
      T.cnt[s] = 1u;
      __threadfence_block();
      *reinterpret_cast<volatile unsigned long long*>(&T.key[s].y) = t.w1;
      return true;
    }
  }
  return false;
}

// Queue the round's misses (m: this lane has one); once 32 are queued, the
// warp inserts the oldest 32 into the global container (WIDTH table slots
// loaded per probe step; the batch kernel, whose many small jobs keep the
// global tables in L2, is faster with one).  qn / qhd: queued entries and
// queue head, warp-uniform.
template <int WIDTH = 2>
__device__ __forceinline__ void mq_push(const JobDev& J, MapWarp& W, bool m, const Tok& t, uint32_t& qn,
                                        uint32_t& qhd) {
  const int lane = threadIdx.x & 31;
  const unsigned mm = __ballot_sync(0xffffffffu, m);
  if (!mm) return;
  if (m) {
    const uint32_t pos = (qhd + qn + (uint32_t)__popc(mm & ((1u << lane) - 1u))) & (MQ - 1);
    W.qw0[pos] = t.w0;
    W.qw1[pos] = t.w1;
    W.qh[pos] = t.h;
  }
  qn += (uint32_t)__popc(mm);
  if (qn >= 32) {
    __syncwarp();
    const uint32_t q = (qhd + (uint32_t)lane) & (MQ - 1);
    global_insert<WIDTH>(J, W.qw0[q], W.qw1[q], W.qh[q], 1);
    qhd = (qhd + 32) & (MQ - 1);
    qn -= 32;
  }
}

// The direct form: a token the cache did not take goes straight to the
// global container.
template <int WIDTH = 2>
__device__ inline void warp_segment(const JobDev& J, uint64_t seg, WarpLocal& L, int& occ) {
  warp_segment_t<WIDTH>(J, seg, L, occ, [&](bool m, const Tok& t) {
    if (m) global_insert<WIDTH>(J, t.w0, t.w1, t.h, 1);
  });
}

}  // namespace wc
}  // namespace mrgb
