// SIMD hashing of variable-length strings (Sec. III-C) on warp lanes.
//
// The paper hashes strings character by character (Listing 1: v = func(v,
// c) per character) and vectorises across strings in two ways; a warp's 32
// lanes play the role of the 16 SIMD lanes:
//   * SIMDH-Padding: a warp takes 32 consecutive strings, one per lane, and
//     runs as many rounds as the longest of them has characters; lanes whose
//     string is shorter are masked off (the paper's "padding").
//   * SIMDH-Stream: a lane whose string is finished takes the next
//     unprocessed string at once, so no lane idles while strings remain; the
//     refill is a warp ballot plus a prefix count (the paper's mask
//     prefix-sum, done here by popc on the ballot).
//   * Wide (GB300-first, not in the paper): Padding's grouping, but each lane
//     reads its string four bytes per load through an aligned word pair and a
//     funnel shift, instead of one byte per load.
// All three compute 64-bit FNV-1a of every token and must agree bit for bit.
#include "mr_internal.h"

namespace mrgb {
namespace {

constexpr int SH_THREADS = 256;
constexpr uint64_t FNV_OFFSET = 0xcbf29ce484222325ull;
constexpr uint64_t FNV_PRIME = 0x100000001b3ull;
constexpr uint64_t STREAM_CHUNK = 32 * 8;  // tokens per warp work unit (Stream)

__device__ __forceinline__ uint64_t fnv_step(uint64_t v, uint32_t c) { return (v ^ c) * FNV_PRIME; }

__global__ void __launch_bounds__(SH_THREADS) simdh_padding_kernel(const uint8_t* __restrict__ text,
                                                                   const uint32_t* __restrict__ off,
                                                                   const uint32_t* __restrict__ len, uint64_t ntok,
                                                                   unsigned long long* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * SH_THREADS + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * SH_THREADS) >> 5;
  for (uint64_t g = warp; g * 32 < ntok; g += nwarps) {
    const uint64_t t = g * 32 + lane;
    const bool act = t < ntok;
    const uint32_t o = act ? off[t] : 0u, L = act ? len[t] : 0u;
    const uint32_t rounds = __reduce_max_sync(0xffffffffu, L);
    uint64_t v = FNV_OFFSET;
    for (uint32_t j = 0; j < rounds; ++j)
      if (j < L) v = fnv_step(v, text[o + j]);
    if (act) out[t] = v;
  }
}

__global__ void __launch_bounds__(SH_THREADS) simdh_stream_kernel(const uint8_t* __restrict__ text,
                                                                  const uint32_t* __restrict__ off,
                                                                  const uint32_t* __restrict__ len, uint64_t ntok,
                                                                  unsigned long long* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const uint64_t warp = ((uint64_t)blockIdx.x * SH_THREADS + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * SH_THREADS) >> 5;
  for (uint64_t c0 = warp * STREAM_CHUNK; c0 < ntok; c0 += nwarps * STREAM_CHUNK) {
    const uint64_t c1 = (c0 + STREAM_CHUNK) < ntok ? c0 + STREAM_CHUNK : ntok;
    uint64_t next = c0, t = 0;
    uint32_t pos = 0, rem = 0;
    uint64_t v = 0;
    bool have = false;
    for (;;) {
      // lanes without a string take the next ones, in lane order
      const unsigned need = __ballot_sync(0xffffffffu, !have);
      if (!have) {
        const uint64_t mine = next + (uint64_t)__popc(need & below);
        if (mine < c1) {
          t = mine;
          pos = off[t];
          rem = len[t];
          v = FNV_OFFSET;
          have = true;
        }
      }
      next += (uint64_t)__popc(need);
      if (!__any_sync(0xffffffffu, have)) break;
      if (have) {
        if (rem) {
          v = fnv_step(v, text[pos]);
          ++pos;
          --rem;
        }
        if (rem == 0) {
          out[t] = v;
          have = false;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(SH_THREADS) simdh_wide_kernel(const uint8_t* __restrict__ text, uint64_t n,
                                                                const uint32_t* __restrict__ off,
                                                                const uint32_t* __restrict__ len, uint64_t ntok,
                                                                unsigned long long* __restrict__ out) {
  // words of the 4-byte-aligned range that holds the text; the first and
  // last words may hold bytes outside the text (never used)
  const uintptr_t a = reinterpret_cast<uintptr_t>(text);
  const uint32_t* __restrict__ words = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
  const uint32_t shift = (uint32_t)(a & 3);
  const uint64_t last_word = n ? (shift + n - 1) / 4 : 0;
  const int lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * SH_THREADS + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * SH_THREADS) >> 5;
  for (uint64_t g = warp; g * 32 < ntok; g += nwarps) {
    const uint64_t t = g * 32 + lane;
    const bool act = t < ntok;
    uint64_t v = FNV_OFFSET;
    if (act) {
      const uint64_t p = (uint64_t)off[t] + shift;
      uint32_t L = len[t];
      uint64_t wi = p >> 2;
      const uint32_t sh = (uint32_t)(p & 3) * 8;
      uint32_t cur = words[wi];
      while (L > 0) {
        const uint32_t nxt = wi + 1 <= last_word ? words[wi + 1] : 0u;
        const uint32_t w = __funnelshift_r(cur, nxt, sh);
        const uint32_t take = L < 4 ? L : 4;
        for (uint32_t b = 0; b < take; ++b) v = fnv_step(v, (w >> (8 * b)) & 0xFFu);
        L -= take;
        cur = nxt;
        ++wi;
      }
      out[t] = v;
    }
  }
}

}  // namespace
}  // namespace mrgb

extern "C" mr_status mr_simdh_hash(const uint8_t* text, uint64_t text_bytes, const uint32_t* tok_off,
                                   const uint32_t* tok_len, uint64_t ntok, int method, uint64_t* hashes,
                                   void* cuda_stream) {
  using namespace mrgb;
  if (method < MR_SIMDH_PADDING || method > MR_SIMDH_WIDE) return MR_EINVAL;
  if (text_bytes >= (1ull << 32)) return MR_EINVAL;
  if (ntok == 0) return MR_OK;
  if (!tok_off || !tok_len || !hashes || (!text && text_bytes)) return MR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_last_error("mr_simdh_hash(device)", e);
    return MR_ECUDA;
  }
  unsigned long long* out = reinterpret_cast<unsigned long long*>(hashes);
  const uint64_t units = method == MR_SIMDH_STREAM ? (ntok + STREAM_CHUNK - 1) / STREAM_CHUNK : (ntok + 31) / 32;
  uint64_t grid = (units + SH_THREADS / 32 - 1) / (SH_THREADS / 32);
  if (grid > (uint64_t)sms * 8) grid = (uint64_t)sms * 8;
  if (grid < 1) grid = 1;
  if (method == MR_SIMDH_PADDING)
    simdh_padding_kernel<<<(unsigned)grid, SH_THREADS, 0, s>>>(text, tok_off, tok_len, ntok, out);
  else if (method == MR_SIMDH_STREAM)
    simdh_stream_kernel<<<(unsigned)grid, SH_THREADS, 0, s>>>(text, tok_off, tok_len, ntok, out);
  else
    simdh_wide_kernel<<<(unsigned)grid, SH_THREADS, 0, s>>>(text, text_bytes, tok_off, tok_len, ntok, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error("mr_simdh_hash", e);
    return MR_ECUDA;
  }
  return MR_OK;
}
