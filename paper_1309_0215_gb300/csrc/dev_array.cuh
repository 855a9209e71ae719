// Device code of the array-container jobs (RGB8 histogram, int8 regression
// sums), shared by the plain kernels (k_array.cu) and the persistent batched
// kernel (k_batch.cu).  See k_array.cu for the design notes.
#pragma once
#include <cstdint>

namespace mrgb {
namespace arr {

constexpr int HIST_BINS = 768;
constexpr int HIST_COLS = 32;
constexpr int HIST_WORDS = HIST_BINS * HIST_COLS;   // 96 KiB of u32 counters
constexpr int CHUNK = 1536;                          // bytes per warp step (3 x 512)
constexpr int CHUNK_VEC = CHUNK / 16;

__device__ __forceinline__ uint4 ldg_stream(const uint4* p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

__device__ __forceinline__ void red_shared_add(uint32_t addr, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// One 32-bit word = 4 bytes; byte b belongs to channel slot (j0 + b) % 3 of
// the rotation cb[]; cb[q] already holds the lane's column base for that
// channel.  Counter address = column base + value * COLS columns * 4 bytes.
template <int J0, int COLS = HIST_COLS>
__device__ __forceinline__ void hist_word(uint32_t w, const uint32_t (&cb)[3]) {
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    uint32_t v = (w >> (8 * b)) & 0xFFu;
    red_shared_add(cb[(J0 + b) % 3] + v * (COLS * 4), 1u);
  }
}

// 16 bytes loaded by one lane for row k of a chunk.  Byte j of row k is at
// chunk offset k*512 + lane*16 + j; its channel is (rot0 + 2k + j) % 3 where
// rot0 = (alignment offset + lane) % 3 (512 = 2 mod 3, 16 = 1 mod 3).
template <int K, int COLS = HIST_COLS>
__device__ __forceinline__ void hist_vec(uint4 a, const uint32_t (&cb)[3]) {
  constexpr int R = (2 * K) % 3;
  // cbk[q] = column base of channel (rot0 + R + q) % 3
  uint32_t cbk[3] = {cb[R % 3], cb[(R + 1) % 3], cb[(R + 2) % 3]};
  hist_word<0, COLS>(a.x, cbk);
  hist_word<4, COLS>(a.y, cbk);
  hist_word<8, COLS>(a.z, cbk);
  hist_word<12, COLS>(a.w, cbk);
}

struct Sums5 { long long v[5]; };

__device__ __forceinline__ void lr_word(uint32_t w, int (&p)[5]) {
  const int wi = (int)w;
  const int xm = (int)(w & 0x00FF00FFu);           // [x0 0 x1 0]
  const int ym = (int)(w & 0xFF00FF00u);           // [0 y0 0 y1]
  const int sw = (int)__byte_perm(w, 0, 0x2301);   // [y0 x0 y1 x1]
  p[0] = __dp4a(wi, 0x00010001, p[0]);
  p[1] = __dp4a(wi, 0x01000100, p[1]);
  p[2] = __dp4a(xm, wi, p[2]);
  p[3] = __dp4a(ym, wi, p[3]);
  p[4] = __dp4a(xm, sw, p[4]);
}


}  // namespace arr
}  // namespace mrgb
