// k-means assignment on the 5th-generation tensor cores (tcgen05): the
// points x centroids contraction in BF16 with FP32 accumulation in tensor
// memory (TMEM), followed by an exact re-check of near ties.
//
// The distance d(x, c) = ||x||^2 - 2 x.c + ||c||^2 needs the cross term x.c,
// a dense (points x D) . (D x K) contraction — the one step of the hot path
// that is a real GEMM.  Per tile of 128 points:
//   * for D = 64 one producer thread moves each FP32 tile (128 rows, 32 KB,
//     contiguous) into a two-deep shared-memory ring with one bulk copy
//     (cp.async.bulk, completion counted on an mbarrier), so loads stay in
//     flight without registers; 8 converter warps read the tile (or load it
//     themselves for other D), compute ||x||^2 in FP32, and write BF16
//     operands in the 128-byte-swizzled K-major layout the MMA reads.  With TERMS = 3 each value is split as
//     x = hi + lo (hi = bf16(x), lo = bf16(x - hi)) and the MMA accumulates
//     hi.hi + hi.lo + lo.hi, so the cross term is good to about 2^-15
//     relative; TERMS = 1 is the plain single BF16 product.
//   * one thread issues tcgen05.mma (M = 128, N = K rounded up to 16, K = 16
//     per instruction, 4 steps over D = 64) into one of two 256-column TMEM
//     accumulators, and commits completion to mbarriers;
//   * 16 epilogue warps read the 128 x N FP32 tile with tcgen05.ld (one
//     TMEM lane per point; four warps per lane quadrant, each on a quarter
//     of the columns), form d~ = fma(-2, acc, ||x||^2) + ||c||^2, pack it
//     with its column into one sortable 32-bit key and keep the two smallest
//     keys with signed min/max (four independent top-2s per thread) plus
//     a lower bound of all other keys, and hand them to
//   * 2 finalizer warps (two lane quadrants each), which merge the four
//     column quarters of each point and apply the margin tests below, so
//     that no epilogue warp carries the per-point tail on its own path.
// Copies, converters, MMA issue, epilogue and finalizers overlap through the
// staging ring, two operand stages, two TMEM accumulators and two hand-off
// buffers.  Every mbarrier wait is bounded; on timeout the
// CTA stops, drains its MMAs, frees TMEM and reports through stats[3].
//
// Margin test (rigorous, per point).  With u_b = 2^-8 (BF16 rounding) the
// split leaves |x.c - (hi.hi + hi.lo + lo.hi)| <= 3.05 * 2^-16 ||x|| ||c||
// (one value: |x - hi - lo| <= u_b^2 |x|; sums by Cauchy-Schwarz); a single
// BF16 product leaves (2 u_b + u_b^2) ||x|| ||c||.  The tensor-core sum of the
// exact BF16 products is charged (products + 8) * 2^-21 ||x|| ||c|| (four
// times the round-to-nearest bound, allowing truncating adders), and the FP32
// norms and the final fma/add (D + 8) * 2^-24 (||x|| + ||c||)^2 (Higham,
// eq. 3.5).  The keys hold d~ truncated to 16 mantissa bits (t <= d~ <
// t (1 + 2^-15)), so with G = 2E + 2^-14 t_1: if t_2 - t_1 > max(1e-3 t_1, G)
// the tensor-core winner is the exact winner.  Otherwise, if b_3 - t_1 > G,
// where b_3 is a lower bound of every key but the top two, every other
// centroid has exact distance above t_1 (1 + 2^-15) + E >= d(k_1), so the
// point only needs an exact FP64 choice between those two (pair list); every
// other point goes to the FP32 pass (and from there, if still close, to
// FP64), so assignments equal the FP64 argmin.
#include <cuda_bf16.h>

#include "dev_pipe.cuh"
#include "mr_internal.h"

namespace mrgb {
namespace {

constexpr int TM = 128;          // points per tile = MMA M = TMEM lanes
constexpr int KD = 64;           // padded dimension: one 128-byte row of BF16
constexpr int NMAX = 256;        // centroids: MMA N
constexpr int EPI_WARPS = 16;     // four per TMEM lane quadrant, each on a quarter of the columns
constexpr int QUARTERS = EPI_WARPS / 4;
constexpr int EPI_COLS = NMAX / QUARTERS;  // 64 columns per epilogue warp
constexpr int MMA_WARP = EPI_WARPS;
constexpr int CVT_WARP0 = MMA_WARP + 1;
constexpr int CVT_WARPS = 8;      // each converts TM / CVT_WARPS rows of a tile
constexpr int CVT_ROWS = TM / CVT_WARPS;
constexpr int FIN_WARP0 = CVT_WARP0 + CVT_WARPS;
constexpr int FIN_WARPS = 2;      // each finalizes 4 / FIN_WARPS TMEM lane quadrants (32 points each)
constexpr int FIN_QUADS = 4 / FIN_WARPS;
constexpr int TMA_WARP = FIN_WARP0 + FIN_WARPS;  // 27
constexpr int TC_THREADS = (EPI_WARPS + 1 + CVT_WARPS + FIN_WARPS + 1) * 32;  // 896
static_assert(CVT_ROWS % 16 == 0 && 4 % FIN_WARPS == 0, "converter rows and finalizer quadrants");
constexpr int STAGES = 2;         // operand stages
constexpr int XST = 2;            // FP32 staging buffers filled by the bulk copy engine
constexpr int ACCS = 2;           // TMEM accumulators
constexpr uint32_t TMEM_COLS = 512;  // two 256-column FP32 accumulators
constexpr int NSET = 4;           // independent running top-2s per epilogue thread
constexpr int CHUNK = 32;         // TMEM columns per tcgen05.ld in the epilogue

struct __align__(1024) TcSmem {
  uint8_t b_hi[NMAX * 128];
  uint8_t b_lo[NMAX * 128];
  uint8_t a_hi[STAGES][TM * 128];
  uint8_t a_lo[STAGES][TM * 128];
  float xs[XST][TM * KD];             // FP32 point tiles (D == 64 path)
  float nx[STAGES][TM];
  float cn[NMAX];
  // per column quarter and row: top-2 keys and the lower bound of the
  // other keys; and the row's ||x||^2 (epilogue -> finalizers)
  uint32_t xw1[ACCS][QUARTERS][TM], xw2[ACCS][QUARTERS][TM], xlb[ACCS][QUARTERS][TM];
  float xnx[ACCS][TM];
  unsigned long long full_a[STAGES], empty_a[STAGES], nx_free[STAGES];
  unsigned long long full_acc[ACCS], empty_acc[ACCS], drained;
  unsigned long long xfull[ACCS], xfree[ACCS];  // epilogue warps hand their keys to the finalizers
  unsigned long long tfull[XST], tempty[XST];   // FP32 staging ring
  uint32_t tmem_base;
  int err;
};

static_assert(sizeof(TcSmem) + 1024 <= 232448, "shared memory of one CTA");

using namespace pipe;

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 D, M = 128.
__host__ __device__ constexpr uint32_t mma_idesc(uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&v)[32]) { tmem_ld32(taddr, v); }

// Sortable key of a distance: its FP32 bit pattern with the low 8 mantissa
// bits replaced by the centroid column, compared as a signed integer.  For
// non-negative floats the pattern is monotonic, so keys order by distance
// truncated to 16 mantissa bits (an under-statement of less than 2^-15 of
// it), then by column; a negative distance (only rounding of a point lying on
// a centroid produces one) orders below every non-negative one, and a point
// whose smallest key is negative is always re-checked.
__device__ __forceinline__ int dist_key(float dist, uint32_t col) {
  return (int)((__float_as_uint(dist) & 0xFFFFFF00u) | col);
}
__device__ __forceinline__ float key_dist(int key) { return __uint_as_float((uint32_t)key & 0xFFFFFF00u); }

// Key of a column that holds no centroid: above every finite distance's key,
// and it decodes to +inf.
constexpr int KEY_NONE = 0x7F8000FF;

// Insert key into the sorted pair (t1 <= t2): three min/max.
__device__ __forceinline__ void top2_insert(int& t1, int& t2, int key) {
  const int h = max(t1, key);
  t1 = min(t1, key);
  t2 = min(t2, h);
}

// Smallest two of two sorted pairs.
__device__ __forceinline__ void top2_merge(int& a1, int& a2, int b1, int b2) {
  const int c2 = min(max(a1, b1), min(a2, b2));
  a1 = min(a1, b1);
  a2 = c2;
}

// Distances of CHUNK columns (ch .. ch + CHUNK - 1) of one point into its
// NSET running top-2s (column j goes to set j mod NSET).  MASK: some columns
// are >= k (their TMEM words are not written by the MMA and may hold
// anything), so those keys are forced to KEY_NONE.
template <bool MASK>
__device__ __forceinline__ void top2_keys(const uint32_t (&acc)[CHUNK], uint32_t ch, float nxv, const float* cn,
                                          uint32_t k, int (&t1)[NSET], int (&t2)[NSET], float* dbg_row) {
#pragma unroll
  for (int j = 0; j < CHUNK; j += 4) {
    const float4 c4 = *reinterpret_cast<const float4*>(cn + ch + j);
    const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const uint32_t kk = ch + (uint32_t)(j + e);
      const float dist = fmaf(-2.f, __uint_as_float(acc[j + e]), nxv) + cv[e];
      int key = dist_key(dist, kk);
      if (MASK) {
        if (kk >= k) key = KEY_NONE;
        else if (dbg_row) dbg_row[kk] = dist;
      }
      top2_insert(t1[(j + e) % NSET], t2[(j + e) % NSET], key);
    }
  }
}

// BF16 hi/lo split of two values, packed little-endian (element 0 low half).
// (one paired round-to-nearest conversion for each of hi and lo)
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Byte offset of 16-byte chunk c of row r in a 128-byte-swizzled tile whose
// base is 1024-byte aligned (chunk index XOR row mod 8).
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

template <int TERMS>
__global__ void __launch_bounds__(TC_THREADS, 1)
km_tc_assign_kernel(const float* __restrict__ x, uint32_t n, uint32_t d, const float* __restrict__ c, uint32_t k,
                    const float* __restrict__ cnorm, const unsigned int* cmax_bits, int32_t* __restrict__ assign,
                    uint32_t* __restrict__ list, uint32_t* nlist, uint2* __restrict__ pairs, uint32_t* npairs,
                    unsigned long long* timeouts, float* dbg, long long polls, uint32_t stop_copies,
                    unsigned int* maxabs) {
  extern __shared__ uint8_t tc_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t npad = (k + 15) & ~15u;
  const uint32_t ntiles = (n + TM - 1) / TM;
  volatile int* err = &S.err;

  if (threadIdx.x == 0) {
    S.err = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&S.full_a[s], CVT_WARPS);
      mbar_init(&S.empty_a[s], 1);
      mbar_init(&S.nx_free[s], EPI_WARPS);
    }
    for (int b = 0; b < ACCS; ++b) {
      mbar_init(&S.full_acc[b], 1);
      mbar_init(&S.empty_acc[b], EPI_WARPS);
      mbar_init(&S.xfull[b], EPI_WARPS);
      mbar_init(&S.xfree[b], FIN_WARPS);
    }
    for (int q = 0; q < XST; ++q) {
      mbar_init(&S.tfull[q], 1);
      mbar_init(&S.tempty[q], CVT_WARPS);
    }
    mbar_init(&S.drained, 1);
    fence_mbar_init();
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // centroid operands (rows >= k and dims >= d are zero) and norms
  for (uint32_t t = threadIdx.x; t < npad * (KD / 2); t += blockDim.x) {
    const uint32_t row = t / (KD / 2), pr = t % (KD / 2);
    const uint32_t d0 = 2 * pr;
    float a = 0.f, b = 0.f;
    if (row < k) {
      if (d0 < d) a = c[(uint64_t)row * d + d0];
      if (d0 + 1 < d) b = c[(uint64_t)row * d + d0 + 1];
    }
    uint32_t hi, lo;
    split2(a, b, hi, lo);
    const uint32_t off = swz((int)row, (int)(pr >> 2)) + (pr & 3) * 4;
    *reinterpret_cast<uint32_t*>(S.b_hi + off) = hi;
    *reinterpret_cast<uint32_t*>(S.b_lo + off) = lo;
  }
  // padded centroid columns get an infinite norm, so they never win
  for (uint32_t t = threadIdx.x; t < NMAX; t += blockDim.x) S.cn[t] = t < k ? cnorm[t] : INFINITY;
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;
  const float cmax = __uint_as_float(*cmax_bits);

  if (warp >= CVT_WARP0 && warp < CVT_WARP0 + CVT_WARPS) {
    // ---------------------------------------------------------- converters
    // Warp cw owns tile rows CVT_ROWS cw .., in parts of 16.  Step q of part
    // hf gives lane l row CVT_ROWS cw + 16 hf + 2q + l / 16 and dims
    // 4 (l % 16) .. + 3, so one warp load reads two whole FP32 rows (512
    // contiguous bytes) and one warp store writes two whole 128-byte
    // swizzled BF16 rows: no shared-memory bank conflicts.
    const int cw = warp - CVT_WARP0;
    const int col = lane & 15, rsub = lane >> 4;
    const bool vec = d == KD && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
    unsigned int mabs = 0;  // bits of max |x| over the values this thread converts (non-negative floats order as ints)
    for (uint32_t i = 0;; ++i) {
      const uint32_t tile = blockIdx.x + i * gridDim.x;
      if (tile >= ntiles) break;
      const int s = (int)(i % STAGES);
      const uint32_t u = i / STAGES;
      const int q2 = (int)(i % XST);
      if (vec) {
        // the tile was staged by the bulk copy engine
        const bool okt = mbar_wait(&S.tfull[q2], (i / XST) & 1, err, polls);
        if (!__all_sync(0xffffffffu, okt)) break;
      }
      bool ok = true;
      for (int hf = 0; hf < CVT_ROWS / 16; ++hf) {
        const int r0 = CVT_ROWS * cw + 16 * hf;
        float4 v[8];
        if (vec) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int rr = r0 + 2 * q + rsub;
            v[q] = tile * TM + rr < n ? *reinterpret_cast<const float4*>(&S.xs[q2][rr * KD + 4 * col])
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const uint32_t p = tile * TM + r0 + 2 * q + rsub;
            const uint32_t d0 = 4 * col;
            const float* row = x + (uint64_t)p * d;
            v[q].x = (p < n && d0 < d) ? row[d0] : 0.f;
            v[q].y = (p < n && d0 + 1 < d) ? row[d0 + 1] : 0.f;
            v[q].z = (p < n && d0 + 2 < d) ? row[d0 + 2] : 0.f;
            v[q].w = (p < n && d0 + 3 < d) ? row[d0 + 3] : 0.f;
          }
        }
        if (hf == 0 && i >= STAGES) {
          ok = mbar_wait(&S.empty_a[s], (u + 1) & 1, err, polls);
          ok = ok && mbar_wait(&S.nx_free[s], (u + 1) & 1, err, polls);
          ok = __all_sync(0xffffffffu, ok);
          if (!ok) break;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int rr = r0 + 2 * q + rsub;
          if (maxabs)
            mabs = max(mabs, max(max(__float_as_uint(fabsf(v[q].x)), __float_as_uint(fabsf(v[q].y))),
                                 max(__float_as_uint(fabsf(v[q].z)), __float_as_uint(fabsf(v[q].w)))));
          float ss = fmaf(v[q].w, v[q].w, fmaf(v[q].z, v[q].z, fmaf(v[q].y, v[q].y, v[q].x * v[q].x)));
          ss += __shfl_xor_sync(0xffffffffu, ss, 8);
          ss += __shfl_xor_sync(0xffffffffu, ss, 4);
          ss += __shfl_xor_sync(0xffffffffu, ss, 2);
          ss += __shfl_xor_sync(0xffffffffu, ss, 1);
          if (col == 0) S.nx[s][rr] = ss;
          uint32_t hi0, lo0, hi1, lo1;
          split2(v[q].x, v[q].y, hi0, lo0);
          split2(v[q].z, v[q].w, hi1, lo1);
          const uint32_t off = swz(rr, col >> 1) + (uint32_t)(col & 1) * 8u;
          *reinterpret_cast<uint2*>(S.a_hi[s] + off) = make_uint2(hi0, hi1);
          if (TERMS == 3) *reinterpret_cast<uint2*>(S.a_lo[s] + off) = make_uint2(lo0, lo1);
        }
      }
      if (!ok) break;
      // The staging buffer is released only here: the bulk copy engine writes
      // through the async proxy, so the shared loads above must be ordered
      // before its next fill by this proxy fence (the stores that consumed
      // them precede it), not just by the mbarrier arrive.
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&S.full_a[s]);
        if (vec) mbar_arrive(&S.tempty[q2]);
      }
    }
    if (maxabs) {
      for (int o = 16; o; o >>= 1) mabs = max(mabs, __shfl_xor_sync(0xffffffffu, mabs, o));
      if (lane == 0) atomicMax(maxabs, mabs);
    }
  } else if (warp == TMA_WARP) {
    // ------------------------------------------------- bulk-copy producer
    if (lane == 0 && d == KD && ((reinterpret_cast<uintptr_t>(x) & 15) == 0)) {
      uint32_t issued = 0;
      for (uint32_t i = 0;; ++i) {
        const uint32_t tile = blockIdx.x + i * gridDim.x;
        if (tile >= ntiles || (stop_copies && i >= stop_copies)) break;
        const int q2 = (int)(i % XST);
        if (i >= XST && !mbar_wait(&S.tempty[q2], ((i / XST) + 1) & 1, err, polls)) break;
        const uint32_t rows = (n - tile * TM) < (uint32_t)TM ? (n - tile * TM) : (uint32_t)TM;
        const uint32_t bytes = rows * KD * 4;
        mbar_expect_tx(&S.tfull[q2], bytes);
        bulk_g2s(S.xs[q2], x + (uint64_t)tile * TM * KD, bytes, &S.tfull[q2]);
        ++issued;
      }
      // No copy may still be landing in shared memory when the CTA exits.
      // Copy i was issued only after the converters released copy i - XST
      // (which they do after its completion), so only the last XST copies
      // can be in flight; wait for them even when a wait gave up elsewhere.
      for (uint32_t i = issued > (uint32_t)XST ? issued - XST : 0; i < issued; ++i)
        mbar_drain(&S.tfull[i % XST], (i / XST) & 1);
    }
    __syncwarp();
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t idesc = mma_idesc(npad);
      const uint32_t bh = su32(S.b_hi), bl = su32(S.b_lo);
      uint32_t issued = 0;
      for (uint32_t i = 0;; ++i) {
        const uint32_t tile = blockIdx.x + i * gridDim.x;
        if (tile >= ntiles) break;
        const int s = (int)(i % STAGES);
        const uint32_t u = i / STAGES;
        const int b = (int)(i & 1);
        const uint32_t v = i >> 1;
        if (!mbar_wait(&S.full_a[s], u & 1, err, polls)) break;
        if (i >= ACCS && !mbar_wait(&S.empty_acc[b], (v + 1) & 1, err, polls)) break;
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)b * 256u;
        const uint32_t ah = su32(S.a_hi[s]), al = su32(S.a_lo[s]);
#pragma unroll
        for (int kk = 0; kk < KD / 16; ++kk) {
          const uint32_t o = kk * 32;  // 16 BF16 = 32 bytes along K inside the swizzle row
          mma_bf16(dt, sw128_desc(ah + o), sw128_desc(bh + o), idesc, kk > 0 ? 1u : 0u);
          if (TERMS == 3) {
            mma_bf16(dt, sw128_desc(ah + o), sw128_desc(bl + o), idesc, 1u);
            mma_bf16(dt, sw128_desc(al + o), sw128_desc(bh + o), idesc, 1u);
          }
        }
        mma_commit(&S.empty_a[s]);
        mma_commit(&S.full_acc[b]);
        ++issued;
      }
      // No MMA may still be running when TMEM is released (or when the
      // operand buffers go away with the CTA): the commit arrives once every
      // MMA issued above has completed, and that is waited for even when a
      // wait gave up elsewhere.
      mma_commit(&S.drained);
      mbar_drain(&S.drained, 0);
      (void)issued;
    }
    __syncwarp();
  } else if (warp >= FIN_WARP0 && warp < FIN_WARP0 + FIN_WARPS) {
    // ------------------------------------------------------------ finalizers
    // Warp f takes the points of TMEM lane quadrants FIN_QUADS f .. (rows
    // 32 q + lane of each): it merges the four column quarters' top-2 keys
    // into the row's exact top-2 (g1, g2) and a lower bound g3 of every other
    // key, then applies the margin tests.
    const int fw = warp - FIN_WARP0;
    const float eps_sum = TERMS == 3 ? (3.05f * 1.52587890625e-05f + (float)(3 * KD + 8) * 4.76837158203125e-07f)
                                     : (2.f * 3.90625e-03f + 1.52587890625e-05f + (float)(KD + 8) * 4.76837158203125e-07f);
    const float eps32 = 1.01f * (float)(d + 8) * 5.9604644775390625e-08f;
    for (uint32_t i = 0;; ++i) {
      const uint32_t tile = blockIdx.x + i * gridDim.x;
      if (tile >= ntiles) break;
      const int b = (int)(i & 1);
      const uint32_t v = i >> 1;
      const bool okx = mbar_wait(&S.xfull[b], v & 1, err, polls);
      if (!__all_sync(0xffffffffu, okx)) break;
      int o1[FIN_QUADS][QUARTERS], o2[FIN_QUADS][QUARTERS], ol[FIN_QUADS][QUARTERS];
      float nxv[FIN_QUADS];
#pragma unroll
      for (int h = 0; h < FIN_QUADS; ++h) {
        const int r = (fw * FIN_QUADS + h) * 32 + lane;
#pragma unroll
        for (int u = 0; u < QUARTERS; ++u) {
          o1[h][u] = (int)S.xw1[b][u][r];
          o2[h][u] = (int)S.xw2[b][u][r];
          ol[h][u] = (int)S.xlb[b][u][r];
        }
        nxv[h] = S.xnx[b][r];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.xfree[b]);
#pragma unroll
      for (int h = 0; h < FIN_QUADS; ++h) {
        int g1 = o1[h][0], g2 = o2[h][0], g3 = ol[h][0];
#pragma unroll
        for (int u = 1; u < QUARTERS; ++u) top2_merge(g1, g2, o1[h][u], o2[h][u]);
        // every key other than g1, g2 is >= g3: the quarters' bounds, and the
        // quarters' top-2 keys that did not make the row's top-2
#pragma unroll
        for (int u = 0; u < QUARTERS; ++u) {
          g3 = min(g3, ol[h][u]);
          g3 = (o1[h][u] != g1 && o1[h][u] != g2) ? min(g3, o1[h][u]) : g3;
          g3 = (o2[h][u] != g1 && o2[h][u] != g2) ? min(g3, o2[h][u]) : g3;
        }
        const uint32_t p = tile * TM + (uint32_t)((fw * FIN_QUADS + h) * 32 + lane);
        bool flag = false, pair = false;
        if (p < n) {
          const float d1 = key_dist(g1), d2 = key_dist(g2), d3 = key_dist(g3);
          const float xn = sqrtf(nxv[h]);
          const float e = 2.f * eps_sum * xn * cmax + eps32 * (xn + cmax) * (xn + cmax);
          // keys under-state a distance by less than 2^-15 of it (2^-14 allowed)
          const float gap = 2.f * e + 6.103515625e-05f * d1;
          if (g1 < 0) flag = true;  // a negative smallest distance: re-check
          else if (d2 - d1 > fmaxf(1e-3f * d1, gap)) assign[p] = g1 & 0xFF;
          else if (d3 - d1 > gap) pair = true;  // only the top two can be the exact minimum
          else flag = true;
        }
        const unsigned pm = __ballot_sync(0xffffffffu, pair);
        if (pm) {
          uint32_t base = 0;
          if (lane == 0) base = atomicAdd(npairs, (uint32_t)__popc(pm));
          base = __shfl_sync(0xffffffffu, base, 0);
          if (pair)
            pairs[base + __popc(pm & ((1u << lane) - 1))] =
                make_uint2(p, ((uint32_t)g1 & 0xFFu) | (((uint32_t)g2 & 0xFFu) << 16));
        }
        const unsigned fm = __ballot_sync(0xffffffffu, flag);
        if (fm) {
          uint32_t base = 0;
          if (lane == 0) base = atomicAdd(nlist, (uint32_t)__popc(fm));
          base = __shfl_sync(0xffffffffu, base, 0);
          if (flag) list[base + __popc(fm & ((1u << lane) - 1))] = p;
        }
      }
    }
  } else {
    // ------------------------------------------------------------- epilogue
    // Warp e reads TMEM lane quadrant e % 4 (rows 32 (e % 4) ..) and column
    // quarter e / 4 (EPI_COLS columns), CHUNK columns per tcgen05.ld.  Each
    // distance becomes one sortable 32-bit key (see dist_key), so a running
    // top-2 costs three min/max; NSET independent top-2s per thread
    // (columns j mod NSET) keep the dependency chains short.  A warp then
    // reduces its sets to its top-2 (w1, w2) and a lower bound lb of all its
    // other keys (per set: the set's smallest key that is not w1 or w2, or
    // its second key when both are, which bounds the rest of that set) and
    // hands (w1, w2, lb) to the finalizer of its lane quadrant.
    const int q = warp & 3, quarter = warp >> 2;
    const int r = q * 32 + lane;
    const uint32_t c_lo = (uint32_t)quarter * EPI_COLS;
    const uint32_t c_hi = min(npad, c_lo + (uint32_t)EPI_COLS);
    for (uint32_t i = 0;; ++i) {
      const uint32_t tile = blockIdx.x + i * gridDim.x;
      if (tile >= ntiles) break;
      const int s = (int)(i % STAGES);
      const int b = (int)(i & 1);
      const uint32_t v = i >> 1;
      const bool ok = mbar_wait(&S.full_acc[b], v & 1, err, polls);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const float nxv = S.nx[s][r];
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.nx_free[s]);
      int t1[NSET], t2[NSET];
#pragma unroll
      for (int a = 0; a < NSET; ++a) t1[a] = t2[a] = KEY_NONE;
      const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * 256u;
      float* dbg_row = (dbg && tile == 0) ? dbg + (uint64_t)r * NMAX : nullptr;
      for (uint32_t ch = c_lo; ch < c_hi; ch += CHUNK) {
        uint32_t acc[CHUNK];
        tmem_ld(ta + ch, acc);
        if (ch + CHUNK <= k && !dbg_row)
          top2_keys<false>(acc, ch, nxv, S.cn, k, t1, t2, nullptr);
        else
          top2_keys<true>(acc, ch, nxv, S.cn, k, t1, t2, dbg_row);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.empty_acc[b]);
      int w1 = t1[0], w2 = t2[0];
#pragma unroll
      for (int a = 1; a < NSET; ++a) top2_merge(w1, w2, t1[a], t2[a]);
      int lb = KEY_NONE;
#pragma unroll
      for (int a = 0; a < NSET; ++a) lb = min(lb, (t1[a] == w1 || t1[a] == w2) ? t2[a] : t1[a]);
      if (i >= ACCS) {
        const bool okf = mbar_wait(&S.xfree[b], (v + 1) & 1, err, polls);
        if (!__all_sync(0xffffffffu, okf)) break;
      }
      S.xw1[b][quarter][r] = (uint32_t)w1;
      S.xw2[b][quarter][r] = (uint32_t)w2;
      S.xlb[b][quarter][r] = (uint32_t)lb;
      if (quarter == 0) S.xnx[b][r] = nxv;
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.xfull[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
  if (threadIdx.x == 0 && S.err) atomicAdd(timeouts, 1ull);
}

}  // namespace

bool km_tc_supported(uint32_t d, uint32_t k) { return d >= 1 && d <= KD && k >= 1 && k <= NMAX; }

size_t km_tc_smem_bytes() { return sizeof(TcSmem) + 1024; }

// Raw launch: list/nlist receive the points to re-check, pairs/npairs the
// two-candidate points; maxabs (when not null) receives the bits of max |x|.
cudaError_t launch_km_tc_kernel(int terms, const float* x, uint32_t n, uint32_t d, const float* c, uint32_t k,
                                const float* cnorm, const unsigned int* cmax_bits, int32_t* assign, uint32_t* list,
                                uint32_t* nlist, uint2* pairs, uint32_t* npairs, unsigned long long* timeouts,
                                float* dbg, int grid, cudaStream_t s, long long polls, uint32_t stop_copies,
                                unsigned int* maxabs) {
  const int smem = (int)km_tc_smem_bytes();
  cudaError_t e;
  if (terms == 3) {
    if ((e = cudaFuncSetAttribute(km_tc_assign_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess)
      return e;
    km_tc_assign_kernel<3><<<grid, TC_THREADS, smem, s>>>(x, n, d, c, k, cnorm, cmax_bits, assign, list, nlist,
                                                           pairs, npairs, timeouts, dbg, polls, stop_copies, maxabs);
  } else {
    if ((e = cudaFuncSetAttribute(km_tc_assign_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess)
      return e;
    km_tc_assign_kernel<1><<<grid, TC_THREADS, smem, s>>>(x, n, d, c, k, cnorm, cmax_bits, assign, list, nlist,
                                                           pairs, npairs, timeouts, dbg, polls, stop_copies, maxabs);
  }
  return cudaGetLastError();
}

cudaError_t launch_kmeans_tc_assign(const float* x, uint32_t n, uint32_t d, const float* c, uint32_t k,
                                    KmBuffers& b, const DevInfo& di, cudaStream_t s, uint64_t* nk, bool maxabs) {
  const uint32_t ntiles = (n + TM - 1) / TM;
  uint32_t grid = ntiles < (uint32_t)di.sms ? ntiles : (uint32_t)di.sms;
  if (b.grid_cap && grid > b.grid_cap) grid = b.grid_cap;
  uint32_t* list = reinterpret_cast<uint32_t*>(b.cent_bf16_norm);
  const int terms = b.precision == MR_KM_BF16X1_TC ? 1 : 3;
  cudaError_t e = kt_begin(b.kt, s);
  if (e != cudaSuccess) return e;
  e = launch_km_tc_kernel(terms, x, n, d, c, k, b.cnorm, b.nflag + 3, b.assign, list, b.nflag + 1, b.pairs,
                          b.nflag + 4, b.stats + 3, nullptr, (int)grid, s, b.polls < 0 ? SPIN_LIMIT : b.polls,
                          b.stop_copies, maxabs ? b.maxabs : nullptr);
  if (e != cudaSuccess || (e = kt_end(b.kt, s)) != cudaSuccess) return e;
  ++*nk;
  // the caller re-checks the pairs and the listed near ties
  return cudaSuccess;
}

}  // namespace mrgb
