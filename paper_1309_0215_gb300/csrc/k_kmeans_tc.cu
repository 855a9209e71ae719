// k-means assignment on the 5th-generation tensor cores (tcgen05): the
// points x centroids contraction in BF16 with FP32 accumulation in tensor
// memory (TMEM), followed by an exact re-check of near ties.
//
// The distance d(x, c) = ||x||^2 - 2 x.c + ||c||^2 needs the cross term x.c,
// a dense (points x D) . (D x K) contraction — the one step of the hot path
// that is a real GEMM.  Per tile of 128 points:
//   * 8 converter warps load the FP32 rows (coalesced 128-bit loads), compute
//     ||x||^2 in FP32, and write BF16 operands in the 128-byte-swizzled
//     K-major layout the MMA reads.  With TERMS = 3 each value is split as
//     x = hi + lo (hi = bf16(x), lo = bf16(x - hi)) and the MMA accumulates
//     hi.hi + hi.lo + lo.hi, so the cross term is good to about 2^-15
//     relative; TERMS = 1 is the plain single BF16 product.
//   * one thread issues tcgen05.mma (M = 128, N = K rounded up to 16, K = 16
//     per instruction, 4 steps over D = 64) into one of two 256-column TMEM
//     accumulators, and commits completion to mbarriers;
//   * 8 epilogue warps read the 128 x N FP32 tile with tcgen05.ld (one TMEM
//     lane per point; two warps per lane quadrant, each on half of the
//     columns), form d~ = fma(-2, acc, ||x||^2) + ||c||^2 and keep the two
//     smallest with four independent branch-free running minima per thread;
//     the upper half hands its pair to the lower half, which applies the
//     margin test below.
// Converters, MMA issue and epilogue overlap through three operand stages
// and two TMEM accumulators.  Every mbarrier wait is bounded; on timeout the
// CTA stops, drains its MMAs, frees TMEM and reports through stats[3].
//
// Margin test (rigorous, per point).  With u_b = 2^-8 (BF16 rounding) the
// split leaves |x.c - (hi.hi + hi.lo + lo.hi)| <= 3.05 * 2^-16 ||x|| ||c||
// (one value: |x - hi - lo| <= u_b^2 |x|; sums by Cauchy-Schwarz); a single
// BF16 product leaves (2 u_b + u_b^2) ||x|| ||c||.  The tensor-core sum of the
// exact BF16 products is charged (products + 8) * 2^-21 ||x|| ||c|| (four
// times the round-to-nearest bound, allowing truncating adders), and the FP32
// norms and the final fma/add (D + 8) * 2^-24 (||x|| + ||c||)^2 (Higham,
// eq. 3.5).  If d~_2 - d~_1 > max(1e-3 d~_1, 2E) the tensor-core winner is
// the exact winner; every other point goes to the FP32 pass (and from there,
// if still close, to the FP64 pass), so assignments equal the FP64 argmin.
#include <cuda_bf16.h>

#include "mr_internal.h"

namespace mrgb {
namespace {

constexpr int TM = 128;          // points per tile = MMA M = TMEM lanes
constexpr int KD = 64;           // padded dimension: one 128-byte row of BF16
constexpr int NMAX = 256;        // centroids: MMA N
constexpr int EPI_WARPS = 8;      // two per TMEM lane quadrant, each on half the columns
constexpr int MMA_WARP = 8;
constexpr int CVT_WARP0 = 9;
constexpr int CVT_WARPS = 8;
constexpr int TC_THREADS = (EPI_WARPS + 1 + CVT_WARPS) * 32;  // 544
constexpr int STAGES = 3;         // operand stages
constexpr int ACCS = 2;           // TMEM accumulators
constexpr uint32_t TMEM_COLS = 512;  // two 256-column FP32 accumulators
constexpr long long SPIN_LIMIT = 1ll << 24;

struct __align__(1024) TcSmem {
  uint8_t b_hi[NMAX * 128];
  uint8_t b_lo[NMAX * 128];
  uint8_t a_hi[STAGES][TM * 128];
  uint8_t a_lo[STAGES][TM * 128];
  float nx[STAGES][TM];
  float cn[NMAX];
  float xd1[ACCS][TM], xd2[ACCS][TM];  // top-2 of the upper column half, per row
  int xk1[ACCS][TM];
  unsigned long long full_a[STAGES], empty_a[STAGES], nx_free[STAGES];
  unsigned long long full_acc[ACCS], empty_acc[ACCS], drained;
  unsigned long long xfull[ACCS], xfree[ACCS];  // upper-half top-2 handed to the lower half
  uint32_t tmem_base;
  int err;
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the completion of the phase with the given parity.
__device__ bool mbar_wait(unsigned long long* b, uint32_t parity, volatile int* err) {
  for (long long i = 0; i < SPIN_LIMIT; ++i) {
    if (mbar_try(b, parity)) return true;
    if ((i & 255) == 255 && *err) return false;
  }
  *err = 1;
  return false;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
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

// BF16 hi/lo split of two values, packed little-endian (element 0 low half).
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
  const __nv_bfloat16 la = __float2bfloat16_rn(a - __bfloat162float(ha));
  const __nv_bfloat16 lb = __float2bfloat16_rn(b - __bfloat162float(hb));
  hi = (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
  lo = (uint32_t)__bfloat16_as_ushort(la) | ((uint32_t)__bfloat16_as_ushort(lb) << 16);
}

// Byte offset of 16-byte chunk c of row r in a 128-byte-swizzled tile whose
// base is 1024-byte aligned (chunk index XOR row mod 8).
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

template <int TERMS>
__global__ void __launch_bounds__(TC_THREADS, 1)
km_tc_assign_kernel(const float* __restrict__ x, uint32_t n, uint32_t d, const float* __restrict__ c, uint32_t k,
                    const float* __restrict__ cnorm, const unsigned int* cmax_bits, int32_t* __restrict__ assign,
                    uint32_t* __restrict__ list, uint32_t* nlist, unsigned long long* timeouts, float* dbg) {
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
      mbar_init(&S.xfull[b], EPI_WARPS / 2);
      mbar_init(&S.xfree[b], EPI_WARPS / 2);
    }
    mbar_init(&S.drained, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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

  if (warp >= CVT_WARP0) {
    // ---------------------------------------------------------- converters
    const int ct = threadIdx.x - CVT_WARP0 * 32;  // 0..255
    const int r = ct >> 1, h = ct & 1;
    const bool vec = d == KD && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
    for (uint32_t i = 0;; ++i) {
      const uint32_t tile = blockIdx.x + i * gridDim.x;
      if (tile >= ntiles) break;
      const int s = (int)(i % STAGES);
      const uint32_t u = i / STAGES;
      const uint32_t p = tile * TM + r;
      float v[32];
      if (p < n && vec) {
        const float4* src = reinterpret_cast<const float4*>(x + (uint64_t)p * KD + h * 32);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 f = __ldg(src + q);
          v[4 * q] = f.x;
          v[4 * q + 1] = f.y;
          v[4 * q + 2] = f.z;
          v[4 * q + 3] = f.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const uint32_t dj = h * 32 + j;
          v[j] = (p < n && dj < d) ? x[(uint64_t)p * d + dj] : 0.f;
        }
      }
      if (i >= STAGES) {
        bool ok = mbar_wait(&S.empty_a[s], (u + 1) & 1, err);
        ok = ok && mbar_wait(&S.nx_free[s], (u + 1) & 1, err);
        if (!__all_sync(0xffffffffu, ok)) break;
      }
      float ss = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) ss = fmaf(v[j], v[j], ss);
      ss += __shfl_xor_sync(0xffffffffu, ss, 1);
      if (h == 0) S.nx[s][r] = ss;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) split2(v[8 * q + 2 * w], v[8 * q + 2 * w + 1], hi[w], lo[w]);
        const uint32_t off = swz(r, h * 4 + q);
        *reinterpret_cast<uint4*>(S.a_hi[s] + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        if (TERMS == 3) *reinterpret_cast<uint4*>(S.a_lo[s] + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.full_a[s]);
    }
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
        if (!mbar_wait(&S.full_a[s], u & 1, err)) break;
        if (i >= ACCS && !mbar_wait(&S.empty_acc[b], (v + 1) & 1, err)) break;
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
      // no MMA may still be running when TMEM is released
      mma_commit(&S.drained);
      mbar_wait(&S.drained, 0, err);
      (void)issued;
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------- epilogue
    // warp e reads TMEM lane quadrant e % 4 (rows 32*(e%4) ..), columns of
    // half e / 4; four independent running top-2s per thread (columns j mod
    // 4) keep the compare chains short.
    const int q = warp & 3, half = warp >> 2;
    const int r = q * 32 + lane;
    const float eps_sum = TERMS == 3 ? (3.05f * 1.52587890625e-05f + (float)(3 * KD + 8) * 4.76837158203125e-07f)
                                     : (2.f * 3.90625e-03f + 1.52587890625e-05f + (float)(KD + 8) * 4.76837158203125e-07f);
    const float eps32 = 1.01f * (float)(d + 8) * 5.9604644775390625e-08f;
    const uint32_t c_lo = (uint32_t)half * 128u;
    const uint32_t c_hi = min(npad, c_lo + 128u);
    for (uint32_t i = 0;; ++i) {
      const uint32_t tile = blockIdx.x + i * gridDim.x;
      if (tile >= ntiles) break;
      const int s = (int)(i % STAGES);
      const int b = (int)(i & 1);
      const uint32_t v = i >> 1;
      const bool ok = mbar_wait(&S.full_acc[b], v & 1, err);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const float nxv = S.nx[s][r];
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.nx_free[s]);
      float d1[4], d2[4];
      int k1[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) d1[a] = d2[a] = INFINITY, k1[a] = 0x7fffffff;
      const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * 256u;
      const uint32_t p = tile * TM + r;
      for (uint32_t ch = c_lo; ch < c_hi; ch += 32) {
        uint32_t acc[32];
        tmem_ld32(ta + ch, acc);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int a = j & 3;
          const uint32_t kk = ch + j;
          const float dist = fmaf(-2.f, __uint_as_float(acc[j]), nxv) + S.cn[kk];
          if (dbg && tile == 0 && kk < k) dbg[(uint64_t)r * NMAX + kk] = dist;
          const bool lt = dist < d1[a];  // columns increase: the first minimum keeps a tie
          d2[a] = fminf(d2[a], fmaxf(d1[a], dist));
          k1[a] = lt ? (int)kk : k1[a];
          d1[a] = fminf(d1[a], dist);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.empty_acc[b]);
#pragma unroll
      for (int a = 1; a < 4; ++a) {
        if (d1[a] < d1[0] || (d1[a] == d1[0] && k1[a] < k1[0])) {
          d2[0] = fminf(d1[0], d2[a]);
          d1[0] = d1[a];
          k1[0] = k1[a];
        } else {
          d2[0] = fminf(d2[0], d1[a]);
        }
      }
      if (half == 1) {
        // hand this half's top-2 to the warp of the other half on the same rows
        if (i >= ACCS) {
          const bool okf = mbar_wait(&S.xfree[b], (v + 1) & 1, err);
          if (!__all_sync(0xffffffffu, okf)) break;
        }
        S.xd1[b][r] = d1[0];
        S.xd2[b][r] = d2[0];
        S.xk1[b][r] = k1[0];
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.xfull[b]);
        continue;
      }
      {
        const bool okx = mbar_wait(&S.xfull[b], v & 1, err);
        if (!__all_sync(0xffffffffu, okx)) break;
        const float e1 = S.xd1[b][r], e2 = S.xd2[b][r];
        const int f1 = S.xk1[b][r];
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.xfree[b]);
        if (e1 < d1[0] || (e1 == d1[0] && f1 < k1[0])) {
          d2[0] = fminf(d1[0], e2);
          d1[0] = e1;
          k1[0] = f1;
        } else {
          d2[0] = fminf(d2[0], e1);
        }
      }
      bool flag = false;
      if (p < n) {
        const float xn = sqrtf(nxv);
        const float e = 2.f * eps_sum * xn * cmax + eps32 * (xn + cmax) * (xn + cmax);
        const float thr = fmaxf(1e-3f * fabsf(d1[0]), 2.f * e);
        if (d2[0] - d1[0] > thr) assign[p] = k1[0];
        else flag = true;
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

cudaError_t launch_kmeans_fp32_list(const float* x, uint32_t n, uint32_t d, const float* c, uint32_t k, KmBuffers& b,
                                    const uint32_t* list, const uint32_t* nlist, const DevInfo& di, cudaStream_t s,
                                    uint64_t* nk);

size_t km_tc_smem_bytes() { return sizeof(TcSmem) + 1024; }

// Raw launch (also used by the diagnostics probe): list/nlist receive the
// points that need the FP32 pass.
cudaError_t launch_km_tc_kernel(int terms, const float* x, uint32_t n, uint32_t d, const float* c, uint32_t k,
                                const float* cnorm, const unsigned int* cmax_bits, int32_t* assign, uint32_t* list,
                                uint32_t* nlist, unsigned long long* timeouts, float* dbg, int grid, cudaStream_t s) {
  const int smem = (int)km_tc_smem_bytes();
  cudaError_t e;
  if (terms == 3) {
    if ((e = cudaFuncSetAttribute(km_tc_assign_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess)
      return e;
    km_tc_assign_kernel<3><<<grid, TC_THREADS, smem, s>>>(x, n, d, c, k, cnorm, cmax_bits, assign, list, nlist,
                                                           timeouts, dbg);
  } else {
    if ((e = cudaFuncSetAttribute(km_tc_assign_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess)
      return e;
    km_tc_assign_kernel<1><<<grid, TC_THREADS, smem, s>>>(x, n, d, c, k, cnorm, cmax_bits, assign, list, nlist,
                                                           timeouts, dbg);
  }
  return cudaGetLastError();
}

cudaError_t launch_kmeans_tc_assign(const float* x, uint32_t n, uint32_t d, const float* c, uint32_t k,
                                    KmBuffers& b, const DevInfo& di, cudaStream_t s, uint64_t* nk) {
  const uint32_t ntiles = (n + TM - 1) / TM;
  const int grid = (int)(ntiles < (uint32_t)di.sms ? ntiles : (uint32_t)di.sms);
  uint32_t* list = reinterpret_cast<uint32_t*>(b.cent_bf16_norm);
  const int terms = b.precision == MR_KM_BF16X1_TC ? 1 : 3;
  cudaError_t e = launch_km_tc_kernel(terms, x, n, d, c, k, b.cnorm, b.nflag + 3, b.assign, list, b.nflag + 1,
                                      b.stats + 3, nullptr, grid, s);
  if (e != cudaSuccess) return e;
  ++*nk;
  // near ties of the tensor-core pass: FP32 pass over the list (its own near
  // ties go on to the FP64 pass launched by the caller)
  return launch_kmeans_fp32_list(x, n, d, c, k, b, list, b.nflag + 1, di, s, nk);
}

}  // namespace mrgb
