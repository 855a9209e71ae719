// k-means (Lloyd) as a MapReduce job with an array container.
//
// map (per point): key = index of the nearest centroid (squared Euclidean,
// lowest index on an exact tie), value = the point; combiner/reduce: per-key
// sum of points and count (K*D + K array); the new centroid is sum / count.
// The paper's array container with local arrays (Sec. III-A, III-E) is a
// per-CTA shared-memory copy of the K*D sums, merged into the global array.
//
// Exactness contract: assignments equal the FP64 argmin of
//   d(x, c) = sum_j ((double)x_j - (double)c_j)^2   (j in order, no FMA),
// and centroids are the exact-sum means rounded to FP32.
//  * FP32 pass: d~ = ||x||^2 - 2 x.c + ||c||^2 with FP32 FMAs.  Its error is
//    at most E = gamma_{D+3} (||x|| + ||c||)^2 (Higham, Accuracy and Stability
//    of Numerical Algorithms, eq. 3.4 / 3.5 for dot products); we use
//    E = 1.01 (D + 8) 2^-24 (||x|| + max_k ||c_k||)^2.  If the two smallest
//    d~ differ by more than 2E the FP32 winner is the FP64 winner.
//  * Every other point is re-checked exactly in FP64 with the same operation
//    order as the definition above, over the centroids that can still win:
//    FP32 direct-difference distances have relative error at most
//    g = gamma_{D+3} (Higham, eq. 3.5 on a sum of squares), so centroid k can
//    be the minimum only if d~_k <= d~_min (1 + g) / (1 - g).
//  * Sums are accumulated as int64 fixed point q = rint(x * 2^s), with s chosen
//    from max|x| and N so no sum can overflow; integer addition is exact and
//    order-independent, so results do not depend on scheduling.  The update
//    first groups points by cluster (counting sort), so each warp adds runs
//    of points of one cluster in registers and issues a handful of atomics
//    per run instead of one per coordinate.
#include <cmath>

#include "dev_pipe.cuh"
#include "mr_internal.h"

namespace mrgb {
namespace {

constexpr int KM_THREADS = 256;   // 8 warps
constexpr int TP = 64;            // points per tile (8 per warp)
constexpr int KC_MAX = 256;       // centroids per chunk (8 per lane)
constexpr int DC_MAX = 64;        // dims per chunk
constexpr int CS_LD = KC_MAX + 1;  // staged centroid row stride: the transposing stores hit distinct banks
constexpr int XS_LD = TP + 4;      // staged point row stride (16-byte rows; see the point loads)

// Running top three distances (the two smallest with their indices);
// between equal distances the lower index ranks first.
struct Top3 {
  float d1, d2, d3;
  int k1, k2;
};
__device__ __forceinline__ void top3_init(Top3& t) {
  t.d1 = t.d2 = t.d3 = INFINITY;
  t.k1 = t.k2 = 0x7fffffff;
}
__device__ __forceinline__ void top3_push(Top3& t, float d, int k) {
  if (d < t.d1 || (d == t.d1 && k < t.k1)) {
    t.d3 = t.d2;
    t.d2 = t.d1;
    t.k2 = t.k1;
    t.d1 = d;
    t.k1 = k;
  } else if (d < t.d2 || (d == t.d2 && k < t.k2)) {
    t.d3 = t.d2;
    t.d2 = d;
    t.k2 = k;
  } else if (d < t.d3) {
    t.d3 = d;
  }
}
// merge another triple in (its third index is never needed: a third value
// can only rank third)
__device__ __forceinline__ void top3_merge(Top3& t, const Top3& o) {
  top3_push(t, o.d1, o.k1);
  top3_push(t, o.d2, o.k2);
  top3_push(t, o.d3, 0x7fffffff);
}

// Sortable keys (K <= 256): the FP32 bits of a distance (negatives, which
// only rounding produces, clamped to 0) with the low 8 mantissa bits replaced
// by the centroid index.  Non-negative floats order like their bits, so keys
// order by the distance truncated to 16 mantissa bits (an under-statement of
// less than 2^-15 of it), then by index; a running top-2 is three unsigned
// min/max.  KEY_NONE (no centroid) decodes to +inf.
constexpr uint32_t KEY_NONE = 0x7F8000FFu;
__device__ __forceinline__ uint32_t dist_key(float dist, uint32_t kk) {
  return ((uint32_t)max((int)__float_as_uint(dist), 0) & 0xFFFFFF00u) | kk;
}
__device__ __forceinline__ float key_dist(uint32_t key) { return __uint_as_float(key & 0xFFFFFF00u); }
__device__ __forceinline__ void top2_insert(uint32_t& t1, uint32_t& t2, uint32_t key) {
  const uint32_t h = max(t1, key);
  t1 = min(t1, key);
  t2 = min(t2, h);
}
// (a1 <= a2, every other key of set a >= la) merged with the same of set b:
// the union's top-2 and a lower bound of its other keys.
__device__ __forceinline__ void top2lb_merge(uint32_t& a1, uint32_t& a2, uint32_t& la, uint32_t b1, uint32_t b2,
                                             uint32_t lb) {
  const uint32_t g1 = min(a1, b1);
  const uint32_t g2 = min(max(a1, b1), min(a2, b2));
  uint32_t g3 = min(la, lb);
  g3 = (a1 != g1 && a1 != g2) ? min(g3, a1) : g3;
  g3 = (a2 != g1 && a2 != g2) ? min(g3, a2) : g3;
  g3 = (b1 != g1 && b1 != g2) ? min(g3, b1) : g3;
  g3 = (b2 != g1 && b2 != g2) ? min(g3, b2) : g3;
  a1 = g1;
  a2 = g2;
  la = g3;
}

// Centroid norms: cn[k] = ||c_k||^2 (FP32, sequential FMA); cmax[0] = max ||c_k||.
__global__ void km_prep_kernel(const float* __restrict__ c, uint32_t k, uint32_t d, float* __restrict__ cn,
                               unsigned int* cmax_bits, long long* sums, unsigned long long* counts, uint32_t* nflag) {
  pdl_wait();
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < (uint64_t)k; i += nth) {
    float s = 0.f;
    for (uint32_t j = 0; j < d; ++j) s = fmaf(c[i * d + j], c[i * d + j], s);
    cn[i] = s;
    atomicMax(cmax_bits, __float_as_uint(sqrtf(s)));
  }
  for (uint64_t i = tid; i < (uint64_t)k * d; i += nth) sums[i] = 0;
  for (uint64_t i = tid; i < (uint64_t)k; i += nth) counts[i] = 0;
  if (tid < 2) nflag[tid] = 0;
  if (tid == 2) nflag[4] = 0;  // pair list
  if (tid == 3) nflag[5] = 0;  // FP64 stage list
}

// FP32 assignment.  A CTA processes tiles of 64 points; warp w owns points
// 8w..8w+7 of the tile, lane l owns centroids l + 32 j (j < 8) of each chunk
// of up to 256 centroids.  Dot products accumulate over dimension chunks
// staged in shared memory (points transposed [dim][point], centroids
// [dim][centroid]).  When K <= 256 and D <= 64 the centroids are loaded once
// per CTA.  idx != nullptr restricts the pass to the listed points.
// KEYS (K <= 256): selection by packed keys (top-2 plus a lower bound of
// the other keys); else a float top-3 with indices.
template <bool KEYS>
__global__ void __launch_bounds__(KM_THREADS, 2)
km_assign_fp32_kernel(const float* __restrict__ x, uint32_t n, uint32_t d, const float* __restrict__ c, uint32_t k,
                      const float* __restrict__ cn, const unsigned int* cmax_bits, const uint32_t* idx,
                      const uint32_t* nidx, int32_t* __restrict__ assign, uint32_t* flagged, uint32_t* nflag,
                      uint2* __restrict__ pairs, uint32_t* npairs, unsigned long long* stat) {
  extern __shared__ float km_sm[];
  const int dc = d < DC_MAX ? (int)d : DC_MAX;
  const int kc = k < KC_MAX ? (int)k : KC_MAX;
  float* cs = km_sm;              // [dc][CS_LD]
  float* xs = km_sm + DC_MAX * CS_LD;  // [dc][XS_LD]
  __shared__ float nx_s[TP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t npts = idx ? *nidx : n;
  const bool resident = k <= KC_MAX && d <= DC_MAX;
  const bool vec4 = (d & 3) == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  const float cmax = __uint_as_float(*cmax_bits);
  const float eps = 1.01f * (float)(d + 8) * 5.9604645e-8f;  // 2^-24
  if (idx && blockIdx.x == 0 && threadIdx.x == 0 && stat) atomicAdd(stat, (unsigned long long)npts);
  if ((uint64_t)blockIdx.x * TP >= npts) return;  // no tile for this CTA (a short list)

  auto load_c = [&](uint32_t k0, uint32_t d0) {
    for (int t = threadIdx.x; t < kc * dc; t += KM_THREADS) {
      const int kk = t / dc, dd = t % dc;
      const uint32_t kg = k0 + kk, dg = d0 + dd;
      cs[dd * CS_LD + kk] = (kg < k && dg < d) ? c[(uint64_t)kg * d + dg] : 0.f;
    }
  };
  if (resident) {
    load_c(0, 0);
    __syncthreads();
  }
  const uint32_t ntiles = (npts + TP - 1) / TP;
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint32_t p0 = tile * TP;
    Top3 tp[KEYS ? 1 : 8];
    uint32_t t1[KEYS ? 8 : 1], t2[KEYS ? 8 : 1];
    if (KEYS) {
#pragma unroll
      for (int i = 0; i < 8; ++i) t1[i] = t2[i] = KEY_NONE;
    } else {
#pragma unroll
      for (int i = 0; i < (KEYS ? 1 : 8); ++i) top3_init(tp[i]);
    }
    float nxacc = 0.f;  // ||x||^2 of point threadIdx.x (threads < TP), FMA over dims in order
    for (uint32_t k0 = 0; k0 < k; k0 += KC_MAX) {
      float acc[8][8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
      for (uint32_t d0 = 0; d0 < d; d0 += DC_MAX) {
        __syncthreads();
        if (!resident) load_c(k0, d0);
        const int dlim = (int)((d - d0) < (uint32_t)dc ? (d - d0) : (uint32_t)dc);
        // A warp item is 16 points x 8 dims: lane l loads point 16 (wi % 4) +
        // l % 16, dims 8 (wi / 4) + 4 (l / 16) .. + 3 (one 16-byte load when
        // rows allow), and stores them transposed; with the row stride TP + 4
        // the 32 lanes of each store hit 32 banks.
        for (int wi = warp; wi < (TP / 16) * ((dc + 7) / 8); wi += KM_THREADS / 32) {
          const int pp = 16 * (wi % (TP / 16)) + (lane & 15);
          const int dd = 8 * (wi / (TP / 16)) + 4 * (lane >> 4);
          const uint32_t pi = p0 + pp;
          float v[4] = {0.f, 0.f, 0.f, 0.f};
          if (pi < npts) {
            const uint32_t p = idx ? idx[pi] : pi;
            const float* row = x + (uint64_t)p * d + d0 + dd;
            if (vec4 && dd + 4 <= dlim) {
              const float4 q = __ldg(reinterpret_cast<const float4*>(row));
              v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
            } else {
#pragma unroll
              for (int m = 0; m < 4; ++m)
                if (dd + m < dlim) v[m] = __ldg(row + m);
            }
          }
#pragma unroll
          for (int m = 0; m < 4; ++m)
            if (dd + m < dc) xs[(dd + m) * XS_LD + pp] = v[m];
        }
        __syncthreads();
        if (k0 == 0 && threadIdx.x < TP)
          for (int dd = 0; dd < dlim; ++dd)
            nxacc = fmaf(xs[dd * XS_LD + threadIdx.x], xs[dd * XS_LD + threadIdx.x], nxacc);
        for (int dd = 0; dd < dlim; ++dd) {
          const float4 xa = *reinterpret_cast<const float4*>(&xs[dd * XS_LD + warp * 8]);
          const float4 xb = *reinterpret_cast<const float4*>(&xs[dd * XS_LD + warp * 8 + 4]);
          const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
          float cv[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) cv[j] = cs[dd * CS_LD + lane + 32 * j];
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(xv[i], cv[j], acc[i][j]);
        }
      }
      if (k0 == 0) {
        __syncthreads();
        if (threadIdx.x < TP) nx_s[threadIdx.x] = nxacc;
        __syncthreads();
      }
      // distances for this chunk
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t kk = k0 + lane + 32 * j;
        if (KEYS) {
          const bool valid = kk < k && lane + 32 * j < kc;
          const float ncv = valid ? cn[kk] : 0.f;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float dist = fmaf(-2.f, acc[i][j], nx_s[warp * 8 + i]) + ncv;
            top2_insert(t1[i], t2[i], valid ? dist_key(dist, kk) : KEY_NONE);
          }
        } else if (kk < k && lane + 32 * j < kc) {
          const float ncv = cn[kk];
#pragma unroll
          for (int i = 0; i < (KEYS ? 1 : 8); ++i) {
            const float dist = fmaf(-2.f, acc[i][j], nx_s[warp * 8 + i]) + ncv;
            top3_push(tp[i], dist, (int)kk);
          }
        }
      }
    }
    // combine the lanes' candidates for each of the warp's 8 points; lane i
    // then decides point i of the warp
    Top3 mt;
    top3_init(mt);
    if (KEYS) {
      uint32_t m1 = KEY_NONE, m2 = KEY_NONE, m3 = KEY_NONE;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        // a lane's keys other than its top-2 are all >= its second key
        uint32_t a1 = t1[i], a2 = t2[i], la = t2[i];
        for (int o = 16; o; o >>= 1) {
          const uint32_t b1 = __shfl_xor_sync(0xffffffffu, a1, o);
          const uint32_t b2 = __shfl_xor_sync(0xffffffffu, a2, o);
          const uint32_t lb = __shfl_xor_sync(0xffffffffu, la, o);
          top2lb_merge(a1, a2, la, b1, b2, lb);
        }
        if (lane == i) m1 = a1, m2 = a2, m3 = la;
      }
      // keys under-state a distance by less than 2^-15 of it: the margin
      // tests below get 2^-14 d1 more
      mt.d1 = key_dist(m1);
      mt.d2 = key_dist(m2);
      mt.d3 = key_dist(m3);
      mt.k1 = (int)(m1 & 0xFFu);
      mt.k2 = (int)(m2 & 0xFFu);
    } else {
#pragma unroll
      for (int i = 0; i < (KEYS ? 1 : 8); ++i) {
        for (int o = 16; o; o >>= 1) {
          Top3 ot;
          ot.d1 = __shfl_xor_sync(0xffffffffu, tp[i].d1, o);
          ot.d2 = __shfl_xor_sync(0xffffffffu, tp[i].d2, o);
          ot.d3 = __shfl_xor_sync(0xffffffffu, tp[i].d3, o);
          ot.k1 = __shfl_xor_sync(0xffffffffu, tp[i].k1, o);
          ot.k2 = __shfl_xor_sync(0xffffffffu, tp[i].k2, o);
          top3_merge(tp[i], ot);
        }
      }
#pragma unroll
      for (int i = 0; i < (KEYS ? 1 : 8); ++i)
        if (lane == i) mt = tp[i];
    }
    const uint32_t pi = p0 + warp * 8 + lane;
    bool flag = false, pair = false;
    if (lane < 8 && pi < npts) {
      const uint32_t p = idx ? idx[pi] : pi;
      const float nxv = sqrtf(nx_s[warp * 8 + lane]);
      const float e = eps * (nxv + cmax) * (nxv + cmax);
      const float gap = 2.f * e + (KEYS ? 6.103515625e-05f * fmaxf(mt.d1, 0.f) : 0.f);
      // only the top two can be the exact minimum when the third is 2E away
      if (mt.d2 - mt.d1 > gap) assign[p] = mt.k1;
      else if (mt.d3 - mt.d1 > gap) pair = true;
      else flag = true;
    }
    const unsigned pm = __ballot_sync(0xffffffffu, pair);
    if (pm) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(npairs, (uint32_t)__popc(pm));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (pair) {
        const uint32_t p = idx ? idx[pi] : pi;
        pairs[base + __popc(pm & ((1u << lane) - 1))] = make_uint2(p, (uint32_t)mt.k1 | ((uint32_t)mt.k2 << 16));
      }
    }
    const unsigned fm = __ballot_sync(0xffffffffu, flag);
    if (fm) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(nflag, (uint32_t)__popc(fm));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (flag) {
        const uint32_t p = idx ? idx[pi] : pi;
        flagged[base + __popc(fm & ((1u << lane) - 1))] = p;
      }
    }
  }
}

__device__ __forceinline__ float warp_dist32(const float* __restrict__ xp, const float* __restrict__ cp, uint32_t d,
                                             int lane) {
  float s = 0.f;
  for (uint32_t j = lane; j < d; j += 32) {
    const float t = xp[j] - cp[j];
    s = fmaf(t, t, s);
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Exact choice between two centroids for the listed points (pairs whose
// other centroids are already ruled out), four pairs per warp: lanes 8g ..
// 8g + 7 take pair g, each lane dimensions s, s + 8, ... of the point and of
// both centroid rows, so a warp has four points' rows in flight at once.
// FP32 direct differences first: their relative error is at most g for any
// summation order (as in the re-check below), so a ratio beyond widen
// decides the exact order; closer pairs (and NaNs) are appended to the FP64
// stage's list (deferred, ndef), which km_fp64_stage_kernel then settles
// with all such points in parallel (the FP64 pipe of this GPU is narrow:
// done here, a few such points kept a few SMs busy long after the rest had
// finished).  stat[0] counts the pairs.
__global__ void km_pair_kernel(const float* __restrict__ x, uint32_t d, const float* __restrict__ c,
                               const uint2* __restrict__ pairs, const uint32_t* npairs, int32_t* assign,
                               unsigned long long* stat, uint32_t* deferred, uint32_t* ndef) {
  const uint32_t np = *npairs;
  const int lane = threadIdx.x & 31, grp = lane >> 3, sl = lane & 7;
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  if (w0 == 0 && lane == 0 && stat) atomicAdd(stat, (unsigned long long)np);
  const float g = 1.01f * (float)(d + 8) * 5.9604644775390625e-08f;
  const float widen = (1.f + g) / (1.f - g) * (1.f + 4.f * 5.9604644775390625e-08f);
  for (uint64_t f0 = 4 * w0; f0 < np; f0 += 4 * nw) {
    const uint64_t f = f0 + (uint64_t)grp;
    const bool live = f < np;
    const uint2 e = live ? pairs[f] : make_uint2(0u, 0u);
    const uint32_t k1 = e.y & 0xffffu, k2 = e.y >> 16;
    const float* xp = x + (uint64_t)e.x * d;
    const float* c1 = c + (uint64_t)k1 * d;
    const float* c2 = c + (uint64_t)k2 * d;
    float f1 = 0.f, f2 = 0.f;
    if (live)
      for (uint32_t j = (uint32_t)sl; j < d; j += 8) {
        const float xv = xp[j];
        const float t1 = xv - c1[j], t2 = xv - c2[j];
        f1 = fmaf(t1, t1, f1);
        f2 = fmaf(t2, t2, f2);
      }
#pragma unroll
    for (int o = 4; o; o >>= 1) {
      f1 += __shfl_xor_sync(0xffffffffu, f1, o);
      f2 += __shfl_xor_sync(0xffffffffu, f2, o);
    }
    if (live && sl == 0) {
      if (f2 > f1 * widen) assign[e.x] = (int32_t)k1;
      else if (f1 > f2 * widen) assign[e.x] = (int32_t)k2;
      else deferred[atomicAdd(ndef, 1u)] = e.x;
    }
  }
}

// Exact FP64 argmin for the listed points, one warp per point.  Pass 1:
// FP32 distance to every centroid with the lanes spread over the dimensions
// (coalesced centroid rows, warp-sum; the bound below holds for any order),
// keeping the smallest.  Pass 2: in FP64, separately rounded subtract,
// multiply and add with the dimensions in order, only for the centroids whose
// FP32 distance is within the relative error bound of that minimum (one lane
// per such centroid).
__global__ void km_recheck_fp64_kernel(const float* __restrict__ x, uint32_t d, const float* __restrict__ c, uint32_t k,
                                       const uint32_t* flagged, const uint32_t* nflag, int32_t* assign,
                                       unsigned long long* stat) {
  pdl_wait();
  const uint32_t nf = *nflag;
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  // every listed point is checked in FP32 and then in FP64 (stat[0], stat[1])
  if (w0 == 0 && lane == 0 && stat) {
    atomicAdd(stat, (unsigned long long)nf);
    atomicAdd(stat + 1, (unsigned long long)nf);
  }
  const float g = 1.01f * (float)(d + 8) * 5.9604644775390625e-08f;
  const float widen = (1.f + g) / (1.f - g) * (1.f + 4.f * 5.9604644775390625e-08f);
  for (uint64_t f = w0; f < nf; f += nw) {
    const uint32_t p = flagged[f];
    const float* xp = x + (uint64_t)p * d;
    float m32 = INFINITY;
    for (uint32_t kk = 0; kk < k; ++kk) m32 = fminf(m32, warp_dist32(xp, c + (uint64_t)kk * d, d, lane));
    const float lim = m32 * widen;
    double best = INFINITY;
    int bk = 0x7fffffff;
    for (uint32_t k0 = 0; k0 < k; k0 += 32) {
      // candidates of this group of 32 centroids, then one lane per candidate
      uint32_t cand = 0;
      for (uint32_t t = 0; t < 32 && k0 + t < k; ++t) {
        const float s32 = warp_dist32(xp, c + (uint64_t)(k0 + t) * d, d, lane);
        if (s32 <= lim || m32 != m32) cand |= 1u << t;
      }
      if ((cand >> lane) & 1u) {
        const uint32_t kk = k0 + lane;
        const float* cp = c + (uint64_t)kk * d;
        double s64 = 0.0;
        for (uint32_t j = 0; j < d; ++j) {
          const double t = __dsub_rn((double)xp[j], (double)cp[j]);
          s64 = __dadd_rn(s64, __dmul_rn(t, t));
        }
        if (s64 < best) best = s64, bk = (int)kk;  // kk increases per lane: the lowest index keeps a tie
      }
    }
    for (int o = 16; o; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
      if (ob < best || (ob == best && ok < bk)) best = ob, bk = ok;
    }
    if (lane == 0) assign[p] = bk == 0x7fffffff ? 0 : bk;  // all-NaN distances: index 0, as the definition
  }
}

// The same re-check with the centroids staged in shared memory (row stride
// D or D + 1 floats, whichever is odd: lanes reading different rows at one
// column hit different banks).  Lane l owns centroids l, l+32, ... (at most KLANE of them): one
// pass computes their FP32 distances into registers and the warp takes the
// minimum; a point with more than one candidate within the bound goes to
// the FP64 stage's list (deferred, ndef).
constexpr int KLANE = 8;  // K <= 256
// Points are handed out in contiguous ranges of at least RC_MIN per CTA, so
// only as many CTAs stage the centroids as there is work for (the lists are
// a few thousand points).  stat[0] counts the listed points (all checked in
// FP32).
constexpr uint32_t RC_MIN = 64;
__global__ void km_recheck_fp64_smem_kernel(const float* __restrict__ x, uint32_t d, const float* __restrict__ c,
                                            uint32_t k, const uint32_t* flagged, const uint32_t* nflag,
                                            int32_t* assign, unsigned long long* stat, uint32_t* deferred,
                                            uint32_t* ndef) {
  pdl_wait();
  extern __shared__ float cs[];  // [k][d | 1]
  const uint32_t nf = *nflag;
  const uint32_t per = max(RC_MIN, (nf + gridDim.x - 1) / gridDim.x);
  const uint64_t f_lo = (uint64_t)blockIdx.x * per;
  const uint64_t f_hi = f_lo + per < nf ? f_lo + per : nf;
  if (blockIdx.x == 0 && threadIdx.x == 0 && stat) atomicAdd(stat, (unsigned long long)nf);
  if (f_lo >= nf) return;  // no work for this CTA: no staging either
  const uint32_t ld = d | 1;
  for (uint32_t t = threadIdx.x; t < k * d; t += blockDim.x) cs[(t / d) * ld + (t % d)] = c[t];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t wpb = blockDim.x >> 5;
  const float g = 1.01f * (float)(d + 8) * 5.9604644775390625e-08f;
  const float widen = (1.f + g) / (1.f - g) * (1.f + 4.f * 5.9604644775390625e-08f);
  for (uint64_t f = f_lo + (threadIdx.x >> 5); f < f_hi; f += wpb) {
    const uint32_t p = flagged[f];
    const float* xp = x + (uint64_t)p * d;
    float dist[KLANE];
#pragma unroll
    for (int q = 0; q < KLANE; ++q) dist[q] = 0.f;
    for (uint32_t j = 0; j < d; ++j) {
      const float xv = __ldg(xp + j);
#pragma unroll
      for (int q = 0; q < KLANE; ++q) {
        const uint32_t kk = lane + 32 * q;
        if (kk < k) {
          const float t = xv - cs[kk * ld + j];
          dist[q] = fmaf(t, t, dist[q]);
        }
      }
    }
    float m32 = INFINITY;
#pragma unroll
    for (int q = 0; q < KLANE; ++q)
      if (lane + 32 * q < k) m32 = fminf(m32, dist[q]);
    for (int o = 16; o; o >>= 1) m32 = fminf(m32, __shfl_xor_sync(0xffffffffu, m32, o));
    const float lim = m32 * widen;
    // one candidate within the bound: it is the argmin, no FP64 needed
    uint32_t ncand = 0;
    int first = -1;
#pragma unroll
    for (int q = 0; q < KLANE; ++q) {
      const uint32_t kk = lane + 32 * q;
      const bool cq = kk < k && (dist[q] <= lim || m32 != m32);
      if (cq && first < 0) first = (int)kk;
      ncand += (uint32_t)__popc(__ballot_sync(0xffffffffu, cq));
    }
    if (ncand == 1) {
      if (first >= 0) assign[p] = first;
    } else if (lane == 0) {
      deferred[atomicAdd(ndef, 1u)] = p;
    }
  }
}

// The FP64 stage: the exact argmin of each point the pair and re-check passes
// deferred, one CTA per point (all of them at once: there are tens to a few
// hundred per iteration).  FP32 direct differences to every centroid (one
// thread per centroid), the block minimum, the candidates within the
// relative bound of it; then the definition in FP64 for the candidates only:
// the products (x_j - c_j)^2, separately rounded, for all dimensions of a
// chunk of candidates at once, and one thread per candidate adding them with
// the dimensions in order, so the FP64 pipe (narrow on this GPU) runs 2
// instructions per (candidate, dimension) spread over the block and one
// dependent chain of D adds per chunk.  The lowest index wins an exact tie;
// all-NaN distances give index 0, as the definition.  stat[1] counts the points.
constexpr int F64_THREADS = 256;
constexpr uint32_t F64_PROD = 8192;  // doubles of product scratch
inline size_t fp64_stage_smem(uint32_t d, uint32_t k) {
  return (size_t)F64_PROD * 8 + (size_t)d * 4 + (size_t)k * 8 + 64;
}
__global__ void __launch_bounds__(F64_THREADS) km_fp64_stage_kernel(const float* __restrict__ x, uint32_t d,
                                                                    const float* __restrict__ c, uint32_t k,
                                                                    const uint32_t* list, const uint32_t* nlist,
                                                                    int32_t* assign, unsigned long long* stat) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char f64_sm[];
  double* prod = reinterpret_cast<double*>(f64_sm);   // [cc][d]
  float* xs = reinterpret_cast<float*>(prod + F64_PROD);  // [d]
  float* dist = xs + d;                               // [k]
  uint32_t* cand = reinterpret_cast<uint32_t*>(dist + k);  // [k]
  __shared__ float red_f[F64_THREADS / 32];
  __shared__ double red_d[F64_THREADS / 32];
  __shared__ int red_k[F64_THREADS / 32];
  __shared__ uint32_t ncand;
  const uint32_t nf = *nlist;
  if (blockIdx.x == 0 && threadIdx.x == 0 && stat) atomicAdd(stat + 1, (unsigned long long)nf);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float g = 1.01f * (float)(d + 8) * 5.9604644775390625e-08f;
  const float widen = (1.f + g) / (1.f - g) * (1.f + 4.f * 5.9604644775390625e-08f);
  // candidates per product chunk (d <= 1024: at least 8), one summing thread each
  const uint32_t cc = F64_PROD / d < (uint32_t)F64_THREADS ? F64_PROD / d : (uint32_t)F64_THREADS;
  for (uint32_t f = blockIdx.x; f < nf; f += gridDim.x) {
    const uint32_t p = list[f];
    const float* xp = x + (uint64_t)p * d;
    __syncthreads();  // the previous point's use of the shared arrays is over
    for (uint32_t j = threadIdx.x; j < d; j += F64_THREADS) xs[j] = xp[j];
    if (threadIdx.x == 0) ncand = 0;
    __syncthreads();
    float m = INFINITY;
    for (uint32_t kk = threadIdx.x; kk < k; kk += F64_THREADS) {
      const float* cp = c + (uint64_t)kk * d;
      float s32 = 0.f;
      for (uint32_t j = 0; j < d; ++j) {
        const float t = xs[j] - __ldg(cp + j);
        s32 = fmaf(t, t, s32);
      }
      dist[kk] = s32;
      m = fminf(m, s32);
    }
    for (int o = 16; o; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red_f[warp] = m;
    __syncthreads();
    float m32 = red_f[0];
    for (int w = 1; w < F64_THREADS / 32; ++w) m32 = fminf(m32, red_f[w]);
    const float lim = m32 * widen;
    for (uint32_t kk = threadIdx.x; kk < k; kk += F64_THREADS)
      if (dist[kk] <= lim || m32 != m32) cand[atomicAdd(&ncand, 1u)] = kk;
    __syncthreads();
    const uint32_t nc = ncand;
    double best = INFINITY;
    int bk = 0x7fffffff;
    for (uint32_t c0 = 0; c0 < nc; c0 += cc) {
      const uint32_t cn = nc - c0 < cc ? nc - c0 : cc;
      for (uint32_t ci = warp; ci < cn; ci += F64_THREADS / 32) {
        const float* cp = c + (uint64_t)cand[c0 + ci] * d;
        for (uint32_t j = lane; j < d; j += 32) {
          const double t = __dsub_rn((double)xs[j], (double)__ldg(cp + j));
          prod[ci * d + j] = __dmul_rn(t, t);
        }
      }
      __syncthreads();
      if (threadIdx.x < cn) {
        double s64 = 0.0;
        for (uint32_t j = 0; j < d; ++j) s64 = __dadd_rn(s64, prod[threadIdx.x * d + j]);
        const int kk = (int)cand[c0 + threadIdx.x];
        if (s64 < best || (s64 == best && kk < bk)) best = s64, bk = kk;
      }
      __syncthreads();
    }
    for (int o = 16; o; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
      if (ob < best || (ob == best && ok < bk)) best = ob, bk = ok;
    }
    if (lane == 0) red_d[warp] = best, red_k[warp] = bk;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < F64_THREADS / 32; ++w)
        if (red_d[w] < best || (red_d[w] == best && red_k[w] < bk)) best = red_d[w], bk = red_k[w];
      assign[p] = bk == 0x7fffffff ? 0 : bk;
    }
  }
}

// max |x| over all coordinates (as float bits; non-negative floats order like ints)
__global__ void km_maxabs_kernel(const float* __restrict__ x, uint64_t cnt, unsigned int* out) {
  unsigned int m = 0;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  uint64_t done = 0;
  if (((uintptr_t)x & 15) == 0) {
    const uint64_t n4 = cnt / 4;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (uint64_t i = tid; i < n4; i += nth) {
      const float4 v = __ldg(x4 + i);
      m = max(m, max(max(__float_as_uint(fabsf(v.x)), __float_as_uint(fabsf(v.y))),
                     max(__float_as_uint(fabsf(v.z)), __float_as_uint(fabsf(v.w)))));
    }
    done = n4 * 4;
  }
  for (uint64_t i = done + tid; i < cnt; i += nth) m = max(m, __float_as_uint(fabsf(x[i])));
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Fixed-point exponent s (at most 60): the largest with max|x| 2^s < 2^39 and
// max|x| 2^s n < 2^62, so every q = rint(x 2^s) fits 40 bits (the update's
// hi/lo split) and no sum of n of them can overflow int64.  s may be
// negative for very large inputs; x 2^s then rounds only where it is far
// below 1/2, and rounds to 0 either way.
__global__ void km_scale_kernel(const unsigned int* maxabs, uint32_t n, int* shift) {
  const float m = __uint_as_float(*maxabs);
  int s = 60;
  if (m > 0.f) {
    const double lim = fmin(ldexp(1.0, 39), ldexp(1.0, 62) / (double)n);
    while (s > -200 && (double)m * ldexp(1.0, s) >= lim) --s;
  }
  *shift = s;
}

__device__ __forceinline__ uint32_t cluster_of(const int32_t* assign, uint64_t i, uint32_t k) {
  const int a = assign[i];
  return (a < 0 || (uint32_t)a >= k) ? 0u : (uint32_t)a;
}

// Cluster sizes (a CTA counts in shared memory, then adds to the global counts).
__global__ void km_count_kernel(const int32_t* __restrict__ assign, uint32_t n, uint32_t k,
                                unsigned long long* counts) {
  extern __shared__ uint32_t hc[];
  for (uint32_t t = threadIdx.x; t < k; t += blockDim.x) hc[t] = 0;
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&hc[cluster_of(assign, i, k)], 1u);
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < k; t += blockDim.x)
    if (hc[t]) atomicAdd(counts + t, (unsigned long long)hc[t]);
}

// Exclusive scan of the counts into each cluster's write cursor (one CTA).
__global__ void km_offsets_kernel(const unsigned long long* counts, uint32_t k, uint32_t* cursor) {
  __shared__ uint32_t carry;
  __shared__ uint32_t wsum[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t b = 0; b < k; b += blockDim.x) {
    const uint32_t i = b + threadIdx.x;
    const uint32_t v = i < k ? (uint32_t)counts[i] : 0;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
      uint32_t wi = w;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      wsum[lane] = wi - w;
    }
    __syncthreads();
    const uint32_t ex = carry + wsum[warp] + incl - v;
    if (i < k) cursor[i] = ex;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = ex + v;
    __syncthreads();
  }
}

// Counting-sort scatter: perm lists the points grouped by cluster (order
// inside a cluster does not matter: the sums are exact integers).  A CTA takes
// a chunk of points, counts them per cluster in shared memory, reserves each
// cluster's range with one global atomic, then places its points with
// shared-memory cursors.
constexpr int SCAT_THREADS = 256;
constexpr int SCAT_PER_THREAD = 16;
__global__ void __launch_bounds__(SCAT_THREADS) km_scatter_kernel(const int32_t* __restrict__ assign, uint32_t n,
                                                                  uint32_t k, uint32_t* cursor,
                                                                  uint32_t* __restrict__ perm) {
  extern __shared__ uint32_t sc[];  // [k] local counts, then local cursors
  const uint64_t chunk = (uint64_t)SCAT_THREADS * SCAT_PER_THREAD;
  const uint64_t b0 = (uint64_t)blockIdx.x * chunk;
  for (uint32_t t = threadIdx.x; t < k; t += SCAT_THREADS) sc[t] = 0;
  __syncthreads();
  uint32_t a[SCAT_PER_THREAD];
#pragma unroll
  for (int r = 0; r < SCAT_PER_THREAD; ++r) {
    const uint64_t i = b0 + (uint64_t)r * SCAT_THREADS + threadIdx.x;
    a[r] = i < n ? cluster_of(assign, i, k) : 0xffffffffu;
    if (a[r] != 0xffffffffu) atomicAdd(&sc[a[r]], 1u);
  }
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < k; t += SCAT_THREADS)
    if (sc[t]) sc[t] = atomicAdd(cursor + t, sc[t]);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < SCAT_PER_THREAD; ++r) {
    const uint64_t i = b0 + (uint64_t)r * SCAT_THREADS + threadIdx.x;
    if (a[r] != 0xffffffffu) perm[atomicAdd(&sc[a[r]], 1u)] = (uint32_t)i;
  }
}

// Per-cluster int64 fixed-point sums.  Warp w adds points perm[64w ..
// 64w+63]; they come in runs of one cluster (ends[c] = one past the last
// position of cluster c in perm, so a run's cluster needs no lookup of the
// point's assignment), summed in registers (lane l holds dimensions l and
// l+32 of the current 64-dimension slice) and added to the global sums once
// per run.  Eight rows are in flight per warp.
constexpr int SUM_RUN = 64;
constexpr int SUM_UNROLL = 8;
// Round-half-even of a finite FP32 value to int64 with FP32 adds and integer
// operations only: the FP32 -> int64 conversion instruction issues on the FP64
// pipe, which is narrow on this GPU and became the sum kernel's limit.
//   |v| < 2^22:  v + 1.5*2^23 rounds (ties to even) to an integer whose value
//                minus 1.5*2^23 sits in the low bits of the sum's encoding;
//   |v| >= 2^23: v is an integer, its significand shifted by e - 150;
//   in between:  one fraction bit, rounded to even by hand.
__device__ __forceinline__ long long rint_i64(float v) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t e = (b >> 23) & 0xFFu;
  if (e < 149u) return (long long)(int32_t)(__float_as_uint(__fadd_rn(v, 12582912.f)) - 0x4B400000u);
  const uint64_t m = (b & 0x7FFFFFu) | 0x800000u;
  const uint64_t q = e == 149u ? (m >> 1) + (m & (m >> 1) & 1u) : m << ((e - 150u) & 63u);
  return (b >> 31) ? -(long long)q : (long long)q;
}
__device__ __forceinline__ void sum_flush(long long* sums, uint32_t cur, uint32_t d, uint32_t dj0, uint32_t dj1,
                                          long long a0, long long a1) {
  if (dj0 < d && a0) atomicAdd(reinterpret_cast<unsigned long long*>(sums + (uint64_t)cur * d + dj0), (unsigned long long)a0);
  if (dj1 < d && a1) atomicAdd(reinterpret_cast<unsigned long long*>(sums + (uint64_t)cur * d + dj1), (unsigned long long)a1);
}
__global__ void __launch_bounds__(256) km_sum_kernel(const float* __restrict__ x, uint32_t n, uint32_t d, uint32_t k,
                                                     const uint32_t* __restrict__ ends,
                                                     const uint32_t* __restrict__ perm, const int* shift,
                                                     long long* sums) {
  const int lane = threadIdx.x & 31;
  const uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t p0 = w * SUM_RUN;
  if (p0 >= n) return;
  const uint64_t p1 = (p0 + SUM_RUN) < n ? p0 + SUM_RUN : n;
  // x * 2^s is exact in FP32 (a power-of-two scale far from overflow), so
  // rounding it to int64 gives the same q as in double precision
  const float scale = ldexpf(1.f, *shift);
  uint32_t idx[2];
  idx[0] = perm[p0 + lane < p1 ? p0 + lane : p0];
  idx[1] = perm[p0 + 32 + lane < p1 ? p0 + 32 + lane : p0];
  // cluster of position p0: the first c with ends[c] > p0
  uint32_t c0 = 0, hi = k - 1;
  while (c0 < hi) {
    const uint32_t mid = (c0 + hi) >> 1;
    if (ends[mid] > p0) hi = mid;
    else c0 = mid + 1;
  }
  for (uint32_t j0 = 0; j0 < d; j0 += 64) {
    const uint32_t dj0 = j0 + lane, dj1 = j0 + 32 + lane;
    long long a0 = 0, a1 = 0;
    uint32_t cur = c0, cend = ends[c0];
    for (uint64_t p = p0; p < p1; p += SUM_UNROLL) {
      float v[SUM_UNROLL][2];
#pragma unroll
      for (int u = 0; u < SUM_UNROLL; ++u) {
        const uint64_t pp = p + u;
        const uint32_t sel = (uint32_t)(pp - p0);
        const uint32_t i = __shfl_sync(0xffffffffu, sel < 32 ? idx[0] : idx[1], (int)(sel & 31));
        const bool ok = pp < p1;
        v[u][0] = (ok && dj0 < d) ? x[(uint64_t)i * d + dj0] : 0.f;
        v[u][1] = (ok && dj1 < d) ? x[(uint64_t)i * d + dj1] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < SUM_UNROLL; ++u) {
        const uint64_t pp = p + u;
        if (pp >= p1) break;
        while (pp >= cend) {  // warp-uniform: the run of cluster cur ended (empty clusters skipped)
          sum_flush(sums, cur, d, dj0, dj1, a0, a1);
          a0 = a1 = 0;
          ++cur;
          cend = ends[cur];
        }
        a0 += rint_i64(v[u][0] * scale);
        a1 += rint_i64(v[u][1] * scale);
      }
    }
    sum_flush(sums, cur, d, dj0, dj1, a0, a1);
  }
}

// Update step with local arrays (Sec. III-E: the array container, privatised
// per thread block).  A CTA's [k][d] fixed-point sums and [k] counts live in
// shared memory; one CTA per SM streams a contiguous range of points in input
// order (coalesced rows: no sort and no gather) and adds each coordinate with
// shared-memory atomics.  A 64-bit sum is kept as two 32-bit words, each
// added by a native 32-bit atomic: the low word's add returns the old value,
// and a carry out of it (new < old) goes into the high word's add, so
// hi * 2^32 + lo is the exact sum modulo 2^64 (which holds it: the scale
// keeps |sum| below 2^62).  The CTA then stores its sums as one partial
// (plain stores) and adds its counts to the global counts;
// km_reduce_finalize_kernel adds the partials.  Integer sums make the result
// independent of the order.
__device__ __forceinline__ void add64_split(uint32_t* lo, uint32_t* hi, long long q) {
  const uint32_t ql = (uint32_t)q;
  const uint32_t old = atomicAdd(lo, ql);
  atomicAdd(hi, (uint32_t)((unsigned long long)q >> 32) + (old + ql < old ? 1u : 0u));
}
constexpr int LS_THREADS = 1024;
constexpr int LS_ROWS = 4;  // rows in flight per warp
constexpr uint32_t LS_MAX_CTAS = 160;  // partials held in scratch
constexpr uint64_t LS_SMEM_MAX = 200 * 1024;
inline bool local_sums_fit(uint64_t d, uint64_t k) { return k * d * 8 + k * 4 <= LS_SMEM_MAX; }
__global__ void __launch_bounds__(LS_THREADS, 1) km_local_sum_kernel(const float* __restrict__ x, uint32_t n,
                                                                     uint32_t d, uint32_t k,
                                                                     const int32_t* __restrict__ assign,
                                                                     const int* shift, long long* __restrict__ part,
                                                                     unsigned long long* counts) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char ls_sm[];
  const uint64_t kd = (uint64_t)k * d;
  uint32_t* SL = reinterpret_cast<uint32_t*>(ls_sm);  // low words [k][d]
  uint32_t* SH = SL + kd;                             // high words [k][d]
  unsigned int* C = SH + kd;
  for (uint64_t i = threadIdx.x; i < 2 * kd; i += LS_THREADS) SL[i] = 0;
  for (uint32_t i = threadIdx.x; i < k; i += LS_THREADS) C[i] = 0;
  __syncthreads();
  const float scale = ldexpf(1.f, *shift);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t per = (((uint64_t)n + gridDim.x - 1) / gridDim.x + 31) & ~31ull;
  const uint64_t p0 = (uint64_t)blockIdx.x * per;
  const uint64_t p1 = p0 + per < (uint64_t)n ? p0 + per : (uint64_t)n;
  for (uint64_t r0 = p0 + 32 * (uint64_t)warp; r0 < p1; r0 += 32 * (LS_THREADS / 32)) {
    // 32 consecutive rows per warp step; lane j holds row r0 + j's cluster
    const uint32_t nr = (uint32_t)(p1 - r0 < 32 ? p1 - r0 : 32);
    const uint32_t cl = (uint32_t)lane < nr ? cluster_of(assign, r0 + lane, k) : 0u;
    if ((uint32_t)lane < nr) atomicAdd(&C[cl], 1u);
    for (uint32_t j0 = 0; j0 < d; j0 += 64) {
      const uint32_t dj0 = j0 + lane, dj1 = j0 + 32 + lane;
      for (uint32_t rr = 0; rr < nr; rr += LS_ROWS) {
        float v[LS_ROWS][2];
        uint32_t c[LS_ROWS];
#pragma unroll
        for (int u = 0; u < LS_ROWS; ++u) {
          const uint32_t j = rr + u;
          c[u] = __shfl_sync(0xffffffffu, cl, (int)(j & 31));
          const bool ok = j < nr;
          const float* row = x + (r0 + j) * d;
          v[u][0] = (ok && dj0 < d) ? row[dj0] : 0.f;
          v[u][1] = (ok && dj1 < d) ? row[dj1] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < LS_ROWS; ++u) {
          if (rr + u >= nr) break;  // warp-uniform
          const uint32_t b = c[u] * d;
          if (dj0 < d) add64_split(SL + b + dj0, SH + b + dj0, rint_i64(v[u][0] * scale));
          if (dj1 < d) add64_split(SL + b + dj1, SH + b + dj1, rint_i64(v[u][1] * scale));
        }
      }
    }
  }
  __syncthreads();
  long long* P = part + (uint64_t)blockIdx.x * kd;
  for (uint64_t i = threadIdx.x; i < kd; i += LS_THREADS)
    P[i] = (long long)(((unsigned long long)SH[i] << 32) | SL[i]);
  for (uint32_t i = threadIdx.x; i < k; i += LS_THREADS)
    if (C[i]) atomicAdd(counts + i, (unsigned long long)C[i]);
}

// Pipelined form of the local-array update, for rows of a multiple of 4
// floats starting 16-byte aligned.  Warp 0 is the producer: its lane 0
// streams chunks of `rows` consecutive points and their cluster ids into an
// LP_ST-deep shared-memory ring with bulk copies (completion counted on one
// mbarrier per stage) and refills a stage as soon as every worker warp has
// released it; warps 1..31 are workers, warp w taking rows w - 1, w - 1 +
// 31, ... of each chunk.  (With a worker refilling the ring only after its
// own rows, the ring ran dry and the kernel waited on DRAM latency.)
//
// Exact sums without 64-bit shared atomics.  The scale keeps |x 2^s| < 2^39
// (km_scale_kernel), so q = rint(x 2^s) = hi 2^20 + lo with hi, lo integers
// of magnitude <= 2^19, both formed by FP32 adds that are exact (lq_split);
// each goes into a 32-bit shared-memory array with a non-returning add.
// Within a window of at most LP_FLUSH_ROWS points no 32-bit sum can overflow,
// so after each window the workers add hi 2^20 + lo of every (cluster, dim)
// into the CTA's own int64 partial in global memory (plain read-modify-
// write: no other CTA touches it) and clear the arrays.  Integer sums stay
// exact and order-independent, equal to the sum of rint(x 2^s) formed any
// other way.
//
// Every wait is bounded.  Workers run the same chunks and barriers whatever
// happens; after a wait gives up, chunks are skipped and the producer issues
// no more copies (it issues into a stage only after every worker released
// the stage's previous chunk with no error raised, i.e. after that chunk
// landed), lets the last copies it issued land, and the CTA counts itself in
// *timeouts.
constexpr int LP_ST = 4;
constexpr int LP_WORKERS = LS_THREADS / 32 - 1;  // warp 0 produces
constexpr uint32_t LP_CHUNK_MAX = 24 * 1024;     // bytes of points per stage, at most
constexpr uint32_t LP_FLUSH_ROWS = 4095;         // 4095 * 2^19 < 2^31
__host__ __device__ constexpr uint64_t lp_fixed_bytes(uint64_t kd, uint64_t k) {
  return (((2 * kd + k) * 4 + 127) & ~127ull) + 2 * LP_ST * 8 + 16;
}
// q = rint(v) for |v| < 2^39 as hi 2^20 + lo (|hi|, |lo| <= 2^19).  hf = v
// rounded to a multiple of 2^20 (adding 1.5 2^43, whose unit in the last
// place is 2^20, and subtracting it back are exact apart from that rounding);
// lf = v - hf is exact (|lf| <= 2^19 on v's own grid); hi = hf / 2^20 and
// lo = rint(lf) are read from the low bits of a sum with 1.5 2^23, whose
// unit in the last place is 1 (ties to even).  hf is an even integer, so
// rint(v) = hf + rint(lf).
__device__ __forceinline__ void lq_split(float v, int& hi, int& lo) {
  const float hf = __fsub_rn(__fadd_rn(v, 0x1.8p43f), 0x1.8p43f);
  const float lf = __fsub_rn(v, hf);
  hi = (int)(__float_as_uint(__fmaf_rn(hf, 0x1p-20f, 0x1.8p23f)) - 0x4B400000u);
  lo = (int)(__float_as_uint(__fadd_rn(lf, 0x1.8p23f)) - 0x4B400000u);
}
__device__ __forceinline__ void red_s32(int* p, int v) { atomicAdd(p, v); }
// barrier 1 among the worker warps only (barrier 0 is __syncthreads)
__device__ __forceinline__ void workers_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(LP_WORKERS * 32) : "memory");
}

template <bool D64>
__global__ void __launch_bounds__(LS_THREADS, 1) km_local_sum_pipe_kernel(
    const float* __restrict__ x, uint32_t n, uint32_t d, uint32_t k, const int32_t* __restrict__ assign,
    const int* shift, long long* __restrict__ part, unsigned long long* counts, uint32_t rows,
    unsigned long long* timeouts, long long polls) {
  pdl_wait();
  using namespace pipe;
  extern __shared__ __align__(128) unsigned char lp_sm[];
  const uint64_t kd = (uint64_t)k * d;
  int* HI = reinterpret_cast<int*>(lp_sm);
  int* LO = HI + kd;
  unsigned int* C = reinterpret_cast<unsigned int*>(LO + kd);
  float* xs = reinterpret_cast<float*>(lp_sm + (((2 * kd + k) * 4 + 127) & ~127ull));
  const uint64_t xst = (uint64_t)rows * d;  // floats per stage
  int32_t* as = reinterpret_cast<int32_t*>(xs + LP_ST * xst);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(as + LP_ST * rows);
  unsigned long long* empty = full + LP_ST;
  volatile int* err = reinterpret_cast<volatile int*>(empty + LP_ST);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // a CTA's range is a whole number of chunks, so every chunk starts 16-byte aligned
  const uint64_t per = ((((uint64_t)n + gridDim.x - 1) / gridDim.x + rows - 1) / rows) * rows;
  const uint64_t p0 = (uint64_t)blockIdx.x * per;
  const uint64_t p1 = p0 + per < (uint64_t)n ? p0 + per : (uint64_t)n;
  const uint32_t nchunks = p0 < p1 ? (uint32_t)((p1 - p0 + rows - 1) / rows) : 0u;
  const uint32_t fc = rows < LP_FLUSH_ROWS ? LP_FLUSH_ROWS / rows : 1u;  // chunks per window
  for (uint64_t i = threadIdx.x; i < 2 * kd; i += LS_THREADS) HI[i] = 0;
  for (uint32_t i = threadIdx.x; i < k; i += LS_THREADS) C[i] = 0;
  if (threadIdx.x == 0) {
    *err = 0;
    for (int q = 0; q < LP_ST; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], LP_WORKERS);
    }
    fence_mbar_init();
  }
  __syncthreads();
  long long* P = part + (uint64_t)blockIdx.x * kd;
  bool written = false;  // this thread's elements of the CTA's partial hold a window already
  auto flush = [&](uint32_t t0, uint32_t nt) {
    for (uint64_t i = t0; i < kd; i += nt) {
      const long long v = (long long)HI[i] * (1ll << 20) + (long long)LO[i];
      P[i] = written ? P[i] + v : v;
      HI[i] = 0;
      LO[i] = 0;
    }
    written = true;
  };
  uint32_t issued = 0;  // thread 0: chunks whose copies were started
  if (warp == 0) {
    // ----------------------------------------------------------- producer
    if (lane == 0) {
      for (uint32_t c = 0; c < nchunks; ++c) {
        const uint32_t q = c % LP_ST;
        // the stage's previous chunk must be released by every worker, with
        // no error raised (so it landed) before the stage is refilled
        if (c >= (uint32_t)LP_ST && (!mbar_wait(&empty[q], ((c / LP_ST) + 1) & 1u, err, polls) || *err)) break;
        const uint64_t r0 = p0 + (uint64_t)c * rows;
        const uint32_t nr = (uint32_t)(p1 - r0 < rows ? p1 - r0 : rows);
        const uint32_t xb = nr * d * 4, ab = ((nr + 3) & ~3u) * 4;  // ids rounded up to 16 bytes (buffer padding)
        mbar_expect_tx(&full[q], xb + ab);
        bulk_g2s(xs + q * xst, x + r0 * d, xb, &full[q]);
        bulk_g2s(as + q * rows, assign + r0, ab, &full[q]);
        issued = c + 1;
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------- workers
    const float scale = ldexpf(1.f, *shift);
    const uint32_t wk = (uint32_t)warp - 1;
    for (uint32_t c = 0; c < nchunks; ++c) {
      const uint32_t q = c % LP_ST, par = (c / LP_ST) & 1u;
      const bool ok = !*err && mbar_wait(&full[q], par, err, polls);
      if (ok) {
        const uint64_t r0 = p0 + (uint64_t)c * rows;
        const uint32_t nr = (uint32_t)(p1 - r0 < rows ? p1 - r0 : rows);
        const float* X = xs + q * xst;
        const int32_t* A = as + q * rows;
        if (D64) {
          // lane holds dimensions lane and lane + 32 of row j
          for (uint32_t j = wk; j < nr; j += LP_WORKERS) {
            const int a = A[j];
            const uint32_t cl = (a < 0 || (uint32_t)a >= k) ? 0u : (uint32_t)a;
            if (lane == 0) atomicAdd(&C[cl], 1u);
            const float* row = X + j * 64u;
            const uint32_t b = cl * 64u + lane;
            int h0, l0, h1, l1;
            lq_split(row[lane] * scale, h0, l0);
            lq_split(row[lane + 32] * scale, h1, l1);
            red_s32(HI + b, h0);
            red_s32(LO + b, l0);
            red_s32(HI + b + 32, h1);
            red_s32(LO + b + 32, l1);
          }
        } else {
          for (uint32_t j = wk; j < nr; j += LP_WORKERS) {
            const int a = A[j];
            const uint32_t cl = (a < 0 || (uint32_t)a >= k) ? 0u : (uint32_t)a;
            if (lane == 0) atomicAdd(&C[cl], 1u);
            const float* row = X + (uint64_t)j * d;
            const uint32_t b = cl * d;
            for (uint32_t dj = lane; dj < d; dj += 32) {
              int h0, l0;
              lq_split(row[dj] * scale, h0, l0);
              red_s32(HI + b + dj, h0);
              red_s32(LO + b + dj, l0);
            }
          }
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[q]);
      if ((c + 1) % fc == 0 && c + 1 < nchunks) {
        workers_sync();
        flush(threadIdx.x - 32, LP_WORKERS * 32);
        workers_sync();
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *err) {
    // a wait gave up somewhere: only the last LP_ST copies the producer
    // issued can still be in flight; let them land before the CTA leaves
    for (uint32_t w = issued > (uint32_t)LP_ST ? issued - LP_ST : 0u; w < issued; ++w)
      mbar_drain(&full[w % LP_ST], (w / LP_ST) & 1u);
    atomicAdd(timeouts, 1ull);
  }
  // the last window, by the workers with the same element-to-thread mapping
  // as the windows before (each thread's `written` covers its own elements)
  if (warp != 0) flush(threadIdx.x - 32, LP_WORKERS * 32);
  for (uint32_t i = threadIdx.x; i < k; i += LS_THREADS)
    if (C[i]) atomicAdd(counts + i, (unsigned long long)C[i]);
}

// Update step for D <= 64 with runs sorted per window (Sec. III-E's array
// container, privatised per thread block as above, with the shared-memory
// atomics taken out of the inner loop).  A CTA walks its contiguous range of
// points in windows of win points (8,192 where the shared memory allows,
// else 4,096: fewer windows, fewer sort phases).  For each window it counting-sorts the point
// indices by cluster in shared memory (a histogram, a scan and a scatter of
// 16-bit indices), then every warp takes an equal slice of the sorted order
// and adds its points run by run in registers: lane l reads up to two
// dimensions of each point (D = 64 with 8-byte-aligned points: 2l and
// 2l + 1 with one 8-byte load, so a warp reads the whole 256-byte row;
// otherwise l and l + 32 where below D) and keeps q = rint(x 2^s) = hi 2^20 + lo (lq_split)
// as two 32-bit sums per dimension; when the cluster changes the run is
// added into the CTA's int64 [k][D] sums with one 64-bit shared-memory add
// per dimension.
// A slice holds at most WS_WIN_MAX / WS_WARPS points, so no 32-bit run sum
// can overflow (256 * 2^19 = 2^27).  The CTA stores its sums as its partial and
// adds its counts to the global counts, like km_local_sum_kernel; the sums are
// the same integers in any order.  No wait of any kind: only plain loads and
// block barriers.
constexpr int WS_THREADS = 1024;
constexpr int WS_WARPS = WS_THREADS / 32;
constexpr uint32_t WS_WIN_MAX = 8192;  // points per window (16-bit positions), or half that
constexpr int WS_UNROLL = 8;       // points in flight per warp
__host__ __device__ constexpr uint64_t ws_smem_bytes(uint64_t k, uint64_t d, uint64_t win) {
  return k * d * 8 + 3 * k * 4 + 3 * win * 2;
}
// add a run's split sums of dimensions j0 and (TWO) j1, when below d, into
// cluster c's int64 sums
template <bool TWO>
__device__ __forceinline__ void ws_flush(long long* S, uint32_t c, uint32_t d, uint32_t j0, uint32_t j1, int h0,
                                         int l0, int h1, int l1) {
  unsigned long long* p = reinterpret_cast<unsigned long long*>(S + (uint64_t)c * d);
  if (j0 < d) atomicAdd(p + j0, (unsigned long long)((long long)h0 * (1ll << 20) + (long long)l0));
  if (TWO && j1 < d) atomicAdd(p + j1, (unsigned long long)((long long)h1 * (1ll << 20) + (long long)l1));
}
// Lanes and dimensions by MODE: WS_D64, D = 64 with 8-byte-aligned rows
// (lane l reads dimensions 2l, 2l + 1 with one 8-byte load); WS_D32,
// D <= 32 (lane l dimension l); WS_DANY, D <= 64 (lane l dimensions l and
// l + 32).
enum { WS_D64 = 0, WS_D32 = 1, WS_DANY = 2 };
template <int MODE>
__global__ void __launch_bounds__(WS_THREADS, 1) km_window_sum_kernel(const float* __restrict__ x, uint32_t n,
                                                                      uint32_t d_arg, uint32_t k, uint32_t win,
                                                                      const int32_t* __restrict__ assign,
                                                                      const int* shift, long long* __restrict__ part,
                                                                      unsigned long long* counts) {
  const uint32_t d = MODE == WS_D64 ? 64u : d_arg;  // a constant on the 64-wide path
  constexpr bool TWO = MODE != WS_D32;            // two dimensions per lane
  pdl_wait();
  extern __shared__ __align__(16) unsigned char ws_sm[];
  long long* S = reinterpret_cast<long long*>(ws_sm);
  uint32_t* hc = reinterpret_cast<uint32_t*>(S + (uint64_t)k * d);
  uint32_t* off = hc + k;
  uint32_t* C = off + k;
  uint16_t* wid = reinterpret_cast<uint16_t*>(C + k);
  uint16_t* perm = wid + win;
  uint16_t* pcl = perm + win;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t i = threadIdx.x; i < (uint64_t)k * d; i += WS_THREADS) S[i] = 0;
  for (uint32_t i = threadIdx.x; i < k; i += WS_THREADS) C[i] = 0;
  const uint32_t j0 = MODE == WS_D64 ? 2 * (uint32_t)lane : (uint32_t)lane;
  const uint32_t j1 = MODE == WS_D64 ? j0 + 1 : j0 + 32;
  const uint64_t per = ((uint64_t)n + gridDim.x - 1) / gridDim.x;
  const uint64_t p0 = (uint64_t)blockIdx.x * per;
  const uint64_t p1 = p0 + per < (uint64_t)n ? p0 + per : (uint64_t)n;
  const float scale = ldexpf(1.f, *shift);
  const uint32_t kl = (k + 31) / 32;  // bins per lane in the scan
  for (uint64_t w0 = p0; w0 < p1; w0 += win) {
    const uint32_t nr = (uint32_t)(p1 - w0 < win ? p1 - w0 : win);
    for (uint32_t t = threadIdx.x; t < k; t += WS_THREADS) hc[t] = 0;
    __syncthreads();  // hc cleared; the previous window's sorted order is no longer read
    for (uint32_t r = threadIdx.x; r < nr; r += WS_THREADS) {
      const uint32_t c = cluster_of(assign, w0 + r, k);
      wid[r] = (uint16_t)c;
      atomicAdd(&hc[c], 1u);
    }
    __syncthreads();
    if (warp == 0) {
      // exclusive scan of the window's cluster sizes (lane l: bins l kl ..)
      uint32_t tot = 0;
      for (uint32_t j = 0; j < kl; ++j) {
        const uint32_t c = (uint32_t)lane * kl + j;
        if (c < k) tot += hc[c];
      }
      uint32_t incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      uint32_t run = incl - tot;
      for (uint32_t j = 0; j < kl; ++j) {
        const uint32_t c = (uint32_t)lane * kl + j;
        if (c < k) {
          const uint32_t h = hc[c];
          off[c] = run;
          run += h;
          C[c] += h;
        }
      }
    }
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < nr; r += WS_THREADS) {
      const uint32_t c = wid[r];
      const uint32_t pos = atomicAdd(&off[c], 1u);
      perm[pos] = (uint16_t)r;
      pcl[pos] = (uint16_t)c;
    }
    __syncthreads();
    // warp slices of the sorted order; runs summed in registers
    const uint32_t pw = (nr + WS_WARPS - 1) / WS_WARPS;
    const uint32_t q0 = (uint32_t)warp * pw;
    const uint32_t q1 = q0 + pw < nr ? q0 + pw : nr;
    if (q0 < q1) {
      const float* X = x + w0 * d;
      uint32_t cur = pcl[q0];
      int h0 = 0, l0 = 0, h1 = 0, l1 = 0;
      for (uint32_t q = q0; q < q1; q += WS_UNROLL) {
        float2 v[WS_UNROLL];
        uint32_t cl[WS_UNROLL];
#pragma unroll
        for (int u = 0; u < WS_UNROLL; ++u) {
          const uint32_t qq = q + (uint32_t)u;
          const bool ok = qq < q1;
          cl[u] = ok ? pcl[qq] : cur;
          const float* row = X + (uint64_t)(ok ? perm[qq] : 0) * d;
          if (MODE == WS_D64) {
            v[u] = ok ? __ldg(reinterpret_cast<const float2*>(row) + lane) : make_float2(0.f, 0.f);
          } else {
            v[u].x = ok && j0 < d ? __ldg(row + j0) : 0.f;
            v[u].y = TWO && ok && j1 < d ? __ldg(row + j1) : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < WS_UNROLL; ++u) {
          if (cl[u] != cur) {  // warp-uniform: the run of cluster cur ended
            ws_flush<TWO>(S, cur, d, j0, j1, h0, l0, h1, l1);
            h0 = l0 = h1 = l1 = 0;
            cur = cl[u];
          }
          int a, b;
          lq_split(v[u].x * scale, a, b);
          h0 += a;
          l0 += b;
          if (TWO) {
            lq_split(v[u].y * scale, a, b);
            h1 += a;
            l1 += b;
          }
        }
      }
      ws_flush<TWO>(S, cur, d, j0, j1, h0, l0, h1, l1);
    }
  }
  __syncthreads();
  long long* P = part + (uint64_t)blockIdx.x * k * d;
  for (uint64_t i = threadIdx.x; i < (uint64_t)k * d; i += WS_THREADS) P[i] = S[i];
  for (uint32_t i = threadIdx.x; i < k; i += WS_THREADS)
    if (C[i]) atomicAdd(counts + i, (unsigned long long)C[i]);
}

// Sum of the g partials of each element (warp w of a CTA adds partials w,
// w + 8, ... of 32 consecutive elements), then the centroid as in
// km_finalize_kernel.
constexpr int RF_THREADS = 256;
__global__ void __launch_bounds__(RF_THREADS) km_reduce_finalize_kernel(const long long* __restrict__ part,
                                                                        uint32_t g, float* c, uint32_t k, uint32_t d,
                                                                        const unsigned long long* counts,
                                                                        const int* shift, unsigned int* cmax_bits) {
  pdl_wait();
  __shared__ long long red[RF_THREADS / 32][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t kd = (uint64_t)k * d;
  const uint64_t e = (uint64_t)blockIdx.x * 32 + lane;
  long long a = 0;
  if (e < kd) {
#pragma unroll 4
    for (uint32_t j = w; j < g; j += RF_THREADS / 32) a += part[(uint64_t)j * kd + e];
  }
  red[w][lane] = a;
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int i = 1; i < RF_THREADS / 32; ++i) a += red[i][lane];
    if (e < kd) {
      const unsigned long long cnt = counts[e / d];
      if (cnt) c[e] = (float)(((double)a * ldexp(1.0, -*shift)) / (double)cnt);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *cmax_bits = 0;
}

// c_k = (sum_k * 2^-s) / count_k in FP64, rounded to FP32; empty clusters keep c_k.
__global__ void km_finalize_kernel(float* c, uint32_t k, uint32_t d, const long long* sums,
                                   const unsigned long long* counts, const int* shift, unsigned int* cmax_bits) {
  const double inv = ldexp(1.0, -*shift);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (uint64_t)k * d;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long cnt = counts[i / d];
    if (cnt) c[i] = (float)(((double)sums[i] * inv) / (double)cnt);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *cmax_bits = 0;
}

__global__ void km_finish_kernel(const float* c, uint64_t kd, float* out_c, const int32_t* assign, uint32_t n,
                                 int32_t* out_a, const unsigned long long* stats, unsigned long long* out_s,
                                 uint32_t iters) {
  pdl_wait();
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < kd; i += nth) out_c[i] = c[i];
  uint64_t done = 0;
  if (((reinterpret_cast<uintptr_t>(out_a) | reinterpret_cast<uintptr_t>(assign)) & 15) == 0) {
    const uint64_t n4 = n / 4;
    for (uint64_t i = tid; i < n4; i += nth)
      reinterpret_cast<int4*>(out_a)[i] = reinterpret_cast<const int4*>(assign)[i];
    done = n4 * 4;
  }
  for (uint64_t i = done + tid; i < n; i += nth) out_a[i] = assign[i];
  if (tid == 0) {
    if ((kd + n) & 1) out_a[n] = 0;  // the zero padding before the 8-byte aligned stats
    out_s[0] = stats[0];
    out_s[1] = stats[1];
    out_s[2] = iters;
    out_s[3] = stats[3];
  }
}

inline uint64_t a256(uint64_t x) { return (x + 255) & ~255ull; }

}  // namespace

size_t km_scratch_bytes(uint32_t n, uint32_t d, uint32_t k, int precision) {
  uint64_t b = 0;
  b += a256((uint64_t)k * d * 4);      // cent
  b += a256((uint64_t)n * 4 + 16);     // assign (+16: the update copies ids in 16-byte units)
  b += a256((uint64_t)k * d * 8);      // sums
  b += a256((uint64_t)k * 8);          // counts
  b += a256(4 * 8);                    // stats
  b += a256((uint64_t)n * 4);          // flagged
  b += a256(8 * 4);                    // counters: nflag[2], maxabs, cmax, pairs
  b += a256((uint64_t)n * 8);          // pair list
  b += a256((uint64_t)n * 4);          // FP64 stage list
  b += a256((uint64_t)k * 4 * 2);      // cnorm (||c||^2) + spare
  b += a256(16);                       // shift
  b += a256((uint64_t)k * 4);          // per-cluster write cursor
  if (precision != MR_KM_FP32) {
    b += a256((uint64_t)n * 4);        // second flag list
    b += a256((uint64_t)k * d * 2 * 2);  // bf16 centroids (hi, lo)
  }
  if (local_sums_fit(d, k)) b += a256((uint64_t)LS_MAX_CTAS * k * d * 8);  // per-CTA partial sums
  return (size_t)b;
}

cudaError_t km_carve(KmBuffers& b, uint8_t* p, size_t bytes) {
  const uint64_t n = b.n, d = b.d, k = b.k;
  uint8_t* q = p;
  auto take = [&](uint64_t sz) { uint8_t* r = q; q += a256(sz); return r; };
  b.cent = reinterpret_cast<float*>(take(k * d * 4));
  b.assign = reinterpret_cast<int32_t*>(take(n * 4 + 16));
  b.sums = reinterpret_cast<long long*>(take(k * d * 8));
  b.counts = reinterpret_cast<unsigned long long*>(take(k * 8));
  b.stats = reinterpret_cast<unsigned long long*>(take(32));
  b.flagged = reinterpret_cast<uint32_t*>(take(n * 4));
  b.nflag = reinterpret_cast<uint32_t*>(take(32));
  b.pairs = reinterpret_cast<uint2*>(take(n * 8));
  b.deferred = reinterpret_cast<uint32_t*>(take(n * 4));
  b.maxabs = reinterpret_cast<unsigned int*>(b.nflag + 2);
  b.cnorm = reinterpret_cast<float*>(take(k * 8));
  b.cent_bf16_norm = nullptr;
  int* shift = reinterpret_cast<int*>(take(16));
  b.kcursor = reinterpret_cast<uint32_t*>(take(k * 4));
  b.fx_shift = 0;
  b.xnorm = reinterpret_cast<float*>(shift);  // holds the device-side shift
  if (b.precision != MR_KM_FP32) {
    b.cent_bf16_norm = reinterpret_cast<float*>(take(n * 4));  // second flag list
    b.cb = reinterpret_cast<uint16_t*>(take(k * d * 4));
  }
  b.part = local_sums_fit(d, k) ? reinterpret_cast<long long*>(take((uint64_t)LS_MAX_CTAS * k * d * 8)) : nullptr;
  if ((uint64_t)(q - p) > bytes) return cudaErrorInvalidValue;
  return cudaSuccess;
}

bool km_tc_supported(uint32_t d, uint32_t k);

cudaError_t launch_kmeans_tc_assign(const float* x, uint32_t n, uint32_t d, const float* c, uint32_t k,
                                    KmBuffers& b, const DevInfo& di, cudaStream_t s, uint64_t* nk, bool maxabs);

cudaError_t launch_kmeans(const float* x, const float* init, uint32_t iters, KmBuffers& b, const DevInfo& di,
                          cudaStream_t s, float* out_c, int32_t* out_a, unsigned long long* out_s, uint64_t* nk) {
  cudaError_t e;
  const uint32_t n = b.n, d = b.d, k = b.k;
  int* shift = reinterpret_cast<int*>(b.xnorm);
  unsigned int* cmax_bits = b.nflag + 3;
  if ((e = cudaMemcpyAsync(b.cent, init, (size_t)k * d * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b.stats, 0, 32, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b.nflag, 0, 32, s)) != cudaSuccess) return e;
  // the fixed-point scale needs max |x|: a pass of its own for the FP32
  // path; the tensor-core pass finds it while converting the first iteration
  const bool tc = b.precision != MR_KM_FP32;
  if (!tc) {
    km_maxabs_kernel<<<di.sms * 4, 256, 0, s>>>(x, (uint64_t)n * d, b.maxabs);
    km_scale_kernel<<<1, 1, 0, s>>>(b.maxabs, n, shift);
    *nk += 2;
  }
  const int asm_bytes = (DC_MAX * CS_LD + DC_MAX * XS_LD) * 4;
  if ((e = cudaFuncSetAttribute(km_assign_fp32_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                asm_bytes)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(km_assign_fp32_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                asm_bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(km_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(k * 4))) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(km_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(k * 4))) !=
      cudaSuccess)
    return e;
  const int ls_bytes = (int)((uint64_t)k * d * 8 + (uint64_t)k * 4);
  const bool local = b.part != nullptr && ls_bytes <= di.smem_optin;
  if (local && (e = cudaFuncSetAttribute(km_local_sum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         ls_bytes)) != cudaSuccess)
    return e;
  // pipelined update: rows of a multiple of 4 floats, 16-byte aligned points, and a ring of >= 4 rows a stage
  uint32_t lp_rows = 0;
  int lp_bytes = 0;
  if (local && d % 4 == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0) {
    const uint64_t fixed = lp_fixed_bytes((uint64_t)k * d, k);
    const uint64_t avail = (uint64_t)di.smem_optin > fixed ? (uint64_t)di.smem_optin - fixed : 0;
    uint64_t r = avail / LP_ST / ((uint64_t)d * 4 + 4);
    if (r > LP_CHUNK_MAX / ((uint64_t)d * 4)) r = LP_CHUNK_MAX / ((uint64_t)d * 4);
    r &= ~3ull;
    if (r >= 4) {
      lp_rows = (uint32_t)r;
      lp_bytes = (int)(fixed + LP_ST * r * ((uint64_t)d * 4 + 4));
      if ((e = cudaFuncSetAttribute(km_local_sum_pipe_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    lp_bytes)) != cudaSuccess ||
          (e = cudaFuncSetAttribute(km_local_sum_pipe_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    lp_bytes)) != cudaSuccess)
        return e;
    }
  }
  // the window-sorted update: D <= 64, sums and window buffers in shared
  // memory (8-byte loads for D = 64 with 8-byte-aligned points)
  const uint32_t ws_win =
      ws_smem_bytes(k, d, WS_WIN_MAX) <= (uint64_t)di.smem_optin ? WS_WIN_MAX : WS_WIN_MAX / 2;
  const bool wsum = local && d <= 64 && ws_smem_bytes(k, d, ws_win) <= (uint64_t)di.smem_optin;
  auto ws_kernel = d == 64 && (reinterpret_cast<uintptr_t>(x) & 7) == 0 ? km_window_sum_kernel<WS_D64>
                   : d <= 32                                               ? km_window_sum_kernel<WS_D32>
                                                                           : km_window_sum_kernel<WS_DANY>;
  if (wsum && (e = cudaFuncSetAttribute(ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)ws_smem_bytes(k, d, ws_win))) != cudaSuccess)
    return e;
  uint32_t ls_grid = (uint32_t)di.sms < LS_MAX_CTAS ? (uint32_t)di.sms : LS_MAX_CTAS;
  if ((uint64_t)ls_grid * 1024 > n) ls_grid = (uint32_t)((n + 1023) / 1024);
  if (b.grid_cap && ls_grid > b.grid_cap) ls_grid = b.grid_cap;
  if (ls_grid < 1) ls_grid = 1;
  const long long polls = b.polls < 0 ? pipe::SPIN_LIMIT : b.polls;
  const int rc_bytes = (int)((uint64_t)k * (d + 1) * 4);
  const bool rc_smem = k <= 32 * KLANE && rc_bytes <= di.smem_optin;
  // as many re-check CTAs per SM as the centroid copies allow (at most 3: 48 warps)
  int rc_per_sm = rc_smem ? (di.smem_optin + 1024) / (rc_bytes + 1024) : 1;
  rc_per_sm = rc_per_sm < 1 ? 1 : (rc_per_sm > 3 ? 3 : rc_per_sm);
  if (rc_smem &&
      (e = cudaFuncSetAttribute(km_recheck_fp64_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, rc_bytes)) !=
          cudaSuccess)
    return e;
  const int f64_bytes = (int)fp64_stage_smem(d, k);
  if ((e = cudaFuncSetAttribute(km_fp64_stage_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, f64_bytes)) !=
      cudaSuccess)
    return e;
  const uint32_t ntiles = (n + TP - 1) / TP;
  uint32_t agrid = ntiles < (uint32_t)di.sms * 2 ? ntiles : (uint32_t)di.sms * 2;
  if (b.grid_cap && agrid > b.grid_cap) agrid = b.grid_cap;
  for (uint32_t it = 0; it < iters; ++it) {
    // kernels that follow another kernel of this job on the stream start
    // while it drains (programmatic dependent launch; each waits first)
    if (it == 0)
      km_prep_kernel<<<64, 256, 0, s>>>(b.cent, k, d, b.cnorm, cmax_bits, b.sums, b.counts, b.nflag);
    else if ((e = launch_pdl(km_prep_kernel, dim3(64), dim3(256), 0, s, (const float*)b.cent, k, d, b.cnorm, cmax_bits,
                             b.sums, b.counts, b.nflag)) != cudaSuccess)
      return e;
    if (b.precision != MR_KM_FP32) {
      if ((e = launch_kmeans_tc_assign(x, n, d, b.cent, k, b, di, s, nk, it == 0)) != cudaSuccess) return e;
      if (it == 0) {
        km_scale_kernel<<<1, 1, 0, s>>>(b.maxabs, n, shift);
        ++*nk;
      }
    } else {
      if ((e = kt_begin(b.kt, s)) != cudaSuccess) return e;
      (k <= 256 ? km_assign_fp32_kernel<true> : km_assign_fp32_kernel<false>)<<<agrid, KM_THREADS, asm_bytes, s>>>(
          x, n, d, b.cent, k, b.cnorm, cmax_bits, nullptr, nullptr, b.assign, b.flagged, b.nflag, b.pairs,
          b.nflag + 4, nullptr);
      if ((e = cudaGetLastError()) != cudaSuccess || (e = kt_end(b.kt, s)) != cudaSuccess) return e;
      ++*nk;
    }
    // one warp per pair, latency-bound: a full SM of warps (32 registers a thread)
    km_pair_kernel<<<di.sms * 8, 256, 0, s>>>(x, d, b.cent, b.pairs, b.nflag + 4, b.assign, b.stats, b.deferred,
                                              b.nflag + 5);
    ++*nk;
    // the points neither pass could decide: from the tensor-core pass its
    // list (re-checked straight away with FP32 direct differences; the points
    // where those leave more than one candidate go to the FP64 stage), from
    // the FP32 pass its own
    const uint32_t* rl = b.precision != MR_KM_FP32 ? reinterpret_cast<const uint32_t*>(b.cent_bf16_norm) : b.flagged;
    const uint32_t* rn = b.precision != MR_KM_FP32 ? b.nflag + 1 : b.nflag;
    if (rc_smem)
      e = launch_pdl(km_recheck_fp64_smem_kernel, dim3(di.sms * rc_per_sm), dim3(512), (size_t)rc_bytes, s, x, d,
                     (const float*)b.cent, k, rl, rn, b.assign, b.stats, b.deferred, b.nflag + 5);
    else
      e = launch_pdl(km_recheck_fp64_kernel, dim3(di.sms * 4), dim3(256), 0, s, x, d, (const float*)b.cent, k, rl, rn,
                     b.assign, b.stats);
    if (e != cudaSuccess) return e;
    // the FP64 stage: the points the pair and re-check passes left to the
    // definition, one CTA each, all at once
    if ((e = launch_pdl(km_fp64_stage_kernel, dim3(di.sms * 2), dim3(F64_THREADS), (size_t)f64_bytes, s, x, d,
                        (const float*)b.cent, k, (const uint32_t*)b.deferred, (const uint32_t*)(b.nflag + 5), b.assign,
                        b.stats)) != cudaSuccess)
      return e;
    *nk += 2;  // re-check, FP64 stage
    if (local) {  // update with local arrays
      if (wsum)
        e = launch_pdl(ws_kernel, dim3(ls_grid),
                       dim3(WS_THREADS), (size_t)ws_smem_bytes(k, d, ws_win), s, x, n, d, k, ws_win,
                       (const int32_t*)b.assign, (const int*)shift, b.part, b.counts);
      else if (lp_rows)
        e = launch_pdl(d == 64 ? km_local_sum_pipe_kernel<true> : km_local_sum_pipe_kernel<false>, dim3(ls_grid),
                       dim3(LS_THREADS), (size_t)lp_bytes, s, x, n, d, k, (const int32_t*)b.assign, (const int*)shift,
                       b.part, b.counts, lp_rows, b.stats + 3, polls);
      else
        e = launch_pdl(km_local_sum_kernel, dim3(ls_grid), dim3(LS_THREADS), (size_t)ls_bytes, s, x, n, d, k,
                       (const int32_t*)b.assign, (const int*)shift, b.part, b.counts);
      if (e != cudaSuccess) return e;
      if ((e = launch_pdl(km_reduce_finalize_kernel, dim3((unsigned)(((uint64_t)k * d + 31) / 32)), dim3(RF_THREADS),
                          0, s, (const long long*)b.part, ls_grid, b.cent, k, d, (const unsigned long long*)b.counts,
                          (const int*)shift, cmax_bits)) != cudaSuccess)
        return e;
      *nk += 3;  // prep, update, reduction
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      continue;
    }
    // update: counting sort of the points by cluster, then run-wise sums
    km_count_kernel<<<di.sms * 2, 512, k * 4, s>>>(b.assign, n, k, b.counts);
    km_offsets_kernel<<<1, 1024, 0, s>>>(b.counts, k, b.kcursor);
    const uint64_t sc_blocks = (n + (uint64_t)SCAT_THREADS * SCAT_PER_THREAD - 1) / ((uint64_t)SCAT_THREADS * SCAT_PER_THREAD);
    km_scatter_kernel<<<(unsigned)sc_blocks, SCAT_THREADS, k * 4, s>>>(b.assign, n, k, b.kcursor, b.flagged);
    const uint64_t sum_warps = (n + SUM_RUN - 1) / SUM_RUN;
    // after the scatter, kcursor[c] is one past the last position of cluster c
    km_sum_kernel<<<(unsigned)((sum_warps * 32 + 255) / 256), 256, 0, s>>>(x, n, d, k, b.kcursor, b.flagged, shift,
                                                                           b.sums);
    km_finalize_kernel<<<64, 256, 0, s>>>(b.cent, k, d, b.sums, b.counts, shift, cmax_bits);
    *nk += 6;  // prep, count, offsets, scatter, sums, finalize
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = launch_pdl(km_finish_kernel, dim3(di.sms * 4), dim3(256), 0, s, (const float*)b.cent, (uint64_t)k * d,
                      out_c, (const int32_t*)b.assign, n, out_a, (const unsigned long long*)b.stats, out_s, iters)) !=
      cudaSuccess)
    return e;
  ++*nk;
  return cudaGetLastError();
}

}  // namespace mrgb
