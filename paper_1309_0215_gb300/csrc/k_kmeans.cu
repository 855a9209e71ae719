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
//  * Every other point is re-checked exactly in FP64 over all K centroids
//    with the same operation order as the definition above.
//  * Sums are accumulated as int64 fixed point q = rint(x * 2^s), with s chosen
//    from max|x| and N so no sum can overflow; integer addition is exact and
//    order-independent, so results do not depend on scheduling.
#include <cmath>

#include "mr_internal.h"

namespace mrgb {
namespace {

constexpr int KM_THREADS = 256;   // 8 warps
constexpr int TP = 64;            // points per tile (8 per warp)
constexpr int KC_MAX = 256;       // centroids per chunk (8 per lane)
constexpr int DC_MAX = 64;        // dims per chunk

__device__ __forceinline__ void best2_push(float d, int k, float& d1, int& k1, float& d2) {
  if (d < d1 || (d == d1 && k < k1)) {
    d2 = d1;
    d1 = d;
    k1 = k;
  } else if (d < d2) {
    d2 = d;
  }
}

__device__ __forceinline__ void best2_merge(float& d1, int& k1, float& d2, float e1, int f1, float e2) {
  if (e1 < d1 || (e1 == d1 && f1 < k1)) {
    d2 = fminf(d1, e2);
    d1 = e1;
    k1 = f1;
  } else {
    d2 = fminf(d2, e1);
  }
}

// Centroid norms: cn[k] = ||c_k||^2 (FP32, sequential FMA); cmax[0] = max ||c_k||.
__global__ void km_prep_kernel(const float* __restrict__ c, uint32_t k, uint32_t d, float* __restrict__ cn,
                               unsigned int* cmax_bits, long long* sums, unsigned long long* counts, uint32_t* nflag) {
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
}

// FP32 assignment.  A CTA processes tiles of 64 points; warp w owns points
// 8w..8w+7 of the tile, lane l owns centroids l + 32 j (j < 8) of each chunk
// of up to 256 centroids.  Dot products accumulate over dimension chunks
// staged in shared memory (points transposed [dim][point], centroids
// [dim][centroid]).  When K <= 256 and D <= 64 the centroids are loaded once
// per CTA.  idx != nullptr restricts the pass to the listed points.
__global__ void __launch_bounds__(KM_THREADS, 2)
km_assign_fp32_kernel(const float* __restrict__ x, uint32_t n, uint32_t d, const float* __restrict__ c, uint32_t k,
                      const float* __restrict__ cn, const unsigned int* cmax_bits, const uint32_t* idx,
                      const uint32_t* nidx, int32_t* __restrict__ assign, uint32_t* flagged, uint32_t* nflag,
                      unsigned long long* stat) {
  extern __shared__ float km_sm[];
  const int dc = d < DC_MAX ? (int)d : DC_MAX;
  const int kc = k < KC_MAX ? (int)k : KC_MAX;
  float* cs = km_sm;              // [dc][KC_MAX]
  float* xs = km_sm + DC_MAX * KC_MAX;  // [dc][TP]
  __shared__ float nx_s[TP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t npts = idx ? *nidx : n;
  const bool resident = k <= KC_MAX && d <= DC_MAX;
  const float cmax = __uint_as_float(*cmax_bits);
  const float eps = 1.01f * (float)(d + 8) * 5.9604645e-8f;  // 2^-24
  if (idx && blockIdx.x == 0 && threadIdx.x == 0 && stat) atomicAdd(stat, (unsigned long long)npts);

  auto load_c = [&](uint32_t k0, uint32_t d0) {
    for (int t = threadIdx.x; t < kc * dc; t += KM_THREADS) {
      const int kk = t / dc, dd = t % dc;
      const uint32_t kg = k0 + kk, dg = d0 + dd;
      cs[dd * KC_MAX + kk] = (kg < k && dg < d) ? c[(uint64_t)kg * d + dg] : 0.f;
    }
  };
  if (resident) {
    load_c(0, 0);
    __syncthreads();
  }
  const uint32_t ntiles = (npts + TP - 1) / TP;
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint32_t p0 = tile * TP;
    float d1[8], d2[8];
    int k1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) d1[i] = d2[i] = INFINITY, k1[i] = 0x7fffffff;
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
        for (int t = threadIdx.x; t < TP * dc; t += KM_THREADS) {
          const int pp = t / dc, dd = t % dc;
          const uint32_t pi = p0 + pp, dg = d0 + dd;
          float v = 0.f;
          if (pi < npts && dg < d) {
            const uint32_t p = idx ? idx[pi] : pi;
            v = x[(uint64_t)p * d + dg];
          }
          xs[dd * TP + pp] = v;
        }
        __syncthreads();
        const int dlim = (int)((d - d0) < (uint32_t)dc ? (d - d0) : (uint32_t)dc);
        if (k0 == 0 && threadIdx.x < TP)
          for (int dd = 0; dd < dlim; ++dd) nxacc = fmaf(xs[dd * TP + threadIdx.x], xs[dd * TP + threadIdx.x], nxacc);
        for (int dd = 0; dd < dlim; ++dd) {
          const float4 xa = *reinterpret_cast<const float4*>(&xs[dd * TP + warp * 8]);
          const float4 xb = *reinterpret_cast<const float4*>(&xs[dd * TP + warp * 8 + 4]);
          const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
          float cv[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) cv[j] = cs[dd * KC_MAX + lane + 32 * j];
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
        if (kk < k && lane + 32 * j < kc) {
          const float ncv = cn[kk];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float dist = fmaf(-2.f, acc[i][j], nx_s[warp * 8 + i]) + ncv;
            best2_push(dist, (int)kk, d1[i], k1[i], d2[i]);
          }
        }
      }
    }
    // combine the lanes' candidates for each of the warp's 8 points
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      for (int o = 16; o; o >>= 1) {
        const float e1 = __shfl_xor_sync(0xffffffffu, d1[i], o);
        const int f1 = __shfl_xor_sync(0xffffffffu, k1[i], o);
        const float e2 = __shfl_xor_sync(0xffffffffu, d2[i], o);
        best2_merge(d1[i], k1[i], d2[i], e1, f1, e2);
      }
    }
    // lane i decides point i of the warp
    float md1 = 0.f, md2 = 0.f;
    int mk1 = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (lane == i) md1 = d1[i], md2 = d2[i], mk1 = k1[i];
    const uint32_t pi = p0 + warp * 8 + lane;
    bool flag = false;
    if (lane < 8 && pi < npts) {
      const uint32_t p = idx ? idx[pi] : pi;
      const float nxv = sqrtf(nx_s[warp * 8 + lane]);
      const float e = eps * (nxv + cmax) * (nxv + cmax);
      if (md2 - md1 > 2.f * e) assign[p] = mk1;
      else flag = true;
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

// Exact FP64 argmin for the listed points: one warp per point, lane l takes
// centroids l, l+32, ...; the distance is the definition's sum in order with
// separately rounded subtract, multiply and add.
__global__ void km_recheck_fp64_kernel(const float* __restrict__ x, uint32_t d, const float* __restrict__ c, uint32_t k,
                                       const uint32_t* flagged, const uint32_t* nflag, int32_t* assign,
                                       unsigned long long* stat) {
  const uint32_t nf = *nflag;
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  if (w0 == 0 && lane == 0 && stat) atomicAdd(stat, (unsigned long long)nf);
  for (uint64_t f = w0; f < nf; f += nw) {
    const uint32_t p = flagged[f];
    const float* xp = x + (uint64_t)p * d;
    double best = INFINITY;
    int bk = 0x7fffffff;
    for (uint32_t kk = lane; kk < k; kk += 32) {
      const float* cp = c + (uint64_t)kk * d;
      double s = 0.0;
      for (uint32_t j = 0; j < d; ++j) {
        const double t = __dsub_rn((double)xp[j], (double)cp[j]);
        s = __dadd_rn(s, __dmul_rn(t, t));
      }
      if (s < best) best = s, bk = (int)kk;  // kk increases: the lowest index keeps a tie
    }
    for (int o = 16; o; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
      if (ob < best || (ob == best && ok < bk)) best = ob, bk = ok;
    }
    if (lane == 0) assign[p] = bk == 0x7fffffff ? 0 : bk;  // all-NaN distances: index 0, as the definition
  }
}

// max |x| over all coordinates (as float bits; non-negative floats order like ints)
__global__ void km_maxabs_kernel(const float* __restrict__ x, uint64_t cnt, unsigned int* out) {
  unsigned int m = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(fabsf(x[i])));
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Fixed-point exponent s: max|x| * 2^s * n < 2^62, capped to [0, 60].
__global__ void km_scale_kernel(const unsigned int* maxabs, uint32_t n, int* shift) {
  const float m = __uint_as_float(*maxabs);
  int s = 60;
  if (m > 0.f) {
    const double lim = ldexp(1.0, 62);
    while (s > 0 && (double)m * ldexp(1.0, s) * (double)n >= lim) --s;
  }
  *shift = s;
}

// Per-cluster int64 fixed-point sums and counts.  A CTA keeps a local copy in
// shared memory when K*D*8 + K*8 fits, else it adds straight into the global
// arrays (the paper's "eliminated local arrays").  A warp takes 8 points per
// step and issues all their loads before the atomics, to keep enough bytes in
// flight; lane l covers dimensions l and l + 32 of each 64-dimension slice.
__global__ void __launch_bounds__(512)
km_update_kernel(const float* __restrict__ x, uint32_t n, uint32_t d, uint32_t k,
                 const int32_t* __restrict__ assign, const int* shift, long long* sums,
                 unsigned long long* counts, int use_smem) {
  extern __shared__ long long up_sm[];
  long long* ls = up_sm;                                         // [k*d]
  unsigned long long* lc = reinterpret_cast<unsigned long long*>(up_sm + (uint64_t)k * d);  // [k]
  long long* ts = use_smem ? ls : sums;
  unsigned long long* tc = use_smem ? lc : counts;
  if (use_smem) {
    for (uint64_t i = threadIdx.x; i < (uint64_t)k * d; i += blockDim.x) ls[i] = 0;
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) lc[i] = 0;
    __syncthreads();
  }
  const double scale = ldexp(1.0, *shift);
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t p0 = w0 * 8; p0 < n; p0 += nw * 8) {
    const int al = (lane < 8 && p0 + lane < n) ? assign[p0 + lane] : -1;
    for (uint32_t j0 = 0; j0 < d; j0 += 64) {
      float v[8][2];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t dj = j0 + lane + 32 * h;
          v[r][h] = (p0 + r < n && dj < d) ? x[(p0 + r) * d + dj] : 0.f;
        }
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int a = __shfl_sync(0xffffffffu, al, r);
        if (a < 0 || (uint32_t)a >= k) continue;
        long long* sp = ts + (uint64_t)a * d;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t dj = j0 + lane + 32 * h;
          if (dj < d) {
            const long long q = __double2ll_rn((double)v[r][h] * scale);
            atomicAdd(reinterpret_cast<unsigned long long*>(sp + dj), (unsigned long long)q);
          }
        }
      }
    }
    if (al >= 0 && (uint32_t)al < k) atomicAdd(tc + al, 1ull);
  }
  if (use_smem) {
    __syncthreads();
    for (uint64_t i = threadIdx.x; i < (uint64_t)k * d; i += blockDim.x)
      if (ls[i]) atomicAdd(reinterpret_cast<unsigned long long*>(sums + i), (unsigned long long)ls[i]);
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x)
      if (lc[i]) atomicAdd(counts + i, lc[i]);
  }
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
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < kd; i += nth) out_c[i] = c[i];
  for (uint64_t i = tid; i < n; i += nth) out_a[i] = assign[i];
  if (tid == 0) {
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
  b += a256((uint64_t)n * 4);          // assign
  b += a256((uint64_t)k * d * 8);      // sums
  b += a256((uint64_t)k * 8);          // counts
  b += a256(4 * 8);                    // stats
  b += a256((uint64_t)n * 4);          // flagged
  b += a256(4 * 4);                    // nflag[2], maxabs, cmax
  b += a256((uint64_t)k * 4 * 2);      // cnorm (||c||^2) + spare
  b += a256(16);                       // shift
  if (precision != MR_KM_FP32) {
    b += a256((uint64_t)n * 4);        // second flag list
    b += a256((uint64_t)k * d * 2 * 2);  // bf16 centroids (hi, lo)
  }
  return (size_t)b;
}

cudaError_t km_carve(KmBuffers& b, uint8_t* p, size_t bytes) {
  const uint64_t n = b.n, d = b.d, k = b.k;
  uint8_t* q = p;
  auto take = [&](uint64_t sz) { uint8_t* r = q; q += a256(sz); return r; };
  b.cent = reinterpret_cast<float*>(take(k * d * 4));
  b.assign = reinterpret_cast<int32_t*>(take(n * 4));
  b.sums = reinterpret_cast<long long*>(take(k * d * 8));
  b.counts = reinterpret_cast<unsigned long long*>(take(k * 8));
  b.stats = reinterpret_cast<unsigned long long*>(take(32));
  b.flagged = reinterpret_cast<uint32_t*>(take(n * 4));
  b.nflag = reinterpret_cast<uint32_t*>(take(16));
  b.maxabs = reinterpret_cast<unsigned int*>(b.nflag + 2);
  b.cnorm = reinterpret_cast<float*>(take(k * 8));
  b.cent_bf16_norm = nullptr;
  int* shift = reinterpret_cast<int*>(take(16));
  b.fx_shift = 0;
  b.xnorm = reinterpret_cast<float*>(shift);  // holds the device-side shift
  if (b.precision != MR_KM_FP32) {
    b.cent_bf16_norm = reinterpret_cast<float*>(take(n * 4));  // second flag list
    b.cb = reinterpret_cast<uint16_t*>(take(k * d * 4));
  }
  if ((uint64_t)(q - p) > bytes) return cudaErrorInvalidValue;
  return cudaSuccess;
}

bool km_tc_supported(uint32_t d, uint32_t k);

cudaError_t launch_kmeans_tc_assign(const float* x, uint32_t n, uint32_t d, const float* c, uint32_t k,
                                    KmBuffers& b, const DevInfo& di, cudaStream_t s, uint64_t* nk);

cudaError_t launch_kmeans(const float* x, const float* init, uint32_t iters, KmBuffers& b, const DevInfo& di,
                          cudaStream_t s, float* out_c, int32_t* out_a, unsigned long long* out_s, uint64_t* nk) {
  cudaError_t e;
  const uint32_t n = b.n, d = b.d, k = b.k;
  int* shift = reinterpret_cast<int*>(b.xnorm);
  unsigned int* cmax_bits = b.nflag + 3;
  if ((e = cudaMemcpyAsync(b.cent, init, (size_t)k * d * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b.stats, 0, 32, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b.nflag, 0, 16, s)) != cudaSuccess) return e;
  km_maxabs_kernel<<<di.sms * 4, 256, 0, s>>>(x, (uint64_t)n * d, b.maxabs);
  km_scale_kernel<<<1, 1, 0, s>>>(b.maxabs, n, shift);
  *nk += 2;
  const int asm_bytes = (DC_MAX * KC_MAX + DC_MAX * TP) * 4;
  if ((e = cudaFuncSetAttribute(km_assign_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, asm_bytes)) !=
      cudaSuccess)
    return e;
  const uint64_t up_bytes = (uint64_t)k * d * 8 + (uint64_t)k * 8;
  const int use_smem = up_bytes <= (uint64_t)di.smem_optin ? 1 : 0;
  if (use_smem) {
    if ((e = cudaFuncSetAttribute(km_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)up_bytes)) !=
        cudaSuccess)
      return e;
  }
  const uint32_t ntiles = (n + TP - 1) / TP;
  const uint32_t agrid = ntiles < (uint32_t)di.sms * 2 ? ntiles : (uint32_t)di.sms * 2;
  for (uint32_t it = 0; it < iters; ++it) {
    km_prep_kernel<<<64, 256, 0, s>>>(b.cent, k, d, b.cnorm, cmax_bits, b.sums, b.counts, b.nflag);
    if (b.precision != MR_KM_FP32) {
      if ((e = launch_kmeans_tc_assign(x, n, d, b.cent, k, b, di, s, nk)) != cudaSuccess) return e;
    } else {
      km_assign_fp32_kernel<<<agrid, KM_THREADS, asm_bytes, s>>>(x, n, d, b.cent, k, b.cnorm, cmax_bits, nullptr,
                                                                 nullptr, b.assign, b.flagged, b.nflag, nullptr);
      ++*nk;
    }
    km_recheck_fp64_kernel<<<di.sms * 4, 256, 0, s>>>(x, d, b.cent, k, b.flagged, b.nflag, b.assign, b.stats + 1);
    km_update_kernel<<<di.sms, 512, use_smem ? up_bytes : 0, s>>>(x, n, d, k, b.assign, shift, b.sums, b.counts,
                                                                  use_smem);
    km_finalize_kernel<<<64, 256, 0, s>>>(b.cent, k, d, b.sums, b.counts, shift, cmax_bits);
    *nk += 4;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  km_finish_kernel<<<di.sms, 256, 0, s>>>(b.cent, (uint64_t)k * d, out_c, b.assign, n, out_a, b.stats, out_s, iters);
  ++*nk;
  return cudaGetLastError();
}

// FP32 re-check of an index list (used after the BF16 tensor-core pass).
cudaError_t launch_kmeans_fp32_list(const float* x, uint32_t n, uint32_t d, const float* c, uint32_t k, KmBuffers& b,
                                    const uint32_t* list, const uint32_t* nlist, const DevInfo& di, cudaStream_t s,
                                    uint64_t* nk) {
  const int asm_bytes = (DC_MAX * KC_MAX + DC_MAX * TP) * 4;
  const uint32_t ntiles = (n + TP - 1) / TP;
  const uint32_t agrid = ntiles < (uint32_t)di.sms * 2 ? ntiles : (uint32_t)di.sms * 2;
  km_assign_fp32_kernel<<<agrid, KM_THREADS, asm_bytes, s>>>(x, n, d, c, k, b.cnorm, b.nflag + 3, list, nlist,
                                                             b.assign, b.flagged, b.nflag, b.stats);
  ++*nk;
  return cudaGetLastError();
}

}  // namespace mrgb
