// Array-container jobs whose key range is large: the 16M-key histogram and
// the k-mer Bloom-filter build (the two applications the paper runs with
// "eliminating local arrays", Sec. III-E and the data-set table of Sec. IV).
//
// Large-key histogram.  Keys are u32; key k < nbins adds one to bin k, any
// other key to bin nbins.  Two containers:
//   * local arrays: one u32 copy of all bins per CTA in shared memory
//     (red.shared), flushed with one global atomic per non-zero bin.  Only
//     possible while nbins + 1 counters fit the opt-in shared memory.
//   * global array (the paper's choice for large arrays): every key is one
//     red.global.add on a single counter array.  While the input has fewer
//     than 2^32 keys the counters are u32, so 16M bins take 64 MiB and stay
//     resident in the 129 MB L2 (the GPU counterpart of the paper's coherent
//     L2 argument); a final pass widens them to the u64 result.
//   Warps combine equal keys first (match.any), which turns the hot keys of
//   a skewed input into one atomic per warp; a warp that sees no repeats over
//   a window of tiles switches the step off and re-probes later.
//
// Bloom-filter build.  Element = every window of L bases of an ASCII DNA
// sequence whose bytes are all A/C/G/T; code = base-4 number of the window,
// first base most significant.  a = mix(code) mod m, b = 1 + mix(code ^
// 0x9E3779B97F4A7C15) mod (m - 1), mix = SplitMix64's output function
// (Steele, Lea & Flood, 2014); bits (a + i b) mod m, i < h, are set with
// atomicOr on u32 words (bit j = bit j%8 of byte j/8 of the result).
// A CTA packs its tile of bases into 2-bit codes (and a 1-bit invalid mask)
// in shared memory, big-endian within each word, so any window's code is one
// 128-bit funnel shift; both reductions mod m use Barrett's method with a
// 64-bit reciprocal computed on the host.
#include "mr_internal.h"

namespace mrgb {
namespace {

constexpr int HK_THREADS = 256;        // global-array kernel
constexpr int HK_SMEM_THREADS = 1024;  // local-array kernel
constexpr int HK_WINDOW = 16;          // tiles per aggregation decision

__device__ __forceinline__ uint4 ldg_nc(const uint4* p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

// L2 policies: the streamed keys are marked evict-first and the counters
// evict-last, so the counter array (64 MiB at 16M bins) stays resident in L2
// instead of being written back and re-read as the input streams through.
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint4 ldg_stream_hint(const uint4* p, uint64_t pol) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p), "l"(pol));
  return r;
}

__device__ __forceinline__ void red_add(uint32_t* p, uint32_t v) { atomicAdd(p, v); }
__device__ __forceinline__ void red_add(unsigned long long* p, uint32_t v) { atomicAdd(p, (unsigned long long)v); }
__device__ __forceinline__ void red_add_hint(uint32_t* p, uint32_t v, uint64_t pol) {
  asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void red_add_hint(unsigned long long* p, uint32_t v, uint64_t pol) {
  asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"((unsigned long long)v),
               "l"(pol)
               : "memory");
}

__device__ __forceinline__ uint32_t key_at(const uint4& w, int e) {
  return e == 0 ? w.x : e == 1 ? w.y : e == 2 ? w.z : w.w;
}

// Keys are read as 16-byte groups from the 16-byte-aligned address at or
// below the input; group g holds keys 4g - off .. 4g - off + 3 (off = the
// input's misalignment in keys), and keys outside [0, n) are masked.  A group
// that holds at least one key lies in the same aligned 16 bytes as that key,
// so no read leaves the pages of the input.
template <typename C>
__global__ void __launch_bounds__(HK_THREADS)
hk_global_kernel(const uint4* __restrict__ base, uint32_t off, uint64_t n, uint32_t nbins, C* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const uint64_t groups = (n + off + 3) / 4;
  const uint64_t tiles = (groups + 31) / 32;  // one group per lane
  const uint64_t warp = ((uint64_t)blockIdx.x * HK_THREADS + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * HK_THREADS) >> 5;
  bool agg = true;
  uint32_t saved = 0, win = 0, off_windows = 0;
  const uint64_t pol_in = l2_policy_evict_first(), pol_cnt = l2_policy_evict_last();
  for (uint64_t t = warp; t < tiles; t += nwarps) {
    const uint64_t g = t * 32 + lane;
    uint4 w = make_uint4(0, 0, 0, 0);
    if (g < groups) w = ldg_stream_hint(base + g, pol_in);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t idx = (int64_t)(4 * g + e) - (int64_t)off;
      const bool valid = g < groups && idx >= 0 && (uint64_t)idx < n;
      const uint32_t key = key_at(w, e);
      const uint32_t k = key < nbins ? key : nbins;
      if (agg) {
        const uint32_t vm = __ballot_sync(0xffffffffu, valid);
        const uint32_t m = __match_any_sync(0xffffffffu, k) & vm;
        if (valid && (__ffs(m) - 1) == lane) {
          red_add_hint(cnt + k, (uint32_t)__popc(m), pol_cnt);
          saved += (uint32_t)__popc(m) - 1;
        }
      } else if (valid) {
        red_add_hint(cnt + k, 1u, pol_cnt);
      }
    }
    if (++win == HK_WINDOW) {
      win = 0;
      if (agg) {
        // keep combining while it saves at least 1 atomic in 16
        const uint32_t s = __reduce_add_sync(0xffffffffu, saved);
        agg = s * 16u >= (uint32_t)(HK_WINDOW * 32 * 4);
        saved = 0;
      } else if (++off_windows == 16) {
        off_windows = 0;
        agg = true;  // re-probe: the key mix may have changed
      }
    }
  }
}

// Local arrays: nbins + 1 u32 counters per CTA in shared memory.
template <typename C>
__global__ void __launch_bounds__(HK_SMEM_THREADS)
hk_smem_kernel(const uint4* __restrict__ base, uint32_t off, uint64_t n, uint32_t nbins, C* __restrict__ cnt) {
  extern __shared__ uint32_t sh_bins[];
  for (uint32_t i = threadIdx.x; i <= nbins; i += blockDim.x) sh_bins[i] = 0;
  __syncthreads();
  const uint64_t groups = (n + off + 3) / 4;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 w = ldg_nc(base + g);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t idx = (int64_t)(4 * g + e) - (int64_t)off;
      if (idx >= 0 && (uint64_t)idx < n) {
        const uint32_t key = key_at(w, e);
        atomicAdd(&sh_bins[key < nbins ? key : nbins], 1u);
      }
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i <= nbins; i += blockDim.x) {
    const uint32_t v = sh_bins[i];
    if (v) red_add(cnt + i, v);
  }
}

// Local arrays spread over a thread-block cluster: the bins are cut into
// HKC slices of `slice` counters, CTA r of a cluster holding slice r in its
// shared memory, so a cluster holds HKC times as many bins as one CTA (the
// paper's local arrays, Sec. III-E, with a cluster of CTAs as the worker).
// Every CTA streams its share of the keys and adds each one to its slice's
// owner through distributed shared memory (red.shared::cluster); a cluster
// barrier before the first add (every slice zeroed) and after the last (every
// add landed), then each CTA adds its slice's non-zero counters to the global
// array.  No CTA touches another's shared memory after the second barrier,
// so CTAs may then exit in any order.
constexpr int HKC = 8;  // CTAs per cluster (the portable maximum)

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

template <typename C>
__global__ void __launch_bounds__(HK_SMEM_THREADS)
hk_cluster_kernel(const uint4* __restrict__ base, uint32_t off, uint64_t n, uint32_t nbins, uint32_t slice,
                  uint32_t slice_mul, C* __restrict__ cnt) {
  extern __shared__ uint32_t sh_bins[];
  const uint32_t rank = cluster_rank();
  for (uint32_t i = threadIdx.x; i < slice; i += blockDim.x) sh_bins[i] = 0;
  cluster_sync_all();
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sh_bins);
  const uint64_t groups = (n + off + 3) / 4;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 w = ldg_nc(base + g);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t idx = (int64_t)(4 * g + e) - (int64_t)off;
      if (idx >= 0 && (uint64_t)idx < n) {
        const uint32_t key = key_at(w, e);
        const uint32_t k = key < nbins ? key : nbins;
        // owner = k / slice: the multiply-high estimate is at most one low
        uint32_t r = __umulhi(k, slice_mul);
        uint32_t loc = k - r * slice;
        if (loc >= slice) {
          ++r;
          loc -= slice;
        }
        uint32_t ra;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(sbase + 4 * loc), "r"(r));
        asm volatile("red.relaxed.cluster.shared::cluster.add.u32 [%0], 1;" ::"r"(ra) : "memory");
      }
    }
  }
  cluster_sync_all();
  const uint64_t b0 = (uint64_t)rank * slice;
  for (uint32_t i = threadIdx.x; i < slice && b0 + i <= nbins; i += blockDim.x) {
    const uint32_t v = sh_bins[i];
    if (v) red_add(cnt + b0 + i, v);
  }
}

__global__ void hk_widen_kernel(const uint32_t* __restrict__ c32, uint64_t nb, unsigned long long* __restrict__ out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = c32[i];
}

// ------------------------------------------------------------ Bloom filter
constexpr int BF_THREADS = 256;
constexpr int BF_TILE = 8192;                     // windows per CTA tile
constexpr int BF_WORDS = BF_TILE / 32 + 2;        // packed words: the tile plus up to 63 more bases

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// x mod m with r = floor((2^64 - 1) / m): q = floor(x r / 2^64) undershoots
// floor(x / m) by at most 2, so at most two corrections.
__device__ __forceinline__ uint64_t mod_barrett(uint64_t x, uint64_t m, uint64_t r) {
  const uint64_t q = __umul64hi(x, r);
  uint64_t rem = x - q * m;
  if (rem >= m) rem -= m;
  if (rem >= m) rem -= m;
  return rem;
}

// 2-bit code and invalid flag of 4 bases packed little-endian in w (first
// base in the low byte): codes A,C,G,T = 0..3 from bits 1..3 of the byte
// ((c >> 1) ^ (c >> 2)) & 3; big-endian 8-bit result (first base on top).
__device__ __forceinline__ void pack4(uint32_t w, uint32_t& code8, uint32_t& bad4) {
  const uint32_t ok = __vcmpeq4(w, 0x41414141u) | __vcmpeq4(w, 0x43434343u) | __vcmpeq4(w, 0x47474747u) |
                      __vcmpeq4(w, 0x54545454u);
  const uint32_t t = ((w >> 1) ^ (w >> 2)) & 0x03030303u;
  code8 = ((t & 3u) << 6) | (((t >> 8) & 3u) << 4) | (((t >> 16) & 3u) << 2) | ((t >> 24) & 3u);
  const uint32_t bad = ~ok;
  bad4 = ((bad & 1u) << 3) | (((bad >> 8) & 1u) << 2) | (((bad >> 16) & 1u) << 1) | ((bad >> 24) & 1u);
}

__global__ void __launch_bounds__(BF_THREADS)
bloom_kernel(const uint8_t* __restrict__ seq, uint64_t n, uint32_t L, uint64_t m, uint64_t rm, uint64_t rm1,
             uint32_t h, uint32_t* __restrict__ bits) {
  __shared__ unsigned long long sc[BF_WORDS];  // 32 bases per word, first base in the top bits
  __shared__ uint32_t sb[BF_WORDS];            // 1 = not A/C/G/T, same order
  if (n < L) return;
  const uint64_t nwin = n - L + 1;
  const uint64_t tiles = (nwin + BF_TILE - 1) / BF_TILE;
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint64_t p0 = t * BF_TILE;
    __syncthreads();  // the previous tile's words are no longer read
    // pack bases p0 .. p0 + 32*BF_WORDS - 1 (beyond n: invalid)
    for (int wi = threadIdx.x; wi < BF_WORDS; wi += BF_THREADS) {
      uint64_t code = 0;
      uint32_t bad = 0;
      const uint64_t b0 = p0 + (uint64_t)wi * 32;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint64_t pos = b0 + (uint64_t)q * 4;
        uint32_t w = 0;
        if (pos + 4 <= n) {
          w = (uint32_t)seq[pos] | ((uint32_t)seq[pos + 1] << 8) | ((uint32_t)seq[pos + 2] << 16) |
              ((uint32_t)seq[pos + 3] << 24);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) w |= (pos + j < n ? (uint32_t)seq[pos + j] : 0u) << (8 * j);
        }
        uint32_t c8, b4;
        pack4(w, c8, b4);
        code = (code << 8) | c8;
        bad = (bad << 4) | b4;
      }
      sc[wi] = code;
      sb[wi] = bad;
    }
    __syncthreads();
    const uint64_t cnt = nwin - p0 < (uint64_t)BF_TILE ? nwin - p0 : (uint64_t)BF_TILE;
    for (uint32_t i = threadIdx.x; i < cnt; i += BF_THREADS) {
      const uint32_t wi = i >> 5, o = i & 31;
      const uint64_t bm = (((uint64_t)sb[wi] << 32) | sb[wi + 1]) << o;
      if (bm >> (64 - L)) continue;  // a base of the window is not A/C/G/T
      const uint64_t hi = sc[wi], lo = sc[wi + 1];
      const uint64_t cat = o ? (hi << (2 * o)) | (lo >> (64 - 2 * o)) : hi;
      const uint64_t code = cat >> (64 - 2 * L);
      uint64_t pos = mod_barrett(mix64(code), m, rm);
      const uint64_t step = 1 + mod_barrett(mix64(code ^ 0x9E3779B97F4A7C15ull), m - 1, rm1);
      for (uint32_t q = 0; q < h; ++q) {
        atomicOr(bits + (pos >> 5), 1u << (pos & 31));
        pos += step;
        if (pos >= m) pos -= m;
      }
    }
  }
}

}  // namespace

int hk_smem_max_bins(const DevInfo& di) { return di.smem_optin / 4 - 1; }
int hk_cluster_max_bins(const DevInfo& di) { return HKC * (di.smem_optin / 4) - 1; }

template <typename C>
static cudaError_t launch_hk_cluster(const uint4* base, uint32_t off, uint64_t n, uint32_t nbins, C* cnt,
                                     const DevInfo& di, cudaStream_t s) {
  const uint32_t slice = (uint32_t)(((uint64_t)nbins + 1 + HKC - 1) / HKC);
  // multiply-high by floor(2^32 / slice) (at most 2^32 - 1) gives
  // floor(k / slice) or one less, for every k < 2^32
  const uint64_t sm64 = (1ull << 32) / slice;
  const uint32_t slice_mul = sm64 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)sm64;
  const int bytes = (int)(slice * 4);
  cudaError_t e = cudaFuncSetAttribute(hk_cluster_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  const uint64_t groups = (n + off + 3) / 4;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = HKC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(HK_SMEM_THREADS, 1, 1);
  cfg.dynamicSmemBytes = (size_t)bytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // as many clusters as fit the GPU at once (each CTA holds one slice)
  int clusters = 0;
  cfg.gridDim = dim3(HKC, 1, 1);
  if ((e = cudaOccupancyMaxActiveClusters(&clusters, hk_cluster_kernel<C>, &cfg)) != cudaSuccess) return e;
  if (clusters < 1) return cudaErrorInvalidConfiguration;
  uint64_t want = (groups + (uint64_t)HK_SMEM_THREADS * 16 * HKC - 1) / ((uint64_t)HK_SMEM_THREADS * 16 * HKC);
  if (want < 1) want = 1;
  if (want > (uint64_t)clusters) want = (uint64_t)clusters;
  cfg.gridDim = dim3((unsigned)(want * HKC), 1, 1);
  return cudaLaunchKernelEx(&cfg, hk_cluster_kernel<C>, base, off, n, nbins, slice, slice_mul, cnt);
}

cudaError_t launch_hist_keys(const uint32_t* keys, uint64_t n, uint32_t nbins, int container, void* counters,
                             bool wide, unsigned long long* out, const DevInfo& di, cudaStream_t s, uint64_t* nk,
                             KTimer* kt) {
  const bool smem = container == MR_C_SMEM_ARRAY;
  const uint64_t nb = (uint64_t)nbins + 1;
  cudaError_t e = cudaMemsetAsync(wide ? (void*)out : counters, 0, nb * (wide ? 8 : 4), s);
  if (e != cudaSuccess) return e;
  const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
  const uint4* base = reinterpret_cast<const uint4*>(addr & ~uintptr_t(15));
  const uint32_t off = (uint32_t)((addr & 15) / 4);
  const uint64_t groups = (n + off + 3) / 4;
  if (n) {
    if ((e = kt_begin(kt, s)) != cudaSuccess) return e;
    if (smem) {
      const int bytes = (int)(nb * 4);
      const int per_sm = bytes <= 48 * 1024 ? 2 : 1;
      uint64_t g = (groups + HK_SMEM_THREADS * 16 - 1) / (HK_SMEM_THREADS * 16);
      g = g < 1 ? 1 : g;
      g = g > (uint64_t)di.sms * per_sm ? (uint64_t)di.sms * per_sm : g;
      if (wide) {
        if ((e = cudaFuncSetAttribute(hk_smem_kernel<unsigned long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      bytes)) != cudaSuccess)
          return e;
        hk_smem_kernel<unsigned long long><<<(int)g, HK_SMEM_THREADS, bytes, s>>>(base, off, n, nbins, out);
      } else {
        if ((e = cudaFuncSetAttribute(hk_smem_kernel<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      bytes)) != cudaSuccess)
          return e;
        hk_smem_kernel<uint32_t><<<(int)g, HK_SMEM_THREADS, bytes, s>>>(base, off, n, nbins,
                                                                        static_cast<uint32_t*>(counters));
      }
    } else if (container == MR_C_CLUSTER_ARRAY) {
      e = wide ? launch_hk_cluster(base, off, n, nbins, out, di, s)
               : launch_hk_cluster(base, off, n, nbins, static_cast<uint32_t*>(counters), di, s);
      if (e != cudaSuccess) return e;
    } else {
      uint64_t g = (groups + HK_THREADS * 8 - 1) / (HK_THREADS * 8);
      g = g < 1 ? 1 : g;
      g = g > (uint64_t)di.sms * 8 ? (uint64_t)di.sms * 8 : g;
      if (wide)
        hk_global_kernel<unsigned long long><<<(int)g, HK_THREADS, 0, s>>>(base, off, n, nbins, out);
      else
        hk_global_kernel<uint32_t><<<(int)g, HK_THREADS, 0, s>>>(base, off, n, nbins, static_cast<uint32_t*>(counters));
    }
    if ((e = cudaGetLastError()) != cudaSuccess || (e = kt_end(kt, s)) != cudaSuccess) return e;
    ++*nk;
  }
  if (!wide) {
    uint64_t g = (nb + 1023) / 1024;
    g = g > (uint64_t)di.sms * 8 ? (uint64_t)di.sms * 8 : (g < 1 ? 1 : g);
    hk_widen_kernel<<<(int)g, 1024, 0, s>>>(static_cast<const uint32_t*>(counters), nb, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nk;
  }
  return cudaSuccess;
}

cudaError_t launch_bloom(const uint8_t* seq, uint64_t n, uint32_t L, uint64_t m, uint32_t h, uint32_t* bits,
                         const DevInfo& di, cudaStream_t s, uint64_t* nk, KTimer* kt) {
  const uint64_t words = (m + 31) / 32;
  cudaError_t e = cudaMemsetAsync(bits, 0, words * 4, s);
  if (e != cudaSuccess || n < L) return e;
  const uint64_t rm = ~0ull / m, rm1 = ~0ull / (m - 1);
  const uint64_t tiles = (n - L + 1 + BF_TILE - 1) / BF_TILE;
  uint64_t g = tiles < (uint64_t)di.sms * 8 ? tiles : (uint64_t)di.sms * 8;
  if ((e = kt_begin(kt, s)) != cudaSuccess) return e;
  bloom_kernel<<<(int)g, BF_THREADS, 0, s>>>(seq, n, L, m, rm, rm1, h, bits);
  if ((e = cudaGetLastError()) != cudaSuccess || (e = kt_end(kt, s)) != cudaSuccess) return e;
  ++*nk;
  return cudaSuccess;
}

}  // namespace mrgb
