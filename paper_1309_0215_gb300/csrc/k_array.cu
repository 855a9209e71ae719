// Array-container jobs: RGB8 histogram and int8 linear-regression sums.
//
// Paper mapping (arXiv:1309.0215):
//  - map + combiner (Sec. III-A): every input byte emits (key, 1) and is
//    combined at once into a local array;
//  - local arrays vs "eliminating local arrays" (Sec. III-E): with local
//    arrays each worker owns a private array that is merged into the global
//    array at the end; without them every emit is an atomic on the global
//    array.  Here a worker is a CTA and its local array lives in shared
//    memory; the "eliminated" form issues global atomics per emit.
//
// GB300 design of the local array (histogram): a CTA keeps 32 copies of the
// 768 bins laid out bin-major, [channel*256 + value][lane], one u32 column per
// lane index, shared by every warp of the CTA.  The word a lane touches is
// always in bank (lane), so a warp-wide update never has a bank conflict
// whatever the data skew, and updates from different warps are resolved by
// the shared-memory atomic unit.  The update is a fire-and-forget
// `red.shared.add.u32`.  Input is streamed with coalesced 128-bit
// non-allocating loads: a warp reads 1536 contiguous bytes (three 512-byte
// rows, 16 bytes per lane per row); 1536 is a multiple of 3, so the channel of
// every byte is a fixed rotation per (row, lane).
#include "mr_internal.h"
#include "dev_array.cuh"

namespace mrgb {
namespace {

using namespace arr;
constexpr int HIST_THREADS = 1024;

// One CTA's share of a histogram job (the grid strides over 1536-byte
// chunks): local array hs in shared memory, merged into bins at the end.
__device__ __forceinline__ void hist_smem_body(const uint8_t* __restrict__ in, uint64_t n,
                                               unsigned long long* __restrict__ bins, uint32_t* hs) {
  for (int i = threadIdx.x; i < HIST_WORDS; i += blockDim.x) hs[i] = 0;
  __syncthreads();

  const uint32_t lane = threadIdx.x & 31;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(hs);
  const uint32_t lb = sbase + lane * 4;

  // 16-byte aligned main region
  uint64_t o0 = (16 - ((uintptr_t)in & 15)) & 15;
  if (o0 > n) o0 = n;
  const uint64_t nchunks = (n - o0) / CHUNK;
  const uint4* vin = reinterpret_cast<const uint4*>(in + o0);

  const uint32_t rot0 = (uint32_t)((o0 + lane) % 3);
  uint32_t cb[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) cb[q] = lb + ((rot0 + q) % 3) * (256u * HIST_COLS * 4);

  const uint64_t w0 = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  uint64_t c = w0;
  for (; c + nw < nchunks; c += 2 * nw) {
    const uint4* p = vin + c * CHUNK_VEC + lane;
    const uint4* q = vin + (c + nw) * CHUNK_VEC + lane;
    uint4 a0 = ldg_stream(p), a1 = ldg_stream(p + 32), a2 = ldg_stream(p + 64);
    uint4 b0 = ldg_stream(q), b1 = ldg_stream(q + 32), b2 = ldg_stream(q + 64);
    hist_vec<0>(a0, cb);
    hist_vec<1>(a1, cb);
    hist_vec<2>(a2, cb);
    hist_vec<0>(b0, cb);
    hist_vec<1>(b1, cb);
    hist_vec<2>(b2, cb);
  }
  if (c < nchunks) {
    const uint4* p = vin + c * CHUNK_VEC + lane;
    uint4 a0 = ldg_stream(p), a1 = ldg_stream(p + 32), a2 = ldg_stream(p + 64);
    hist_vec<0>(a0, cb);
    hist_vec<1>(a1, cb);
    hist_vec<2>(a2, cb);
  }
  // unaligned head and ragged tail: the last CTA, byte by byte
  if (blockIdx.x == gridDim.x - 1) {
    const uint64_t tail0 = o0 + nchunks * CHUNK;
    const uint64_t nscalar = o0 + (n - tail0);
    for (uint64_t t = threadIdx.x; t < nscalar; t += blockDim.x) {
      uint64_t i = t < o0 ? t : tail0 + (t - o0);
      uint32_t ch = (uint32_t)(i % 3);
      red_shared_add(lb + ch * (256u * HIST_COLS * 4) + (uint32_t)in[i] * (HIST_COLS * 4), 1u);
    }
  }
  __syncthreads();
  // merge the local array into the global array (in the fused launch, once
  // the kernel that clears the results has finished)
  pdl_wait();
  for (int bin = threadIdx.x; bin < HIST_BINS; bin += blockDim.x) {
    unsigned long long s = 0;
#pragma unroll 8
    for (int l = 0; l < HIST_COLS; ++l) s += hs[bin * HIST_COLS + ((l + bin) & 31)];
    if (s) atomicAdd(bins + bin, s);
  }
}

__global__ void __launch_bounds__(HIST_THREADS, 1)
hist_smem_kernel(const uint8_t* __restrict__ in, uint64_t n, unsigned long long* __restrict__ bins) {
  extern __shared__ uint32_t hs[];
  hist_smem_body(in, n, bins, hs);
}

// "Eliminated local arrays": every emit is a 64-bit atomic on the global bins.
__global__ void hist_global_kernel(const uint8_t* __restrict__ in, uint64_t n, unsigned long long* __restrict__ bins) {
  uint64_t o0 = (16 - ((uintptr_t)in & 15)) & 15;
  if (o0 > n) o0 = n;
  const uint64_t nvec = (n - o0) / 16;
  const uint4* vin = reinterpret_cast<const uint4*>(in + o0);
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = tid; v < nvec; v += nth) {
    uint4 a = ldg_stream(vin + v);
    uint32_t w[4] = {a.x, a.y, a.z, a.w};
    uint32_t ch = (uint32_t)((o0 + 16 * v) % 3);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      uint32_t val = (w[j >> 2] >> (8 * (j & 3))) & 0xFFu;
      atomicAdd(bins + ch * 256 + val, 1ull);
      ch = ch == 2 ? 0 : ch + 1;
    }
  }
  const uint64_t tail0 = o0 + nvec * 16;
  const uint64_t nscalar = o0 + (n - tail0);
  for (uint64_t t = tid; t < nscalar; t += nth) {
    uint64_t i = t < o0 ? t : tail0 + (t - o0);
    atomicAdd(bins + (i % 3) * 256 + in[i], 1ull);
  }
}

// ------------------------------------------------------------- regression
// Σx, Σy, Σx², Σy², Σxy over int8 pairs with dp4a on 32-bit words holding
// two pairs [x0 y0 x1 y1].  Per-thread partials are int32 for at most
// LR_FLUSH vectors (|partial| <= 4096 * 4 words * 2 * 16384 < 2^31), then
// widened to int64.
constexpr int LR_THREADS = 512;
constexpr int LR_FLUSH = 4096;

__device__ __forceinline__ void block_add_sums(long long (&acc)[5], long long* out) {
  __shared__ long long part[32][5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    long long v = acc[i];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[warp][i] = v;
  }
  __syncthreads();
  if (warp == 0) {
    const int nwarps = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      long long v = lane < nwarps ? part[lane][i] : 0;
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && v) atomicAdd(reinterpret_cast<unsigned long long*>(out + i), (unsigned long long)v);
    }
  }
}

// One CTA's share of a regression job (the grid strides over 16-byte words).
__device__ __forceinline__ void linreg_body(const int8_t* __restrict__ in, uint64_t n, long long* __restrict__ sums) {
  long long acc[5] = {0, 0, 0, 0, 0};
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t npairs = n / 2;
  if (((uintptr_t)in & 1) == 0) {
    uint64_t o0 = (16 - ((uintptr_t)in & 15)) & 15;  // even
    if (o0 > n) o0 = n & ~1ull;
    const uint64_t nvec = (n - o0) / 16;
    const uint4* vin = reinterpret_cast<const uint4*>(in + o0);
    uint64_t v = tid;
    while (v < nvec) {
      int p[5] = {0, 0, 0, 0, 0};
      int it = 0;
      // eight 16-byte loads in flight per thread (four left the regression
      // alone at 0.75 of the HBM copy rate)
      for (; v + 7 * nth < nvec && it + 8 <= LR_FLUSH; v += 8 * nth, it += 8) {
        uint4 w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) w[u] = ldg_stream(vin + v + u * nth);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          lr_word(w[u].x, p);
          lr_word(w[u].y, p);
          lr_word(w[u].z, p);
          lr_word(w[u].w, p);
        }
      }
      for (; v < nvec && it < LR_FLUSH; v += nth, ++it) {
        uint4 a = ldg_stream(vin + v);
        lr_word(a.x, p); lr_word(a.y, p); lr_word(a.z, p); lr_word(a.w, p);
      }
#pragma unroll
      for (int i = 0; i < 5; ++i) acc[i] += p[i];
    }
    // head pairs [0, o0/2) and tail pairs from o0 + 16*nvec
    const uint64_t head = o0 / 2;
    const uint64_t tail0 = (o0 + nvec * 16) / 2;
    const uint64_t nscalar = head + (npairs - tail0);
    for (uint64_t t = tid; t < nscalar; t += nth) {
      uint64_t i = t < head ? t : tail0 + (t - head);
      long long x = in[2 * i], y = in[2 * i + 1];
      acc[0] += x; acc[1] += y; acc[2] += x * x; acc[3] += y * y; acc[4] += x * y;
    }
  } else {
    for (uint64_t i = tid; i < npairs; i += nth) {
      long long x = in[2 * i], y = in[2 * i + 1];
      acc[0] += x; acc[1] += y; acc[2] += x * x; acc[3] += y * y; acc[4] += x * y;
    }
  }
  pdl_wait();  // (fused launch: the results are cleared)
  block_add_sums(acc, sums);
}

__global__ void __launch_bounds__(LR_THREADS)
linreg_kernel(const int8_t* __restrict__ in, uint64_t n, long long* __restrict__ sums) {
  linreg_body(in, n, sums);
}

// Several independent array jobs (shared-memory histograms, regressions) as
// one launch: every CTA takes its share of each job in turn, so the GPU
// streams the jobs' inputs back to back, with one launch, one ramp and one
// tail instead of one per job, and no job's CTAs competing with another's
// for the SMs and HBM while both run.  The jobs' results are cleared by
// array_zero_kernel just before; the fused kernel is a programmatic dependent
// launch that reads and combines its inputs at once and waits for the
// clearing only before its first global add.
__global__ void array_zero_kernel(ArrayJobs J) {
  for (uint32_t i = 0; i < J.n; ++i) {
    unsigned long long* o = static_cast<unsigned long long*>(J.out[i]);
    const uint32_t words = J.kind[i] == MR_HIST_RGB8 ? 768u : 5u;
    for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) o[w] = 0ull;
  }
}

__global__ void __launch_bounds__(HIST_THREADS, 1) array_fused_kernel(ArrayJobs J) {
  extern __shared__ uint32_t hs[];
  for (uint32_t i = 0; i < J.n; ++i) {
    __syncthreads();  // the previous job's merge has read the local array
    if (J.kind[i] == MR_HIST_RGB8)
      hist_smem_body(J.in[i], J.bytes[i], static_cast<unsigned long long*>(J.out[i]), hs);
    else
      linreg_body(reinterpret_cast<const int8_t*>(J.in[i]), J.bytes[i], static_cast<long long*>(J.out[i]));
  }
}

}  // namespace

int hist_smem_bytes() { return HIST_WORDS * 4; }
int hist_block_threads() { return HIST_THREADS; }

cudaError_t launch_hist_smem(const uint8_t* in, uint64_t n, uint64_t* bins, int grid, cudaStream_t s) {
  static bool attr_done = false;  // per process; the attribute is per function
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(hist_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, HIST_WORDS * 4);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  if (grid < 1) grid = 1;
  hist_smem_kernel<<<grid, HIST_THREADS, HIST_WORDS * 4, s>>>(in, n, reinterpret_cast<unsigned long long*>(bins));
  return cudaGetLastError();
}

cudaError_t launch_hist_global(const uint8_t* in, uint64_t n, uint64_t* bins, int grid, cudaStream_t s) {
  if (grid < 1) grid = 1;
  hist_global_kernel<<<grid, 512, 0, s>>>(in, n, reinterpret_cast<unsigned long long*>(bins));
  return cudaGetLastError();
}

cudaError_t launch_array_fused(const ArrayJobs& jobs, int grid, cudaStream_t s) {
  static bool attr_done = false;  // per process; the attribute is per function
  if (!attr_done) {
    cudaError_t e =
        cudaFuncSetAttribute(array_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, HIST_WORDS * 4);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  if (grid < 1) grid = 1;
  array_zero_kernel<<<1, 256, 0, s>>>(jobs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_pdl(array_fused_kernel, dim3(grid), dim3(HIST_THREADS), (size_t)HIST_WORDS * 4, s, jobs);
}

cudaError_t launch_linreg(const int8_t* in, uint64_t n, int64_t* sums, int grid, cudaStream_t s) {
  if (grid < 1) grid = 1;
  linreg_kernel<<<grid, LR_THREADS, 0, s>>>(in, n, reinterpret_cast<long long*>(sums));
  return cudaGetLastError();
}

}  // namespace mrgb
