// Batched execution: many independent jobs of uneven sizes in ONE persistent
// launch.
//
// Every pending histogram / regression / word-count job is cut into fixed
// tiles (array jobs: a multiple of 1536 bytes; word count: a multiple of the
// 512-byte segment), and the tiles of all jobs are laid end to end in one
// tile space.  Persistent CTAs (one per SM) pull tile indices from a global
// atomic cursor, so large and small jobs share the GPU without per-job launch
// or tail costs.  A CTA keeps the local container of the job it is working on
// (the paper's combiner, Sec. III-A) across consecutive tiles of that job —
// lane-column shared-memory arrays for a histogram, registers for the
// regression sums, a CTA-shared hash table for word count — and
// merges it into the job's global container when it moves to a tile of
// another job and at the end.  The word-count jobs' merge and sort then run
// once for all of them (k_wordcount.cu, sort keyed by job).
//
// Per-job choices (tile sizes, histogram local arrays vs global atomics) come
// from the planner / autotuner in mr_api.cu.
#include "mr_internal.h"
#include "dev_array.cuh"
#include "dev_wordcount.cuh"

namespace mrgb {
namespace {

// 32 warps per CTA, one CTA per SM: the large-input word-count map kernel's
// shape.  A word-count tile runs as in that kernel: one local table per CTA
// shared by its warps (wc::CtaTableBig), each warp's misses queued and
// inserted 32 at a time, each warp's next segment loaded ahead.  Histogram
// tiles use 32 lane columns per bin (96 KiB), as the plain histogram kernel.
constexpr int BT = 1024;
constexpr int BWARPS = BT / 32;
constexpr int BCTAS = 1;                 // CTAs per SM
constexpr int BH_COLS = 32;              // histogram lane columns per bin
constexpr int BH_WORDS = arr::HIST_BINS * BH_COLS;
constexpr int B_SMEM_HIST = BH_WORDS * 4;
constexpr int B_SMEM_WC = (int)(sizeof(wc::CtaTableBig) + BWARPS * sizeof(wc::MapWarp));
constexpr int B_SMEM = B_SMEM_HIST > B_SMEM_WC ? B_SMEM_HIST : B_SMEM_WC;
static_assert(BCTAS * (B_SMEM + 1024) + 4096 <= 232448, "BCTAS batch CTAs must fit one SM's shared memory");

__device__ __forceinline__ uint32_t find_job(const BatchJob* jobs, uint32_t njobs, uint64_t t) {
  uint32_t lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile_begin <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void block_reduce_add5(long long (&acc)[5], long long* out, long long (*part)[5]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    long long v = acc[i];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[warp][i] = v;
    acc[i] = 0;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      long long v = lane < BWARPS ? part[lane][i] : 0;
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && v) atomicAdd(reinterpret_cast<unsigned long long*>(out + i), (unsigned long long)v);
    }
  }
  __syncthreads();
}

// Bytes before the first 16-byte aligned address of a job's input (at most n).
__device__ __forceinline__ uint64_t arr_head(const uint8_t* in, uint64_t n) {
  const uint64_t h = (16 - ((uintptr_t)in & 15)) & 15;
  return h < n ? h : n;
}

// histogram tile with local arrays.  Array tiles are counted from the job's
// first aligned address B = in + h: [t0, t1) is relative to B (t0 a multiple
// of 1536), and tile 0 also takes the h head bytes, so every tile streams
// aligned 128-bit loads whatever the input's alignment.  Byte k of B has
// channel (h + k) % 3, hence the rotation (h + lane) % 3.
__device__ void hist_tile_smem(const BatchJob& J, uint64_t h, uint64_t t0, uint64_t t1, bool first, uint32_t sbase) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lb = sbase + (lane % BH_COLS) * 4;
  const uint8_t* in = J.in;
  const uint8_t* B = in + h;
  const uint32_t rot0 = (uint32_t)((h + lane) % 3);
  uint32_t cb[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) cb[q] = lb + ((rot0 + q) % 3) * (256u * BH_COLS * 4);
  const uint64_t c0 = t0 / arr::CHUNK, c1 = t1 > t0 ? c0 + (t1 - t0) / arr::CHUNK : c0;
  const uint4* vin = reinterpret_cast<const uint4*>(B);
  uint64_t c = c0 + warp;
  for (; c + BWARPS < c1; c += BWARPS) {
    const uint4* p = vin + c * arr::CHUNK_VEC + lane;
    uint4 a0 = arr::ldg_stream(p), a1 = arr::ldg_stream(p + 32), a2 = arr::ldg_stream(p + 64);
    arr::hist_vec<0, BH_COLS>(a0, cb);
    arr::hist_vec<1, BH_COLS>(a1, cb);
    arr::hist_vec<2, BH_COLS>(a2, cb);
  }
  if (c < c1) {
    const uint4* p = vin + c * arr::CHUNK_VEC + lane;
    uint4 a0 = arr::ldg_stream(p), a1 = arr::ldg_stream(p + 32), a2 = arr::ldg_stream(p + 64);
    arr::hist_vec<0, BH_COLS>(a0, cb);
    arr::hist_vec<1, BH_COLS>(a1, cb);
    arr::hist_vec<2, BH_COLS>(a2, cb);
  }
  // ragged tail of the tile (job offsets h + [c1 * CHUNK, t1)) and, in tile 0, the head [0, h)
  const uint64_t tail0 = h + c1 * arr::CHUNK, tail1 = t1 > t0 ? h + t1 : tail0;
  const uint64_t nhead = first ? h : 0;
  for (uint64_t t = threadIdx.x; t < nhead + (tail1 - tail0); t += BT) {
    const uint64_t i = t < nhead ? t : tail0 + (t - nhead);
    arr::red_shared_add(lb + (uint32_t)(i % 3) * (256u * BH_COLS * 4) + (uint32_t)in[i] * (BH_COLS * 4), 1u);
  }
}

// histogram tile without local arrays: 64-bit atomics on the global bins
__device__ void hist_tile_global(const BatchJob& J, uint64_t t0, uint64_t t1) {
  unsigned long long* bins = static_cast<unsigned long long*>(J.out);
  for (uint64_t i = t0 + threadIdx.x; i < t1; i += BT) atomicAdd(bins + (i % 3) * 256 + J.in[i], 1ull);
}

// Regression tile.  With an even head h the tile is [t0, t1) relative to
// B = in + h (aligned 128-bit loads of whole pairs; tile 0 also takes the
// head); an odd-aligned input (h odd) keeps job offsets and reads bytes.
__device__ void linreg_tile(const BatchJob& J, uint64_t h, uint64_t t0, uint64_t t1, bool first, long long (&acc)[5]) {
  const int8_t* in = reinterpret_cast<const int8_t*>(J.in);
  uint64_t s0 = t0, s1 = t1;  // byte range still to do (job offsets)
  if ((h & 1) == 0) {
    const uint64_t v0 = t0 / 16, v1 = t1 > t0 ? t0 / 16 + (t1 - t0) / 16 : v0;  // t0 is a multiple of 16
    const uint4* vin = reinterpret_cast<const uint4*>(in + h);
    int p[5] = {0, 0, 0, 0, 0};  // at most a tile per flush: far below the int32 limit
    uint64_t v = v0 + threadIdx.x;
    // four 16-byte loads in flight per thread, then pairs
    for (; v + 3 * BT < v1; v += 4 * BT) {
      uint4 w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) w[u] = arr::ldg_stream(vin + v + u * BT);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        arr::lr_word(w[u].x, p);
        arr::lr_word(w[u].y, p);
        arr::lr_word(w[u].z, p);
        arr::lr_word(w[u].w, p);
      }
    }
    for (; v + BT < v1; v += 2 * BT) {
      uint4 a = arr::ldg_stream(vin + v);
      uint4 b = arr::ldg_stream(vin + v + BT);
      arr::lr_word(a.x, p); arr::lr_word(a.y, p); arr::lr_word(a.z, p); arr::lr_word(a.w, p);
      arr::lr_word(b.x, p); arr::lr_word(b.y, p); arr::lr_word(b.z, p); arr::lr_word(b.w, p);
    }
    if (v < v1) {
      uint4 a = arr::ldg_stream(vin + v);
      arr::lr_word(a.x, p); arr::lr_word(a.y, p); arr::lr_word(a.z, p); arr::lr_word(a.w, p);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) acc[i] += p[i];
    s0 = h + v1 * 16;
    s1 = t1 > t0 ? h + t1 : s0;
    if (first) {  // the head pairs [0, h)
      for (uint64_t i = threadIdx.x; 2 * i < h; i += BT) {
        const long long x = in[2 * i], y = in[2 * i + 1];
        acc[0] += x; acc[1] += y; acc[2] += x * x; acc[3] += y * y; acc[4] += x * y;
      }
    }
  }
  for (uint64_t i = s0 / 2 + threadIdx.x; 2 * i + 1 < s1; i += BT) {
    const long long x = in[2 * i], y = in[2 * i + 1];
    acc[0] += x; acc[1] += y; acc[2] += x * x; acc[3] += y * y; acc[4] += x * y;
  }
}

__global__ void __launch_bounds__(BT, BCTAS)
batch_kernel(const BatchJob* __restrict__ jobs, uint32_t njobs, uint64_t total_tiles, unsigned long long* cursor,
             uint64_t arr_tile, uint64_t wc_tile) {
  extern __shared__ __align__(16) unsigned char bsm[];
  __shared__ unsigned long long s_tile[2];
  __shared__ uint32_t s_job[2];
  __shared__ long long part[BWARPS][5];
  __shared__ wc::JobDev s_jd;  // the current word-count job
  uint32_t* hs = reinterpret_cast<uint32_t*>(bsm);
  wc::CtaTableBig& T = *reinterpret_cast<wc::CtaTableBig*>(bsm);
  wc::MapWarp& W = reinterpret_cast<wc::MapWarp*>(bsm + sizeof(wc::CtaTableBig))[threadIdx.x >> 5];
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(hs);
  const int lane = threadIdx.x & 31;
  int64_t cur = -1;
  uint32_t kind = 0, cont = 0;
  uint32_t qn = 0, qhd = 0;  // this warp's queued misses (word count)

  auto flush = [&](const BatchJob& J) {
    if (kind == MR_HIST_RGB8 && cont != MR_C_GLOBAL_ARRAY) {
      __syncthreads();
      unsigned long long* bins = static_cast<unsigned long long*>(J.out);
      for (int bin = threadIdx.x; bin < arr::HIST_BINS; bin += BT) {
        unsigned long long s = 0;
#pragma unroll 8
        for (int l = 0; l < BH_COLS; ++l) s += hs[bin * BH_COLS + ((l + bin) & (BH_COLS - 1))];
        if (s) atomicAdd(bins + bin, s);
      }
      __syncthreads();
    } else if (kind == MR_WORDCOUNT) {
      // every warp's queued misses, then the CTA's table, into the job's
      // global container
      __syncwarp();
      if ((uint32_t)lane < qn) {
        const uint32_t q = (qhd + (uint32_t)lane) & (wc::MQ - 1);
        wc::global_insert(s_jd, W.qw0[q], W.qw1[q], W.qh[q], 1);
      }
      qn = qhd = 0;
      __syncthreads();
      for (int i = threadIdx.x; i < wc::CtaTableBig::SLOTS; i += BT) {
        const ulonglong2 k = T.key[i];
        if (k.y != 0) wc::global_insert(s_jd, k.x, k.y, T.h[i], T.cnt[i]);
      }
      __syncthreads();
    }
  };
  auto init = [&](const BatchJob& J) {
    kind = J.kind;
    cont = J.container;
    if (kind == MR_HIST_RGB8 && cont != MR_C_GLOBAL_ARRAY) {
      for (int i = threadIdx.x; i < BH_WORDS; i += BT) hs[i] = 0;
      __syncthreads();
    } else if (kind == MR_WORDCOUNT) {
      if (threadIdx.x == 0) s_jd = J.wc;
      for (int i = threadIdx.x; i < wc::CtaTableBig::SLOTS; i += BT) T.key[i] = make_ulonglong2(0ull, 0ull);
      qn = qhd = 0;
      __syncthreads();
    }
  };

  for (int it = 0;; ++it) {
    const int b = it & 1;  // double-buffered broadcast: one barrier per tile
    if (threadIdx.x == 0) {
      const unsigned long long t = atomicAdd(cursor, 1ull);
      s_tile[b] = t;
      s_job[b] = t < total_tiles ? find_job(jobs, njobs, t) : 0xffffffffu;
    }
    __syncthreads();
    const uint64_t t = s_tile[b];
    if (t >= total_tiles) break;
    const uint32_t j = s_job[b];
    const BatchJob& J = jobs[j];
    if ((int64_t)j != cur) {
      if (cur >= 0) flush(jobs[cur]);
      init(J);
      cur = j;
    }
    const uint64_t local = t - J.tile_begin;
    if (J.kind == MR_WORDCOUNT) {
      const uint64_t s0 = local * (wc_tile / wc::SEG);
      uint64_t s1 = s0 + wc_tile / wc::SEG;
      const uint64_t nseg = (J.n + wc::SEG - 1) / wc::SEG;
      if (s1 > nseg) s1 = nseg;
      // the job's descriptor from shared memory (copied at the job switch):
      // through a reference to global memory every use in the hot loop would
      // be a global reload, and a register copy would not fit
      const uint64_t w0 = s0 + (threadIdx.x >> 5);
      uint4 pre[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
      bool have = w0 < s1 && wc::seg_prefetchable(s_jd, w0);
      if (have) wc::seg_prefetch(s_jd, w0, pre);
      for (uint64_t sg = w0; sg < s1; sg += BWARPS) {
        const uint64_t base = sg * wc::SEG;
        uint4 cp[2] = {pre[0], pre[1]};
        const bool cp_ok = have;
        have = sg + BWARPS < s1 && wc::seg_prefetchable(s_jd, sg + BWARPS);
        if (have) wc::seg_prefetch(s_jd, sg + BWARPS, pre);
        const int total = wc::stage_tokens(s_jd, sg, W, cp_ok ? cp : nullptr);
        for (int r0 = 0; r0 < total; r0 += 32) {
          const int i = r0 + lane;
          bool m = false;
          wc::Tok tk{0, 0, 0};
          if (i < total) {
            tk = wc::read_token(s_jd.in, s_jd.n, base, W, W.starts[i]);
            m = !wc::cta_add(T, tk);
          }
          wc::mq_push<1>(s_jd, W, m, tk, qn, qhd);
          __syncwarp();
        }
      }
    } else {
      const uint64_t t0 = local * arr_tile;
      if (J.kind == MR_HIST_RGB8 && cont == MR_C_GLOBAL_ARRAY) {
        hist_tile_global(J, t0, (t0 + arr_tile) < J.n ? t0 + arr_tile : J.n);
      } else {
        // tiles counted from the first aligned address (odd-aligned regression inputs: from the start)
        uint64_t h = arr_head(J.in, J.n);
        if (J.kind == MR_LINREG_I8 && (h & 1)) h = 0;
        const uint64_t bn = J.n - h;
        const uint64_t t1 = (t0 + arr_tile) < bn ? t0 + arr_tile : bn;
        if (J.kind == MR_HIST_RGB8) {
          hist_tile_smem(J, h, t0, t1, local == 0, sbase);
        } else {
          // sums reduced per tile: no registers stay reserved across tiles
          long long acc[5] = {0, 0, 0, 0, 0};
          linreg_tile(J, (((uintptr_t)J.in & 1) == 0) ? h : 1, t0, t1, local == 0, acc);
          block_reduce_add5(acc, static_cast<long long*>(J.out), part);
        }
      }
    }
  }
  if (cur >= 0) flush(jobs[cur]);
}

// Zero every container the batch accumulates into: histogram bins,
// regression sums, word-count tables and state words.  The containers are
// cut into chunks of BATCH_ZCHUNK bytes numbered across the jobs (zchunk0),
// so a large word-count table is cleared by many CTAs at once instead of one.
__device__ __forceinline__ uint32_t find_zjob(const BatchJob* jobs, uint32_t njobs, uint64_t c) {
  uint32_t lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (jobs[mid].zchunk0 <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ uint64_t zero_bytes(const BatchJob& J) {
  return J.kind == MR_WORDCOUNT ? J.wc.cap * 24 : (J.kind == MR_HIST_RGB8 ? 768 * 8 : 48);
}
__global__ void batch_init_kernel(const BatchJob* __restrict__ jobs, uint32_t njobs, uint64_t nchunks) {
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const BatchJob& J = jobs[find_zjob(jobs, njobs, c)];
    const uint64_t off = (c - J.zchunk0) * BATCH_ZCHUNK;
    const uint64_t bytes = zero_bytes(J);
    if (off >= bytes) continue;
    const uint64_t end = off + BATCH_ZCHUNK < bytes ? off + BATCH_ZCHUNK : bytes;
    uint4* p = static_cast<uint4*>(J.kind == MR_WORDCOUNT ? static_cast<void*>(J.wc.key) : J.out);
    for (uint64_t i = off / 16 + threadIdx.x; i < end / 16; i += blockDim.x) p[i] = make_uint4(0, 0, 0, 0);
    if (J.kind == MR_WORDCOUNT && off == 0)
      for (uint32_t i = threadIdx.x; i < 64 / 4; i += blockDim.x) J.wc.state[i] = 0;
  }
}

}  // namespace

uint64_t batch_zero_chunks(uint32_t kind, uint64_t wc_cap) {
  const uint64_t bytes = kind == MR_WORDCOUNT ? wc_cap * 24 : (kind == MR_HIST_RGB8 ? 768 * 8 : 48);
  return (bytes + BATCH_ZCHUNK - 1) / BATCH_ZCHUNK;
}

uint64_t batch_tiles_for(uint32_t kind, uint64_t n, uint64_t arr_tile, uint64_t wc_tile) {
  const uint64_t t = kind == MR_WORDCOUNT ? wc_tile : arr_tile;
  return (n + t - 1) / t;
}

cudaError_t batch_prepare() {
  return cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SMEM);
}

cudaError_t launch_batch(const BatchJob* jobs_dev, uint32_t njobs, uint64_t total_tiles, unsigned long long* cursor,
                         uint64_t arr_tile, uint64_t wc_tile, uint64_t total_zchunks, const DevInfo& di,
                         cudaStream_t s, uint64_t* nk) {
  cudaError_t e;
  batch_init_kernel<<<di.sms * 4, 256, 0, s>>>(jobs_dev, njobs, total_zchunks);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(cursor, 0, 8, s)) != cudaSuccess) return e;
  uint64_t grid = (uint64_t)BCTAS * di.sms;
  if (grid > total_tiles) grid = total_tiles ? total_tiles : 1;
  batch_kernel<<<(unsigned)grid, BT, B_SMEM, s>>>(jobs_dev, njobs, total_tiles, cursor, arr_tile, wc_tile);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *nk += 2;
  return cudaSuccess;
}

}  // namespace mrgb
