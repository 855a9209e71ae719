/*
 * Seeded synthetic input generators for the four job kinds (word count text,
 * interleaved RGB8 image, int8 (x,y) regression pairs, Gaussian-mixture points).
 *
 * This module only PRODUCES inputs.  It contains none of the map/reduce
 * arithmetic (no tokenising, counting, hashing or summing of the data it
 * writes); the oracle and the CUDA path both consume its output.
 *
 * Randomness: xoshiro256** (Blackman & Vigna, 2018) seeded through SplitMix64
 * (Steele, Lea & Flood, 2014).  Large outputs are cut into fixed chunks, each
 * with its own stream derived from (seed, chunk index), so the bytes do not
 * depend on the number of threads used.  Normals use the Marsaglia polar
 * method on top of the uniform stream.
 *
 * Portable C11 + pthreads: no intrinsics, no reliance on char signedness.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

typedef struct { uint64_t s[4]; int have_spare; double spare; } rng_t;

static uint64_t splitmix64(uint64_t* x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static void rng_seed(rng_t* r, uint64_t seed, uint64_t stream) {
  uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ull + 0x8CB92BA72F3D8DD7ull);
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
  r->have_spare = 0;
  r->spare = 0.0;
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(rng_t* r) {
  uint64_t* s = r->s;
  uint64_t result = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl(s[3], 45);
  return result;
}

/* uniform double in [0, 1) with 53 random bits */
static inline double rng_u01(rng_t* r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, n), Lemire's multiply-shift with rejection (unbiased) */
static inline uint32_t rng_below(rng_t* r, uint32_t n) {
  uint64_t m = (rng_next(r) >> 32) * (uint64_t)n;
  uint32_t lo = (uint32_t)m;
  if (lo < n) {
    uint32_t t = (uint32_t)(-n) % n;
    while (lo < t) {
      m = (rng_next(r) >> 32) * (uint64_t)n;
      lo = (uint32_t)m;
    }
  }
  return (uint32_t)(m >> 32);
}

/* standard normal, Marsaglia polar method */
static double rng_normal(rng_t* r) {
  if (r->have_spare) { r->have_spare = 0; return r->spare; }
  double u, v, s;
  do {
    u = 2.0 * rng_u01(r) - 1.0;
    v = 2.0 * rng_u01(r) - 1.0;
    s = u * u + v * v;
  } while (s >= 1.0 || s == 0.0);
  double f = sqrt(-2.0 * log(s) / s);
  r->spare = v * f;
  r->have_spare = 1;
  return u * f;
}

static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ------------------------------------------------------------------ */
/* chunked parallel driver                                             */
/* ------------------------------------------------------------------ */
typedef void (*chunk_fn)(void* ctx, uint64_t chunk, uint64_t begin, uint64_t end);
typedef struct { chunk_fn fn; void* ctx; uint64_t n, chunk, nchunks; int tid, nthreads; } job_t;

static void* worker(void* p) {
  job_t* j = (job_t*)p;
  for (uint64_t c = (uint64_t)j->tid; c < j->nchunks; c += (uint64_t)j->nthreads) {
    uint64_t b = c * j->chunk, e = b + j->chunk;
    if (e > j->n) e = j->n;
    j->fn(j->ctx, c, b, e);
  }
  return NULL;
}

static void run_chunks(chunk_fn fn, void* ctx, uint64_t n, uint64_t chunk, int nthreads) {
  uint64_t nchunks = (n + chunk - 1) / chunk;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 64) nthreads = 64;
  if ((uint64_t)nthreads > nchunks) nthreads = nchunks ? (int)nchunks : 1;
  job_t jobs[64];
  pthread_t th[64];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].n = n; jobs[t].chunk = chunk;
    jobs[t].nchunks = nchunks; jobs[t].tid = t; jobs[t].nthreads = nthreads;
  }
  int started = 0;
  for (int t = 1; t < nthreads; ++t) {
    if (pthread_create(&th[t], NULL, worker, &jobs[t]) != 0) break;
    started = t;
  }
  worker(&jobs[0]);
  for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
  /* chunks of threads that failed to start are done serially */
  for (int t = started + 1; t < nthreads; ++t) worker(&jobs[t]);
}

#define CHUNK (1ull << 20)

/* ------------------------------------------------------------------ */
/* RGB8 image: per pixel, with probability p_uniform three independent */
/* uniform bytes; otherwise one of n_clusters colour clusters whose     */
/* channel value is clamp(round(centre + sigma * N(0,1)), 0, 255).      */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t seed; double p_uniform; uint32_t ncl; double sigma; int centre[64][3]; uint8_t* out; } hist_ctx;

static void hist_chunk(void* p, uint64_t chunk, uint64_t b, uint64_t e) {
  hist_ctx* c = (hist_ctx*)p;
  rng_t r; rng_seed(&r, c->seed, chunk + 1);
  for (uint64_t i = b; i < e; ++i) {
    uint8_t* px = c->out + 3 * i;
    if (c->ncl == 0 || rng_u01(&r) < c->p_uniform) {
      uint64_t w = rng_next(&r);
      px[0] = (uint8_t)(w >> 8); px[1] = (uint8_t)(w >> 24); px[2] = (uint8_t)(w >> 40);
    } else {
      uint32_t k = rng_below(&r, c->ncl);
      for (int ch = 0; ch < 3; ++ch) {
        double v = (double)c->centre[k][ch] + c->sigma * rng_normal(&r);
        px[ch] = (uint8_t)clampi((int)lround(v), 0, 255);
      }
    }
  }
}

int synth_hist_rgb8(uint64_t seed, uint64_t n_pixels, double p_uniform, uint32_t n_clusters,
                    double sigma, uint8_t* out, int nthreads) {
  if (!out && n_pixels) return 1;
  if (n_clusters > 64) return 1;
  hist_ctx c;
  c.seed = seed; c.p_uniform = p_uniform; c.ncl = n_clusters; c.sigma = sigma; c.out = out;
  rng_t r; rng_seed(&r, seed, 0);
  for (uint32_t k = 0; k < n_clusters; ++k)
    for (int ch = 0; ch < 3; ++ch) c.centre[k][ch] = (int)rng_below(&r, 256);
  run_chunks(hist_chunk, &c, n_pixels, CHUNK, nthreads);
  return 0;
}

/* ------------------------------------------------------------------ */
/* int8 regression pairs: x uniform on [xmin, xmax], y = clamp(slope*x +  */
/* round(sigma * N(0,1)), -128, 127); stored interleaved x0 y0 x1 y1 ...  */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t seed; int xmin, xmax, slope; double sigma; int8_t* out; } lr_ctx;

static void lr_chunk(void* p, uint64_t chunk, uint64_t b, uint64_t e) {
  lr_ctx* c = (lr_ctx*)p;
  rng_t r; rng_seed(&r, c->seed, chunk + 1);
  uint32_t span = (uint32_t)(c->xmax - c->xmin + 1);
  for (uint64_t i = b; i < e; ++i) {
    int x = c->xmin + (int)rng_below(&r, span);
    int y = c->slope * x + (int)lround(c->sigma * rng_normal(&r));
    c->out[2 * i] = (int8_t)clampi(x, -128, 127);
    c->out[2 * i + 1] = (int8_t)clampi(y, -128, 127);
  }
}

int synth_linreg_i8(uint64_t seed, uint64_t n_pairs, int xmin, int xmax, int slope, double sigma,
                    int8_t* out, int nthreads) {
  if ((!out && n_pairs) || xmax < xmin) return 1;
  lr_ctx c = {seed, xmin, xmax, slope, sigma, out};
  run_chunks(lr_chunk, &c, n_pairs, CHUNK, nthreads);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Gaussian mixture: ncomp means uniform in [lo, hi]^d; each point picks */
/* a component uniformly and adds sigma * N(0,1) per coordinate (FP32).  */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t seed; uint32_t d, ncomp; double sigma; const double* means; float* out; int32_t* comp; } km_ctx;

static void km_chunk(void* p, uint64_t chunk, uint64_t b, uint64_t e) {
  km_ctx* c = (km_ctx*)p;
  rng_t r; rng_seed(&r, c->seed, chunk + 1);
  for (uint64_t i = b; i < e; ++i) {
    uint32_t k = rng_below(&r, c->ncomp);
    if (c->comp) c->comp[i] = (int32_t)k;
    const double* mu = c->means + (uint64_t)k * c->d;
    float* x = c->out + i * c->d;
    for (uint32_t j = 0; j < c->d; ++j) x[j] = (float)(mu[j] + c->sigma * rng_normal(&r));
  }
}

int synth_kmeans_f32(uint64_t seed, uint64_t n, uint32_t d, uint32_t ncomp, double lo, double hi,
                     double sigma, float* out, int32_t* comp_out, double* means_out, int nthreads) {
  if ((!out && n) || d == 0 || ncomp == 0 || !means_out) return 1;
  rng_t r; rng_seed(&r, seed, 0);
  for (uint64_t i = 0; i < (uint64_t)ncomp * d; ++i) means_out[i] = lo + (hi - lo) * rng_u01(&r);
  km_ctx c = {seed, d, ncomp, sigma, means_out, out, comp_out};
  /* 4096 points per chunk keeps chunk sizes moderate for any d */
  run_chunks(km_chunk, &c, n, 4096, nthreads);
  return 0;
}

/* ------------------------------------------------------------------ */
/* u32 keys for the large-key histogram.                                */
/* dist 0: uniform on [0, nbins).                                       */
/* dist 1: skewed: rank j = min(floor((nbins + 1)^u) - 1, nbins - 1)     */
/* with u uniform on [0, 1), so P(j) falls off roughly like 1/(j + 1)   */
/* (a continuous stand-in for Zipf, s = 1); ranks are spread over the   */
/* key range by j -> (j * 2654435761) mod nbins, a bijection because    */
/* 2654435761 is prime and larger than any u32 nbins it could divide.   */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t seed; uint32_t nbins; int dist; double lg; uint32_t* out; } keys_ctx;

static void keys_chunk(void* p, uint64_t chunk, uint64_t b, uint64_t e) {
  keys_ctx* c = (keys_ctx*)p;
  rng_t r; rng_seed(&r, c->seed, chunk + 1);
  for (uint64_t i = b; i < e; ++i) {
    if (c->dist == 0) {
      c->out[i] = rng_below(&r, c->nbins);
    } else {
      double v = floor(exp(rng_u01(&r) * c->lg)) - 1.0;
      uint64_t j = v < 0.0 ? 0 : (uint64_t)v;
      if (j > c->nbins - 1) j = c->nbins - 1;
      c->out[i] = (uint32_t)((j * 2654435761ull) % c->nbins);
    }
  }
}

int synth_keys_u32(uint64_t seed, uint64_t n, uint32_t nbins, int dist, uint32_t* out, int nthreads) {
  if ((!out && n) || nbins == 0 || dist < 0 || dist > 1) return 1;
  keys_ctx c = {seed, nbins, dist, log((double)nbins + 1.0), out};
  run_chunks(keys_chunk, &c, n, CHUNK, nthreads);
  return 0;
}

/* ------------------------------------------------------------------ */
/* DNA sequence for the Bloom-filter build: bases 'A','C','G','T'       */
/* uniform and independent; optionally n_runs runs of 'N' (length      */
/* uniform on [1, max_run]) written over uniformly drawn positions, as  */
/* assemblies carry gaps.                                               */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t seed; uint8_t* out; } dna_ctx;

static void dna_chunk(void* p, uint64_t chunk, uint64_t b, uint64_t e) {
  dna_ctx* c = (dna_ctx*)p;
  static const uint8_t base[4] = {'A', 'C', 'G', 'T'};
  rng_t r; rng_seed(&r, c->seed, chunk + 1);
  uint64_t i = b;
  while (i < e) {
    uint64_t w = rng_next(&r);
    for (int q = 0; q < 32 && i < e; ++q, ++i) c->out[i] = base[(w >> (2 * q)) & 3];
  }
}

int synth_dna(uint64_t seed, uint64_t n, uint32_t n_runs, uint32_t max_run, uint8_t* out, int nthreads) {
  if ((!out && n) || (n_runs && (max_run == 0 || n == 0))) return 1;
  dna_ctx c = {seed, out};
  run_chunks(dna_chunk, &c, n, CHUNK, nthreads);
  rng_t r; rng_seed(&r, seed, 0xDA7Aull);
  for (uint32_t k = 0; k < n_runs; ++k) {
    uint64_t at = rng_next(&r) % n;
    uint32_t len = 1 + rng_below(&r, max_run);
    for (uint32_t j = 0; j < len && at + j < n; ++j) out[at + j] = 'N';
  }
  return 0;
}

/* k distinct indices in [0, n) by a partial Fisher-Yates shuffle; scratch holds n u32 */
int synth_sample_distinct(uint64_t seed, uint32_t n, uint32_t k, uint32_t* scratch, uint32_t* out) {
  if (k > n || !scratch || !out) return 1;
  rng_t r; rng_seed(&r, seed, 0xFEEDull);
  for (uint32_t i = 0; i < n; ++i) scratch[i] = i;
  for (uint32_t i = 0; i < k; ++i) {
    uint32_t j = i + rng_below(&r, n - i);
    uint32_t t = scratch[i]; scratch[i] = scratch[j]; scratch[j] = t;
    out[i] = scratch[i];
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Word-count text.                                                     */
/* Vocabulary candidates: length uniform on [minlen, maxlen], letters   */
/* uniform on 'a'..'z'.  The caller removes duplicates (rejection) and   */
/* keeps drawing until it has enough distinct words.                     */
/* ------------------------------------------------------------------ */
int synth_wc_candidates(uint64_t seed, uint64_t stream, uint32_t count, uint32_t minlen, uint32_t maxlen,
                        uint8_t* buf /* count * maxlen */, uint32_t* lens) {
  if (minlen == 0 || maxlen < minlen || !buf || !lens) return 1;
  rng_t r; rng_seed(&r, seed, 0x5EED0000ull + stream);
  for (uint32_t i = 0; i < count; ++i) {
    uint32_t L = minlen + rng_below(&r, maxlen - minlen + 1);
    lens[i] = L;
    for (uint32_t j = 0; j < L; ++j) buf[(uint64_t)i * maxlen + j] = (uint8_t)('a' + rng_below(&r, 26));
  }
  return 0;
}

/*
 * Zipf text.  cdf[r] (r = 0..nvocab-1) is the cumulative probability of ranks
 * 0..r; a draw u in [0,1) selects the first rank with cdf > u.  Words are
 * separated by ' ', except that after every n-th word (n uniform on
 * [nl_min, nl_max], redrawn after each newline) the separator is '\n'.
 * Words are appended while word + separator still leave room for one final
 * byte; the rest of the buffer (at least one byte) is filled with '\n'.
 * ranks_out (optional) receives the rank of every emitted word in order.
 * Returns the number of words emitted, or -1 on bad arguments / small ranks_cap.
 */
int64_t synth_wc_text(uint64_t seed, const uint8_t* vocab, const uint64_t* voff, const uint32_t* vlen,
                      uint32_t nvocab, const double* cdf, uint64_t nbytes, uint32_t nl_min, uint32_t nl_max,
                      uint8_t* out, uint32_t* ranks_out, uint64_t ranks_cap) {
  if (!vocab || !voff || !vlen || !cdf || !out || nvocab == 0 || nl_min == 0 || nl_max < nl_min) return -1;
  if (nbytes == 0) return 0;
  rng_t r; rng_seed(&r, seed, 0x7E47ull);
  uint64_t pos = 0, nw = 0;
  uint32_t until_nl = nl_min + rng_below(&r, nl_max - nl_min + 1);
  for (;;) {
    double u = rng_u01(&r);
    uint32_t lo = 0, hi = nvocab - 1;
    while (lo < hi) {
      uint32_t mid = lo + (hi - lo) / 2;
      if (cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    uint32_t L = vlen[lo];
    if (pos + L + 1 > nbytes - 1) break;
    memcpy(out + pos, vocab + voff[lo], L);
    pos += L;
    if (--until_nl == 0) {
      out[pos++] = '\n';
      until_nl = nl_min + rng_below(&r, nl_max - nl_min + 1);
    } else {
      out[pos++] = ' ';
    }
    if (ranks_out) {
      if (nw >= ranks_cap) return -1;
      ranks_out[nw] = lo;
    }
    ++nw;
  }
  while (pos < nbytes) out[pos++] = '\n';
  return (int64_t)nw;
}
