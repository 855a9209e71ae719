/*
 * CPU ORACLE — test infrastructure only.
 *
 * Plain, serial, obviously-correct restatements of what each MapReduce job
 * computes.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg load this library; the product path (the CUDA library) never does, and
 * the two share no code, headers, tables or helpers.
 *
 * What the paper fixes (arXiv:1309.0215):
 *   - the MapReduce programming model (Sec. II-A "Programming model"): map is
 *     applied to every input element and emits intermediate key/value pairs,
 *     reduce folds all values of one key, and the result pairs may be ordered;
 *   - the basic workflow (Sec. II-A, Fig. 1): split -> map -> partition by key
 *     -> reduce -> merge -> output;
 *   - the two container kinds (Sec. III-A): a hash table for open-ended keys
 *     (Word Count) and an array for integer keys in a fixed range (Histogram).
 * Each function below therefore runs map over the input in order, groups by
 * key in a std::unordered_map or a plain array (the "container"), applies the
 * reduce (a sum) and, for word count, orders the output.
 *
 * The linear-regression and k-means jobs are not in the paper; their
 * definitions (five int64 sums; Lloyd iterations in FP64 with FP32 centroid
 * state) are the textbook ones.
 *
 * Parity pins (tests/test_oracle.py): brute force on tiny inputs in Python,
 * closed forms, exact rational nearest-centroid search, generator ground
 * truth and conservation invariants.  No function here is "parity unpinned".
 *
 * Build: g++ -O2 -std=c++17 -ffp-contract=off (no fused multiply-add, so the
 * FP64 sums are the same on every host).
 */
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>
#include <algorithm>

extern "C" {

/* 0 = ok, 1 = invalid argument, 2 = output buffer too small */

/* Word count (Sec. II-A programming model; Table I: hash-table container).
 * map: a token is a maximal run of bytes that are not ASCII whitespace
 * (space, \t, \n, \v, \f, \r); each token emits (token, 1).
 * reduce: sum of the values of one key.
 * output order: count descending, then key bytes ascending (unsigned,
 * a proper prefix first).
 * Output layout: u64 n_records, u64 n_key_bytes,
 *                n_records x {u64 count, u64 key_off, u64 key_len},
 *                key bytes concatenated in record order. */
static inline bool is_ws(uint8_t c) {
  return c == ' ' || c == '\t' || c == '\n' || c == '\v' || c == '\f' || c == '\r';
}

int oracle_wordcount(const uint8_t* text, uint64_t n, uint8_t* out, uint64_t out_cap, uint64_t* needed) {
  if (!text && n) return 1;
  std::unordered_map<std::string, uint64_t> container;
  uint64_t i = 0;
  while (i < n) {
    while (i < n && is_ws(text[i])) ++i;
    if (i >= n) break;
    uint64_t b = i;
    while (i < n && !is_ws(text[i])) ++i;
    container[std::string(reinterpret_cast<const char*>(text + b), i - b)] += 1;  // emit + combine
  }
  std::vector<std::pair<std::string, uint64_t>> recs(container.begin(), container.end());
  std::sort(recs.begin(), recs.end(), [](const auto& a, const auto& b) {
    if (a.second != b.second) return a.second > b.second;
    return a.first < b.first;  // char_traits<char>::lt compares as unsigned char
  });
  uint64_t kb = 0;
  for (auto& r : recs) kb += r.first.size();
  uint64_t total = 16 + 24 * (uint64_t)recs.size() + kb;
  if (needed) *needed = total;
  if (!out) return 0;
  if (out_cap < total) return 2;
  uint64_t hdr[2] = {(uint64_t)recs.size(), kb};
  std::memcpy(out, hdr, 16);
  uint64_t off = 0;
  uint8_t* rec = out + 16;
  uint8_t* keys = out + 16 + 24 * (uint64_t)recs.size();
  for (auto& r : recs) {
    uint64_t f[3] = {r.second, off, (uint64_t)r.first.size()};
    std::memcpy(rec, f, 24);
    rec += 24;
    std::memcpy(keys + off, r.first.data(), r.first.size());
    off += r.first.size();
  }
  return 0;
}

/* RGB histogram (Sec. II-A; Table I: array container).
 * Input: interleaved R,G,B bytes; map emits (channel c, value) for each
 * byte, key = c*256 + value; reduce sums.  bins[c*256 + v], u64. */
int oracle_hist_rgb8(const uint8_t* px, uint64_t n, uint64_t* bins) {
  if ((!px && n) || !bins || n % 3 != 0) return 1;
  for (int i = 0; i < 768; ++i) bins[i] = 0;
  for (uint64_t p = 0; p < n / 3; ++p)
    for (int c = 0; c < 3; ++c) bins[c * 256 + px[3 * p + c]] += 1;
  return 0;
}

/* Linear regression sums over int8 pairs (x = b[2i], y = b[2i+1]):
 * sums = {Σx, Σy, Σx², Σy², Σxy} in int64. */
int oracle_linreg_i8(const int8_t* xy, uint64_t n, int64_t* sums) {
  if ((!xy && n) || !sums || n % 2 != 0) return 1;
  int64_t sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0;
  for (uint64_t i = 0; i < n / 2; ++i) {
    int64_t x = xy[2 * i], y = xy[2 * i + 1];
    sx += x; sy += y; sxx += x * x; syy += y * y; sxy += x * y;
  }
  sums[0] = sx; sums[1] = sy; sums[2] = sxx; sums[3] = syy; sums[4] = sxy;
  return 0;
}

/* Large-key histogram (the Histogram application of Sec. IV: 16M unique
 * keys, 256M elements; array container of Sec. III-A, held as one global
 * array per Sec. III-E "eliminating local arrays").
 * map: element i is a u32 key and emits (key, 1); reduce: sum.
 * Output u64[nbins + 1]: out[k] = number of elements equal to k (k < nbins),
 * out[nbins] = number of elements >= nbins. */
int oracle_hist_u32(const uint32_t* keys, uint64_t n, uint32_t nbins, uint64_t* out) {
  if ((!keys && n) || !out || nbins == 0) return 1;
  std::vector<uint64_t> bins((size_t)nbins + 1, 0);
  for (uint64_t i = 0; i < n; ++i) {
    const uint32_t key = keys[i];
    bins[key < nbins ? key : nbins] += 1;
  }
  std::memcpy(out, bins.data(), bins.size() * sizeof(uint64_t));
  return 0;
}

/* The SplitMix64 output function (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as the Bloom filter's
 * base hash: applied to a state value it gives that state's output. */
uint64_t oracle_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Bloom-filter build (the Bloom Filter application of Sec. IV: 30M elements
 * into 300M entries, k-mers of a chromosome; array container, Sec. III-E).
 * Elements: every window of L consecutive bytes that are all in {A,C,G,T};
 * its code is the base-4 number of the window (A=0, C=1, G=2, T=3, first
 * base most significant), L <= 32.  Hashes (double hashing, Kirsch and
 * Mitzenmacher, ESA 2006): a = mix(code) mod m, b = 1 + mix(code ^
 * 0x9E3779B97F4A7C15) mod (m - 1); the element sets bits (a + i*b) mod m for
 * i = 0..h-1.  Output: ceil(m/8) bytes, bit j = bit (j mod 8) of byte j/8.
 * A window containing any other byte (N, lower case, newline) is skipped. */
static int base_code(uint8_t c) {
  switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'T': return 3;
    default: return -1;
  }
}

static void bloom_insert(uint64_t code, uint64_t m, uint32_t h, uint8_t* bits) {
  const uint64_t a = oracle_mix64(code) % m;
  const uint64_t b = 1 + oracle_mix64(code ^ 0x9E3779B97F4A7C15ull) % (m - 1);
  for (uint32_t i = 0; i < h; ++i) {
    const uint64_t j = (a + (uint64_t)i * b) % m;
    bits[j / 8] |= (uint8_t)(1u << (j % 8));
  }
}

int oracle_bloom_dna(const uint8_t* seq, uint64_t n, uint32_t L, uint64_t m, uint32_t h, uint8_t* bits) {
  if ((!seq && n) || !bits || L == 0 || L > 32 || m < 2 || m > (1ull << 32) || h == 0 || h > 32) return 1;
  std::memset(bits, 0, (size_t)((m + 7) / 8));
  for (uint64_t p = 0; p + L <= n; ++p) {
    uint64_t code = 0;
    bool ok = true;
    for (uint32_t j = 0; j < L; ++j) {
      const int v = base_code(seq[p + j]);
      if (v < 0) {
        ok = false;
        break;
      }
      code = code * 4 + (uint64_t)v;
    }
    if (ok) bloom_insert(code, m, h, bits);
  }
  return 0;
}

/* The same insertion for explicit element codes (used to pin the window
 * encoding from outside). */
int oracle_bloom_codes(const uint64_t* codes, uint64_t n, uint64_t m, uint32_t h, uint8_t* bits) {
  if ((!codes && n) || !bits || m < 2 || m > (1ull << 32) || h == 0 || h > 32) return 1;
  std::memset(bits, 0, (size_t)((m + 7) / 8));
  for (uint64_t i = 0; i < n; ++i) bloom_insert(codes[i], m, h, bits);
  return 0;
}

/* Hash computation for strings (Sec. III-C, Listing 1): a string is hashed
 * character by character, v = func(v, c).  The paper names FNV; this is
 * 64-bit FNV-1a (Fowler, Noll, Vo): v = 0xcbf29ce484222325, then for each
 * byte v = (v xor byte) * 0x100000001b3 mod 2^64.  Tokens are the word-count
 * tokens (maximal runs of non-whitespace bytes), in input order.  With
 * out_* null only *ntok is set. */
uint64_t oracle_fnv1a64(const uint8_t* s, uint64_t len) {
  uint64_t v = 0xcbf29ce484222325ull;
  for (uint64_t i = 0; i < len; ++i) v = (v ^ s[i]) * 0x100000001b3ull;
  return v;
}

int oracle_token_hashes(const uint8_t* text, uint64_t n, uint64_t* out_off, uint64_t* out_len, uint64_t* out_hash,
                        uint64_t cap, uint64_t* ntok) {
  if ((!text && n) || !ntok) return 1;
  uint64_t t = 0, i = 0;
  while (i < n) {
    while (i < n && is_ws(text[i])) ++i;
    if (i >= n) break;
    const uint64_t b = i;
    while (i < n && !is_ws(text[i])) ++i;
    if (out_off) {
      if (t >= cap) return 2;
      out_off[t] = b;
      out_len[t] = i - b;
      out_hash[t] = oracle_fnv1a64(text + b, i - b);
    }
    ++t;
  }
  *ntok = t;
  return 0;
}

/* Squared Euclidean distance in FP64: Σ_j (x_j - c_j)², j in order, no FMA. */
static double dist2_f64(const float* x, const float* c, uint32_t d) {
  double s = 0.0;
  for (uint32_t j = 0; j < d; ++j) {
    double t = (double)x[j] - (double)c[j];
    s += t * t;
  }
  return s;
}

/* k-means assignment step: a[i] = argmin_k dist2_f64(x_i, c_k); the lowest k
 * wins a tie.  Optionally returns the minimum distance per point. */
int oracle_kmeans_assign(const float* X, uint64_t n, uint32_t d, const float* C, uint32_t k,
                         int32_t* assign, double* dmin) {
  if ((!X && n) || !C || !assign || d == 0 || k == 0) return 1;
  for (uint64_t i = 0; i < n; ++i) {
    const float* x = X + i * d;
    double best = dist2_f64(x, C, d);
    int32_t bk = 0;
    for (uint32_t j = 1; j < k; ++j) {
      double v = dist2_f64(x, C + (uint64_t)j * d, d);
      if (v < best) { best = v; bk = (int32_t)j; }
    }
    assign[i] = bk;
    if (dmin) dmin[i] = best;
  }
  return 0;
}

/* k-means update step: for each cluster, the FP64 sum of its points (point
 * order) divided by its count, rounded to FP32; an empty cluster keeps its
 * previous centroid.  counts (optional) receives the cluster sizes. */
int oracle_kmeans_update(const float* X, uint64_t n, uint32_t d, const int32_t* assign, uint32_t k,
                         const float* C_prev, float* C_new, uint64_t* counts) {
  if ((!X && n) || !assign || !C_prev || !C_new || d == 0 || k == 0) return 1;
  std::vector<double> sum((uint64_t)k * d, 0.0);
  std::vector<uint64_t> cnt(k, 0);
  for (uint64_t i = 0; i < n; ++i) {
    int32_t a = assign[i];
    if (a < 0 || (uint32_t)a >= k) return 1;
    cnt[a] += 1;
    for (uint32_t j = 0; j < d; ++j) sum[(uint64_t)a * d + j] += (double)X[i * d + j];
  }
  for (uint32_t c = 0; c < k; ++c) {
    for (uint32_t j = 0; j < d; ++j) {
      uint64_t o = (uint64_t)c * d + j;
      C_new[o] = cnt[c] ? (float)(sum[o] / (double)cnt[c]) : C_prev[o];
    }
    if (counts) counts[c] = cnt[c];
  }
  return 0;
}

/* Lloyd's algorithm, a fixed number of iterations: each iteration assigns
 * every point to its nearest centroid, then recomputes the centroids.  The
 * returned assignments are those of the last iteration (made against the
 * centroids it started from). */
int oracle_kmeans(const float* X, uint64_t n, uint32_t d, const float* init, uint32_t k, uint32_t iters,
                  float* C_out, int32_t* assign_out) {
  if ((!X && n) || !init || !C_out || !assign_out || d == 0 || k == 0) return 1;
  std::vector<float> cur(init, init + (uint64_t)k * d), nxt((uint64_t)k * d);
  for (uint32_t t = 0; t < iters; ++t) {
    int rc = oracle_kmeans_assign(X, n, d, cur.data(), k, assign_out, nullptr);
    if (rc) return rc;
    rc = oracle_kmeans_update(X, n, d, assign_out, k, cur.data(), nxt.data(), nullptr);
    if (rc) return rc;
    cur.swap(nxt);
  }
  std::memcpy(C_out, cur.data(), sizeof(float) * (uint64_t)k * d);
  return 0;
}

}  // extern "C"
