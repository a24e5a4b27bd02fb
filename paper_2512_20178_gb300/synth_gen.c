/*
 * synth_gen.c -- fast seeded input generation for synth.py (inputs only: no unique-column sets,
 * no packing, no SpMM).  The same counter-based SplitMix64 stream as synth.py (Steele, Lea and
 * Flood, OOPSLA 2014): output i of stream (seed, s) is mix(state + (i + 1) * GAMMA) with
 * state = mix(seed * GAMMA + s).  Every element is computed from its own counter, so the result
 * does not depend on the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GAMMA 0x9E3779B97F4A7C15ULL

static const double TWO_PI = 6.283185307179586476925286766559;

static inline uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t stream_state(uint64_t seed, uint64_t stream) {
  return mix(seed * GAMMA + stream);
}

int synth_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* N(0, std^2) values by Box-Muller, two outputs per 64-bit draw: draw k gives outputs 2k and
 * 2k + 1 from u1 = (hi32 + 0.5) / 2^32 and u2 = (lo32 + 0.5) / 2^32. */
void synth_normal_f32(uint64_t seed, uint64_t stream, int64_t count, double std, float* out) {
  const uint64_t st = stream_state(seed, stream);
  const int64_t pairs = (count + 1) / 2;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < pairs; ++k) {
    const uint64_t z = mix(st + (uint64_t)(k + 1) * GAMMA);
    const double u1 = ((double)(z >> 32) + 0.5) * (1.0 / 4294967296.0);
    const double u2 = ((double)(z & 0xFFFFFFFFULL) + 0.5) * (1.0 / 4294967296.0);
    const double r = sqrt(-2.0 * log(u1)) * std;
    const double t = TWO_PI * u2;
    out[2 * k] = (float)(r * cos(t));
    if (2 * k + 1 < count) out[2 * k + 1] = (float)(r * sin(t));
  }
}

/* R-MAT edge samples start .. start + count - 1 as keys row * n + col (no dedup), most significant
 * bit first, one 32-bit uniform per level: level pair l2 uses stream base_stream + l2, the high
 * half for level 2*l2 and the low half for level 2*l2 + 1.  Quadrant by thresholds ta < tab < tabc
 * (a: top-left, b: top-right, c: bottom-left, d: bottom-right).  Samples with an endpoint >= n get
 * key -1 (rejected by the caller). */
void synth_rmat_keys(uint64_t seed, uint64_t base_stream, int32_t scale, int64_t n, int64_t start,
                     int64_t count, uint64_t ta, uint64_t tab, uint64_t tabc, int64_t* keys) {
  uint64_t st[32];
  const int pairs = (scale + 1) / 2;
  for (int l2 = 0; l2 < pairs && l2 < 32; ++l2) st[l2] = stream_state(seed, base_stream + l2);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) {
    int64_t r = 0, c = 0;
    const uint64_t ctr = (uint64_t)(start + i + 1) * GAMMA;
    for (int l2 = 0; l2 < pairs; ++l2) {
      const uint64_t z = mix(st[l2] + ctr);
      for (int half = 0; half < 2; ++half) {
        const int lvl = 2 * l2 + half;
        if (lvl >= scale) break;
        const uint64_t u = half == 0 ? (z >> 32) : (z & 0xFFFFFFFFULL);
        const int64_t rb = u >= tab;
        const int64_t cb = (u >= ta && u < tab) || u >= tabc;
        const int sh = scale - 1 - lvl;
        r |= rb << sh;
        c |= cb << sh;
      }
    }
    keys[i] = (r < n && c < n) ? r * n + c : -1;
  }
}

/* U[0,1) floats from the top 24 bits of outputs start .. start + count - 1. */
void synth_uniform_f32(uint64_t seed, uint64_t stream, int64_t start, int64_t count, float* out) {
  const uint64_t st = stream_state(seed, stream);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) {
    const uint64_t z = mix(st + (uint64_t)(start + i + 1) * GAMMA);
    out[i] = (float)(z >> 40) * (1.0f / 16777216.0f);
  }
}

static int cmp_i32(const void* a, const void* b) {
  const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* CSR pattern (rows ascending, columns ascending and distinct within a row) of the keys
 * row * n + col (keys < 0 are skipped; duplicates merged).  rowptr has n + 1 entries; col needs
 * room for `count` entries (the scratch of the bucket pass).  Returns the number of nonzeros. */
int64_t synth_keys_to_csr(const int64_t* keys, int64_t count, int64_t n, int64_t* rowptr,
                          int32_t* col) {
  for (int64_t i = 0; i <= n; ++i) rowptr[i] = 0;
  for (int64_t k = 0; k < count; ++k)
    if (keys[k] >= 0) rowptr[keys[k] / n + 1] += 1;
  for (int64_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) fill[i] = rowptr[i];
  for (int64_t k = 0; k < count; ++k)
    if (keys[k] >= 0) {
      const int64_t r = keys[k] / n;
      col[fill[r]++] = (int32_t)(keys[k] - r * n);
    }
  /* Sort and deduplicate each row in place; fill[i] becomes its distinct count. */
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    int32_t* c = col + rowptr[i];
    const int64_t len = rowptr[i + 1] - rowptr[i];
    if (len > 1) qsort(c, (size_t)len, sizeof(int32_t), cmp_i32);
    int64_t u = 0;
    for (int64_t j = 0; j < len; ++j)
      if (u == 0 || c[j] != c[u - 1]) c[u++] = c[j];
    fill[i] = u;
  }
  /* Compact the rows to the front. */
  int64_t w = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t s = rowptr[i];
    const int64_t u = fill[i];
    for (int64_t j = 0; j < u; ++j) col[w + j] = col[s + j];
    rowptr[i] = w;
    w += u;
  }
  rowptr[n] = w;
  free(fill);
  return w;
}

/* FP32 -> BF16 bit patterns, round to nearest with ties to even (finite inputs). */
void synth_f32_to_bf16(const uint32_t* in, int64_t count, uint16_t* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) {
    const uint32_t b = in[i];
    out[i] = (uint16_t)((b + 0x7FFFu + ((b >> 16) & 1u)) >> 16);
  }
}
