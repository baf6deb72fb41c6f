/*
 * Seeded synthetic input generators shared by the oracle tests and the CUDA
 * path.  This file holds no threshold or counting arithmetic: it only draws
 * random bitmaps, position lists and query parameters.
 *
 * Random numbers: xoshiro256** (Blackman and Vigna, "Scrambled linear
 * pseudorandom number generators", 2018), each stream seeded by four outputs
 * of splitmix64 (Steele, Lea and Flood, 2014), both written from their
 * published definitions.  Stream s of seed S is seeded with
 * S + golden * (s + 1), so bitmaps can be generated in parallel and still be
 * deterministic.
 *
 * Bit layout of a dense bitmap (the paper's "Uncompressed Bitmaps", Sec. 2.1):
 * row i lives in 64-bit word i / 64 at bit position i % 64, least significant
 * bit first.  Rows >= r are never set.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9e3779b97f4a7c15ULL

typedef struct {
    uint64_t s[4];
} dg_rng;

static uint64_t splitmix64(uint64_t *state) {
    uint64_t z = (*state += GOLDEN);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(dg_rng *g) {
    uint64_t *s = g->s;
    const uint64_t out = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

static void rng_seed(dg_rng *g, uint64_t seed, uint64_t stream) {
    uint64_t sm = seed + GOLDEN * (stream + 1);
    for (int i = 0; i < 4; ++i) g->s[i] = splitmix64(&sm);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double rng_u01(dg_rng *g) { return (double)(rng_next(g) >> 11) * 0x1.0p-53; }

/* Number of failures before the first success of a Bernoulli(p) trial
 * sequence (inverse-CDF sampling), saturated at 2^62. */
static uint64_t rng_geometric0(dg_rng *g, double p) {
    if (p >= 1.0) return 0;
    double u = 1.0 - rng_u01(g); /* (0, 1] */
    double x = floor(log(u) / log1p(-p));
    if (!(x < 4.6e18)) return (uint64_t)1 << 62;
    return (uint64_t)x;
}

/* Fill `n` doubles uniform in [0, 1) from stream `stream`. */
void dg_uniform(uint64_t seed, uint64_t stream, uint64_t n, double *out) {
    dg_rng g;
    rng_seed(&g, seed, stream);
    for (uint64_t i = 0; i < n; ++i) out[i] = rng_u01(&g);
}

/* Raw 64-bit outputs of stream `stream` (used by tests of the generator). */
void dg_raw(uint64_t seed, uint64_t stream, uint64_t n, uint64_t *out) {
    dg_rng g;
    rng_seed(&g, seed, stream);
    for (uint64_t i = 0; i < n; ++i) out[i] = rng_next(&g);
}

/*
 * nbm bitmaps of r bits, bitmap k drawn i.i.d. Bernoulli(p[k]) per bit, by
 * geometric gaps between consecutive ones.  Bitmap k uses stream
 * stream0 + k and is written to out + k * stride_words; words beyond
 * ceil(r/64) up to stride_words are zeroed.
 */
void dg_bernoulli(uint64_t seed, uint64_t stream0, uint32_t nbm, uint64_t r_bits,
                  const double *p, uint64_t *out, uint64_t stride_words) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < (int64_t)nbm; ++k) {
        uint64_t *w = out + (uint64_t)k * stride_words;
        memset(w, 0, stride_words * sizeof(uint64_t));
        if (p[k] <= 0.0) continue;
        dg_rng g;
        rng_seed(&g, seed, stream0 + (uint64_t)k);
        uint64_t pos = rng_geometric0(&g, p[k]);
        while (pos < r_bits) {
            w[pos >> 6] |= (uint64_t)1 << (pos & 63);
            uint64_t gap = rng_geometric0(&g, p[k]);
            if (gap >= r_bits) break;
            pos += gap + 1;
        }
    }
}

/*
 * nbm bitmaps of r bits whose ones come in runs: repeatedly draw a start
 * uniform in [0, r) and a length 1 + Geometric0(1 / mean_len) (support >= 1,
 * mean mean_len), set the rows [start, min(start + len, r)), until the
 * bitmap holds at least round(density[k] * r) ones (the last run may
 * overshoot).  Bitmap k uses stream stream0 + k.
 */
void dg_runs(uint64_t seed, uint64_t stream0, uint32_t nbm, uint64_t r_bits,
             const double *density, double mean_len, uint64_t *out,
             uint64_t stride_words) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < (int64_t)nbm; ++k) {
        uint64_t *w = out + (uint64_t)k * stride_words;
        memset(w, 0, stride_words * sizeof(uint64_t));
        double target_d = floor(density[k] * (double)r_bits + 0.5);
        uint64_t target = target_d > (double)r_bits ? r_bits : (uint64_t)target_d;
        dg_rng g;
        rng_seed(&g, seed, stream0 + (uint64_t)k);
        uint64_t have = 0;
        const double p = 1.0 / mean_len;
        while (have < target) {
            uint64_t start = (uint64_t)(rng_u01(&g) * (double)r_bits);
            if (start >= r_bits) start = r_bits - 1;
            uint64_t len = 1 + rng_geometric0(&g, p);
            uint64_t end = start + len;
            if (end > r_bits || end < start) end = r_bits;
            for (uint64_t i = start; i < end; ++i) {
                uint64_t m = (uint64_t)1 << (i & 63);
                if (!(w[i >> 6] & m)) {
                    w[i >> 6] |= m;
                    ++have;
                }
            }
        }
    }
}

/*
 * Sorted positions of the ones of nbm bitmaps (r bits each, bitmap k at
 * words + k * stride_words).  Pass 1 (out == NULL) writes the list lengths to
 * offsets[1..nbm] as a running total with offsets[0] = 0; pass 2 (out != NULL)
 * writes list k to out[offsets[k] .. offsets[k+1]).  Representation change
 * only.
 */
void dg_positions(const uint64_t *words, uint32_t nbm, uint64_t stride_words,
                  uint64_t r_bits, uint64_t *offsets, uint32_t *out) {
    const uint64_t nw = (r_bits + 63) / 64;
    if (!out) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t k = 0; k < (int64_t)nbm; ++k) {
            const uint64_t *w = words + (uint64_t)k * stride_words;
            uint64_t n = 0;
            for (uint64_t j = 0; j < nw; ++j) {
                uint64_t x = w[j];
                while (x) {
                    uint64_t i = j * 64 + (uint64_t)__builtin_ctzll(x);
                    if (i < r_bits) ++n;
                    x &= x - 1;
                }
            }
            offsets[k + 1] = n;
        }
        offsets[0] = 0;
        for (uint32_t k = 0; k < nbm; ++k) offsets[k + 1] += offsets[k];
        return;
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t k = 0; k < (int64_t)nbm; ++k) {
        const uint64_t *w = words + (uint64_t)k * stride_words;
        uint32_t *o = out + offsets[k];
        for (uint64_t j = 0; j < nw; ++j) {
            uint64_t x = w[j];
            while (x) {
                uint64_t i = j * 64 + (uint64_t)__builtin_ctzll(x);
                if (i < r_bits) *o++ = (uint32_t)i;
                x &= x - 1;
            }
        }
    }
}

/*
 * k distinct integers from [0, n) (Floyd's sampling algorithm, as published
 * in Bentley and Floyd, CACM 1987), written in the order they are drawn.
 * Uses stream `stream`.  `seen` is caller scratch of n bytes.
 */
void dg_floyd(uint64_t seed, uint64_t stream, uint32_t n, uint32_t k, uint32_t *out,
              uint8_t *seen) {
    dg_rng g;
    rng_seed(&g, seed, stream);
    memset(seen, 0, n);
    uint32_t m = 0;
    for (uint32_t j = n - k; j < n; ++j) {
        uint32_t t = (uint32_t)(rng_u01(&g) * (double)(j + 1));
        if (t > j) t = j;
        if (seen[t]) t = j;
        seen[t] = 1;
        out[m++] = t;
    }
}
