/*
 * ORACLE — test infrastructure only.  Nothing in the product path links,
 * loads or calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.
 *
 * A plain, slow, obviously correct CPU statement of what a threshold or
 * symmetric-function query over bitmaps computes (Kaser and Lemire, Sec. 1
 * "Formulation" and Sec. 2.2-2.3):
 *
 *   for every row i < r:  c_i = sum over k of bit i of bitmap ids[k]
 *   threshold query:      output bit i = [c_i >= theta]
 *   symmetric query:      output bit i = f(c_i), f given as bits 0..N
 *   cardinality:          number of ones in the output bitmap
 *   weighted threshold:   output bit i = [sum of weights[k] over inputs k
 *                         holding row i >= theta] (Sec. 2.3: a weight is the
 *                         number of copies of an input), then optionally
 *                         combined with one more bitmap by AND, OR or AND NOT
 *
 * A repeated id counts once per repeat (the paper's weighting by replication,
 * Sec. 2.3).  Rows >= r are never set in the output and input bits at rows
 * >= r are ignored.  Bit i of a bitmap is bit (i mod 64) of 64-bit word i/64
 * (Sec. 2.1, "Uncompressed Bitmaps").
 *
 * The counting is literal: one integer counter per row, incremented once per
 * input that has the row's bit set, then compared.  No word-level tricks.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Threads of the oracle's OpenMP loops (the host's cores by default). */
void oracle_set_threads(int n) {
    if (n > 0) omp_set_num_threads(n);
}

int oracle_get_threads(void) { return omp_get_max_threads(); }

static inline int oracle_bit(const uint64_t *words, uint64_t i) {
    return (int)((words[i / 64] >> (i % 64)) & 1u);
}

/* Number of ones among the first r bits of a bitmap, one bit at a time. */
uint64_t oracle_cardinality(const uint64_t *words, uint64_t r_bits) {
    uint64_t card = 0;
    for (uint64_t i = 0; i < r_bits; ++i) card += (uint64_t)oracle_bit(words, i);
    return card;
}

/*
 * Per-row counts c_i for rows [64*w0, min(64*w1, r)).  counts[i - 64*w0].
 * Bitmap ids[k] starts at base + ids[k] * stride_words.
 */
void oracle_counts(const uint64_t *base, uint64_t stride_words, const uint32_t *ids,
                   uint32_t n, uint64_t r_bits, uint64_t w0, uint64_t w1,
                   uint32_t *counts) {
    uint64_t row_end = w1 * 64 < r_bits ? w1 * 64 : r_bits;
#pragma omp parallel for schedule(static)
    for (int64_t i = (int64_t)(w0 * 64); i < (int64_t)row_end; ++i) {
        uint32_t c = 0;
        for (uint32_t k = 0; k < n; ++k)
            c += (uint32_t)oracle_bit(base + (uint64_t)ids[k] * stride_words, (uint64_t)i);
        counts[(uint64_t)i - w0 * 64] = c;
    }
}

/*
 * Output words w0..w1-1 of a symmetric query whose truth table is `table`
 * (bit c of the word array = f(c), c = 0..n) written to out[0 .. w1-w0), and
 * the number of ones among them in *card.
 */
void oracle_symmetric(const uint64_t *base, uint64_t stride_words, const uint32_t *ids,
                      uint32_t n, uint64_t r_bits, const uint64_t *table, uint64_t w0,
                      uint64_t w1, uint64_t *out, uint64_t *card) {
    uint64_t total = 0;
#pragma omp parallel for schedule(static) reduction(+ : total)
    for (int64_t w = (int64_t)w0; w < (int64_t)w1; ++w) {
        uint32_t counts[64];
        memset(counts, 0, sizeof counts);
        for (uint32_t k = 0; k < n; ++k) {
            const uint64_t *bm = base + (uint64_t)ids[k] * stride_words;
            for (int b = 0; b < 64; ++b) {
                uint64_t i = (uint64_t)w * 64 + (uint64_t)b;
                if (i < r_bits) counts[b] += (uint32_t)oracle_bit(bm, i);
            }
        }
        uint64_t word = 0;
        for (int b = 0; b < 64; ++b) {
            uint64_t i = (uint64_t)w * 64 + (uint64_t)b;
            if (i >= r_bits) continue;
            if (oracle_bit(table, counts[b])) {
                word |= (uint64_t)1 << b;
                total += 1;
            }
        }
        out[(uint64_t)w - w0] = word;
    }
    *card = total;
}

/*
 * Output words w0..w1-1 of the threshold query "at least theta of the n
 * inputs", and the number of ones among them.  theta = 0 selects every row;
 * theta > n selects none.
 */
void oracle_threshold(const uint64_t *base, uint64_t stride_words, const uint32_t *ids,
                      uint32_t n, uint64_t r_bits, uint64_t theta, uint64_t w0, uint64_t w1,
                      uint64_t *out, uint64_t *card) {
    uint64_t total = 0;
#pragma omp parallel for schedule(static) reduction(+ : total)
    for (int64_t w = (int64_t)w0; w < (int64_t)w1; ++w) {
        uint32_t counts[64];
        memset(counts, 0, sizeof counts);
        for (uint32_t k = 0; k < n; ++k) {
            const uint64_t *bm = base + (uint64_t)ids[k] * stride_words;
            for (int b = 0; b < 64; ++b) {
                uint64_t i = (uint64_t)w * 64 + (uint64_t)b;
                if (i < r_bits) counts[b] += (uint32_t)oracle_bit(bm, i);
            }
        }
        uint64_t word = 0;
        for (int b = 0; b < 64; ++b) {
            uint64_t i = (uint64_t)w * 64 + (uint64_t)b;
            if (i >= r_bits) continue;
            if ((uint64_t)counts[b] >= theta) {
                word |= (uint64_t)1 << b;
                total += 1;
            }
        }
        out[(uint64_t)w - w0] = word;
    }
    *card = total;
}

/*
 * ScanCount over sorted position lists (Sec. 4.2 and App. D): one counter per
 * row, every listed position increments its row's counter, then a final pass
 * compares each counter with theta (or looks f up).  List of bitmap id k is
 * positions[offsets[k] .. offsets[k+1]).  Only rows [64*w0, 64*w1) are
 * produced; positions outside that range are skipped.  `table` may be NULL
 * for a threshold query.
 */
void oracle_scancount(const uint32_t *positions, const uint64_t *offsets, const uint32_t *ids,
                      uint32_t n, uint64_t r_bits, uint64_t theta, const uint64_t *table,
                      uint64_t w0, uint64_t w1, uint64_t *out, uint64_t *card) {
    uint64_t row0 = w0 * 64;
    uint64_t row1 = w1 * 64 < r_bits ? w1 * 64 : r_bits;
    uint64_t nrows = row1 > row0 ? row1 - row0 : 0;
    uint32_t *counts = (uint32_t *)calloc(nrows ? nrows : 1, sizeof(uint32_t));
    for (uint32_t k = 0; k < n; ++k) {
        const uint32_t id = ids[k];
        for (uint64_t j = offsets[id]; j < offsets[id + 1]; ++j) {
            uint64_t p = positions[j];
            if (p >= row0 && p < row1) counts[p - row0] += 1;
        }
    }
    memset(out, 0, (w1 - w0) * sizeof(uint64_t));
    uint64_t total = 0;
    for (uint64_t i = 0; i < nrows; ++i) {
        int hit = table ? oracle_bit(table, counts[i]) : ((uint64_t)counts[i] >= theta);
        if (hit) {
            out[i / 64] |= (uint64_t)1 << (i % 64);
            total += 1;
        }
    }
    free(counts);
    *card = total;
}

/*
 * Weighted threshold (Sec. 2.3) with an optional combining step: for each row
 * i < r, w_i = sum of weights[k] over inputs k whose bit i is 1 (64-bit sum);
 * t_i = [w_i >= theta]; then out_i = t_i (post_op 0), t_i AND m_i (1),
 * t_i OR m_i (2) or t_i AND NOT m_i (3), m being the bitmap `post` (ignored
 * for post_op 0).  Output words w0..w1-1 and their number of ones.
 */
void oracle_weighted(const uint64_t *base, uint64_t stride_words, const uint32_t *ids,
                     const uint32_t *weights, uint32_t n, uint64_t r_bits, uint64_t theta,
                     uint32_t post_op, const uint64_t *post, uint64_t w0, uint64_t w1,
                     uint64_t *out, uint64_t *card) {
    uint64_t total = 0;
#pragma omp parallel for schedule(static) reduction(+ : total)
    for (int64_t w = (int64_t)w0; w < (int64_t)w1; ++w) {
        uint64_t word = 0;
        for (int b = 0; b < 64; ++b) {
            uint64_t i = (uint64_t)w * 64 + (uint64_t)b;
            if (i >= r_bits) continue;
            uint64_t sum = 0;
            for (uint32_t k = 0; k < n; ++k)
                if (oracle_bit(base + (uint64_t)ids[k] * stride_words, i)) sum += weights[k];
            int t = sum >= theta;
            if (post_op != 0) {
                int m = oracle_bit(post, i);
                if (post_op == 1) t = t && m;
                else if (post_op == 2) t = t || m;
                else t = t && !m;
            }
            if (t) {
                word |= (uint64_t)1 << b;
                total += 1;
            }
        }
        out[(uint64_t)w - w0] = word;
    }
    *card = total;
}
