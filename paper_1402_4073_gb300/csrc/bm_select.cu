// Per-query kernel choice: features, fixed rule, learned selector.
#include <algorithm>
#include <cmath>

#include "bm_select.h"

namespace bm {

const Candidate kCandidateTable[kCandidates] = {{BM_PATH_DENSE, 0, 0},
                                                {BM_PATH_SPARSE, 16384, 0},
                                                {BM_PATH_SPARSE, 32768, 0},
                                                {BM_PATH_SPARSE, 65536, 0},
                                                {BM_PATH_DENSE, 0, 1},
                                                {BM_PATH_RLE, 0, 0}};

void query_features(const bm_pool* p, const uint32_t* ids, uint32_t n,
                    const std::vector<uint8_t>& f, float out[kFeatures]) {
    double sum = 0.0, mx = 0.0;
    for (uint32_t k = 0; k < n; ++k) {
        const double d = (double)p->card[ids[k]] / (double)p->r_bits;
        sum += d;
        mx = d > mx ? d : mx;
    }
    uint32_t first = 0;  // first count where f changes (0 if f is constant)
    for (uint32_t c = 1; c <= n; ++c)
        if ((f[c] != 0) != (f[c - 1] != 0)) {
            first = c;
            break;
        }
    out[0] = (float)std::log2((double)n);
    out[1] = (float)((double)first / (double)n);
    out[2] = (float)std::log10(std::max(sum / n, 1e-9));
    out[3] = (float)std::log10(std::max(mx, 1e-9));
    out[4] = (float)std::log2((double)p->r_bits);
    // run-length forms: summaries (8 bytes per input and tile) and containers
    bool rle = true;
    uint64_t units = 0;
    for (uint32_t k = 0; k < n && rle; ++k) {
        rle = p->rle_present[ids[k]] != 0;
        if (rle) units += p->rle_units[ids[k]];
    }
    const double tiles = (double)((p->words + kRleTileWords - 1) / kRleTileWords);
    const double rle_bytes = 16.0 * (double)units + 8.0 * (double)n * tiles;
    const double dense_bytes = (double)n * (double)p->r_bits / 8.0;
    out[5] = rle ? (float)std::log2(std::max(rle_bytes, 1.0) / std::max(dense_bytes, 1.0)) : 0.f;
}

static bool all_have(const std::vector<uint8_t>& present, const uint32_t* ids, uint32_t n) {
    for (uint32_t k = 0; k < n; ++k)
        if (!present[ids[k]]) return false;
    return true;
}

int pick_candidate(const bm_pool* p, const uint32_t* ids, uint32_t n, const float* y,
                   float dense_discount) {
    const bool lists = all_have(p->list_present, ids, n);
    const bool dense = all_have(p->dense_present, ids, n);
    const bool rle = all_have(p->rle_present, ids, n);
    int best = -1, rle_c = -1;
    for (int c = 0; c < kCandidates; ++c) {
        const Candidate& k = kCandidateTable[c];
        if (k.path == BM_PATH_RLE) {
            if (rle) rle_c = c;
            continue;
        }
        if ((k.path == BM_PATH_DENSE && !dense) || (k.path == BM_PATH_SPARSE && !lists)) continue;
        if (best < 0 || y[c] < y[best]) best = c;
    }
    if (best < 0) return rle_c < 0 ? 0 : rle_c;
    // the run-length path runs as a launch of its own: against a dense pick
    // it must beat the dense prediction less the batch's discount
    const float other =
        y[best] - (kCandidateTable[best].path == BM_PATH_DENSE ? dense_discount : 0.f);
    return rle_c >= 0 && y[rle_c] < other ? rle_c : best;
}

Candidate rule_choice(const bm_pool* p, const uint32_t* ids, uint32_t n) {
    const bool lists = all_have(p->list_present, ids, n);
    const bool dense = all_have(p->dense_present, ids, n);
    if (!lists) return kCandidateTable[0];
    uint64_t b = 0;
    for (uint32_t k = 0; k < n; ++k) b += p->list_len[ids[k]];
    const double dense_bytes = (double)n * (double)p->r_bits / 8.0;
    if (!dense || 4.0 * 4.0 * (double)b < dense_bytes)
        return Candidate{BM_PATH_SPARSE, p->sparse_cfg.tile_rows, 0};
    return kCandidateTable[0];
}

void mlp_forward_host(const float* P, int C, const float* x, float* y) {
    const int F = kFeatures, H = kHidden;
    const float* W1 = P;
    const float* b1 = W1 + F * H;
    const float* W2 = b1 + H;
    const float* b2 = W2 + H * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + H * C;
    float h1[kHidden], h2[kHidden];
    for (int j = 0; j < H; ++j) {
        float s = b1[j];
        for (int i = 0; i < F; ++i) s += x[i] * W1[i * H + j];
        h1[j] = s > 0.f ? s : 0.f;
    }
    for (int j = 0; j < H; ++j) {
        float s = b2[j];
        for (int i = 0; i < H; ++i) s += h1[i] * W2[i * H + j];
        h2[j] = s > 0.f ? s : 0.f;
    }
    for (int j = 0; j < C; ++j) {
        float s = b3[j];
        for (int i = 0; i < H; ++i) s += h2[i] * W3[i * C + j];
        y[j] = s;
    }
}

Candidate select_candidate(const bm_pool* p, const uint32_t* ids, uint32_t n,
                           const std::vector<uint8_t>& f) {
    if (!selector_installed(p)) return rule_choice(p, ids, n);
    float x[kFeatures], y[kCandidates];
    query_features(p, ids, n, f, x);
    for (int i = 0; i < kFeatures; ++i) x[i] = (x[i] - p->sel_mean[i]) / p->sel_std[i];
    mlp_forward_host(p->sel_params.data(), kCandidates, x, y);
    return kCandidateTable[pick_candidate(p, ids, n, y, 0.f)];
}

// Cost of a single query on GB300 (device time with L2 flushed), fitted to
// the measured kernels: the dense counter streams N r/8 bytes at about
// 7 TB/s after a fixed 9 us (N = 16..256, r = 2^20..2^26); the run-length
// kernel pays about 12.5 us of launch and set-up, 1.3 us per round of tiles
// across the GPU (three CTAs per SM below 8192 inputs, two above) and 1.05 us
// per MB of summaries and containers read (N = 32..256, r = 2^20..2^26, runs
// of mean 4096, 256 and 8 rows: 13-299 us).
constexpr double kDenseUsPerMB = 0.14, kDenseFixedUs = 9.0;
constexpr double kRleUsPerMB = 1.05, kRleRoundUs = 1.3, kRleFixedUs = 12.5;

Candidate with_rle(const bm_pool* p, const uint32_t* ids, uint32_t n, Candidate c,
                   double dense_speedup) {
    if (c.path != BM_PATH_DENSE || !all_have(p->rle_present, ids, n)) return c;
    uint64_t units = 0;  // container bytes (masks and literal words) / 16
    for (uint32_t k = 0; k < n; ++k) units += p->rle_units[ids[k]];
    const double tiles = (double)((p->words + kRleTileWords - 1) / kRleTileWords);
    const double rle_mb = (16.0 * (double)units + 8.0 * (double)n * tiles) / 1e6;
    const double dense_mb = (double)n * (double)p->r_bits / 8.0 / 1e6;
    const double per_sm = n < 8192 ? 3.0 : 2.0;
    const double rounds = std::ceil(tiles / (per_sm * (double)std::max(1, p->sm_count)));
    if (kRleFixedUs + kRleRoundUs * rounds + kRleUsPerMB * rle_mb <
        (kDenseFixedUs + kDenseUsPerMB * dense_mb) / dense_speedup)
        return Candidate{BM_PATH_RLE, 0, 0};
    return c;
}

Candidate single_query_candidate(const bm_pool* p, const uint32_t* ids, uint32_t n,
                                 const std::vector<uint8_t>& f) {
    if (selector_installed(p)) return select_candidate(p, ids, n, f);
    return with_rle(p, ids, n, rule_choice(p, ids, n));
}

}  // namespace bm
