// Kernel selection per query: query features, the fixed density rule, and
// the learned selector (a small MLP predicting each candidate's log time).
#pragma once

#include <stdint.h>

#include <vector>

#include "bm_internal.cuh"

namespace bm {

constexpr int kFeatures = 6;
constexpr int kHidden = 64;

// The kernel configurations a query can run on (the selector's outputs).
struct Candidate {
    int path;              // BM_PATH_DENSE, BM_PATH_SPARSE or BM_PATH_RLE
    uint32_t tile_rows;    // sparse tile (0 for dense)
    uint32_t dense_words;  // dense: 1 = one 64-bit word per thread, 0 = the pool's shape
};
constexpr int kCandidates = 6;
extern const Candidate kCandidateTable[kCandidates];

// Features of a query: log2 n, first transition of f over n, log10 of the
// mean and of the largest input density, log2 r, log2 of the run-length
// forms' bytes over the dense bytes (0 unless every input has one).
void query_features(const bm_pool* p, const uint32_t* ids, uint32_t n,
                    const std::vector<uint8_t>& f, float out[kFeatures]);

// Fixed rule: ScanCount when every input has a position list and the lists
// are at least 128x smaller than the dense words (mean density < 1/128),
// else the dense counter.
Candidate rule_choice(const bm_pool* p, const uint32_t* ids, uint32_t n);

// Learned choice if a selector is installed, else the rule; candidates whose
// inputs are missing (no lists, no dense words, no run-length forms) are
// never chosen.
Candidate select_candidate(const bm_pool* p, const uint32_t* ids, uint32_t n,
                           const std::vector<uint8_t>& f);
// Index of the smallest prediction y[0..kCandidates) among the candidates
// the query's inputs allow.  The run-length candidate is compared last, with
// dense_discount (log scale) taken off a dense pick's prediction first: in a
// batch the dense kernel shares the pool's reads, while a run-length query
// runs as a launch of its own (0 for a single query).
int pick_candidate(const bm_pool* p, const uint32_t* ids, uint32_t n, const float* y,
                   float dense_discount);
// True when a selector with the current candidates is installed.
inline bool selector_installed(const bm_pool* p) {
    return !p->sel_params.empty() && p->sel_outputs == kCandidates;
}

// The run-length path in place of a dense choice c when every input has a
// run-length form and the estimated time of reading its runs, literal words
// and tile summaries is below that of reading the dense words; else c.
// dense_speedup divides the dense estimate: a query left in a batch's dense
// kernel shares the pool's slabs through L2 with the other queries
// (kBatchDenseSpeedup), while a run-length query runs as a launch of its own.
Candidate with_rle(const bm_pool* p, const uint32_t* ids, uint32_t n, Candidate c,
                   double dense_speedup = 1.0);
// Queries per second of the batch's dense kernel over one launch per query
// on the mixed batch workload (measured on GB300: 38.0k vs 15.2k).
constexpr double kBatchDenseSpeedup = 2.5;

// A single query's choice: the installed selector's pick, else the rule
// followed by with_rle.
Candidate single_query_candidate(const bm_pool* p, const uint32_t* ids, uint32_t n,
                                 const std::vector<uint8_t>& f);

// MLP forward on the host for one feature vector (fp32), all C outputs.
void mlp_forward_host(const float* params, int C, const float* x, float* y);

inline size_t mlp_param_count(int F, int H, int C) {
    return (size_t)F * H + H + (size_t)H * H + H + (size_t)H * C + C;
}

}  // namespace bm
