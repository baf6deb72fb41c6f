// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "../../include/bm.h"

#define BM_CUDA_TRY(expr)                                  \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) {                           \
            bm_note_cuda_error(e_, #expr, __FILE__, __LINE__); \
            return BM_ECUDA;                               \
        }                                                  \
    } while (0)

void bm_note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

namespace bm {

// Rows covered by one entry of a position list's tile index.
constexpr uint32_t kListTileRows = 8192;
// Bit of a list's device begin offset marking a list of zeros (the rows where
// the bitmap is 0): ScanCount subtracts its positions from counters that
// start at the number of such inputs (Sec. 2.3, the complement identity).
constexpr uint64_t kListComplement = 1ull << 63;
// Most threshold transitions a predicate evaluates as comparators before it
// switches to a per-row table lookup.
constexpr int kMaxTransitions = 8;
// Bounded device waits give up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;
// Device error word bits.
constexpr int kErrTimeout = 1;

// A symmetric predicate f over counts 0..n, compiled on the host
// (Sec. 4.3: intervals and general symmetric functions from thresholds).
//   mode 0: constant v0.
//   mode 1: f(c) = v0 XOR [c >= t_1] XOR ... XOR [c >= t_m]  (t strictly
//           increasing, 1 <= t <= n).  Because the threshold sets are nested,
//           an interval [L, U] is T_L AND NOT T_{U+1}.
//   mode 2: per-row lookup of bit c of `table` (m > kMaxTransitions).
struct Pred {
    uint32_t mode;
    uint32_t v0;
    uint32_t ntrans;
    uint32_t table_words32;  // mode 2: 32-bit words of the table
    uint32_t trans[kMaxTransitions];
    const uint32_t* table;   // mode 2: device, bit c of word c/32
};

// Compile a truth table f(0..n) (host bytes 0/1) into a predicate.  The
// caller places the table on the device for mode 2.
Pred compile_pred(const uint8_t* f, uint32_t n);
// f for the threshold theta / the interval [lo, hi], as bytes f(0..n).
void threshold_truth(uint32_t n, uint32_t theta, std::vector<uint8_t>& f);
void interval_truth(uint32_t n, uint32_t lo, uint32_t hi, std::vector<uint8_t>& f);

// Ids of a query of at most kInlineIds inputs travel in the kernel's
// parameter block (copied to shared memory by each CTA) instead of a staged
// host-to-device copy: a small query is then a single launch.
constexpr uint32_t kInlineIds = 256;

// Arguments of one dense query launch.
struct DenseArgs {
    const uint64_t* base;     // pool dense storage
    uint64_t stride_words;    // words between bitmaps (multiple of 32)
    uint64_t words;           // ceil(r / 64)
    uint64_t r_bits;
    const uint32_t* ids;      // device, n ids
    uint32_t n;
    Pred pred;
    uint64_t* out;            // device, `words` words
    unsigned long long* card; // device cardinality (may be null): a pre-zeroed
                              // accumulator, or, with LaunchExtra::acc, stored
    int* err;                 // device error word
};

// Second parameter of the single-query kernels: a small query's ids inline
// and the cardinality's completion state.
struct LaunchExtra {
    unsigned long long* acc;  // device, zero on entry and on exit (null: card is
                              // a pre-zeroed accumulator that the kernel adds to)
    unsigned int* ticket;     // device, zero on entry and on exit (with acc)
    uint32_t n_inline;        // ids in inl[] (the Args' ids pointer is then unused), else 0
    uint32_t inl[kInlineIds];
};

// Dense kernel variants (the autotuner picks one per shape).
struct DenseConfig {
    int variant;   // 0 = direct 128-bit loads, 1 = bulk-copy (TMA) pipeline in shared memory
    int threads;   // consumer threads per CTA
    int stages;    // pipeline depth (variant 1)
    int ctas_per_sm;
    int adder = 0;             // sideways-sum block: 0 = 16 inputs, 1 = 8 inputs (variant 0)
    int words_per_thread = 2;  // 64-bit words per thread per input: 2 or 1 (variant 0)
};

int launch_dense(const DenseArgs& a, const LaunchExtra& x, const DenseConfig& cfg, int sm_count,
                 cudaStream_t s);

// The Looped recurrence (Sec. 4.4) for a plain threshold whose T, or whose
// complement N - T + 1 (Sec. 2.3, corrected), is at most kLoopedMaxT.
constexpr uint32_t kLoopedMaxT = 3;
struct LoopedForm {
    uint32_t t;     // accumulators: min(T, N - T + 1)
    bool neg;       // through the complement identity (negated inputs and result)
    uint32_t flip;  // ~0u: the predicate is "count < T"
};
// True (and *form set) if pred over n inputs is such a threshold with t <= max_t.
bool looped_form(const Pred& pred, uint32_t n, uint32_t max_t, LoopedForm* form);
int launch_looped(const DenseArgs& a, const LaunchExtra& x, const LoopedForm& f, int sm_count,
                  cudaStream_t s);

// Arguments of one sparse (ScanCount) query launch.
struct SparseArgs {
    const uint32_t* positions;   // pool list arena
    const uint64_t* list_begin;  // device, per id: first entry in the arena (| kListComplement)
    const uint32_t* tile_index;  // device, per id: tiles_per_list + 1 entries
    uint32_t tiles_per_list;     // ceil(r / kListTileRows)
    uint32_t tile_rows;          // rows per CTA tile, a multiple of kListTileRows
    uint64_t r_bits;
    const uint32_t* ids;         // device, n ids
    uint32_t n;
    uint32_t d_fill;             // inputs given by their zeros: the counters' start value
    Pred pred;
    uint64_t* out;
    unsigned long long* card;    // as DenseArgs
};

struct SparseConfig {
    uint32_t tile_rows;  // multiple of kListTileRows
    int threads;
    int ctas_per_sm;
    int unroll = 4;      // list slices a warp has in flight: 4 or 8
};

int launch_sparse(const SparseArgs& a, const LaunchExtra& x, const SparseConfig& cfg, int sm_count,
                  cudaStream_t s);

// Word-aligned run-length form of a bitmap (EWAH-like, Sec. 2.1), tiled for
// the GPU: every word is clean-0 (all zeros), clean-1 (all ones) or literal.
// Per tile of kRleTileWords words, one summary (uint2): the tile's class
// (clean-0 or clean-1 when one clean run covers it, else mixed) and, for a
// mixed tile, where its container starts in the pool's container arena, in
// 16-byte units (bits 0..29 in x below the class, bits 30.. in y above the
// container's size in 16-byte units, which is at most 133).  A container
// (16-byte aligned, padded to 16 bytes) is: L[0..7] (32-bit; bit b of L[s]:
// word 32 s + b is literal), O[0..7] (bit b of O[s]: that word is clean-1),
// R[0..7] (bytes; R[s]: literal words in slices before s), 8 bytes of
// padding, then the tile's literal words in order.  Summaries are stored
// tile-major (tile t of id j at t * capacity + j), so a tile's summaries of
// consecutive ids are adjacent.
constexpr uint32_t kTileClean0 = 0, kTileClean1 = 1, kTileMixed = 2;
constexpr uint32_t kTileOffsetMask = (1u << 30) - 1u;
// Container start (16-byte units) and size (16-byte units) of a summary.
__host__ __device__ inline uint64_t tile_container(uint2 s) {
    return ((uint64_t)(s.y >> 8) << 30) | (s.x & kTileOffsetMask);
}
__host__ __device__ inline uint32_t tile_units(uint2 s) { return s.y & 0xFFu; }
constexpr uint32_t kRleTileWords = 256;   // words per tile of the summaries and kernel
constexpr uint32_t kRleSliceWords = 32;   // words per mask of a container (one per warp)
constexpr uint32_t kRleHeaderBytes = 80;  // container bytes before the literal words

// Arguments of one run-length query launch.
struct RleArgs {
    const uint8_t* arena;         // pool container arena (16-byte aligned)
    const uint2* tile_index;      // device, tiles x capacity summaries (tile-major)
    uint32_t capacity;            // summaries between consecutive tiles
    uint64_t words, r_bits;
    const uint32_t* ids;
    uint32_t n;
    Pred pred;
    uint64_t* out;
    unsigned long long* card;    // as DenseArgs
    int* err;                    // pool error word (bounded waits)
};

int launch_rle(const RleArgs& a, const LaunchExtra& x, int sm_count, cudaStream_t s);
// Run-length form of `nwords` words (host): the containers of the mixed tiles
// (appended to `containers`) and one summary per tile (written to
// summary[0], summary[stride], ...), whose container starts count from
// `first_unit` for the arena unit where `containers` will be placed.  Also
// counts the maximal runs of equal word kind and the literal words.
void rle_encode(const uint64_t* words, uint64_t nwords, std::vector<uint4>& containers,
                uint64_t first_unit, uint2* summary, size_t stride, uint64_t* runs,
                uint64_t* literal_words);
int launch_cardinality(const uint64_t* words, uint64_t r_bits, unsigned long long* out,
                       int sm_count, cudaStream_t s);
int planes_for(uint32_t n);  // counter planes needed for counts 0..n

}  // namespace bm

// Per-call host->device staging: pinned host block + device block + event.
// The device block starts with a header of kStageHeader bytes that is never
// copied over: the cardinality accumulator (uint64) and the arrival ticket
// (uint32) of the call's kernel (see CardOut in bm_device.cuh), zero between
// calls; h and d point past it, at the staged payload.
constexpr size_t kStageHeader = 16;
struct bm_stage_slot {
    void* h = nullptr;       // payload, pinned host
    void* d = nullptr;       // payload, device
    void* h_base = nullptr;  // allocations
    void* d_base = nullptr;
    size_t cap = 0;          // payload bytes
    cudaEvent_t ev = nullptr;
    bool used = false;
    unsigned long long* acc() const { return static_cast<unsigned long long*>(d_base); }
    unsigned int* ticket() const {
        return reinterpret_cast<unsigned int*>(static_cast<uint8_t*>(d_base) + 8);
    }
};

struct bm_pool {
    int device = 0;
    int sm_count = 0;
    uint64_t r_bits = 0, words = 0, stride_words = 0;
    uint32_t capacity = 0;
    uint64_t mem_budget = 0, device_bytes = 0;

    uint64_t* d_dense = nullptr;          // capacity * stride_words
    std::vector<uint8_t> dense_present;
    std::vector<uint64_t> card;           // per id cardinality, host copy

    // position lists: one growable device arena
    uint32_t* d_pos = nullptr;
    uint64_t pos_cap = 0, pos_used = 0;
    std::vector<uint64_t> list_begin, list_len;  // host, per id
    std::vector<uint8_t> list_present;
    std::vector<uint8_t> list_complement;  // the list holds the zeros of the bitmap
    uint32_t* d_tile_index = nullptr;     // capacity * tiles_per_list (+1)
    uint64_t* d_list_begin = nullptr;     // per id, device copy
    uint32_t tiles_per_list = 0;

    // run-length form: one growable container arena, per-id bases, tile-major
    // summaries
    uint4* d_rle_arena = nullptr;
    uint64_t rle_cap = 0, rle_used = 0;   // arena 16-byte units allocated / in use
    uint2* d_rle_tiles = nullptr;         // rle_tiles x capacity
    uint32_t rle_tiles = 0;               // ceil(words / kRleTileWords)
    std::vector<uint8_t> rle_present;
    std::vector<uint64_t> rle_runs, rle_lits;  // host, per id: runs and literal words
    std::vector<uint64_t> rle_units;           // host, per id: container 16-byte units

    int* d_err = nullptr;
    static constexpr int kSlots = 8;
    bm_stage_slot slots[kSlots];
    int next_slot = 0;
    bm::DenseConfig dense_cfg{0, 256, 4, 2};
    bm::SparseConfig sparse_cfg{32768, 512, 2};
    uint32_t looped_max = 0;  // plain thresholds with min(T, N-T+1) <= this run Looped
    // learned selector (empty: fixed density rule)
    std::vector<float> sel_params;
    float sel_mean[8] = {}, sel_std[8] = {};
    int sel_outputs = 0;
    void* batch = nullptr;  // batched-query state (descriptor slots, graphs)
    std::mutex mu;
};

namespace bm {
// Truth table f(0..n) of a query descriptor.
int query_truth(const bm_query* q, std::vector<uint8_t>& f);
// Host validation of ids for a path (BM_PATH_*).
int validate_ids(const bm_pool* p, const uint32_t* ids, uint32_t n, int path);
// Inputs of ids[0..n) whose position list holds their zeros (with repeats).
uint32_t complement_inputs(const bm_pool* p, const uint32_t* ids, uint32_t n);
// Reserve a staging slot of at least `bytes` of payload, waiting for its
// previous use; a new device block gets its header zeroed on stream `s`.
int stage_acquire(bm_pool* p, size_t bytes, bm_stage_slot** out, cudaStream_t s);
// Copy the slot's first `bytes` to the device on `s` and mark its reuse point.
int stage_commit(bm_stage_slot* slot, size_t bytes, cudaStream_t s);
int stage_release(bm_stage_slot* slot, cudaStream_t s);
int track_alloc(bm_pool* p, void** ptr, size_t bytes);
void track_free(bm_pool* p, void* ptr, size_t bytes);
// Raise kernel fn's dynamic shared-memory limit on the current device to at
// least `bytes`.  The runtime is called only when a launch needs more than
// any earlier one of fn on that device (the call costs more than a small
// query's kernel).
int ensure_smem_limit(const void* fn, size_t bytes);
// Largest dynamic shared memory a CTA may opt in to on the current device.
int smem_optin(int* bytes);
void batch_state_free(bm_pool* p);
}  // namespace bm
