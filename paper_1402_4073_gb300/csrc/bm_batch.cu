// Batched queries: many queries of uneven n, predicate and path in one
// CUDA-graph launch of two persistent kernels.
//
//  * Dense items are (column tile, query) pairs taken tile-major from an
//    atomic work counter, so at any moment the CTAs of the GPU work on the
//    same 32768-row slab of the pool: each input slab is read from HBM once
//    and then served from L2 to every other query that reads it.
//  * Sparse items are (query, row tile) pairs of the ScanCount kernel with
//    16-bit shared-memory counters and each query's own tile size.
//  * A zeroing kernel resets the work counters and the caller's
//    cardinalities.  All three read their arguments from a device-side
//    descriptor block, so the captured graph is replayed unchanged for every
//    batch; only the block is copied to the device before each replay.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "bm_dense_common.cuh"
#include "bm_scan_common.cuh"
#include "bm_select.h"

namespace bm {

constexpr int kBatchThreads = 256;        // dense: one 16-byte column per thread
constexpr int kSparseBatchThreads = 384;
// Batched sparse items use at most 16384 counter words (32768 rows of 16-bit
// counters, 65536 rows of 8-bit ones), so that two sparse CTAs fit on an SM
// whatever tile a query would take alone.
constexpr uint32_t kSparseMaxWords = 16384;
// Pieces per load batch of a warp in batched ScanCount items (two batches
// in flight; they fit in the 64 registers two 512-thread CTAs per SM leave).
constexpr int kSparseBatchUnroll = 2;

struct QueryDesc {
    const uint32_t* ids;
    uint32_t n;
    uint32_t tile_rows;
    uint64_t* out;
    uint32_t d_fill;  // sparse: inputs given by their zeros (ScanCount counters start here)
    uint32_t pad;
    Pred pred;
};

struct BatchHeader {
    uint64_t* out_cards;
    const QueryDesc* desc;
    const uint32_t* dense_list;
    const uint32_t* sparse_list;
    const uint64_t* sparse_off;  // n_sparse + 1 prefix sums of sparse items
    uint32_t nq, n_dense, n_sparse, pad;
    uint64_t dense_items;
    unsigned long long dense_next, sparse_next;
};

struct BatchPoolArgs {
    const uint64_t* base;
    uint64_t stride_words, words, r_bits;
    const uint32_t* positions;
    const uint64_t* list_begin;
    const uint32_t* tile_index;
    uint32_t tiles_per_list;
};

namespace {

using namespace dev;

__global__ void batch_zero_kernel(BatchHeader* h) {
    for (uint32_t i = threadIdx.x; i < h->nq; i += blockDim.x) h->out_cards[i] = 0;
    if (threadIdx.x == 0) {
        h->dense_next = 0;
        h->sparse_next = 0;
    }
}

__device__ __forceinline__ void block_card_add(unsigned long long card, unsigned long long* dst,
                                               unsigned long long* part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) card += __shfl_xor_sync(0xFFFFFFFFu, card, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = card;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        if (t) atomicAdd(dst, t);
    }
}

// One-word columns (L = 2) hold half the planes: three CTAs fit per SM.
// Thread 0 fetches the next item while the current one is counted, and each
// warp adds its own share of the cardinality: one barrier per item.
template <int K, int G, int L>
__global__ void __launch_bounds__(kBatchThreads, L == 2 ? 3 : 2)
    dense_batch_kernel(BatchHeader* h, BatchPoolArgs pa) {
    __shared__ unsigned long long item_s[2];
    constexpr uint64_t W = L / 2;  // 64-bit words per thread per input
    const uint64_t ncols = (pa.words + W - 1) / W;
    const uint32_t nd = h->n_dense;
    const uint64_t total = h->dense_items;
    if (threadIdx.x == 0) item_s[0] = atomicAdd(&h->dense_next, 1ull);
    __syncthreads();
    for (uint32_t it = 0;; ++it) {
        // item_s[it & 1] was published by the barrier that ended the last
        // iteration; it is overwritten only after the next barrier
        const uint64_t item = item_s[it & 1];
        if (item >= total) break;
        unsigned long long next = 0;
        if (threadIdx.x == 0) next = atomicAdd(&h->dense_next, 1ull);
        const uint64_t tile = item / nd;
        const uint32_t qi = h->dense_list[item % nd];
        const QueryDesc* d = h->desc + qi;
        const uint64_t col = tile * kBatchThreads + threadIdx.x;
        unsigned long long card = 0;
        if (col < ncols) {
            const Pred pred = d->pred;
            uint64_t* out = d->out;
            uint32_t P[L][K];
            zero_planes<K, L>(P);
            count_column<K, G, L, false, true>(P, pa.base + W * col, d->ids, d->n,
                                                 pa.stride_words);
            const bool vec_ok = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
            card = finish_column<K, L>(P, pred, pred.table, pa.r_bits, pa.words, out, col, vec_ok);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) card += __shfl_xor_sync(0xFFFFFFFFu, card, o);
        if ((threadIdx.x & 31) == 0 && card)
            atomicAdd(reinterpret_cast<unsigned long long*>(h->out_cards + qi), card);
        if (threadIdx.x == 0) item_s[(it + 1) & 1] = next;
        __syncthreads();
    }
}

// One (query, row tile) item of ScanCount with BITS-bit counters.
template <int BITS>
__device__ __forceinline__ unsigned long long sparse_item(const QueryDesc* d, const Pred& pred,
                                                          const uint32_t* tab, uint32_t* scratch,
                                                          uint32_t* s_next,
                                                          uint32_t* cnt, uint32_t cnt_words,
                                                          uint64_t tile, const BatchPoolArgs& pa) {
    constexpr uint32_t kPer = 32 / BITS;
    const uint32_t n = d->n, tile_rows = d->tile_rows;
    const uint64_t rlo = tile * tile_rows;
    const uint64_t rhi = min(rlo + tile_rows, pa.r_bits);
    const uint32_t sub = tile_rows / kListTileRows;
    const uint64_t t0 = tile * sub;
    const uint64_t t1 = (t0 + sub < pa.tiles_per_list) ? t0 + sub : (uint64_t)pa.tiles_per_list;
    const uint32_t* ids = d->ids;
    count_tile<BITS, kSparseBatchUnroll>(cnt, scratch, s_next,
                                         [ids](uint32_t j) { return __ldg(ids + j); }, n,
                                         reinterpret_cast<const uint4*>(pa.positions),
                                         pa.list_begin, pa.tile_index, pa.tiles_per_list, t0, t1,
                                         (uint32_t)rlo, (uint32_t)(rhi - rlo),
                                         cnt_words * kPer,  // spares past every item's counters
                                         d->d_fill);
    __syncthreads();
    const uint32_t lanes = (uint32_t)((rhi - rlo + 31) / 32);
    uint32_t* out32 = reinterpret_cast<uint32_t*>(d->out);
    unsigned long long card = 0;
    for (uint32_t l = threadIdx.x; l < lanes; l += blockDim.x) {
        uint32_t o = counters_to_lane<BITS>(cnt + l * (32 / kPer), pred, tab);
        const uint64_t row0 = rlo + 32ull * l;
        if (row0 + 32 > pa.r_bits) o &= (1u << (pa.r_bits - row0)) - 1u;
        out32[row0 / 32] = o;
        card += __popc(o);
    }
    // the upper half of the last 64-bit word when r ends in its lower half
    if (rhi == pa.r_bits && threadIdx.x == 0 && ((pa.r_bits + 31) / 32) % 2 == 1)
        out32[(pa.r_bits + 31) / 32] = 0u;
    return card;
}

__global__ void __launch_bounds__(kSparseBatchThreads, 2)
    sparse_batch_kernel(BatchHeader* h, BatchPoolArgs pa) {
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ unsigned long long item_s;
    __shared__ unsigned long long part[kSparseBatchThreads / 32];
    uint32_t* tab = sm;                      // up to 2048 words (n <= 65535)
    __shared__ uint32_t s_next;  // next group of lists to count
    uint32_t* scratch = sm + 2048;
    uint32_t* cnt = scratch + kScanWarpWords * (kSparseBatchThreads / 32);  // counters
    const uint32_t ns = h->n_sparse;
    const uint64_t total = ns ? h->sparse_off[ns] : 0;
    // counters start at zero; evaluating an item clears the ones it used.  The
    // launch sized the counters for its largest tile: zero what it allocated.
    const uint32_t cnt_words =
        dynamic_smem_bytes() / 4 - 2048 - kScanWarpWords * (kSparseBatchThreads / 32) - 32;
    for (uint32_t i = threadIdx.x; i < cnt_words; i += blockDim.x) cnt[i] = 0u;
    __shared__ uint32_t query_s;  // the query of this CTA's current (then previous) item
    // thread 0 fetches each next item while the current one is counted
    unsigned long long pending = 0;
    if (threadIdx.x == 0) {
        query_s = 0;
        pending = atomicAdd(&h->sparse_next, 1ull);
    }
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long it = pending;
            item_s = it;
            if (it < total) {
                pending = atomicAdd(&h->sparse_next, 1ull);
                // the query of this item is the last prefix entry <= it.  A CTA's
                // items increase, so gallop forward from its previous query, then
                // bisect: a few dependent loads instead of log2(n_sparse)
                uint32_t lo = query_s, hi = lo + 1, step = 1;
                while (hi < ns && h->sparse_off[hi] <= it) {
                    lo = hi;
                    step *= 2;
                    hi = lo + step;
                }
                if (hi > ns) hi = ns;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) / 2;
                    if (h->sparse_off[mid] <= it)
                        lo = mid;
                    else
                        hi = mid;
                }
                query_s = lo;
            }
        }
        __syncthreads();
        const uint64_t item = item_s;
        const uint32_t lo = query_s;
        __syncthreads();
        if (item >= total) break;
        const uint32_t qi = h->sparse_list[lo];
        const QueryDesc* d = h->desc + qi;
        const uint32_t n = d->n;
        const uint64_t tile = item - h->sparse_off[lo];
        const Pred& pred = d->pred;  // read in place: no registers held across the count
        // truth table of f over 0..n (a plain threshold is compared directly)
        const bool plain = pred.mode == 1 && pred.ntrans == 1 && pred.v0 == 0;
        const uint32_t tab_words = plain ? 0u : (n + 1 + 31) / 32;
        for (uint32_t w = threadIdx.x; w < tab_words; w += blockDim.x) {
            uint32_t bits = 0;
            if (pred.mode == 2) {
                bits = pred.table[w];
            } else {
                for (uint32_t b = 0; b < 32; ++b) {
                    const uint32_t c = w * 32 + b;
                    if (c > n) break;
                    uint32_t v = pred.v0;
                    if (pred.mode == 1)
#pragma unroll
                        for (int i = 0; i < kMaxTransitions; ++i)
                            if ((uint32_t)i < pred.ntrans) v ^= (c >= pred.trans[i]) ? 1u : 0u;
                    bits |= v << b;
                }
            }
            tab[w] = bits;
        }
        // 8-bit counters hold every count when n <= 255 (the counter-width switch by N)
        const unsigned long long card =
            n <= 255 ? sparse_item<8>(d, pred, tab, scratch, &s_next, cnt, cnt_words, tile, pa)
                     : sparse_item<16>(d, pred, tab, scratch, &s_next, cnt, cnt_words, tile, pa);
        block_card_add(card, reinterpret_cast<unsigned long long*>(h->out_cards + qi), part);
        __syncthreads();
    }
}

// Shared memory of the sparse batch kernel with `words` 32-bit counter words
// (rows x counter bits / 32 of its largest item).
size_t sparse_batch_smem(uint32_t words) {
    // truth table, scratch, 16-bit counters and one spare word per lane
    return (2048 + (size_t)kScanWarpWords * (kSparseBatchThreads / 32) + (size_t)words + 32) * 4;
}

}  // namespace

// One descriptor slot: pinned host block, device block, completion event and
// the graphs captured on it (one per counter-plane count).
struct BatchSlot {
    void* h = nullptr;
    void* d = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool used = false;
    std::map<int, cudaGraphExec_t> graphs;  // key: planes K * 16 + adder
};

struct BatchState {
    static constexpr int kSlots = 4;
    BatchSlot slots[kSlots];
    int next = 0;
    cudaStream_t capture = nullptr, capture2 = nullptr;  // fork/join capture of the graph
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaStream_t infer = nullptr;
    float* d_sel = nullptr;  // selector inference buffers
    size_t sel_cap = 0;
    DenseConfig cfg{0, kBatchThreads, 0, 2, 0};
};

void batch_state_free(bm_pool* p) {
    BatchState* b = static_cast<BatchState*>(p->batch);
    if (!b) return;
    for (auto& sl : b->slots) {
        for (auto& kv : sl.graphs) cudaGraphExecDestroy(kv.second);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.h) cudaFreeHost(sl.h);
        if (sl.d) cudaFree(sl.d);
    }
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->capture2) cudaStreamDestroy(b->capture2);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    if (b->infer) cudaStreamDestroy(b->infer);
    if (b->d_sel) cudaFree(b->d_sel);
    delete b;
    p->batch = nullptr;
}

static BatchState* state(bm_pool* p) {
    if (!p->batch) p->batch = new BatchState();
    return static_cast<BatchState*>(p->batch);
}

static int slot_reserve(bm_pool* p, BatchSlot& sl, size_t bytes) {
    if (sl.used) BM_CUDA_TRY(cudaEventSynchronize(sl.ev));
    sl.used = false;
    if (!sl.ev) BM_CUDA_TRY(cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming));
    if (sl.cap >= bytes) return BM_OK;
    for (auto& kv : sl.graphs) cudaGraphExecDestroy(kv.second);
    sl.graphs.clear();
    if (sl.h) cudaFreeHost(sl.h);
    if (sl.d) {
        cudaFree(sl.d);
        p->device_bytes -= std::min<uint64_t>(p->device_bytes, sl.cap);
    }
    sl.h = sl.d = nullptr;
    sl.cap = 0;
    size_t cap = std::max<size_t>(bytes + bytes / 4, 1 << 20);
    cap = (cap + 4095) & ~(size_t)4095;
    if (cudaHostAlloc(&sl.h, cap, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        sl.h = nullptr;
        return BM_ENOMEM;
    }
    int rc = track_alloc(p, &sl.d, cap);
    if (rc) {
        cudaFreeHost(sl.h);
        sl.h = nullptr;
        return rc;
    }
    sl.cap = cap;
    return BM_OK;
}

static int graph_for(bm_pool* p, BatchState* b, BatchSlot& sl, int K, uint32_t max_words,
                     const BatchPoolArgs& pa, cudaGraphExec_t* out) {
    const int adder = b->cfg.adder, L = b->cfg.words_per_thread == 1 ? 2 : 4;
    // counter words of the largest sparse item: 8192 or kSparseMaxWords
    const int tile_code = max_words <= kSparseMaxWords / 2 ? 0 : 1;
    const uint32_t words_cap = (kSparseMaxWords / 2) << tile_code;
    const int key = ((K * 64 + adder * 8 + L) << 2) | tile_code;
    auto it = sl.graphs.find(key);
    if (it != sl.graphs.end()) {
        *out = it->second;
        return BM_OK;
    }
    if (!b->capture) {
        BM_CUDA_TRY(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
        BM_CUDA_TRY(cudaStreamCreateWithFlags(&b->capture2, cudaStreamNonBlocking));
        BM_CUDA_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        BM_CUDA_TRY(cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming));
    }
    BatchHeader* h = static_cast<BatchHeader*>(sl.d);
    const size_t sp_smem = sparse_batch_smem(words_cap);
    int optin = 0;
    BM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    const unsigned dense_grid = (unsigned)(p->sm_count * std::max(1, b->cfg.ctas_per_sm));
    const unsigned sparse_grid =
        (unsigned)p->sm_count * (2 * sp_smem + 2048 <= (size_t)optin ? 2u : 1u);
    auto dense_fn = [&](auto fn) -> int {
        // the dense and the sparse persistent kernels run side by side
        BM_CUDA_TRY(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
        batch_zero_kernel<<<1, 256, 0, b->capture>>>(h);
        BM_CUDA_TRY(cudaEventRecord(b->fork, b->capture));
        BM_CUDA_TRY(cudaStreamWaitEvent(b->capture2, b->fork, 0));
        fn<<<dense_grid, kBatchThreads, 0, b->capture>>>(h, pa);
        sparse_batch_kernel<<<sparse_grid, kSparseBatchThreads, sp_smem, b->capture2>>>(h, pa);
        BM_CUDA_TRY(cudaEventRecord(b->join, b->capture2));
        BM_CUDA_TRY(cudaStreamWaitEvent(b->capture, b->join, 0));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->capture, &g);
        if (e != cudaSuccess) {
            bm_note_cuda_error(e, "batch graph capture", __FILE__, __LINE__);
            return BM_ECUDA;
        }
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            bm_note_cuda_error(e, "batch graph instantiate", __FILE__, __LINE__);
            return BM_ECUDA;
        }
        sl.graphs[key] = ex;
        *out = ex;
        return BM_OK;
    };
    BM_CUDA_TRY(cudaFuncSetAttribute(sparse_batch_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sparse_batch_smem(kSparseMaxWords)));
#define BM_BATCH_DISPATCH(LL)                                                      \
    if (adder == 2) {                                                              \
        if (K <= 5) return dense_fn(dense_batch_kernel<5, 16, LL>);                \
        if (K <= 9) return dense_fn(dense_batch_kernel<9, 32, LL>);                \
        if (K <= 11) return dense_fn(dense_batch_kernel<11, 32, LL>);              \
        if (K <= 13) return dense_fn(dense_batch_kernel<13, 32, LL>);              \
        return dense_fn(dense_batch_kernel<17, 32, LL>);                           \
    }                                                                              \
    if (adder == 1) {                                                              \
        if (K <= 5) return dense_fn(dense_batch_kernel<5, 8, LL>);                 \
        if (K <= 9) return dense_fn(dense_batch_kernel<9, 8, LL>);                 \
        if (K <= 11) return dense_fn(dense_batch_kernel<11, 8, LL>);               \
        if (K <= 13) return dense_fn(dense_batch_kernel<13, 8, LL>);               \
        return dense_fn(dense_batch_kernel<17, 8, LL>);                            \
    }                                                                              \
    if (K <= 5) return dense_fn(dense_batch_kernel<5, 16, LL>);                    \
    if (K <= 9) return dense_fn(dense_batch_kernel<9, 16, LL>);                    \
    if (K <= 11) return dense_fn(dense_batch_kernel<11, 16, LL>);                  \
    if (K <= 13) return dense_fn(dense_batch_kernel<13, 16, LL>);                  \
    return dense_fn(dense_batch_kernel<17, 16, LL>);
    if (L == 4) {
        BM_BATCH_DISPATCH(4)
    }
    BM_BATCH_DISPATCH(2)
#undef BM_BATCH_DISPATCH
}

// The learned selector's predictions for every AUTO query of a batch, on the
// device: y[i * kCandidates + c].
static int batch_select(bm_pool* p, BatchState* b, const std::vector<std::vector<float>>& feats,
                        std::vector<float>& y) {
    const uint32_t B = (uint32_t)feats.size();
    if (!B) return BM_OK;
    const int F = kFeatures, H = kHidden, C = kCandidates;
    const size_t np = mlp_param_count(F, H, C);
    const size_t need = np + (size_t)B * (F + 2 * H + C);
    if (!b->infer) BM_CUDA_TRY(cudaStreamCreateWithFlags(&b->infer, cudaStreamNonBlocking));
    if (b->sel_cap < need) {
        if (b->d_sel) {
            cudaFree(b->d_sel);
            p->device_bytes -= std::min<uint64_t>(p->device_bytes, b->sel_cap * 4);
        }
        b->d_sel = nullptr;
        b->sel_cap = 0;
        int rc = track_alloc(p, (void**)&b->d_sel, need * 4);
        if (rc) return rc;
        b->sel_cap = need;
    }
    std::vector<float> x((size_t)B * F);
    y.assign((size_t)B * C, 0.f);
    for (uint32_t i = 0; i < B; ++i)
        for (int f = 0; f < F; ++f) x[(size_t)i * F + f] = (feats[i][f] - p->sel_mean[f]) / p->sel_std[f];
    float* dP = b->d_sel;
    float* dx = dP + np;
    float* dh1 = dx + (size_t)B * F;
    float* dh2 = dh1 + (size_t)B * H;
    float* dy = dh2 + (size_t)B * H;
    BM_CUDA_TRY(cudaMemcpyAsync(dP, p->sel_params.data(), np * 4, cudaMemcpyHostToDevice, b->infer));
    BM_CUDA_TRY(cudaMemcpyAsync(dx, x.data(), x.size() * 4, cudaMemcpyHostToDevice, b->infer));
    int rc = bm_mlp_forward(dP, F, H, C, dx, B, dh1, dh2, dy, b->infer);
    if (rc) return rc;
    BM_CUDA_TRY(cudaMemcpyAsync(y.data(), dy, y.size() * 4, cudaMemcpyDeviceToHost, b->infer));
    BM_CUDA_TRY(cudaStreamSynchronize(b->infer));
    return BM_OK;
}

}  // namespace bm

using namespace bm;

extern "C" int bm_threshold_batch(bm_pool* p, const bm_query* q, uint32_t nq, uint64_t* out_cards,
                                  int32_t* chosen_paths, void* stream) {
    if (!p || !q || nq == 0 || !out_cards) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    BM_CUDA_TRY(cudaSetDevice(p->device));
    BatchState* b = state(p);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // validate, truth tables, candidate choice
    std::vector<std::vector<uint8_t>> truth(nq);
    std::vector<Candidate> cand(nq);
    std::vector<uint32_t> auto_idx;
    std::vector<std::vector<float>> feats;
    uint64_t total_ids = 0, total_tab = 0;
    uint32_t max_dense_n = 1;
    for (uint32_t i = 0; i < nq; ++i) {
        const bm_query& qi = q[i];
        if (!qi.out_words || qi.reserved || qi.path < BM_PATH_AUTO || qi.path > BM_PATH_RLE)
            return BM_EINVAL;
        int rc = validate_ids(p, qi.ids, qi.n, qi.path);
        if (!rc) rc = query_truth(&qi, truth[i]);
        if (rc) return rc;
        total_ids += (qi.n + 3) & ~3u;  // each query's ids start 16-byte aligned
        if (qi.path == BM_PATH_AUTO) {
            if (selector_installed(p)) {
                auto_idx.push_back(i);
                feats.emplace_back(kFeatures);
                query_features(p, qi.ids, qi.n, truth[i], feats.back().data());
            } else {
                cand[i] = with_rle(p, qi.ids, qi.n, rule_choice(p, qi.ids, qi.n),
                                   kBatchDenseSpeedup);
            }
        } else {
            cand[i] = Candidate{qi.path, qi.path == BM_PATH_SPARSE ? p->sparse_cfg.tile_rows : 0u, 0u};
        }
    }
    if (!auto_idx.empty()) {
        std::vector<float> y;
        int rc = batch_select(p, b, feats, y);
        if (rc) return rc;
        // the smallest prediction among the candidates whose inputs are
        // loaded; a query left in the batch's dense kernel shares the pool's
        // reads with the others, so the dense predictions shrink by its gain
        const float discount = (float)std::log(kBatchDenseSpeedup);
        for (size_t j = 0; j < auto_idx.size(); ++j) {
            const uint32_t i = auto_idx[j];
            cand[i] = kCandidateTable[pick_candidate(p, q[i].ids, q[i].n,
                                                     y.data() + j * kCandidates, discount)];
        }
    }
    std::vector<Pred> preds(nq);
    std::vector<uint32_t> dense_list, sparse_list, rle_list;
    std::vector<uint64_t> sparse_off(1, 0);
    uint32_t max_words = 0;
    for (uint32_t i = 0; i < nq; ++i) {
        preds[i] = compile_pred(truth[i].data(), q[i].n);
        if (preds[i].mode == 2) total_tab += preds[i].table_words32;
        if (cand[i].path == BM_PATH_SPARSE) {
            // 8-bit items (n <= 255) fit twice the rows in the same counter words
            const uint32_t bits = q[i].n <= 255 ? 8u : 16u;
            const uint32_t cap = kSparseMaxWords * (32 / bits);
            if (cand[i].tile_rows > cap) cand[i].tile_rows = cap;
            max_words = std::max(max_words, cand[i].tile_rows * bits / 32);
            sparse_list.push_back(i);
            sparse_off.push_back(sparse_off.back() +
                                 (p->r_bits + cand[i].tile_rows - 1) / cand[i].tile_rows);
        } else if (cand[i].path == BM_PATH_RLE) {
            rle_list.push_back(i);
        } else {
            dense_list.push_back(i);
            max_dense_n = std::max(max_dense_n, q[i].n);
        }
        if (chosen_paths) chosen_paths[i] = cand[i].path;
    }

    // descriptor block: header | descs | dense list | sparse list | sparse off | ids | tables
    auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
    const size_t o_desc = al(sizeof(BatchHeader));
    const size_t o_dl = o_desc + al(sizeof(QueryDesc) * nq);
    const size_t o_sl = o_dl + al(4 * dense_list.size());
    const size_t o_so = o_sl + al(4 * sparse_list.size());
    const size_t o_ids = o_so + al(8 * sparse_off.size());
    const size_t o_tab = o_ids + al(4 * total_ids);
    const size_t bytes = o_tab + al(4 * total_tab);
    BatchSlot& sl = b->slots[b->next];
    b->next = (b->next + 1) % BatchState::kSlots;
    int rc = slot_reserve(p, sl, bytes);
    if (rc) return rc;
    uint8_t* hb = static_cast<uint8_t*>(sl.h);
    uint8_t* db = static_cast<uint8_t*>(sl.d);
    BatchHeader* hh = reinterpret_cast<BatchHeader*>(hb);
    memset(hh, 0, sizeof(BatchHeader));
    hh->out_cards = out_cards;
    hh->desc = reinterpret_cast<const QueryDesc*>(db + o_desc);
    hh->dense_list = reinterpret_cast<const uint32_t*>(db + o_dl);
    hh->sparse_list = reinterpret_cast<const uint32_t*>(db + o_sl);
    hh->sparse_off = reinterpret_cast<const uint64_t*>(db + o_so);
    hh->nq = nq;
    hh->n_dense = (uint32_t)dense_list.size();
    hh->n_sparse = (uint32_t)sparse_list.size();
    const uint64_t wpt = b->cfg.words_per_thread == 1 ? 1 : 2;
    const uint64_t ncols = (p->words + wpt - 1) / wpt;
    const uint64_t dense_tiles = (ncols + kBatchThreads - 1) / kBatchThreads;
    hh->dense_items = dense_tiles * dense_list.size();
    QueryDesc* hd = reinterpret_cast<QueryDesc*>(hb + o_desc);
    uint32_t* hids = reinterpret_cast<uint32_t*>(hb + o_ids);
    uint32_t* htab = reinterpret_cast<uint32_t*>(hb + o_tab);
    uint64_t id_pos = 0, tab_pos = 0;
    for (uint32_t i = 0; i < nq; ++i) {
        memcpy(hids + id_pos, q[i].ids, 4ull * q[i].n);
        hd[i].ids = reinterpret_cast<const uint32_t*>(db + o_ids) + id_pos;
        hd[i].n = q[i].n;
        hd[i].tile_rows = cand[i].tile_rows;
        hd[i].out = q[i].out_words;
        hd[i].d_fill = cand[i].path == BM_PATH_SPARSE ? complement_inputs(p, q[i].ids, q[i].n) : 0u;
        hd[i].pad = 0;
        hd[i].pred = preds[i];
        if (preds[i].mode == 2) {
            uint32_t* t = htab + tab_pos;
            memset(t, 0, 4ull * preds[i].table_words32);
            for (uint32_t c = 0; c <= q[i].n; ++c)
                if (truth[i][c]) t[c >> 5] |= 1u << (c & 31);
            hd[i].pred.table = reinterpret_cast<const uint32_t*>(db + o_tab) + tab_pos;
            tab_pos += preds[i].table_words32;
        }
        id_pos += (q[i].n + 3) & ~3u;
    }
    if (!dense_list.empty())
        memcpy(hb + o_dl, dense_list.data(), 4 * dense_list.size());
    if (!sparse_list.empty())
        memcpy(hb + o_sl, sparse_list.data(), 4 * sparse_list.size());
    memcpy(hb + o_so, sparse_off.data(), 8 * sparse_off.size());

    BatchPoolArgs pa{};
    pa.base = p->d_dense;
    pa.stride_words = p->stride_words;
    pa.words = p->words;
    pa.r_bits = p->r_bits;
    pa.positions = p->d_pos;
    pa.list_begin = p->d_list_begin;
    pa.tile_index = p->d_tile_index;
    pa.tiles_per_list = p->tiles_per_list;
    const int K = planes_for(max_dense_n);
    const int kk = K <= 5 ? 5 : K <= 9 ? 9 : K <= 11 ? 11 : K <= 13 ? 13 : 17;
    cudaGraphExec_t ex = nullptr;
    rc = graph_for(p, b, sl, kk, max_words, pa, &ex);
    if (rc) return rc;
    BM_CUDA_TRY(cudaMemcpyAsync(sl.d, sl.h, bytes, cudaMemcpyHostToDevice, s));
    BM_CUDA_TRY(cudaGraphLaunch(ex, s));
    // run-length queries: one launch each of the run-length kernel after the
    // graph, reading their ids and tables from the descriptor block and adding
    // to the cardinalities the graph zeroed
    for (uint32_t i : rle_list) {
        RleArgs a{};
        a.arena = reinterpret_cast<const uint8_t*>(p->d_rle_arena);
        a.tile_index = p->d_rle_tiles;
        a.capacity = p->capacity;
        a.err = p->d_err;
        a.words = p->words;
        a.r_bits = p->r_bits;
        a.ids = hd[i].ids;
        a.n = hd[i].n;
        a.pred = hd[i].pred;  // a table, if any, in the descriptor block
        a.out = q[i].out_words;
        a.card = reinterpret_cast<unsigned long long*>(out_cards + i);
        const LaunchExtra none{};  // ids staged; the graph zeroed the cardinality
        rc = launch_rle(a, none, p->sm_count, s);
        if (rc) return rc;
    }
    BM_CUDA_TRY(cudaEventRecord(sl.ev, s));
    sl.used = true;
    return BM_OK;
}

extern "C" int bm_pool_set_batch_config(bm_pool* p, const bm_batch_config_t* c) {
    if (!p || !c || c->ctas_per_sm < 1 || c->ctas_per_sm > 3 || c->adder < 0 || c->adder > 2 ||
        (c->words_per_thread != 1 && c->words_per_thread != 2))
        return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    BatchState* b = state(p);
    if (b->cfg.ctas_per_sm != c->ctas_per_sm || b->cfg.adder != c->adder ||
        b->cfg.words_per_thread != c->words_per_thread) {
        for (auto& sl : b->slots) {
            if (sl.used) cudaEventSynchronize(sl.ev);
            for (auto& kv : sl.graphs) cudaGraphExecDestroy(kv.second);
            sl.graphs.clear();
        }
    }
    b->cfg.ctas_per_sm = c->ctas_per_sm;
    b->cfg.adder = c->adder;
    b->cfg.words_per_thread = c->words_per_thread;
    return BM_OK;
}

extern "C" int bm_pool_get_batch_config(bm_pool* p, bm_batch_config_t* c) {
    if (!p || !c) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    BatchState* b = state(p);
    c->ctas_per_sm = b->cfg.ctas_per_sm;
    c->adder = b->cfg.adder;
    c->words_per_thread = b->cfg.words_per_thread;
    return BM_OK;
}
