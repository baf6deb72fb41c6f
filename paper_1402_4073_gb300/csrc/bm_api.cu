// Single-query entry points: host validation, predicate compilation,
// staging of ids and truth tables, path choice and kernel launch.
#include <algorithm>
#include <cstring>

#include "bm_device.cuh"
#include "bm_select.h"

namespace bm {

void threshold_truth(uint32_t n, uint32_t theta, std::vector<uint8_t>& f) {
    f.assign((size_t)n + 1, 0);
    for (uint32_t c = 0; c <= n; ++c) f[c] = c >= theta;
}

void interval_truth(uint32_t n, uint32_t lo, uint32_t hi, std::vector<uint8_t>& f) {
    f.assign((size_t)n + 1, 0);
    for (uint32_t c = 0; c <= n; ++c) f[c] = c >= lo && c <= hi;
}

Pred compile_pred(const uint8_t* f, uint32_t n) {
    Pred p{};
    p.v0 = f[0] ? 1u : 0u;
    uint32_t m = 0;
    for (uint32_t c = 1; c <= n; ++c)
        if ((f[c] != 0) != (f[c - 1] != 0)) ++m;
    if (m == 0) {
        p.mode = 0;
        return p;
    }
    if (m <= (uint32_t)kMaxTransitions) {
        p.mode = 1;
        for (uint32_t c = 1; c <= n; ++c)
            if ((f[c] != 0) != (f[c - 1] != 0)) p.trans[p.ntrans++] = c;
        return p;
    }
    p.mode = 2;
    p.table_words32 = (n + 1 + 31) / 32;
    return p;
}

int query_truth(const bm_query* q, std::vector<uint8_t>& f) {
    switch (q->kind) {
        case BM_KIND_THRESHOLD: threshold_truth(q->n, q->theta, f); return BM_OK;
        case BM_KIND_INTERVAL: interval_truth(q->n, q->lo, q->hi, f); return BM_OK;
        case BM_KIND_TABLE:
            if (!q->table) return BM_EINVAL;
            f.assign((size_t)q->n + 1, 0);
            for (uint32_t c = 0; c <= q->n; ++c)
                f[c] = (uint8_t)((q->table[c >> 6] >> (c & 63)) & 1u);
            return BM_OK;
        default: return BM_EINVAL;
    }
}

int validate_ids(const bm_pool* p, const uint32_t* ids, uint32_t n, int path) {
    if (!ids || n == 0 || n > BM_N_MAX) return BM_EINVAL;
    for (uint32_t k = 0; k < n; ++k) {
        if (ids[k] >= p->capacity) return BM_ERANGE;
        if (path == BM_PATH_DENSE && !p->dense_present[ids[k]]) return BM_ERANGE;
        if (path == BM_PATH_SPARSE && !p->list_present[ids[k]]) return BM_ERANGE;
        if (path == BM_PATH_RLE && !p->rle_present[ids[k]]) return BM_ERANGE;
        if (path == BM_PATH_AUTO && !p->dense_present[ids[k]] && !p->list_present[ids[k]])
            return BM_ERANGE;
    }
    return BM_OK;
}

uint32_t complement_inputs(const bm_pool* p, const uint32_t* ids, uint32_t n) {
    uint32_t d = 0;
    for (uint32_t k = 0; k < n; ++k) d += p->list_complement[ids[k]];
    return d;
}

// Stage ids (and a table-mode truth table) and launch the chosen kernel.
// A query of at most kInlineIds inputs whose predicate needs no table passes
// its ids in the kernel's parameter block: nothing is copied to the device.
// The cardinality is stored by the kernel itself through the staging slot's
// header (no memset), so such a query is one launch.
// dense_words = 1 runs the dense counter with one 64-bit word per thread
// (twice the threads of the pool's shape: more parallelism for few rows).
int run_single(bm_pool* p, const uint32_t* ids, uint32_t n, const std::vector<uint8_t>& f,
               int path, uint32_t tile_rows, uint64_t* out_words, uint64_t* out_card,
               cudaStream_t s, uint32_t dense_words = 0) {
    Pred pred = compile_pred(f.data(), n);
    const bool inl = pred.mode != 2 && n <= kInlineIds;
    const size_t ids_bytes = inl ? 0 : ((size_t)n * 4 + 15) & ~(size_t)15;
    const size_t tab_bytes = pred.mode == 2 ? (size_t)pred.table_words32 * 4 : 0;
    bm_stage_slot* sl = nullptr;
    int rc = stage_acquire(p, ids_bytes + tab_bytes, &sl, s);
    if (rc) return rc;
    if (!inl) memcpy(sl->h, ids, (size_t)n * 4);
    if (tab_bytes) {
        uint32_t* t = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(sl->h) + ids_bytes);
        memset(t, 0, tab_bytes);
        for (uint32_t c = 0; c <= n; ++c)
            if (f[c]) t[c >> 5] |= 1u << (c & 31);
        pred.table = reinterpret_cast<const uint32_t*>(static_cast<uint8_t*>(sl->d) + ids_bytes);
    }
    if (ids_bytes + tab_bytes) {
        rc = stage_commit(sl, ids_bytes + tab_bytes, s);
        if (rc) return rc;
    }
    const uint32_t* d_ids = inl ? nullptr : static_cast<const uint32_t*>(sl->d);
    unsigned long long* acc = out_card ? sl->acc() : nullptr;
    LaunchExtra x{};
    x.acc = acc;
    x.ticket = sl->ticket();
    x.n_inline = inl ? n : 0u;
    if (inl) memcpy(x.inl, ids, (size_t)n * 4);
    unsigned long long* card = reinterpret_cast<unsigned long long*>(out_card);
    if (path == BM_PATH_SPARSE) {
        SparseArgs a{};
        a.positions = p->d_pos;
        a.list_begin = p->d_list_begin;
        a.tile_index = p->d_tile_index;
        a.tiles_per_list = p->tiles_per_list;
        a.tile_rows = tile_rows ? tile_rows : p->sparse_cfg.tile_rows;
        a.r_bits = p->r_bits;
        a.ids = d_ids;
        a.n = n;
        a.d_fill = complement_inputs(p, ids, n);
        a.pred = pred;
        a.out = out_words;
        a.card = card;
        rc = launch_sparse(a, x, p->sparse_cfg, p->sm_count, s);
    } else if (path == BM_PATH_RLE) {
        RleArgs a{};
        a.arena = reinterpret_cast<const uint8_t*>(p->d_rle_arena);
        a.tile_index = p->d_rle_tiles;
        a.capacity = p->capacity;
        a.err = p->d_err;
        a.words = p->words;
        a.r_bits = p->r_bits;
        a.ids = d_ids;
        a.n = n;
        a.pred = pred;
        a.out = out_words;
        a.card = card;
        rc = launch_rle(a, x, p->sm_count, s);
    } else {
        DenseArgs a{};
        a.base = p->d_dense;
        a.stride_words = p->stride_words;
        a.words = p->words;
        a.r_bits = p->r_bits;
        a.ids = d_ids;
        a.n = n;
        a.pred = pred;
        a.out = out_words;
        a.err = p->d_err;
        a.card = card;
        LoopedForm lf{};
        DenseConfig cfg = p->dense_cfg;
        if (dense_words == 1) {  // direct loads, 8-byte columns (32-input blocks need two words)
            cfg.variant = 0;
            cfg.words_per_thread = 1;
            if (cfg.adder == 2) cfg.adder = 0;
        }
        if (looped_form(pred, n, p->looped_max, &lf))
            rc = launch_looped(a, x, lf, p->sm_count, s);
        else
            rc = launch_dense(a, x, cfg, p->sm_count, s);
    }
    int rc2 = stage_release(sl, s);
    return rc ? rc : rc2;
}

}  // namespace bm

using namespace bm;

extern "C" {

int bm_threshold(bm_pool* p, const uint32_t* ids, uint32_t n, uint32_t theta,
                 uint64_t* out_words, uint64_t* out_card, void* stream) {
    if (!p || !out_words) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    int rc = validate_ids(p, ids, n, BM_PATH_DENSE);
    if (rc) return rc;
    BM_CUDA_TRY(cudaSetDevice(p->device));
    std::vector<uint8_t> f;
    threshold_truth(n, theta, f);
    return run_single(p, ids, n, f, BM_PATH_DENSE, 0, out_words, out_card,
                      static_cast<cudaStream_t>(stream));
}

int bm_symmetric(bm_pool* p, const uint32_t* ids, uint32_t n, const uint64_t* table,
                 uint64_t* out_words, uint64_t* out_card, void* stream) {
    if (!p || !out_words || !table) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    int rc = validate_ids(p, ids, n, BM_PATH_DENSE);
    if (rc) return rc;
    BM_CUDA_TRY(cudaSetDevice(p->device));
    std::vector<uint8_t> f((size_t)n + 1);
    for (uint32_t c = 0; c <= n; ++c) f[c] = (uint8_t)((table[c >> 6] >> (c & 63)) & 1u);
    return run_single(p, ids, n, f, BM_PATH_DENSE, 0, out_words, out_card,
                      static_cast<cudaStream_t>(stream));
}

int bm_query_run(bm_pool* p, const bm_query* q, uint64_t* out_card, int32_t* chosen_path,
                 void* stream) {
    if (!p || !q || !q->out_words || q->reserved) return BM_EINVAL;
    if (q->path < BM_PATH_AUTO || q->path > BM_PATH_RLE) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    int rc = validate_ids(p, q->ids, q->n, q->path);
    if (rc) return rc;
    std::vector<uint8_t> f;
    rc = query_truth(q, f);
    if (rc) return rc;
    BM_CUDA_TRY(cudaSetDevice(p->device));
    Candidate c{q->path, 0, 0};
    if (q->path == BM_PATH_AUTO) c = single_query_candidate(p, q->ids, q->n, f);
    if (chosen_path) *chosen_path = c.path;
    return run_single(p, q->ids, q->n, f, c.path, c.tile_rows, q->out_words, out_card,
                      static_cast<cudaStream_t>(stream), c.dense_words);
}

int bm_pool_set_sparse_config(bm_pool* p, const bm_sparse_config_t* c) {
    if (!p || !c || c->tile_rows == 0 || c->tile_rows % kListTileRows || c->tile_rows > 65536)
        return BM_EINVAL;
    if (c->threads < 64 || c->threads > 512 || c->threads % 32 || c->ctas_per_sm < 1 ||
        c->ctas_per_sm > 8 || (c->unroll != 2 && c->unroll != 4))
        return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    p->sparse_cfg = SparseConfig{c->tile_rows, c->threads, c->ctas_per_sm, c->unroll};
    return BM_OK;
}

int bm_pool_get_sparse_config(bm_pool* p, bm_sparse_config_t* c) {
    if (!p || !c) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    c->tile_rows = p->sparse_cfg.tile_rows;
    c->threads = p->sparse_cfg.threads;
    c->ctas_per_sm = p->sparse_cfg.ctas_per_sm;
    c->unroll = p->sparse_cfg.unroll;
    return BM_OK;
}

}  // extern "C"
