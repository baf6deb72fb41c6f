// Autotuner: measure candidate kernel shapes on the pool's own bitmaps and
// install the fastest; results can be cached in a text file keyed by GPU
// model and pool shape.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <functional>
#include <sstream>
#include <string>

#include "bm_internal.cuh"

namespace {

struct Tuned {
    bm_dense_config_t dense{0, 256, 4, 2, 0, 2};
    bm_sparse_config_t sparse{32768, 512, 2, 4};
    bm_batch_config_t batch{2, 0, 2};
    bool has_sparse = false;
};

// Bumped whenever kernel shapes or their parameters change meaning, so that
// entries tuned for other kernels are not reused.
constexpr int kTuneVersion = 3;

std::string cache_key(const bm_pool* p, bool lists) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, p->device);
    std::ostringstream k;
    std::string name = prop.name;
    std::replace(name.begin(), name.end(), ' ', '_');
    k << "v" << kTuneVersion << "/" << name << "/sm" << prop.multiProcessorCount << "/r" << p->r_bits << "/lists" << (lists ? 1 : 0);
    return k.str();
}

bool cache_load(const char* path, const std::string& key, Tuned& t) {
    if (!path) return false;
    std::ifstream f(path);
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        std::istringstream ls(line);
        std::string k;
        if (!(ls >> k) || k != key) continue;
        Tuned x;
        std::string tag;
        int ok = 0;
        while (ls >> tag) {
            if (sscanf(tag.c_str(), "dense=%d,%d,%d,%d,%d,%d", &x.dense.variant, &x.dense.threads,
                       &x.dense.stages, &x.dense.ctas_per_sm, &x.dense.adder,
                       &x.dense.words_per_thread) == 6)
                ok |= 1;
            else if (sscanf(tag.c_str(), "sparse=%u,%d,%d,%d", &x.sparse.tile_rows,
                            &x.sparse.threads, &x.sparse.ctas_per_sm, &x.sparse.unroll) == 4) {
                x.has_sparse = true;
            } else if (sscanf(tag.c_str(), "batch=%d,%d,%d", &x.batch.ctas_per_sm, &x.batch.adder,
                              &x.batch.words_per_thread) == 3)
                ok |= 2;
        }
        if (ok == 3) {
            t = x;
            found = true;  // the last matching line wins
        }
    }
    return found;
}

void cache_store(const char* path, const std::string& key, const Tuned& t) {
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s dense=%d,%d,%d,%d,%d,%d batch=%d,%d,%d", key.c_str(), t.dense.variant,
            t.dense.threads, t.dense.stages, t.dense.ctas_per_sm, t.dense.adder,
            t.dense.words_per_thread, t.batch.ctas_per_sm, t.batch.adder,
            t.batch.words_per_thread);
    if (t.has_sparse)
        fprintf(f, " sparse=%u,%d,%d,%d", t.sparse.tile_rows, t.sparse.threads,
                t.sparse.ctas_per_sm, t.sparse.unroll);
    fprintf(f, "\n");
    fclose(f);
}

// Median time in microseconds of `fn` on stream s (1 warm-up, 5 timed runs).
int time_us(cudaStream_t s, const std::function<int()>& fn, double* out) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int rc = fn();
    std::vector<double> t;
    for (int r = 0; r < 5 && !rc; ++r) {
        cudaEventRecord(a, s);
        rc = fn();
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        t.push_back(ms * 1e3);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    std::sort(t.begin(), t.end());
    *out = t[t.size() / 2];
    return BM_OK;
}

}  // namespace

extern "C" int bm_pool_autotune(bm_pool* p, const char* cache_path, char* report,
                                uint64_t report_len) {
    if (!p) return BM_EINVAL;
    std::vector<uint32_t> dense_ids, list_ids;
    for (uint32_t i = 0; i < p->capacity; ++i) {
        if (p->dense_present[i]) dense_ids.push_back(i);
        if (p->list_present[i]) list_ids.push_back(i);
    }
    if (dense_ids.empty()) return BM_EINVAL;
    const std::string key = cache_key(p, !list_ids.empty());
    Tuned t;
    std::ostringstream rep;
    if (cache_load(cache_path, key, t)) {
        rep << "cached " << key;
    } else {
        BM_CUDA_TRY(cudaSetDevice(p->device));
        cudaStream_t s = nullptr;
        BM_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        uint64_t* out = nullptr;
        uint64_t* cards = nullptr;
        const int nbatch = 32;
        if (cudaMalloc(&out, (size_t)nbatch * p->words * 8) != cudaSuccess ||
            cudaMalloc(&cards, nbatch * 8) != cudaSuccess) {
            cudaGetLastError();
            cudaStreamDestroy(s);
            if (out) cudaFree(out);
            return BM_ENOMEM;
        }
        int rc = BM_OK;
        // dense single query: up to 256 loaded bitmaps, theta = 2
        std::vector<uint32_t> ids(std::min<size_t>(256, dense_ids.size()));
        for (size_t i = 0; i < ids.size(); ++i) ids[i] = dense_ids[i];
        bm_query q{};
        q.ids = ids.data();
        q.n = (uint32_t)ids.size();
        q.kind = BM_KIND_THRESHOLD;
        q.theta = 2;
        q.out_words = out;
        q.path = BM_PATH_DENSE;
        std::vector<bm_dense_config_t> dense_c = {
            {0, 256, 4, 2, 0, 2}, {0, 256, 4, 3, 0, 2}, {0, 256, 4, 2, 1, 2}, {0, 256, 4, 3, 1, 2},
            {0, 256, 4, 2, 2, 2},
            {0, 256, 4, 2, 0, 1}, {0, 256, 4, 4, 0, 1}, {0, 256, 4, 4, 1, 1}, {1, 256, 3, 1, 0, 2},
            {1, 256, 2, 1, 0, 2}, {1, 128, 4, 1, 0, 2}, {1, 64, 6, 2, 0, 2}};
        double best = 1e30, tt = 0;
        for (auto& c : dense_c) {
            if (bm_pool_set_dense_config(p, &c)) continue;
            rc = time_us(s, [&] { return bm_query_run(p, &q, cards, nullptr, s); }, &tt);
            if (rc) break;
            if (tt < best) {
                best = tt;
                t.dense = c;
            }
        }
        rep << "dense=" << t.dense.variant << "," << t.dense.ctas_per_sm << "," << t.dense.adder
            << "," << t.dense.words_per_thread << " (" << best << " us, n=" << q.n << ")";
        // sparse single query
        if (!rc && !list_ids.empty()) {
            std::vector<uint32_t> sids(std::min<size_t>(512, list_ids.size()));
            for (size_t i = 0; i < sids.size(); ++i) sids[i] = list_ids[i];
            bm_query sq = q;
            sq.ids = sids.data();
            sq.n = (uint32_t)sids.size();
            sq.path = BM_PATH_SPARSE;
            best = 1e30;
            for (uint32_t tile : {16384u, 32768u, 65536u})
                for (int th : {256, 512})
                    for (int ct : {1, 2, 4})
                    for (int un : {2, 4}) {
                        bm_sparse_config_t c{tile, th, ct, un};
                        if (bm_pool_set_sparse_config(p, &c)) continue;
                        rc = time_us(s, [&] { return bm_query_run(p, &sq, cards, nullptr, s); }, &tt);
                        if (rc) break;
                        if (tt < best) {
                            best = tt;
                            t.sparse = c;
                        }
                    }
            t.has_sparse = true;
            rep << " sparse=" << t.sparse.tile_rows << "," << t.sparse.threads << ","
                << t.sparse.ctas_per_sm << "," << t.sparse.unroll << " (" << best << " us, n="
                << sq.n << ")";
        }
        // batch: 32 dense queries over rotating subsets of up to 64 bitmaps
        if (!rc) {
            const uint32_t n = (uint32_t)std::min<size_t>(64, dense_ids.size());
            std::vector<std::vector<uint32_t>> bids(nbatch, std::vector<uint32_t>(n));
            std::vector<bm_query> bq(nbatch);
            for (int i = 0; i < nbatch; ++i) {
                for (uint32_t k = 0; k < n; ++k)
                    bids[i][k] = dense_ids[(i * 7 + k * 13) % dense_ids.size()];
                bq[i] = bm_query{};
                bq[i].ids = bids[i].data();
                bq[i].n = n;
                bq[i].kind = BM_KIND_THRESHOLD;
                bq[i].theta = n / 4 + 1;
                bq[i].out_words = out + (size_t)i * p->words;
                bq[i].path = BM_PATH_DENSE;
            }
            best = 1e30;
            for (int ct : {1, 2, 3})
                for (int ad : {0, 1, 2})
                    for (int w : {2, 1}) {
                        if (ct == 3 && w != 1) continue;  // three CTAs per SM only fit one-word columns
                        bm_batch_config_t c{ct, ad, w};
                        if (bm_pool_set_batch_config(p, &c)) continue;
                        rc = time_us(s, [&] {
                            return bm_threshold_batch(p, bq.data(), nbatch, cards, nullptr, s);
                        }, &tt);
                        if (rc) break;
                        if (tt < best) {
                            best = tt;
                            t.batch = c;
                        }
                    }
            rep << " batch=" << t.batch.ctas_per_sm << "," << t.batch.adder << ","
                << t.batch.words_per_thread << " (" << best << " us, " << nbatch << "x" << n << ")";
        }
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
        cudaFree(out);
        cudaFree(cards);
        if (rc) return rc;
        cache_store(cache_path, key, t);
    }
    int rc = bm_pool_set_dense_config(p, &t.dense);
    if (!rc && t.has_sparse) rc = bm_pool_set_sparse_config(p, &t.sparse);
    if (!rc) rc = bm_pool_set_batch_config(p, &t.batch);
    if (report && report_len) {
        const std::string r = rep.str();
        const size_t n = std::min<size_t>(r.size(), report_len - 1);
        memcpy(report, r.data(), n);
        report[n] = 0;
    }
    return rc;
}
