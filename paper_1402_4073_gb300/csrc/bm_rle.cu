// Threshold and symmetric queries over run-length compressed bitmaps: the
// word-aligned run form (EWAH-like, Sec. 2.1) with the clean-run pruning of
// RBMrg (Sec. 4.1): where an input is a clean run, it adds 0 or 1 to every
// row and needs no bitwise work; only the literal ("dirty") words are added
// bit by bit.
//
// GPU form: a CTA owns a tile of 256 words (one 64-bit word column per
// thread).  For every input it reads one summary word of the tile (the run
// holding the tile's first word, and whether that clean run covers the whole
// tile).  An input that is one clean run over the whole tile costs nothing
// more: a clean-0 run is skipped, a clean-1 run adds one to a per-tile
// constant c1.  The other inputs are decoded, a half-warp per input, 16 at a
// time: their clean-0 runs add nothing, their clean-1 runs add one to the
// coverage of the columns they span (a difference array, two shared-memory
// updates per run), and only their literal words go to a shared stage, with
// one mask bit per (column, input).  Each thread then adds its column's
// literal words into K counter planes (the sixteen-input sideways-sum block
// of the dense kernel when all sixteen are literal, else two at a time), and
// at the end of the tile evaluates the predicate on count + c1 + coverage of
// its column: thresholds move down by that offset, a table is read past it.
// Only the runs and literal words of the tile are read from HBM, and clean
// words cost neither stores nor additions.
#include <algorithm>
#include <vector>

#include "bm_dense_common.cuh"

namespace bm {

void rle_encode(const uint64_t* w, uint64_t nw, std::vector<uint2>& runs,
                std::vector<uint64_t>& lits, std::vector<uint32_t>& tile_index) {
    runs.clear();
    lits.clear();
    auto type_of = [](uint64_t x) {
        return x == 0ull ? kRunClean0 : (x == ~0ull ? kRunClean1 : kRunLiteral);
    };
    uint64_t i = 0;
    while (i < nw) {
        const uint32_t t = type_of(w[i]);
        uint64_t j = i + 1;
        while (j < nw && type_of(w[j]) == t) ++j;
        runs.push_back(make_uint2((uint32_t)i | (t << 30),
                                  t == kRunLiteral ? (uint32_t)lits.size() : 0u));
        if (t == kRunLiteral) lits.insert(lits.end(), w + i, w + j);
        i = j;
    }
    runs.push_back(make_uint2((uint32_t)nw, 0u));  // sentinel: start = word count
    const uint64_t tiles = (nw + kRleTileWords - 1) / kRleTileWords;
    tile_index.assign(tiles + 1, 0u);
    uint32_t r = 0;
    for (uint64_t t = 0; t <= tiles; ++t) {
        const uint64_t w0 = std::min<uint64_t>(t * kRleTileWords, nw);
        const uint64_t w1 = std::min<uint64_t>(w0 + kRleTileWords, nw);
        while (r + 1 < runs.size() && (runs[r + 1].x & kRunStartMask) <= w0) ++r;
        // last run starting at or before the tile's first word, and whether the
        // tile lies in that one clean run
        const uint32_t type = runs[r].x >> 30;
        const bool one_run = r + 1 < runs.size() && (runs[r + 1].x & kRunStartMask) >= w1;
        const uint32_t cls = (type != kRunLiteral && one_run) ? type : kRunLiteral;
        tile_index[t] = r | (cls << 30);
    }
}

namespace {

using namespace dev;

constexpr uint32_t kRleThreads = kRleTileWords;  // one word column per thread
constexpr uint32_t kRleGroup = 2 * kRleThreads / 32;  // inputs staged per round: one per half-warp
constexpr uint32_t kRleChunk = 1024;             // inputs classified per pass

// Decode words [w0, w1) of one input (runs from index r0 of the input's runs)
// with the 16 lanes of a half-warp, so that a warp decodes two inputs at
// once.  Clean-0 runs add nothing; a clean-1 run adds one to the coverage of
// its columns (two updates of the difference array cov); a literal word w is
// stored at dst[w - w0] with bit `slot` of lmask[w - w0] set.  The lanes read
// 16 runs at a time; a lane handles its own run when the run's part of the
// tile is short, and the half-warp then spreads the long literal runs.
__device__ __forceinline__ void decode_tile(const RleArgs& a, uint32_t id, uint32_t r0,
                                            uint32_t w0, uint32_t w1, uint64_t* dst,
                                            uint32_t slot, uint32_t* lmask, int* cov,
                                            uint32_t lane) {
    constexpr uint32_t kShort = 8;  // literal words a lane stores alone
    const uint32_t seg = lane & 15, half = lane >> 4;
    const uint32_t hmask = 0xFFFFu << (16 * half);
    const uint32_t bit = 1u << slot;
    const uint2* runs = a.runs + __ldg(a.run_begin + id);
    const uint64_t* lits = a.lits + __ldg(a.lit_begin + id);
    const uint32_t nruns = __ldg(a.run_count + id);  // including the sentinel
    for (uint32_t r = r0;; r += 16) {
        uint32_t st = kRunStartMask, nx = kRunStartMask, type = kRunClean0, lo = 0;
        if (r + seg + 1 < nruns) {
            const uint2 run = __ldg(runs + r + seg);
            st = run.x & kRunStartMask;
            type = run.x >> 30;
            lo = run.y;
            nx = __ldg(&runs[r + seg + 1].x) & kRunStartMask;
        }
        const uint32_t b = max(st, w0), e = min(nx, w1);  // this run's words in the tile
        const bool live = st < w1;
        if (live && type == kRunClean1) {
            atomicAdd(&cov[b - w0], 1);
            atomicAdd(&cov[e - w0], -1);
        }
        const bool lit = live && type == kRunLiteral;
        if (lit && e - b <= kShort) {
            for (uint32_t w = b; w < e; ++w) {
                dst[w - w0] = __ldg(lits + lo + (w - st));
                atomicOr(&lmask[w - w0], bit);
            }
        }
        uint32_t big = (__ballot_sync(hmask, lit && e - b > kShort) >> (16 * half)) & 0xFFFFu;
        while (big) {
            const uint32_t j = __ffs(big) - 1;
            big &= big - 1;
            const uint32_t sj = __shfl_sync(hmask, st, j, 16);
            const uint32_t bj = __shfl_sync(hmask, b, j, 16);
            const uint32_t ej = __shfl_sync(hmask, e, j, 16);
            const uint32_t lj = __shfl_sync(hmask, lo, j, 16);
            for (uint32_t w = bj + seg; w < ej; w += 16) {
                dst[w - w0] = __ldg(lits + lj + (w - sj));
                atomicOr(&lmask[w - w0], bit);
            }
        }
        // runs start in increasing order: once one starts past the tile, all later do
        if (__ballot_sync(hmask, !live) & hmask) return;
    }
}

// Output word of one column: the predicate on count + off per row, where the
// planes P hold the literal words' count and `off` the inputs covering the
// column with ones (c1 + clean-1 coverage).  Thresholds move down by off
// (those at or below it always hold); a table is read at count + off.
template <int K>
__device__ __forceinline__ uint64_t eval_offset(const uint32_t (&P)[2][K], const Pred& p,
                                                const uint32_t* tab, uint32_t off) {
    if (p.mode == 2) {
        uint64_t word = 0;
#pragma unroll
        for (int l = 0; l < 2; ++l)
            for (int b = 0; b < 32; ++b) {
                uint32_t c = 0;
#pragma unroll
                for (int j = 0; j < K; ++j) c |= ((P[l][j] >> b) & 1u) << j;
                c += off;
                word |= (uint64_t)((tab[c >> 5] >> (c & 31u)) & 1u) << (32 * l + b);
            }
        return word;
    }
    Pred q = p;
    if (p.mode == 1) {
        uint32_t k = 0;
#pragma unroll
        for (int i = 0; i < kMaxTransitions; ++i) {
            if ((uint32_t)i < p.ntrans) {
                if (p.trans[i] <= off)
                    q.v0 ^= 1u;
                else
                    q.trans[k++] = p.trans[i] - off;
            }
        }
        q.ntrans = k;
    }
    return (uint64_t)eval_pred<K>(P[0], q, tab) | ((uint64_t)eval_pred<K>(P[1], q, tab) << 32);
}

// The pruning of RBMrg over a whole tile (Sec. 4.1): every row's count lies
// in [lo, hi], lo = the inputs that are one clean-1 run over the tile (k in
// the paper), hi = lo + the inputs left to decode.  When f takes one value
// over [lo, hi] (for a threshold T: T - k <= 0, or T - k beyond the inputs
// left), that value is the tile's output and nothing needs decoding.
// Returns it, or -1.  tab: f over 0..n (mode 2).
__device__ __forceinline__ int constant_over(const Pred& p, const uint32_t* tab, uint32_t lo,
                                             uint32_t hi) {
    if (p.mode == 0) return (int)p.v0;
    if (p.mode == 1) {
        uint32_t v = p.v0;
#pragma unroll
        for (int i = 0; i < kMaxTransitions; ++i) {
            if ((uint32_t)i >= p.ntrans) break;
            if (p.trans[i] <= lo) v ^= 1u;
            else if (p.trans[i] <= hi) return -1;
        }
        return (int)v;
    }
    const uint32_t v = (tab[lo >> 5] >> (lo & 31u)) & 1u;
    for (uint32_t w = lo >> 5; w <= (hi >> 5); ++w) {
        uint32_t m = ~0u;
        if (w == (lo >> 5)) m &= ~0u << (lo & 31u);
        if (w == (hi >> 5) && (hi & 31u) != 31u) m &= (2u << (hi & 31u)) - 1u;
        if ((tab[w] ^ (v ? ~0u : 0u)) & m) return -1;
    }
    return (int)v;
}

template <int K>
__global__ void __launch_bounds__(kRleThreads, K <= 9 ? 4 : (K <= 13 ? 3 : 2))
    rle_kernel(RleArgs a, const __grid_constant__ LaunchExtra x) {
    extern __shared__ __align__(16) uint64_t sm64[];
    uint64_t* stage = sm64;                                                    // [kRleGroup][256]
    uint2* dirty = reinterpret_cast<uint2*>(stage + kRleGroup * kRleThreads);  // [kRleChunk]
    uint32_t* tab = reinterpret_cast<uint32_t*>(dirty + kRleChunk);           // f over 0..n
    __shared__ uint32_t s_c1, s_nd;
    __shared__ uint32_t lmask[kRleThreads];  // per column: staged inputs with a literal word
    __shared__ int cov[kRleThreads + 1];     // clean-1 coverage, as differences
    __shared__ int warp_tot[kRleThreads / 32];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t tab_words = a.pred.mode == 2 ? (a.n + 1 + 31) / 32 : 0u;
    for (uint32_t w = tid; w < tab_words; w += kRleThreads) tab[w] = a.pred.table[w];
    lmask[tid] = 0u;
    const uint64_t ntiles = (a.words + kRleTileWords - 1) / kRleTileWords;
    unsigned long long card = 0;
    // ids and tile summaries of up to four inputs per thread.  With one chunk
    // (n <= kRleChunk) the ids stay in registers for every tile and the next
    // tile's summaries are loaded while this tile is decoded.
    constexpr uint32_t kPer = kRleChunk / kRleThreads;
    const bool one_chunk = a.n <= kRleChunk;
    uint32_t id[kPer], sum_next[kPer];
    auto load_ids = [&](uint32_t c0, uint32_t m) {
#pragma unroll
        for (uint32_t u = 0; u < kPer; ++u) {
            const uint32_t i = tid + u * kRleThreads;
            id[u] = i >= m ? 0u : x.n_inline ? x.inl[c0 + i] : __ldg(a.ids + c0 + i);
        }
    };
    auto load_sums = [&](uint32_t m, uint64_t tile, uint32_t (&sum)[kPer]) {
#pragma unroll
        for (uint32_t u = 0; u < kPer; ++u) {
            const uint32_t i = tid + u * kRleThreads;
            sum[u] = i < m && tile < ntiles
                         ? __ldg(a.tile_index + (uint64_t)id[u] * a.tiles_plus_one + tile)
                         : 0u;  // clean-0: nothing to add
        }
    };
    if (one_chunk) {
        load_ids(0, a.n);
        load_sums(a.n, blockIdx.x, sum_next);
    }
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t w0 = (uint32_t)(tile * kRleTileWords);
        const uint32_t w1 = (uint32_t)min((uint64_t)w0 + kRleTileWords, a.words);
        uint32_t P[2][K];
        zero_planes<K, 2>(P);
        int konst = -1;  // the tile's output when it needs no decoding
        if (tid == 0) {
            s_c1 = 0u;
            cov[kRleThreads] = 0;
        }
        cov[tid] = 0;
        for (uint32_t c0 = 0; c0 < a.n; c0 += kRleChunk) {
            const uint32_t m = min(kRleChunk, a.n - c0);
            if (tid == 0) s_nd = 0u;
            __syncthreads();
            // classify by the tile summary: one clean run over the whole tile,
            // or to be decoded
            uint32_t sum[kPer];
            if (one_chunk) {
#pragma unroll
                for (uint32_t u = 0; u < kPer; ++u) sum[u] = sum_next[u];
            } else {
                load_ids(c0, m);
                load_sums(m, tile, sum);
            }
#pragma unroll
            for (uint32_t u = 0; u < kPer; ++u) {
                const uint32_t cls = sum[u] >> 30;
                if (cls == kRunClean1) atomicAdd(&s_c1, 1u);
                if (cls == kRunLiteral)
                    dirty[atomicAdd(&s_nd, 1u)] = make_uint2(id[u], sum[u] & kRunStartMask);
            }
            __syncthreads();
            if (one_chunk) load_sums(m, tile + gridDim.x, sum_next);  // in flight while decoding
            const uint32_t nd = s_nd;
            if (one_chunk) konst = constant_over(a.pred, tab, s_c1, s_c1 + nd);
            __syncthreads();  // every thread has nd before the next chunk resets it
            if (konst >= 0) break;  // the whole tile is one value: no decoding
            for (uint32_t g0 = 0; g0 < nd; g0 += kRleGroup) {
                const uint32_t gn = min(kRleGroup, nd - g0);
                // half-warp h of the CTA decodes entry h of the group into stage row h
                const uint32_t e = 2 * warp + (lane >> 4);
                if (e < gn) {
                    const uint2 d = dirty[g0 + e];
                    decode_tile(a, d.x, d.y, w0, w1, stage + e * kRleThreads, e, lmask, cov, lane);
                }
                __syncthreads();
                // add this column's literal words: a full group through the
                // sixteen-input tree, otherwise two at a time
                uint32_t mk = lmask[tid];
                lmask[tid] = 0u;
                auto get = [&](uint32_t row) {
                    const uint64_t x = stage[row * kRleThreads + tid];
                    Slice<2> v;
                    v.v[0] = (uint32_t)x;
                    v.v[1] = (uint32_t)(x >> 32);
                    return v;
                };
                if (mk == 0xFFFFu) {
                    Slice<2> v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = get(i);
                    add_group<K, 2, 16>(P, v);
                } else {
                    while (mk) {
                        const uint32_t i0 = __ffs(mk) - 1;
                        mk &= mk - 1;
                        const Slice<2> u = get(i0);
                        if (mk) {
                            const uint32_t i1 = __ffs(mk) - 1;
                            mk &= mk - 1;
                            const Slice<2> v = get(i1);
                            add2<K>(P[0], u.v[0], v.v[0]);
                            add2<K>(P[1], u.v[1], v.v[1]);
                        } else {
                            add1<K>(P[0], u.v[0]);
                            add1<K>(P[1], u.v[1]);
                        }
                    }
                }
                __syncthreads();
            }
        }
        if (konst >= 0) {
            const uint64_t col = (uint64_t)w0 + tid;
            if (col < a.words) {
                uint64_t word = konst ? ~0ull : 0ull;
                if (col == a.words - 1 && (a.r_bits & 63u)) word &= (1ull << (a.r_bits & 63u)) - 1ull;
                a.out[col] = word;
                card += (unsigned long long)__popcll(word);
            }
            __syncthreads();  // s_c1, s_nd are reused by the next tile
            continue;
        }
        __syncthreads();  // c1 and the coverage differences are final
        // coverage of this thread's column: inclusive prefix sum of cov
        int x = cov[tid];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        for (uint32_t w = 0; w < warp; ++w) x += warp_tot[w];
        const uint32_t off = s_c1 + (uint32_t)x;
        const uint64_t col = (uint64_t)w0 + tid;
        if (col < a.words) {
            uint64_t word = eval_offset<K>(P, a.pred, tab, off);
            if (col == a.words - 1 && (a.r_bits & 63u)) word &= (1ull << (a.r_bits & 63u)) - 1ull;
            a.out[col] = word;
            card += (unsigned long long)__popcll(word);
        }
        __syncthreads();  // s_c1, s_nd, cov and warp_tot are reused by the next tile
    }
    flush_card_block(card, a.card, x.acc, x.ticket);
}

template <int K>
int launch_k(const RleArgs& a, const LaunchExtra& x, int sm_count, cudaStream_t s) {
    const size_t tab_words = a.pred.mode == 2 ? (a.n + 1 + 31) / 32 : 0;
    const size_t smem = (size_t)kRleGroup * kRleThreads * 8 + (size_t)kRleChunk * 8 + tab_words * 4;
    BM_CUDA_TRY(
        cudaFuncSetAttribute(rle_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // persistent: as many CTAs as fit at once (tiles are latency-bound, so all
    // of them count), or one per tile
    int per_sm = 0;
    BM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rle_kernel<K>,
                                                              (int)kRleThreads, smem));
    const uint64_t ntiles = (a.words + kRleTileWords - 1) / kRleTileWords;
    const unsigned grid = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>(ntiles, (uint64_t)sm_count * (uint64_t)std::max(1, per_sm)));
    rle_kernel<K><<<grid, kRleThreads, smem, s>>>(a, x);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

}  // namespace

int launch_rle(const RleArgs& a, const LaunchExtra& x, int sm_count, cudaStream_t s) {
    if (a.words == 0) return BM_OK;
    const int k = planes_for(a.n);
    if (k <= 5) return launch_k<5>(a, x, sm_count, s);
    if (k <= 9) return launch_k<9>(a, x, sm_count, s);
    if (k <= 13) return launch_k<13>(a, x, sm_count, s);
    return launch_k<17>(a, x, sm_count, s);
}

}  // namespace bm

using namespace bm;

extern "C" {

int bm_pool_put_rle(bm_pool* p, uint32_t first_id, uint32_t count) {
    if (!p || count == 0) return BM_EINVAL;
    if ((uint64_t)first_id + count > p->capacity) return BM_ERANGE;
    for (uint32_t j = 0; j < count; ++j)
        if (!p->dense_present[first_id + j]) return BM_ERANGE;
    std::lock_guard<std::mutex> lk(p->mu);
    BM_CUDA_TRY(cudaSetDevice(p->device));
    const uint64_t tiles1 = (uint64_t)p->rle_tiles + 1;
    if (!p->d_run_begin) {
        int rc = track_alloc(p, (void**)&p->d_run_begin, (size_t)p->capacity * 8);
        if (!rc) rc = track_alloc(p, (void**)&p->d_lit_begin, (size_t)p->capacity * 8);
        if (!rc) rc = track_alloc(p, (void**)&p->d_run_count, (size_t)p->capacity * 4);
        if (!rc) rc = track_alloc(p, (void**)&p->d_rle_tiles, (size_t)p->capacity * tiles1 * 4);
        if (rc) return rc;
        BM_CUDA_TRY(cudaMemset(p->d_run_begin, 0, (size_t)p->capacity * 8));
        BM_CUDA_TRY(cudaMemset(p->d_lit_begin, 0, (size_t)p->capacity * 8));
        BM_CUDA_TRY(cudaMemset(p->d_run_count, 0, (size_t)p->capacity * 4));
        BM_CUDA_TRY(cudaMemset(p->d_rle_tiles, 0, (size_t)p->capacity * tiles1 * 4));
    }
    // grow an arena of `elem` bytes per entry to hold `need` entries
    auto grow = [&](void** arena, uint64_t* cap, uint64_t used, uint64_t need, size_t elem) -> int {
        if (need <= *cap) return BM_OK;
        const uint64_t ncap = std::max<uint64_t>({need, *cap + *cap / 2, 1u << 16});
        void* nd = nullptr;
        int rc = track_alloc(p, &nd, ncap * elem);
        if (rc) return rc;
        if (used) BM_CUDA_TRY(cudaMemcpy(nd, *arena, used * elem, cudaMemcpyDeviceToDevice));
        track_free(p, *arena, *cap * elem);
        *arena = nd;
        *cap = ncap;
        return BM_OK;
    };
    std::vector<uint64_t> host(p->words);
    std::vector<uint2> runs;
    std::vector<uint64_t> lits;
    std::vector<uint32_t> tidx;
    for (uint32_t j = 0; j < count; ++j) {
        const uint32_t id = first_id + j;
        BM_CUDA_TRY(cudaMemcpy(host.data(), p->d_dense + (uint64_t)id * p->stride_words,
                               p->words * 8, cudaMemcpyDeviceToHost));
        rle_encode(host.data(), p->words, runs, lits, tidx);
        int rc = grow((void**)&p->d_runs, &p->runs_cap, p->runs_used, p->runs_used + runs.size(), 8);
        if (!rc)
            rc = grow((void**)&p->d_lits, &p->lits_cap, p->lits_used,
                      p->lits_used + std::max<size_t>(lits.size(), 1), 8);
        if (rc) return rc;
        BM_CUDA_TRY(cudaMemcpy(p->d_runs + p->runs_used, runs.data(), runs.size() * 8,
                               cudaMemcpyHostToDevice));
        if (!lits.empty())
            BM_CUDA_TRY(cudaMemcpy(p->d_lits + p->lits_used, lits.data(), lits.size() * 8,
                                   cudaMemcpyHostToDevice));
        BM_CUDA_TRY(cudaMemcpy(p->d_rle_tiles + (uint64_t)id * tiles1, tidx.data(), tiles1 * 4,
                               cudaMemcpyHostToDevice));
        const uint64_t rb = p->runs_used, lb = p->lits_used;
        const uint32_t nr = (uint32_t)runs.size();
        BM_CUDA_TRY(cudaMemcpy(p->d_run_begin + id, &rb, 8, cudaMemcpyHostToDevice));
        BM_CUDA_TRY(cudaMemcpy(p->d_lit_begin + id, &lb, 8, cudaMemcpyHostToDevice));
        BM_CUDA_TRY(cudaMemcpy(p->d_run_count + id, &nr, 4, cudaMemcpyHostToDevice));
        p->runs_used += runs.size();
        p->lits_used += lits.size();
        p->rle_runs[id] = runs.size() - 1;
        p->rle_lits[id] = lits.size();
        p->rle_present[id] = 1;
    }
    return BM_OK;
}

int bm_pool_rle_info(const bm_pool* p, uint32_t id, uint64_t* runs, uint64_t* literal_words) {
    if (!p) return BM_EINVAL;
    if (id >= p->capacity || !p->rle_present[id]) return BM_ERANGE;
    if (runs) *runs = p->rle_runs[id];
    if (literal_words) *literal_words = p->rle_lits[id];
    return BM_OK;
}

}  // extern "C"
