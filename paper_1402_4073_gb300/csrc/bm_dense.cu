// Dense bit-sliced carry-save counter (the adder-circuit family of Sec. 4.3
// evaluated word-parallel, 32 rows per register), its predicate and the
// output/cardinality epilogue.
//
// Each thread owns a column of 128 rows (one 16-byte slice: two 64-bit
// words, four 32-bit lanes) of every input bitmap and streams the N inputs of
// that column through K counter planes held in registers.  Sixteen inputs
// at a time go through a 15-full-adder sideways-sum tree (one LOP3 for each
// sum and each carry).  After the last input the predicate (threshold
// comparator, interval, or table lookup) turns the planes into the output
// slice, which is stored and popcounted.
//
// Two ways of feeding the inputs:
//  * variant 0 ("direct"): each thread issues 16 streaming 128-bit loads per
//    step, coalesced across the warp (consecutive threads read consecutive
//    16-byte slices of the same bitmap).
//  * variant 1 ("bulk"): a producer warp moves each (tile, group of 16
//    bitmaps) into a shared-memory stage with bulk copies (cp.async.bulk, the
//    non-tensor TMA form; one lane per bitmap) completing on an mbarrier; the
//    consumer warps read 128-bit slices from shared memory.  Stages are
//    recycled through a second mbarrier per stage.  All waits are bounded.
#include <algorithm>

#include "bm_dense_common.cuh"

namespace bm {

int planes_for(uint32_t n) {
    int k = 0;
    while ((1ull << k) <= n) ++k;  // counts 0..n need k bits
    return k;
}

namespace {

using namespace dev;

__device__ __forceinline__ void load_table(const DenseArgs& a, uint32_t* tab, int tid, int nthr) {
    if (a.pred.mode == 2)
        for (uint32_t i = tid; i < a.pred.table_words32; i += nthr) tab[i] = a.pred.table[i];
}

// ---------------------------------------------------------------------------
// variant 0: direct streaming loads

template <int K, int G, int L>
__global__ void __launch_bounds__(256, (K <= 13 ? 2 : 1))
    csa_direct_kernel(DenseArgs a, const __grid_constant__ LaunchExtra x) {
    extern __shared__ uint32_t tab[];
    __shared__ __align__(16) uint32_t s_ids[kInlineIds];
    const uint32_t* ids = launch_ids(a.ids, x, s_ids);
    load_table(a, tab, threadIdx.x, blockDim.x);
    __syncthreads();
    constexpr uint64_t W = L / 2;  // 64-bit words per thread per input
    const uint64_t ncols = (a.words + W - 1) / W;
    const bool vec_ok = ((reinterpret_cast<uintptr_t>(a.out) & 15u) == 0);
    unsigned long long card = 0;
    for (uint64_t col = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; col < ncols;
         col += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t P[L][K];
        zero_planes<K, L>(P);
        count_column<K, G, L, true>(P, a.base + W * col, ids, a.n, a.stride_words);
        card += finish_column<K, L>(P, a.pred, tab, a.r_bits, a.words, a.out, col, vec_ok);
    }
    flush_card_block(card, a.card, x.acc, x.ticket);
}

// ---------------------------------------------------------------------------
// variant 1: bulk-copy pipeline through shared memory

template <int K, int NT>
__global__ void __launch_bounds__(NT + 32, 1)
    csa_bulk_kernel(DenseArgs a, const __grid_constant__ LaunchExtra x, int stages) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint4* buf = reinterpret_cast<uint4*>(smem);  // [stages][16][NT]
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)stages * 16 * NT * 16);
    uint64_t* empty = full + stages;
    uint32_t* tab = reinterpret_cast<uint32_t*>(empty + stages);
    __shared__ __align__(16) uint32_t s_ids[kInlineIds];
    const uint32_t* ids = launch_ids(a.ids, x, s_ids);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kConsumerWarps = NT / 32;
    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        fence_barrier_init();
    }
    load_table(a, tab, tid, blockDim.x);
    __syncthreads();

    const uint64_t ncols = (a.words + 1) / 2;
    const uint64_t ntiles = (ncols + NT - 1) / NT;
    const uint32_t ngroups = (a.n + 15) / 16;
    const uint64_t stride_bytes = a.stride_words * 8;

    if (warp == kConsumerWarps) {
        // producer warp: lane 0 waits for free stages and posts the expected
        // bytes; lane b then issues the bulk copy of bitmap b of the group,
        // so the 16 copies of a stage go out in parallel
        const uint64_t pol = policy_evict_first();
        uint64_t it = 0;
        bool ok = true;
        for (uint64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const uint64_t off = tile * (uint64_t)NT * 16;
            const uint32_t bytes = (uint32_t)min((uint64_t)NT * 16, stride_bytes - off);
            for (uint32_t g = 0; g < ngroups; ++g, ++it) {
                const int s = (int)(it % (uint64_t)stages);
                bool free_stage = true;
                if (lane == 0 && it >= (uint64_t)stages)
                    free_stage = mbar_wait_bounded(&empty[s], (uint32_t)((it / stages - 1) & 1), a.err);
                if (!__shfl_sync(0xFFFFFFFFu, free_stage, 0)) {
                    ok = false;
                    break;
                }
                const uint32_t nb = min(16u, a.n - g * 16);
                if (lane == 0) mbar_arrive_expect_tx(&full[s], nb * bytes);
                __syncwarp();
                if ((uint32_t)lane < nb) {
                    const uint8_t* src = reinterpret_cast<const uint8_t*>(a.base) +
                                         (uint64_t)ids[g * 16 + lane] * stride_bytes + off;
                    bulk_g2s(buf + ((size_t)s * 16 + lane) * NT, src, bytes, &full[s], pol);
                }
                __syncwarp();
            }
        }
        // every issued copy must land before this CTA may exit
        if (lane == 0) {
            const uint64_t first = it > (uint64_t)stages ? it - stages : 0;
            for (uint64_t j = first; j < it; ++j)
                mbar_wait_bounded(&full[j % stages], (uint32_t)((j / stages) & 1), a.err);
        }
        return;
    }

    // consumers
    const bool vec_ok = ((reinterpret_cast<uintptr_t>(a.out) & 15u) == 0);
    unsigned long long card = 0;
    uint64_t it = 0;
    bool ok = true;
    for (uint64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        uint32_t P[4][K];
        zero_planes<K, 4>(P);
        for (uint32_t g = 0; g < ngroups; ++g, ++it) {
            const int s = (int)(it % (uint64_t)stages);
            // every lane waits; the warp proceeds only if all lanes saw the stage land
            const bool landed = mbar_wait_bounded(&full[s], (uint32_t)((it / stages) & 1), a.err);
            if (!__all_sync(0xFFFFFFFFu, landed)) {
                ok = false;
                break;
            }
            const Slice<4>* st = reinterpret_cast<const Slice<4>*>(buf + (size_t)s * 16 * NT) + tid;
            const uint32_t nb = min(16u, a.n - g * 16);
            if (nb == 16) {
                Slice<4> v[16];
#pragma unroll
                for (int b = 0; b < 16; ++b) v[b] = st[b * NT];
                add_group<K, 4, 16>(P, v);
            } else {
                add_partial<K, 4>(P, nb, [&](uint32_t b) { return st[b * NT]; });
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        if (!ok) break;
        const uint64_t col = tile * NT + tid;
        if (col < ncols)
            card += finish_column<K, 4>(P, a.pred, tab, a.r_bits, a.words, a.out, col, vec_ok);
    }
    // every consumer warp contributes (nothing if its waits gave up, which
    // the error word reports), so the last one completes the cardinality
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) card += __shfl_xor_sync(0xFFFFFFFFu, card, o);
    if (lane == 0)
        card_contribute(ok ? card : 0ull, a.card, x.acc, x.ticket, gridDim.x * kConsumerWarps);
}

template <int K>
int launch_k(const DenseArgs& a, const LaunchExtra& x, const DenseConfig& cfg, int sm_count,
             cudaStream_t s) {
    const uint64_t ncols = (a.words + 1) / 2;
    const size_t tab_bytes = a.pred.mode == 2 ? (size_t)a.pred.table_words32 * 4 : 0;
    if (cfg.variant == 0) {
        const int threads = 256;
        const int L = cfg.words_per_thread == 1 ? 2 : 4;
        const uint64_t cols = L == 4 ? ncols : a.words;
        const uint64_t blocks_needed = (cols + threads - 1) / threads;
        const uint64_t cap = (uint64_t)sm_count * (uint64_t)std::max(1, cfg.ctas_per_sm);
        const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min(blocks_needed, cap));
        constexpr int G32 = K >= 6 ? 32 : 16;  // 32-input blocks need a sixth plane
        auto fn = L == 4 ? (cfg.adder == 1   ? csa_direct_kernel<K, 8, 4>
                            : cfg.adder == 2 ? csa_direct_kernel<K, G32, 4>
                                             : csa_direct_kernel<K, 16, 4>)
                         : (cfg.adder == 1 ? csa_direct_kernel<K, 8, 2> : csa_direct_kernel<K, 16, 2>);
        const int rc = ensure_smem_limit((const void*)fn, tab_bytes);
        if (rc) return rc;
        fn<<<grid, threads, tab_bytes, s>>>(a, x);
        BM_CUDA_TRY(cudaGetLastError());
        return BM_OK;
    }
    int optin = 0;
    const int orc = smem_optin(&optin);
    if (orc) return orc;
    auto run = [&](auto fn, int nt) -> int {
        // stages of 16 bitmaps x nt 16-byte slices, plus two mbarriers each
        const int fit = (int)(((size_t)optin - tab_bytes) / ((size_t)256 * nt + 16));
        const int stages = std::max(2, std::min({8, cfg.stages, fit}));
        if (fit < 2) return BM_EINVAL;
        const size_t bytes = (size_t)stages * 16 * nt * 16 + 2 * (size_t)stages * 8 + tab_bytes;
        const int rc = ensure_smem_limit((const void*)fn, bytes);
        if (rc) return rc;
        const uint64_t ntiles = (ncols + nt - 1) / nt;
        const uint64_t cap = (uint64_t)sm_count * (uint64_t)std::max(1, cfg.ctas_per_sm);
        const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min(ntiles, cap));
        fn<<<grid, nt + 32, bytes, s>>>(a, x, stages);
        BM_CUDA_TRY(cudaGetLastError());
        return BM_OK;
    };
    if (cfg.threads <= 64) return run(csa_bulk_kernel<K, 64>, 64);
    if (cfg.threads <= 128) return run(csa_bulk_kernel<K, 128>, 128);
    return run(csa_bulk_kernel<K, 256>, 256);
}

}  // namespace

int launch_dense(const DenseArgs& a, const LaunchExtra& x, const DenseConfig& cfg, int sm_count,
                 cudaStream_t s) {
    if (a.words == 0) return BM_OK;
    const int k = planes_for(a.n);
    if (k <= 5) return launch_k<5>(a, x, cfg, sm_count, s);
    if (k <= 9) return launch_k<9>(a, x, cfg, sm_count, s);
    if (k <= 13) return launch_k<13>(a, x, cfg, sm_count, s);
    return launch_k<17>(a, x, cfg, sm_count, s);
}

// ---------------------------------------------------------------------------
// cardinality of one bitmap (the paper's |B_i|, Sec. 2.1)

namespace {
__global__ void __launch_bounds__(256) cardinality_kernel(const uint64_t* w, uint64_t words,
                                                          uint64_t r_bits,
                                                          unsigned long long* out) {
    unsigned long long c = 0;
    const uint32_t tail = (uint32_t)(r_bits & 63u);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t x = w[i];
        if (tail && i == words - 1) x &= (1ull << tail) - 1ull;
        c += (unsigned long long)__popcll(x);
    }
    flush_card(c, out);
}
}  // namespace

int launch_cardinality(const uint64_t* words, uint64_t r_bits, unsigned long long* out,
                       int sm_count, cudaStream_t s) {
    BM_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(unsigned long long), s));
    const uint64_t nw = (r_bits + 63) / 64;
    if (nw == 0) return BM_OK;
    const uint64_t blocks = std::min<uint64_t>((nw + 255) / 256, (uint64_t)sm_count * 8);
    cardinality_kernel<<<(unsigned)std::max<uint64_t>(1, blocks), 256, 0, s>>>(words, nw, r_bits,
                                                                                out);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

}  // namespace bm
