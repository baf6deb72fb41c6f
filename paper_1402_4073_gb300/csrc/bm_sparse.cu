// ScanCount over sorted position lists (Sec. 4.2, and App. D for the form
// over BitSets): one counter per row, every listed position increments its
// row's counter, then one pass evaluates f on each counter.
//
// GPU form: the rows are cut into tiles; a CTA owns one tile's counters in
// shared memory (8-bit counters when n <= 255, else 16-bit: the paper's
// width switch by N, packed four or two to a 32-bit word and incremented
// with shared-memory atomics).  The tile's slice of a list comes from the
// pool's per-list tile index (first entry at every multiple of 8192 rows), so
// a list is never searched; warps take groups of 32 lists and read their
// slices, laid end to end, as one stream of 16-byte vectors
// (bm_scan_common.cuh).  Then each thread turns 32 counters into one 32-bit
// output lane (a plain threshold by SIMD compares, any other f through its
// truth table in shared memory), stores it and popcounts it.
#include <algorithm>

#include "bm_scan_common.cuh"

namespace bm {
namespace {

using namespace dev;

// Truth table bits of the predicate for counts 0..n, into shared memory.
__device__ void build_truth(const Pred& pr, uint32_t n, uint32_t* tab, uint32_t words32) {
    for (uint32_t w = threadIdx.x; w < words32; w += blockDim.x) {
        uint32_t bits = 0;
        if (pr.mode == 2) {
            bits = pr.table[w];
        } else {
            for (uint32_t b = 0; b < 32; ++b) {
                const uint32_t c = w * 32 + b;
                if (c > n) break;
                uint32_t v = pr.v0;
                if (pr.mode == 1)
#pragma unroll
                    for (int i = 0; i < kMaxTransitions; ++i)
                        if ((uint32_t)i < pr.ntrans) v ^= (c >= pr.trans[i]) ? 1u : 0u;
                bits |= v << b;
            }
        }
        tab[w] = bits;
    }
}

// Two 512-thread CTAs per SM: the pipelined loads need the 64 registers
// that leaves.
template <int BITS, int U>  // counter width: 8 or 16; pieces per load batch
__global__ void __launch_bounds__(512, 2)
    scancount_kernel(SparseArgs a, const __grid_constant__ LaunchExtra x) {
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ uint32_t s_next;  // next group of lists to count
    __shared__ __align__(16) uint32_t s_ids[kInlineIds];
    launch_ids(a.ids, x, s_ids);
    constexpr uint32_t kPer = 32 / BITS;  // counters per 32-bit word
    const uint32_t tab_words = (a.n + 1 + 31) / 32;
    uint32_t* tab = sm;
    uint32_t* scratch = sm + ((tab_words + 3) & ~3u);
    uint32_t* cnt = scratch + kScanWarpWords * (blockDim.x / 32);
    const uint32_t cnt_words = a.tile_rows / kPer;
    build_truth(a.pred, a.n, tab, tab_words);

    const uint64_t ntiles = (a.r_bits + a.tile_rows - 1) / a.tile_rows;
    const uint32_t sub = a.tile_rows / kListTileRows;  // index entries per tile
    unsigned long long card = 0;
    // counters start at zero; evaluating a tile clears them for the next one
    for (uint32_t i = threadIdx.x; i < cnt_words; i += blockDim.x) cnt[i] = 0u;
    __syncthreads();
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t lo = tile * a.tile_rows;
        const uint64_t hi = min(lo + a.tile_rows, a.r_bits);
        const uint64_t t0 = tile * sub;
        const uint64_t t1 = (t0 + sub < a.tiles_per_list) ? t0 + sub : (uint64_t)a.tiles_per_list;
        count_tile<BITS, U>(cnt, scratch, &s_next,
                            [&](uint32_t j) { return x.n_inline ? s_ids[j] : __ldg(a.ids + j); }, a.n,
                            reinterpret_cast<const uint4*>(a.positions),
                            a.list_begin, a.tile_index, a.tiles_per_list, t0, t1, (uint32_t)lo,
                            (uint32_t)(hi - lo), a.tile_rows, a.d_fill);
        __syncthreads();
        // 32 rows per thread -> one 32-bit output lane
        const uint32_t lanes = (uint32_t)((hi - lo + 31) / 32);
        uint32_t* out32 = reinterpret_cast<uint32_t*>(a.out);
        for (uint32_t l = threadIdx.x; l < lanes; l += blockDim.x) {
            uint32_t o = counters_to_lane<BITS>(cnt + l * (32 / kPer), a.pred, tab);
            const uint64_t row0 = lo + 32ull * l;
            if (row0 + 32 > a.r_bits) o &= (1u << (a.r_bits - row0)) - 1u;  // rows >= r
            out32[row0 / 32] = o;
            card += __popc(o);
        }
        __syncthreads();
    }
    // rows between r and the end of the last 64-bit word
    if (blockIdx.x == 0 && threadIdx.x == 0 && ((a.r_bits + 31) / 32) % 2 == 1)
        reinterpret_cast<uint32_t*>(a.out)[(a.r_bits + 31) / 32] = 0u;
    flush_card_block(card, a.card, x.acc, x.ticket);
}

}  // namespace

int launch_sparse(const SparseArgs& a, const LaunchExtra& x, const SparseConfig& cfg, int sm_count,
                  cudaStream_t s) {
    if (a.r_bits == 0) return BM_OK;
    // padded lists keep their padding out of every tile of at most 65536 rows
    if (a.tile_rows == 0 || a.tile_rows % kListTileRows || a.tile_rows > 65536) return BM_EINVAL;
    const int bits = a.n <= 255 ? 8 : 16;
    // tile_rows is sized for 16-bit counters: 8-bit counters take twice the
    // rows in the same shared memory (at most 65536, where the list padding
    // stays outside every tile), halving the tiles of a small query
    SparseArgs b = a;
    if (bits == 8) b.tile_rows = std::min<uint32_t>(65536u, 2 * a.tile_rows);
    const size_t tab_words = ((size_t)(a.n + 1 + 31) / 32 + 3) & ~(size_t)3;
    const int threads = std::max(64, std::min(512, cfg.threads)) & ~31;
    const size_t scratch_words = (size_t)dev::kScanWarpWords * (size_t)(threads / 32);
    // counters, then one spare word per lane
    const size_t smem = (tab_words + scratch_words + (size_t)b.tile_rows * bits / 32 + 32) * 4;
    const uint64_t ntiles = (b.r_bits + b.tile_rows - 1) / b.tile_rows;
    const uint64_t cap = (uint64_t)sm_count * (uint64_t)std::max(1, cfg.ctas_per_sm);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min(ntiles, cap));
    auto go = [&](auto fn) -> int {
        const int rc = ensure_smem_limit((const void*)fn, smem);
        if (rc) return rc;
        fn<<<grid, threads, smem, s>>>(b, x);
        BM_CUDA_TRY(cudaGetLastError());
        return BM_OK;
    };
    if (cfg.unroll <= 2)
        return bits == 8 ? go(scancount_kernel<8, 2>) : go(scancount_kernel<16, 2>);
    return bits == 8 ? go(scancount_kernel<8, 4>) : go(scancount_kernel<16, 4>);
}

}  // namespace bm
