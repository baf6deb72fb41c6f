// Counting one row tile of ScanCount (Sec. 4.2) in shared memory, shared by
// the single-query and the batch kernels.
//
// The tile's slice of every list is found from the pool's per-list tile
// index.  Lists are taken in chunks of kScanChunk: the CTA first loads the
// slice bounds of the whole chunk at once (all independent loads), then each
// warp takes kSlices slices at a time, its lanes loading 32 consecutive
// positions of each (coalesced; kSlices independent loads in flight per lane)
// and adding them into the counters with shared-memory atomics.  Slices
// longer than 32 positions continue in a loop.
#pragma once

#include "bm_device.cuh"

namespace bm {
namespace dev {

constexpr uint32_t kScanChunk = 1024;
constexpr int kSlices = 4;  // slices a warp loads at once
// shared words the helper needs besides the counters
constexpr uint32_t kScanSmemWords = 2 * kScanChunk;

// Add every position of rows [lo, lo + tile) of lists ids[0..n) into
// BITS-bit counters cnt (packed 32 / BITS per word).  t0, t1: tile-index
// entries bounding the tile.  scratch: kScanSmemWords shared words.
template <int BITS>
__device__ __forceinline__ void count_tile(uint32_t* cnt, uint32_t* scratch, const uint32_t* ids,
                                           uint32_t n, const uint32_t* positions,
                                           const uint64_t* list_begin,
                                           const uint32_t* tile_index, uint32_t tiles_per_list,
                                           uint64_t t0, uint64_t t1, uint32_t lo) {
    constexpr uint32_t kPer = 32 / BITS;
    uint32_t* s_len = scratch;              // kScanChunk
    uint32_t* s_base = s_len + kScanChunk;  // kScanChunk
    const uint32_t T = blockDim.x;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
    auto add = [&](uint32_t p) {
        const uint32_t row = p - lo;
        atomicAdd(&cnt[row / kPer], 1u << (BITS * (row % kPer)));
    };
    for (uint32_t c0 = 0; c0 < n; c0 += kScanChunk) {
        const uint32_t m = min(kScanChunk, n - c0);
        for (uint32_t j = threadIdx.x; j < m; j += T) {
            const uint32_t id = __ldg(ids + c0 + j);
            const uint32_t* idx = tile_index + (uint64_t)id * (tiles_per_list + 1);
            const uint32_t b = __ldg(idx + t0), e = __ldg(idx + t1);
            s_len[j] = e - b;
            s_base[j] = (uint32_t)(__ldg(list_begin + id) + b);
        }
        __syncthreads();
        for (uint32_t j0 = warp; j0 < m; j0 += kSlices * nw) {
            uint32_t len[kSlices], base[kSlices], p[kSlices];
#pragma unroll
            for (int u = 0; u < kSlices; ++u) {
                const uint32_t j = j0 + u * nw;
                len[u] = j < m ? s_len[j] : 0u;
                base[u] = j < m ? s_base[j] : 0u;
                p[u] = lane < len[u] ? __ldg(positions + base[u] + lane) : 0u;
            }
#pragma unroll
            for (int u = 0; u < kSlices; ++u)
                if (lane < len[u]) add(p[u]);
#pragma unroll
            for (int u = 0; u < kSlices; ++u) {
                for (uint32_t k = 32 + lane; k < len[u]; k += 128) {
                    uint32_t q[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        q[v] = (k + 32 * v < len[u]) ? __ldg(positions + base[u] + k + 32 * v) : 0u;
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        if (k + 32 * v < len[u]) add(q[v]);
                }
            }
        }
        __syncthreads();
    }
}

// One 32-bit output lane from 32 counters (words cw[0 .. kWords)).  Lane l
// reads its words starting at word l mod kWords, so at each step the 32
// lanes of a warp hit (at most two-way) distinct banks instead of all
// reading the same two banks.  A plain threshold (v0 = 0, one transition
// theta) compares packed counters with SIMD byte/halfword compares; every
// other predicate looks f up.
template <int BITS>
__device__ __forceinline__ uint32_t counters_to_lane(const uint32_t* cw, const Pred& pred,
                                                     const uint32_t* tab) {
    constexpr uint32_t kPer = 32 / BITS, kWords = 32 / kPer;
    const uint32_t rot = threadIdx.x;
    uint32_t o = 0;
    if (pred.mode == 1 && pred.ntrans == 1 && pred.v0 == 0) {
        const uint32_t th = pred.trans[0];
        if (BITS == 8) {
            const uint32_t t4 = th * 0x01010101u;  // theta <= 255 whenever 8-bit counters are used
#pragma unroll
            for (uint32_t k = 0; k < kWords; ++k) {
                const uint32_t w = (k + rot) & (kWords - 1);
                const uint32_t ge = __vcmpgeu4(cw[w], t4);  // 0xFF per byte where count >= theta
                const uint32_t b = ge & 0x01010101u;
                o |= ((b | (b >> 7) | (b >> 14) | (b >> 21)) & 0xFu) << (4 * w);
            }
        } else {
            const uint32_t t2 = th * 0x00010001u;
#pragma unroll
            for (uint32_t k = 0; k < kWords; ++k) {
                const uint32_t w = (k + rot) & (kWords - 1);
                const uint32_t ge = __vcmpgeu2(cw[w], t2);  // 0xFFFF per half where count >= theta
                o |= ((ge & 1u) | ((ge >> 15) & 2u)) << (2 * w);
            }
        }
        return o;
    }
#pragma unroll
    for (uint32_t k = 0; k < kWords; ++k) {
        const uint32_t w = (k + rot) & (kWords - 1);
        const uint32_t word = cw[w];
#pragma unroll
        for (uint32_t s = 0; s < kPer; ++s) {
            const uint32_t c = (word >> (BITS * s)) & ((1u << BITS) - 1u);
            o |= ((tab[c >> 5] >> (c & 31u)) & 1u) << (w * kPer + s);
        }
    }
    return o;
}

}  // namespace dev
}  // namespace bm
