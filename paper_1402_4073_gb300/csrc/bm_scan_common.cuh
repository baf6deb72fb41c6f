// Counting one row tile of ScanCount (Sec. 4.2) in shared memory, shared by
// the single-query and the batch kernels.
//
// The tile's slice of every list is found from the pool's per-list tile
// index.  Lists are taken in chunks of kScanChunk.  For each, the CTA loads
// all slice bounds at once, cuts every slice into pieces of at most 32
// consecutive positions, prefix-sums the piece counts and writes a
// piece -> slice table in shared memory.  Warps then take pieces in turn,
// U at a time: the lanes of a warp load one piece's positions (coalesced)
// and add them into the counters with shared-memory atomics.  Every warp
// gets the same number of pieces (+-1), however skewed the list lengths
// are, and no lane searches for its slice.
#pragma once

#include "bm_device.cuh"

namespace bm {
namespace dev {

constexpr uint32_t kScanChunk = 1024;  // lists per chunk
constexpr uint32_t kPieceTable = 4096; // pieces per pass (uint16 slice ids)
// shared words the helper needs besides the counters
constexpr uint32_t kScanSmemWords = 4 * kScanChunk + 1 + 32 + kPieceTable / 2;

// Exclusive prefix sum of len[0..m) into off[0..m], off[m] = total
// (m <= kScanChunk, blockDim.x a multiple of 32, at most 1024).
__device__ __forceinline__ void block_exclusive_scan(const uint32_t* len, uint32_t* off, uint32_t m,
                                                     uint32_t* warp_tot) {
    const uint32_t T = blockDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t nw = T >> 5;
    const uint32_t E = (kScanChunk + T - 1) / T;
    uint32_t s = 0;
    for (uint32_t e = 0; e < E; ++e) {
        const uint32_t i = t * E + e;
        if (i < m) s += len[i];
    }
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= (uint32_t)o) w += y;
        }
        if (lane < nw) warp_tot[lane] = w;  // inclusive totals per warp
    }
    __syncthreads();
    uint32_t prefix = (warp ? warp_tot[warp - 1] : 0u) + x - s;
    for (uint32_t e = 0; e < E; ++e) {
        const uint32_t i = t * E + e;
        if (i < m) {
            off[i] = prefix;
            prefix += len[i];
        }
    }
    if (t == 0) off[m] = warp_tot[nw - 1];
    __syncthreads();
}

// Add every position of rows [lo, lo + tile) of lists ids[0..n) into
// BITS-bit counters cnt (packed 32 / BITS per word).  t0, t1: tile-index
// entries bounding the tile.  scratch: kScanSmemWords shared words.
template <int BITS, int U>
__device__ __forceinline__ void count_tile(uint32_t* cnt, uint32_t* scratch, const uint32_t* ids,
                                           uint32_t n, const uint32_t* positions,
                                           const uint64_t* list_begin,
                                           const uint32_t* tile_index, uint32_t tiles_per_list,
                                           uint64_t t0, uint64_t t1, uint32_t lo) {
    constexpr uint32_t kPer = 32 / BITS;
    uint32_t* s_len = scratch;                  // kScanChunk: slice lengths
    uint32_t* s_np = s_len + kScanChunk;        // kScanChunk: pieces of each slice
    uint32_t* s_base = s_np + kScanChunk;       // kScanChunk: arena offset of each slice
    uint32_t* s_off = s_base + kScanChunk;      // kScanChunk + 1: first piece of each slice
    uint32_t* s_wt = s_off + kScanChunk + 1;    // 32
    uint16_t* s_piece = reinterpret_cast<uint16_t*>(s_wt + 32);  // kPieceTable
    const uint32_t T = blockDim.x;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
    for (uint32_t c0 = 0; c0 < n; c0 += kScanChunk) {
        const uint32_t m = min(kScanChunk, n - c0);
        for (uint32_t j = threadIdx.x; j < m; j += T) {
            const uint32_t id = __ldg(ids + c0 + j);
            const uint32_t* idx = tile_index + (uint64_t)id * (tiles_per_list + 1);
            const uint32_t b = __ldg(idx + t0), en = __ldg(idx + t1);
            s_len[j] = en - b;
            s_np[j] = (en - b + 31) / 32;
            s_base[j] = (uint32_t)(__ldg(list_begin + id) + b);
        }
        __syncthreads();
        block_exclusive_scan(s_np, s_off, m, s_wt);
        const uint32_t pieces = s_off[m];
        for (uint32_t p0 = 0; p0 < pieces; p0 += kPieceTable) {
            const uint32_t p1 = min(pieces, p0 + kPieceTable);
            __syncthreads();  // previous pass done with the table; lengths visible
            for (uint32_t j = threadIdx.x; j < m; j += T) {
                const uint32_t a = max(s_off[j], p0), z = min(s_off[j + 1], p1);
                for (uint32_t q = a; q < z; ++q) s_piece[q - p0] = (uint16_t)j;
            }
            __syncthreads();
            for (uint32_t q0 = p0 + warp * U; q0 < p1; q0 += nw * U) {
                uint32_t p[U];
                bool have[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t q = q0 + u;
                    have[u] = false;
                    p[u] = 0;
                    if (q < p1) {  // uniform across the warp
                        const uint32_t j = s_piece[q - p0];
                        const uint32_t k = (q - s_off[j]) * 32 + lane;
                        have[u] = k < s_len[j];
                        if (have[u]) p[u] = __ldg(positions + s_base[j] + k);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (have[u]) {
                        const uint32_t row = p[u] - lo;
                        atomicAdd(&cnt[row / kPer], 1u << (BITS * (row % kPer)));
                    }
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
