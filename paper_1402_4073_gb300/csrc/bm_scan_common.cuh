// Counting one row tile of ScanCount (Sec. 4.2) in shared memory, shared by
// the single-query and the batch kernels.
//
// Position lists sit in the pool 16-byte aligned and padded to a multiple of
// four entries with values outside every tile that could read them, so any
// aligned 16-byte vector of a list may be read and its four entries filtered
// by the tile's row range alone.  The tile's slice of every list is found
// from the pool's per-list tile index and widened to whole vectors.  Lists
// are taken in chunks of kScanChunk: the CTA loads all slice bounds of a
// chunk at once, prefix-sums the vector counts (and the number of non-empty
// slices) in one scan, and so lays the slices end to end as one stream of
// vectors.  The stream is cut into pieces of 32 vectors; per piece a table
// holds the slice of its first vector and a bit mask of the slices that
// start inside it, so lane l of a warp finds the slice of vector 32q + l with
// one population count.  Warps take pieces in turn, U at a time, each lane
// loading one 16-byte vector per piece: all lanes are busy however short the
// slices are, and no lane searches.
#pragma once

#include "bm_device.cuh"

namespace bm {
namespace dev {

constexpr uint32_t kScanChunk = 1024;   // lists per chunk
constexpr uint32_t kPieceTable = 1024;  // pieces per pass of the piece table
// shared words the helper needs besides the counters: packed scan values
// (64-bit, kScanChunk + 1), warp totals (64-bit, 32), slice starts by list,
// slice starts and stream offsets by rank (+1), piece masks, piece bases
// (16-bit)
constexpr uint32_t kScanSmemWords = 2 * (kScanChunk + 1) + 2 * 32 + kScanChunk + kScanChunk +
                                    (kScanChunk + 1) + kPieceTable + kPieceTable / 2;

// In-place exclusive prefix sum of v[0..m) (64-bit), v[m] = total
// (m <= kScanChunk, blockDim.x a multiple of 32, at most 1024).
__device__ __forceinline__ void block_exclusive_scan64(uint64_t* v, uint32_t m,
                                                       uint64_t* warp_tot) {
    const uint32_t T = blockDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t nw = T >> 5;
    const uint32_t E = (kScanChunk + T - 1) / T;
    uint64_t s = 0;
    for (uint32_t e = 0; e < E; ++e) {
        const uint32_t i = t * E + e;
        if (i < m) s += v[i];
    }
    uint64_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < nw ? warp_tot[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= (uint32_t)o) w += y;
        }
        if (lane < nw) warp_tot[lane] = w;  // inclusive totals per warp
    }
    __syncthreads();
    uint64_t prefix = (warp ? warp_tot[warp - 1] : 0ull) + x - s;
    for (uint32_t e = 0; e < E; ++e) {
        const uint32_t i = t * E + e;
        if (i < m) {
            const uint64_t a = v[i];
            v[i] = prefix;
            prefix += a;
        }
    }
    if (t == 0) v[m] = warp_tot[nw - 1];
    __syncthreads();
}

// Add the four entries of a vector that lie in rows [lo, lo + nrows).  An
// entry outside the range (alignment or padding of a slice) goes to the
// lane's own spare counter word past the tile instead, so the four atomics
// are issued without branches; the spare words are never read.
template <int BITS>
__device__ __forceinline__ void count_vec(uint32_t* cnt, const uint4& x, uint32_t lo,
                                          uint32_t nrows, uint32_t spare_row) {
    constexpr uint32_t kPer = 32 / BITS;
    const uint32_t e[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t row = e[i] - lo;
        row = row < nrows ? row : spare_row;
        atomicAdd(&cnt[row / kPer], 1u << (BITS * (row % kPer)));
    }
}

// Add every position of rows [lo, lo + nrows) of lists ids[0..n) into
// BITS-bit counters cnt (packed 32 / BITS per word; cnt_rows / (32 / BITS)
// words for rows, then 32 spare words).  t0, t1: tile-index
// entries bounding the tile.  vpos: the pool's list arena as 16-byte
// vectors.  scratch: kScanSmemWords shared words, 16-byte aligned.
template <int BITS, int U>
__device__ __forceinline__ void count_tile(uint32_t* cnt, uint32_t* scratch, const uint32_t* ids,
                                           uint32_t n, const uint4* vpos,
                                           const uint64_t* list_begin,
                                           const uint32_t* tile_index, uint32_t tiles_per_list,
                                           uint64_t t0, uint64_t t1, uint32_t lo,
                                           uint32_t nrows, uint32_t cnt_rows) {
    uint64_t* s_scan = reinterpret_cast<uint64_t*>(scratch);  // kScanChunk + 1: (vectors, non-empty)
    uint64_t* s_wt = s_scan + kScanChunk + 1;                  // 32
    uint32_t* s_vsj = reinterpret_cast<uint32_t*>(s_wt + 32);  // kScanChunk: first vector, by list
    uint32_t* s_vs = s_vsj + kScanChunk;                       // kScanChunk: first vector, by rank
    uint32_t* s_off = s_vs + kScanChunk;                       // kScanChunk + 1: stream offset, by rank
    uint32_t* s_mask = s_off + kScanChunk + 1;                 // kPieceTable: slice starts in a piece
    uint16_t* s_base = reinterpret_cast<uint16_t*>(s_mask + kPieceTable);  // kPieceTable
    const uint32_t T = blockDim.x;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
    const uint32_t below = ((2u << lane) - 1u) & ~1u;  // lanes 1..lane of a piece
    const uint32_t spare = cnt_rows + lane * (32 / BITS);  // this lane's spare counter word
    for (uint32_t c0 = 0; c0 < n; c0 += kScanChunk) {
        const uint32_t m = min(kScanChunk, n - c0);
        for (uint32_t j = threadIdx.x; j < m; j += T) {
            const uint32_t id = __ldg(ids + c0 + j);
            const uint32_t* idx = tile_index + (uint64_t)id * (tiles_per_list + 1);
            const uint32_t b = __ldg(idx + t0), en = __ldg(idx + t1);
            const uint64_t base = __ldg(list_begin + id);
            const uint32_t vs = (uint32_t)((base + b) >> 2);
            const uint32_t nv = b < en ? (uint32_t)((base + en + 3) >> 2) - vs : 0u;
            s_vsj[j] = vs;
            s_scan[j] = ((uint64_t)nv << 32) | (nv ? 1u : 0u);
        }
        __syncthreads();
        block_exclusive_scan64(s_scan, m, s_wt);
        const uint32_t total = (uint32_t)(s_scan[m] >> 32);  // vectors in the stream
        const uint32_t slices = (uint32_t)s_scan[m];         // non-empty slices
        for (uint32_t j = threadIdx.x; j < m; j += T) {
            const uint64_t a = s_scan[j];
            if (s_scan[j + 1] != a) {  // non-empty: rank = slices before it
                s_vs[(uint32_t)a] = s_vsj[j];
                s_off[(uint32_t)a] = (uint32_t)(a >> 32);
            }
        }
        if (threadIdx.x == 0) s_off[slices] = total;
        const uint32_t pieces = (total + 31) / 32;
        for (uint32_t p0 = 0; p0 < pieces; p0 += kPieceTable) {
            const uint32_t p1 = min(pieces, p0 + kPieceTable);
            __syncthreads();  // offsets visible; the previous pass is done with the tables
            for (uint32_t q = threadIdx.x; q < p1 - p0; q += T) s_mask[q] = 0u;
            __syncthreads();
            for (uint32_t r = threadIdx.x; r < slices; r += T) {
                const uint32_t a = s_off[r], z = s_off[r + 1];  // a < z
                if (a / 32 >= p0 && a / 32 < p1) atomicOr(&s_mask[a / 32 - p0], 1u << (a % 32));
                // pieces whose first vector lies in this slice
                const uint32_t qa = max((a + 31) / 32, p0), qz = min((z - 1) / 32 + 1, p1);
                for (uint32_t q = qa; q < qz; ++q) s_base[q - p0] = (uint16_t)r;
            }
            __syncthreads();
            for (uint32_t q0 = p0 + warp * U; q0 < p1; q0 += nw * U) {
                uint4 x[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t q = q0 + u;
                    const uint32_t v = q * 32 + lane;
                    x[u] = make_uint4(lo - 1u, lo - 1u, lo - 1u, lo - 1u);  // outside the tile
                    if (q < p1 && v < total) {
                        const uint32_t r = s_base[q - p0] + __popc(s_mask[q - p0] & below);
                        x[u] = ld_stream(vpos + s_vs[r] + (v - s_off[r]));
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) count_vec<BITS>(cnt, x[u], lo, nrows, spare);
            }
        }
        __syncthreads();
    }
}

// One 32-bit output lane from 32 counters (words cw[0 .. kWords)), which
// are cleared as they are read, ready for the next tile.  Lane l
// reads its words starting at word l mod kWords, so at each step the 32
// lanes of a warp hit (at most two-way) distinct banks instead of all
// reading the same two banks.  A plain threshold (v0 = 0, one transition
// theta) compares packed counters with SIMD byte/halfword compares; every
// other predicate looks f up.
template <int BITS>
__device__ __forceinline__ uint32_t counters_to_lane(uint32_t* cw, const Pred& pred,
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
                cw[w] = 0u;
                const uint32_t b = ge & 0x01010101u;
                o |= ((b | (b >> 7) | (b >> 14) | (b >> 21)) & 0xFu) << (4 * w);
            }
        } else {
            const uint32_t t2 = th * 0x00010001u;
#pragma unroll
            for (uint32_t k = 0; k < kWords; ++k) {
                const uint32_t w = (k + rot) & (kWords - 1);
                const uint32_t ge = __vcmpgeu2(cw[w], t2);  // 0xFFFF per half where count >= theta
                cw[w] = 0u;
                o |= ((ge & 1u) | ((ge >> 15) & 2u)) << (2 * w);
            }
        }
        return o;
    }
#pragma unroll
    for (uint32_t k = 0; k < kWords; ++k) {
        const uint32_t w = (k + rot) & (kWords - 1);
        const uint32_t word = cw[w];
        cw[w] = 0u;
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
