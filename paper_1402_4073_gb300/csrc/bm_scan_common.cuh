// Counting one row tile of ScanCount (Sec. 4.2) in shared memory, shared by
// the single-query and the batch kernels.
//
// Position lists sit in the pool 16-byte aligned and padded to a multiple of
// four entries with values outside every tile that could read them, so any
// aligned 16-byte vector of a list may be read and its four entries filtered
// by the tile's row range alone.  The tile's slice of a list is found from
// the pool's per-list tile index and widened to whole vectors.
//
// Warps take groups of 32 lists: each warp's first group is fixed, the rest
// come from a shared counter, so warps that drew short slices take more
// groups; with fewer groups than warps, teams of warps share a group's
// pieces.  In a group, lane k loads the slice bounds of list k (the next
// group's bounds are in flight while this one is counted), a warp scan lays
// the 32 slices end to end as one stream of vectors, and the stream is read
// in pieces of 32 vectors, one per lane: the slice holding lane l's vector
// is found with one ballot (slices begun before the piece), one OR-reduction
// (slices beginning inside it) and a population count, so all lanes load
// whatever the slice lengths.  The loads of the next U pieces are issued
// before the increments of the current U.  No block-wide barrier is taken
// while counting.
#pragma once

#include "bm_device.cuh"

namespace bm {
namespace dev {

constexpr uint32_t kScanWarpWords = 64;  // shared words per warp: a group's slices
// shared words the helper needs besides the counters (up to 32 warps)
constexpr uint32_t kScanSmemWords = kScanWarpWords * 32;

// Add (sub: subtract) one for each of the four entries of a vector that lie
// in rows [lo, lo + nrows).  An entry outside the range (alignment or padding
// of a slice) goes to the lane's own spare counter word past the tile
// instead, so the four atomics are issued without branches; the spare words
// are never read.  A subtraction never borrows across packed counters: a row
// is decremented at most once per input given by its zeros, and its counter
// started at the number of such inputs.
template <int BITS>
__device__ __forceinline__ void count_vec(uint32_t* cnt, const uint4& x, uint32_t lo,
                                          uint32_t nrows, uint32_t spare_row, bool sub) {
    constexpr uint32_t kPer = 32 / BITS;
    const uint32_t e[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t row = e[i] - lo;
        row = row < nrows ? row : spare_row;
        const uint32_t inc = 1u << (BITS * (row % kPer));
        atomicAdd(&cnt[row / kPer], sub ? 0u - inc : inc);
    }
}

// Count rows [lo, lo + nrows) of lists ids[0..n) into BITS-bit counters cnt
// (packed 32 / BITS per word; cnt_rows / (32 / BITS) words for rows, then 32
// spare words), which hold zero on entry: every position of a list of ones
// adds one; the counters first take d_fill, the number of inputs given by a
// list of their zeros, and every position of such a list subtracts one, so
// each counter ends at the number of inputs holding its row (the complement
// identity of Sec. 2.3 applied input by input).  t0, t1: tile-index entries
// bounding the tile.  vpos: the pool's list arena as 16-byte vectors.
// scratch: kScanWarpWords shared words per warp.  s_next: a shared word.
// id(j) returns the query's j-th id.
// Every thread of the block calls this; it begins with a block barrier.
template <int BITS, int U, typename IdOf>
__device__ __forceinline__ void count_tile(uint32_t* cnt, uint32_t* scratch, uint32_t* s_next,
                                           IdOf id_of, uint32_t n, const uint4* vpos,
                                           const uint64_t* list_begin,
                                           const uint32_t* tile_index, uint32_t tiles_per_list,
                                           uint64_t t0, uint64_t t1, uint32_t lo,
                                           uint32_t nrows, uint32_t cnt_rows, uint32_t d_fill) {
    constexpr uint32_t kFull = 0xFFFFFFFFu;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t le = (2u << lane) - 1u, lt = (1u << lane) - 1u;
    const uint32_t spare = cnt_rows + lane * (32 / BITS);  // this lane's spare counter word
    const uint32_t ngroups = (n + 31) / 32;
    uint32_t* ws = scratch + warp * kScanWarpWords;  // [0,32): first vector | zeros bit, [32,64): offset
    if (threadIdx.x == 0) *s_next = nw;
    if (d_fill) {  // the rows' counters (those evaluated) start at d_fill
        const uint32_t fill = BITS == 8 ? d_fill * 0x01010101u : d_fill * 0x00010001u;
        const uint32_t words = (nrows + 31) / 32 * BITS;  // BITS words per 32 rows
        for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) cnt[i] = fill;
    }
    __syncthreads();
    // slice of list 32 g + lane: first vector vs, vectors nv (0: empty)
    auto bounds = [&](uint32_t g, uint32_t& vs, uint32_t& nv) {
        vs = 0u;
        nv = 0u;
        const uint32_t j = g * 32 + lane;
        if (g < ngroups && j < n) {
            const uint32_t id = id_of(j);
            const uint32_t* idx = tile_index + (uint64_t)id * (tiles_per_list + 1);
            const uint32_t b = __ldg(idx + t0), en = __ldg(idx + t1);
            const uint64_t begin = __ldg(list_begin + id);
            const uint64_t base = begin & ~kListComplement;
            vs = (uint32_t)((base + b) >> 2);
            nv = b < en ? (uint32_t)((base + en + 3) >> 2) - vs : 0u;
            vs |= (uint32_t)(begin >> 32) & 0x80000000u;  // bit 31: a list of zeros
        }
    };
    // With fewer groups than warps, a team of `team` warps shares each group,
    // member m taking pieces m, m + team, ...: work unit u = (group u / team,
    // member u % team).
    uint32_t team = 1;
    while (ngroups && team * 2 * ngroups <= nw) team *= 2;
    const uint32_t units = ngroups * team;
    uint32_t u = warp, vs, nv;
    bounds(u / team, vs, nv);
    while (u < units) {
        uint32_t un = 0;
        if (lane == 0) un = atomicAdd(s_next, 1u);
        un = __shfl_sync(kFull, un, 0);
        uint32_t vs_n, nv_n;
        bounds(un < units ? un / team : ngroups, vs_n, nv_n);  // in flight while this unit is counted
        uint32_t inc = nv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, inc, o);
            if (lane >= (uint32_t)o) inc += y;
        }
        const uint32_t start = inc - nv;                      // stream offset of this slice
        const uint32_t total = __shfl_sync(kFull, inc, 31);   // vectors in the stream
        const uint32_t ne = __ballot_sync(kFull, nv != 0u);   // non-empty slices
        if (nv) {  // non-empty slices by rank
            const uint32_t rk = __popc(ne & lt);
            ws[rk] = vs;
            ws[32 + rk] = start;
        }
        __syncwarp();
        const uint32_t pieces = (total + 31) / 32;
        const uint32_t member = u % team;
        // this warp's pieces: member + k * team, k = 0, 1, ...
        const uint32_t mine = pieces > member ? (pieces - member + team - 1) / team : 0u;
        auto fetch = [&](uint32_t k0, uint4 (&x)[U], uint32_t& subs) {
            subs = 0u;
#pragma unroll
            for (int i = 0; i < U; ++i) {
                const uint32_t q = member + (k0 + i) * team;
                x[i] = make_uint4(lo - 1u, lo - 1u, lo - 1u, lo - 1u);  // outside the tile
                if (k0 + i < mine) {  // uniform across the warp
                    // rank of the slice holding vector 32 q + lane
                    const uint32_t before = __popc(__ballot_sync(kFull, nv != 0u && start < q * 32));
                    const uint32_t inside = __reduce_or_sync(
                        kFull, (nv != 0u && (start >> 5) == q) ? (1u << (start & 31)) : 0u);
                    const uint32_t r = before + __popc(inside & le) - 1u;
                    const uint32_t v = q * 32 + lane;
                    if (v < total) {
                        const uint32_t first = ws[r];
                        x[i] = ld_stream(vpos + (first & 0x7FFFFFFFu) + (v - ws[32 + r]));
                        subs |= (first >> 31) << i;
                    }
                }
            }
        };
        auto add = [&](const uint4 (&x)[U], uint32_t subs) {
#pragma unroll
            for (int i = 0; i < U; ++i) count_vec<BITS>(cnt, x[i], lo, nrows, spare, (subs >> i) & 1u);
        };
        uint4 xa[U], xb[U];
        uint32_t sa, sb;
        fetch(0, xa, sa);
        for (uint32_t k0 = 0; k0 < mine; k0 += 2 * U) {
            if (k0 + U < mine) fetch(k0 + U, xb, sb);
            add(xa, sa);
            if (k0 + U >= mine) break;
            if (k0 + 2 * U < mine) fetch(k0 + 2 * U, xa, sa);
            add(xb, sb);
        }
        __syncwarp();  // the group's slices are read before the next unit writes them
        u = un;
        vs = vs_n;
        nv = nv_n;
    }
}

// One 32-bit output lane from 32 counters (words cw[0 .. kWords), 16-byte
// aligned), which are cleared as they are read, ready for the next tile.
// The words are read 16 bytes at a time; a chunk whose counters are all zero
// (most of them, in a sparse tile) yields f(0) for its rows and needs no
// compare and no clear.  Lane l starts at chunk l mod kChunks, spreading the
// warp over the banks.  A plain threshold (v0 = 0, one transition theta)
// compares packed counters with SIMD byte/halfword compares; every other
// predicate looks f up in `tab`.
template <int BITS>
__device__ __forceinline__ uint32_t counters_to_lane(uint32_t* cw, const Pred& pred,
                                                     const uint32_t* tab) {
    constexpr uint32_t kPer = 32 / BITS, kWords = 32 / kPer, kChunks = kWords / 4;
    constexpr uint32_t kChunkRows = 4 * kPer;  // rows per 16-byte chunk
    uint4* c4 = reinterpret_cast<uint4*>(cw);
    const uint32_t rot = threadIdx.x;
    const bool plain = pred.mode == 1 && pred.ntrans == 1 && pred.v0 == 0;
    const uint32_t th = pred.trans[0];  // plain: 1 <= theta <= n
    const uint32_t tw = BITS == 8 ? th * 0x01010101u : th * 0x00010001u;
    // rows nobody counted: f(0) (0 for a plain threshold)
    const uint32_t zero_rows = (!plain && (tab[0] & 1u)) ? (1u << kChunkRows) - 1u : 0u;
    uint32_t o = 0;
#pragma unroll
    for (uint32_t k = 0; k < kChunks; ++k) {
        const uint32_t c = (k + rot) & (kChunks - 1);
        const uint4 v = c4[c];
        if ((v.x | v.y | v.z | v.w) == 0u) {
            o |= zero_rows << (c * kChunkRows);
            continue;
        }
        c4[c] = make_uint4(0u, 0u, 0u, 0u);
        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) {
            const uint32_t word = wv[j];
            const uint32_t shift = (c * 4 + j) * kPer;  // first row of this word in the lane
            uint32_t bits = 0;
            if (plain) {
                if (BITS == 8) {
                    const uint32_t b = __vcmpgeu4(word, tw) & 0x01010101u;  // per byte: count >= theta
                    bits = (b | (b >> 7) | (b >> 14) | (b >> 21)) & 0xFu;
                } else {
                    const uint32_t ge = __vcmpgeu2(word, tw);  // 0xFFFF per half where count >= theta
                    bits = (ge & 1u) | ((ge >> 15) & 2u);
                }
            } else {
#pragma unroll
                for (uint32_t s = 0; s < kPer; ++s) {
                    const uint32_t cnt = (word >> (BITS * s)) & ((1u << BITS) - 1u);
                    bits |= ((tab[cnt >> 5] >> (cnt & 31u)) & 1u) << s;
                }
            }
            o |= bits << shift;
        }
    }
    return o;
}

}  // namespace dev
}  // namespace bm
