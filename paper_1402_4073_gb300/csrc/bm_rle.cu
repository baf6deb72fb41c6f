// Threshold and symmetric queries over run-length compressed bitmaps: the
// word-aligned form of Sec. 2.1 (every word clean-0, clean-1 or literal, as
// in EWAH) with the clean-run pruning of RBMrg (Sec. 4.1): where an input is
// a clean run, it adds 0 or 1 to every row and needs no bitwise work, and
// only the tiles where an input mixes kinds are added word by word.
//
// GPU form: a CTA owns a tile of 256 words at a time (one 64-bit word column
// per consumer thread, a 32-word slice per consumer warp) and one producer
// warp feeds it.  The producer reads the tile's summary of every input: a
// clean-0 input is skipped, a clean-1 one adds one to a per-tile constant c1
// (k in the paper), a mixed one is listed.  When the predicate takes one
// value over every count the tile can still reach, [c1, c1 + mixed inputs],
// the tile is that value: the producer writes it and nothing else is read.
// Otherwise the producer streams the mixed inputs' containers (masks, ranks,
// literal words) into a ring of shared-memory stages, up to 32 per stage, one
// lane per container issuing 16-byte asynchronous copies (cp.async) whose
// completion the stage's mbarrier tracks, and runs ahead into the next tiles
// while the consumers work (it also loads the next tiles' summaries while
// posting this one).  Containers are a few hundred bytes: the lanes' copies
// issue faster than one bulk copy (TMA) per container.  A consumer warp first
// finds which containers of the stage have a word of its slice that is not
// zero; a lane then reads its word of each of them from shared memory (the literal at the slice's rank plus the lane's
// place among the literal bits, or all ones), the words go through the
// eight-input sideways-sum block of the dense counter, and at the tile's
// last stage the predicate is evaluated on count + c1.  Only summaries and
// the containers of mixed tiles are read from HBM, each once.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "bm_dense_common.cuh"

namespace bm {

void rle_encode(const uint64_t* w, uint64_t nw, std::vector<uint4>& containers,
                uint64_t first_unit, uint2* summary, size_t stride, uint64_t* runs,
                uint64_t* literal_words) {
    auto kind = [](uint64_t x) -> uint32_t {
        return x == 0ull ? kTileClean0 : (x == ~0ull ? kTileClean1 : kTileMixed);
    };
    uint64_t nr = 0, nl = 0;
    uint32_t prev = 3;
    for (uint64_t i = 0; i < nw; ++i) {
        const uint32_t k = kind(w[i]);
        nr += k != prev;
        nl += k == kTileMixed;
        prev = k;
    }
    *runs = nr;
    *literal_words = nl;
    const uint64_t base = containers.size();
    const uint64_t tiles = (nw + kRleTileWords - 1) / kRleTileWords;
    constexpr uint32_t kSlices = kRleTileWords / kRleSliceWords;
    std::vector<uint64_t> lits;
    lits.reserve(kRleTileWords);
    for (uint64_t t = 0; t < tiles; ++t) {
        const uint64_t w0 = t * kRleTileWords, w1 = std::min<uint64_t>(w0 + kRleTileWords, nw);
        uint32_t L[kSlices] = {}, O[kSlices] = {};
        uint32_t nones = 0;
        lits.clear();
        for (uint64_t i = w0; i < w1; ++i) {
            const uint32_t k = kind(w[i]);
            const uint32_t s = (uint32_t)(i - w0) / kRleSliceWords;
            const uint32_t b = (uint32_t)(i - w0) % kRleSliceWords;
            if (k == kTileMixed) {
                L[s] |= 1u << b;
                lits.push_back(w[i]);
            }
            if (k == kTileClean1) {
                O[s] |= 1u << b;
                ++nones;
            }
        }
        uint2& sum = summary[t * stride];
        if (lits.empty() && nones == 0) {
            sum = make_uint2(kTileClean0 << 30, 0u);
            continue;
        }
        if (lits.empty() && nones == w1 - w0) {
            sum = make_uint2(kTileClean1 << 30, 0u);
            continue;
        }
        // header and literal words, padded to 16 bytes (at most 133 units)
        const size_t units = (kRleHeaderBytes + 8 * lits.size() + 15) / 16;
        const uint64_t at = containers.size();
        const uint64_t start = first_unit + (at - base);
        sum = make_uint2((kTileMixed << 30) | (uint32_t)(start & kTileOffsetMask),
                         (uint32_t)((start >> 30) << 8) | (uint32_t)units);
        containers.resize(at + units, make_uint4(0u, 0u, 0u, 0u));
        uint8_t* c = reinterpret_cast<uint8_t*>(containers.data() + at);
        uint8_t R[kSlices];
        uint32_t before = 0;
        for (uint32_t s = 0; s < kSlices; ++s) {
            R[s] = (uint8_t)before;
            before += (uint32_t)__builtin_popcount(L[s]);
        }
        std::memcpy(c, L, sizeof(L));
        std::memcpy(c + sizeof(L), O, sizeof(O));
        std::memcpy(c + sizeof(L) + sizeof(O), R, sizeof(R));
        std::memcpy(c + kRleHeaderBytes, lits.data(), 8 * lits.size());
    }
}

namespace {

using namespace dev;

// Global -> shared copy of 16 bytes by one thread, cached in L2 only.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}
// Arrive on `bar` once every cp.async this thread issued so far has landed;
// the arrival counts against the barrier's expected count.
__device__ __forceinline__ void cp_async_mbar_arrive_noinc(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}


constexpr uint32_t kRleSlices = kRleTileWords / kRleSliceWords;  // consumer warps
constexpr uint32_t kRleThreads = kRleTileWords + 32;             // + the producer warp
constexpr uint32_t kRleChunk = 1024;        // inputs classified per pass
constexpr uint32_t kRleStageMax = 32;       // containers per stage: one per producer lane
constexpr uint32_t kRleStageBytes = 8192;   // bytes per stage (a container is at most 2128)
constexpr uint32_t kRleStages = 4;
constexpr uint32_t kRleAhead = 4;  // tiles whose first 256 summaries are in flight (one chunk)

// What the producer posts with each stage.
constexpr uint32_t kRleNoTile = 0xFFFFFFFFu;  // the terminal stage: no tiles left
struct RleStage {
    uint32_t tile;                // the tile the containers belong to, or kRleNoTile
    uint32_t count;               // containers in the stage
    uint32_t last;                // the tile's last stage
    uint32_t c1;                  // inputs clean-1 over the tile so far (all of them on the last)
    uint16_t off[kRleStageMax];   // byte offset of each container in the stage
};

// Output word of one column: the predicate on count + off per row, where the
// planes P hold the count of the mixed inputs and `off` the inputs that are
// clean-1 over the tile.  Thresholds move down by off (those at or below it
// always hold); a table is read at count + off.
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
    if (p.mode == 1) {
        // a transition at or below off holds on every row: it flips the
        // constant; one above it is the threshold count >= t - off
        uint32_t r0 = p.v0 ? 0xFFFFFFFFu : 0u, r1 = r0;
#pragma unroll 1
        for (int i = 0; i < kMaxTransitions; ++i) {
            if ((uint32_t)i < p.ntrans) {
                const uint32_t t = p.trans[i];
                if (t <= off) {
                    r0 = ~r0;
                    r1 = ~r1;
                } else {
                    r0 ^= greater_than<K>(P[0], t - off - 1u);
                    r1 ^= greater_than<K>(P[1], t - off - 1u);
                }
            }
        }
        return (uint64_t)r0 | ((uint64_t)r1 << 32);
    }
    return (uint64_t)eval_pred<K>(P[0], p, tab) | ((uint64_t)eval_pred<K>(P[1], p, tab) << 32);
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
__global__ void __launch_bounds__(kRleThreads, K <= 13 ? 3 : 2)
    rle_kernel(RleArgs a, const __grid_constant__ LaunchExtra x) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t* ring = smem;                                                // [stages][bytes]
    uint64_t* full = reinterpret_cast<uint64_t*>(ring + kRleStages * kRleStageBytes);
    uint64_t* empty = full + kRleStages;
    RleStage* desc = reinterpret_cast<RleStage*>(empty + kRleStages);   // [stages]
    uint64_t* list_at = reinterpret_cast<uint64_t*>(desc + kRleStages);  // [chunk]: arena bytes
    uint32_t* s_ids = reinterpret_cast<uint32_t*>(list_at + kRleChunk);  // [chunk]
    uint16_t* list_units = reinterpret_cast<uint16_t*>(s_ids + kRleChunk);  // [chunk]
    uint2* s_sum = reinterpret_cast<uint2*>(list_units + kRleChunk);      // [ahead][256]
    uint32_t* tab = reinterpret_cast<uint32_t*>(s_sum + kRleAhead * 256);  // f over 0..n
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t tab_words = a.pred.mode == 2 ? (a.n + 1 + 31) / 32 : 0u;
    for (uint32_t w = tid; w < tab_words; w += kRleThreads) tab[w] = a.pred.table[w];
    // with one chunk (n <= kRleChunk) the ids are read once
    const bool one_chunk = a.n <= kRleChunk;
    if (one_chunk)
        for (uint32_t i = tid; i < a.n; i += kRleThreads)
            s_ids[i] = x.n_inline ? x.inl[i] : __ldg(a.ids + i);
    if (tid == 0) {
        for (uint32_t s = 0; s < kRleStages; ++s) {
            // full: each producer lane's copies (tracked by cp.async) and the
            // post of the stage's descriptor
            mbar_init(&full[s], 33);
            mbar_init(&empty[s], kRleSlices);
        }
        fence_barrier_init();
    }
    __syncthreads();
    const uint64_t ntiles = (a.words + kRleTileWords - 1) / kRleTileWords;

    if (warp == kRleSlices) {
        // producer: classify each tile's inputs; write a constant tile, or
        // post its mixed inputs' containers in stages (the tile's last is
        // marked), then a terminal stage
        // with one chunk, the summaries of the first 256 inputs of the next
        // kRleAhead tiles are in flight to s_sum (a lane copies its own eight)
        auto fetch_first = [&](uint64_t tile, uint32_t slot) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t i = 32 * u + lane;
                uint2* dst = s_sum + slot * 256 + i;
                if (i < a.n && tile < ntiles)
                    cp_async8(dst, a.tile_index + tile * a.capacity + s_ids[i]);
                else
                    *dst = make_uint2(0u, 0u);  // clean-0: nothing to add
            }
            cp_async_commit();
        };
        if (one_chunk)
            for (uint32_t d = 0; d < kRleAhead; ++d)
                fetch_first(blockIdx.x + (uint64_t)d * gridDim.x, d);
        uint32_t ti = 0;  // tiles of this CTA so far
        uint64_t it = 0;
        bool ok = true;
        unsigned long long card = 0;  // of the tiles the producer writes
        // wait until stage st is free (its previous use consumed)
        auto free_stage = [&](uint32_t st) -> bool {
            bool f = true;
            if (lane == 0 && it >= kRleStages)
                f = mbar_wait_bounded(&empty[st], (uint32_t)((it / kRleStages - 1) & 1), a.err);
            ok = __shfl_sync(0xFFFFFFFFu, f, 0) && ok;
            return ok;
        };
        for (uint64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const uint2* row = a.tile_index + tile * a.capacity;
            uint32_t c1 = 0;
            for (uint32_t c0 = 0; c0 < a.n && ok; c0 += kRleChunk) {
                const uint32_t m = min(kRleChunk, a.n - c0);
                const bool final = c0 + m >= a.n;
                uint32_t nd = 0;
                for (uint32_t k0 = 0; k0 < m; k0 += 256) {
                    // eight inputs per lane in flight; with one chunk the first
                    // 256 were loaded while the previous tile was posted
                    uint2 sm[8];
                    if (one_chunk && k0 == 0) {
                        const uint32_t slot = ti % kRleAhead;
                        cp_async_wait<kRleAhead - 1>();
#pragma unroll
                        for (int u = 0; u < 8; ++u) sm[u] = s_sum[slot * 256 + 32 * u + lane];
                        fetch_first(tile + (uint64_t)kRleAhead * gridDim.x, slot);
                    } else {
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const uint32_t i = k0 + 32 * u + lane;
                            sm[u] = make_uint2(0u, 0u);  // clean-0: nothing to add
                            if (i < m) {
                                const uint32_t id = one_chunk      ? s_ids[i]
                                                    : x.n_inline ? x.inl[c0 + i]
                                                                 : __ldg(a.ids + c0 + i);
                                sm[u] = __ldg(row + id);
                            }
                        }
                    }
                    // counts by lane, summed over the warp; the mixed inputs are
                    // listed lane after lane (a scan of the lanes' counts places
                    // them), unless one pass of at most 256 inputs finds the tile
                    // constant first
                    uint32_t ones = 0, mixed = 0;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const uint32_t cls = sm[u].x >> 30;
                        ones += cls == kTileClean1;
                        mixed += cls == kTileMixed;
                    }
                    c1 += __reduce_add_sync(0xFFFFFFFFu, ones);
                    const uint32_t tot = __reduce_add_sync(0xFFFFFFFFu, mixed);
                    if (one_chunk && m <= 256 && tot &&
                        constant_over(a.pred, tab, c1, c1 + tot) >= 0) {
                        nd = tot;  // the tile is constant: no list needed
                        break;
                    }
                    if (tot) {
                        uint32_t incl = mixed;
#pragma unroll
                        for (uint32_t o = 1; o < 32; o <<= 1) {
                            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                            if (lane >= o) incl += y;
                        }
                        uint32_t at = nd + incl - mixed;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            if ((sm[u].x >> 30) == kTileMixed) {
                                list_at[at] = tile_container(sm[u]) * 16;
                                list_units[at] = (uint16_t)tile_units(sm[u]);
                                ++at;
                            }
                        }
                    }
                    nd += tot;
                }
                __syncwarp();
                if (one_chunk) {
                    const int konst = constant_over(a.pred, tab, c1, c1 + nd);
                    if (konst >= 0) {
                        // the whole tile is one value: the producer writes it,
                        // the consumers never see the tile
                        const uint64_t w0 = tile * kRleTileWords;
                        const uint64_t fill = konst ? ~0ull : 0ull;
                        if (w0 + kRleTileWords <= a.words &&
                            (reinterpret_cast<uintptr_t>(a.out) & 15u) == 0) {
                            // a whole tile: two words per 16-byte store
#pragma unroll
                            for (uint32_t u = 0; u < kRleTileWords / 64; ++u)
                                asm volatile("st.global.v2.u64 [%0], {%1, %2};" ::"l"(
                                                 a.out + w0 + 64 * u + 2 * lane),
                                             "l"(fill), "l"(fill)
                                             : "memory");
                            if (konst && lane == 0) card += 64ull * kRleTileWords;
                        } else {
#pragma unroll
                            for (uint32_t u = 0; u < kRleTileWords / 32; ++u) {
                                const uint64_t col = w0 + 32 * u + lane;
                                if (col < a.words) {
                                    uint64_t word = fill;
                                    if (col == a.words - 1 && (a.r_bits & 63u))
                                        word &= (1ull << (a.r_bits & 63u)) - 1ull;
                                    a.out[col] = word;
                                    card += (unsigned long long)__popcll(word);
                                }
                            }
                        }
                        break;
                    }
                }
                // post the listed containers in stages; the final pass posts
                // at least one (which carries c1 and ends the tile)
                uint32_t e = 0;
                while (ok && (e < nd || (final && e == 0 && nd == 0))) {
                    const uint32_t st = (uint32_t)(it % kRleStages);
                    if (!free_stage(st)) break;
                    // the next containers that fit: lanes take one each, an
                    // inclusive sum of their sizes places them
                    const bool valid = lane < kRleStageMax && e + lane < nd;
                    const uint32_t units = valid ? list_units[e + lane] : 0u;
                    uint32_t incl = units;
#pragma unroll
                    for (uint32_t o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const uint32_t count =
                        __popc(__ballot_sync(0xFFFFFFFFu, valid && incl * 16 <= kRleStageBytes));
                    const uint32_t off = 16 * (incl - units);
                    RleStage& d = desc[st];
                    if (lane < count) {
                        d.off[lane] = (uint16_t)off;
                        const uint8_t* src = a.arena + list_at[e + lane];
                        uint8_t* dst = ring + st * kRleStageBytes + off;
                        for (uint32_t q = 0; q < units; ++q) cp_async16(dst + 16 * q, src + 16 * q);
                    }
                    cp_async_mbar_arrive_noinc(&full[st]);
                    __syncwarp();
                    if (lane == 0) {
                        d.tile = (uint32_t)tile;
                        d.count = count;
                        d.last = final && e + count >= nd;
                        d.c1 = c1;
                        mbar_arrive(&full[st]);
                    }
                    __syncwarp();
                    e += count;
                    ++it;
                    if (count == 0) break;  // the empty final stage
                }
            }
            ++ti;
        }
        // the terminal stage
        if (ok && free_stage((uint32_t)(it % kRleStages))) {
            const uint32_t st = (uint32_t)(it % kRleStages);
            cp_async_mbar_arrive_noinc(&full[st]);
            __syncwarp();
            if (lane == 0) {
                desc[st].tile = kRleNoTile;
                desc[st].count = 0;
                mbar_arrive(&full[st]);
            }
            ++it;
        }
        // the producer's part of the cardinality
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) card += __shfl_xor_sync(0xFFFFFFFFu, card, o);
        if (lane == 0) card_contribute(card, a.card, x.acc, x.ticket, gridDim.x * (kRleSlices + 1));
        // every issued copy must land before this CTA may exit
        cp_async_wait<0>();
        if (lane == 0) {
            const uint64_t first = it > kRleStages ? it - kRleStages : 0;
            for (uint64_t j = first; j < it; ++j)
                mbar_wait_bounded(&full[j % kRleStages], (uint32_t)((j / kRleStages) & 1), a.err);
        }
        return;
    }

    // consumers: stages in the producer's order, each for one tile; a tile's
    // last stage ends it
    unsigned long long card = 0;
    uint64_t it = 0;
    bool ok = true;
    uint32_t P[2][K];
    zero_planes<K, 2>(P);
    for (;;) {
        const uint32_t st = (uint32_t)(it % kRleStages);
        // every lane waits; the warp goes on only if all lanes saw the stage land
        const bool landed = mbar_wait_bounded(&full[st], (uint32_t)((it / kRleStages) & 1), a.err);
        if (!__all_sync(0xFFFFFFFFu, landed)) {
            ok = false;
            break;
        }
        const RleStage& d = desc[st];
        const uint32_t tile = d.tile;
        if (tile == kRleNoTile) break;
        const uint32_t count = d.count;
        const bool last = d.last != 0;
        const uint32_t c1 = d.c1;
        if (count) {
            // lane k reads container k's masks and rank for this warp's
            // slice; only containers with a word of the slice that is not
            // zero are added, eight at a time
            const uint8_t* buf = ring + st * kRleStageBytes;
            uint32_t lwk = 0, owk = 0, pos = 0;
            if (lane < count) {
                const uint32_t off = d.off[lane];
                const uint8_t* c = buf + off;
                lwk = reinterpret_cast<const uint32_t*>(c)[warp];
                owk = reinterpret_cast<const uint32_t*>(c)[kRleSlices + warp];
                pos = off | (uint32_t)c[8 * kRleSlices + warp] << 16;
            }
            uint32_t rem = __ballot_sync(0xFFFFFFFFu, (lwk | owk) != 0u);
            while (rem) {
                Slice<2> v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    uint64_t word = 0;
                    if (rem) {
                        const int j = __ffs(rem) - 1;
                        rem &= rem - 1;
                        const uint32_t lw = __shfl_sync(0xFFFFFFFFu, lwk, j);
                        const uint32_t ow = __shfl_sync(0xFFFFFFFFu, owk, j);
                        const uint32_t pj = __shfl_sync(0xFFFFFFFFu, pos, j);
                        if ((lw >> lane) & 1u)
                            word = reinterpret_cast<const uint64_t*>(
                                buf + (pj & 0xFFFFu) + kRleHeaderBytes)[(pj >> 16) +
                                                                        __popc(lw & below)];
                        else if ((ow >> lane) & 1u)
                            word = ~0ull;
                    }
                    v[k].v[0] = (uint32_t)word;
                    v[k].v[1] = (uint32_t)(word >> 32);
                }
                add_group<K, 2, 8>(P, v);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
        ++it;
        if (last) {
            const uint64_t col = (uint64_t)tile * kRleTileWords + tid;
            if (col < a.words) {
                uint64_t word = eval_offset<K>(P, a.pred, tab, c1);
                if (col == a.words - 1 && (a.r_bits & 63u))
                    word &= (1ull << (a.r_bits & 63u)) - 1ull;
                a.out[col] = word;
                card += (unsigned long long)__popcll(word);
            }
            zero_planes<K, 2>(P);
        }
    }
    // every consumer warp contributes (nothing if its waits gave up, which the
    // error word reports), so the last of them and the producers completes
    // the cardinality
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) card += __shfl_xor_sync(0xFFFFFFFFu, card, o);
    if (lane == 0)
        card_contribute(ok ? card : 0ull, a.card, x.acc, x.ticket,
                        gridDim.x * (kRleSlices + 1));
}

constexpr size_t kRleFixedSmem = (size_t)kRleStages * (kRleStageBytes + 16 + sizeof(RleStage)) +
                                 (size_t)kRleChunk * (8 + 4 + 2) +
                                 (size_t)kRleAhead * 256 * 8;
constexpr size_t kRleMaxSmem = kRleFixedSmem + ((size_t)BM_N_MAX + 1 + 31) / 32 * 4;
constexpr int kRleMaxDevices = 64;

// CTAs per SM of rle_kernel<K> on the current device.  The first call on a
// device raises the kernel's dynamic shared-memory limit to the largest
// request (the largest table) and looks the occupancy up at that size; later
// launches reuse both (the host calls cost more than a small query).
template <int K>
int rle_ctas_per_sm(int* per_sm) {
    static std::atomic<int> cached[kRleMaxDevices];
    int dev = 0;
    BM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < kRleMaxDevices && (*per_sm = cached[dev].load()) > 0) return BM_OK;
    BM_CUDA_TRY(cudaFuncSetAttribute(rle_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRleMaxSmem));
    int v = 0;
    BM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, rle_kernel<K>,
                                                              (int)kRleThreads, kRleMaxSmem));
    *per_sm = std::max(1, v);
    if (dev >= 0 && dev < kRleMaxDevices) cached[dev].store(*per_sm);
    return BM_OK;
}

template <int K>
int launch_k(const RleArgs& a, const LaunchExtra& x, int sm_count, cudaStream_t s) {
    const size_t tab_bytes = a.pred.mode == 2 ? (size_t)(a.n + 1 + 31) / 32 * 4 : 0;
    const size_t bytes = kRleFixedSmem + tab_bytes;
    // persistent: as many CTAs as fit at once, or one per tile
    int per_sm = 1;
    const int rc = rle_ctas_per_sm<K>(&per_sm);
    if (rc) return rc;
    const uint64_t ntiles = (a.words + kRleTileWords - 1) / kRleTileWords;
    const unsigned grid = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>(ntiles, (uint64_t)sm_count * (uint64_t)per_sm));
    rle_kernel<K><<<grid, kRleThreads, bytes, s>>>(a, x);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

}  // namespace

int launch_rle(const RleArgs& a, const LaunchExtra& x, int sm_count, cudaStream_t s) {
    if (a.words == 0) return BM_OK;
    if (a.n == 0) return BM_EINVAL;  // every tile needs at least one pass of inputs
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
    const uint64_t tiles = p->rle_tiles;
    if (!p->d_rle_tiles) {
        const size_t sum_bytes = (size_t)p->capacity * std::max<uint64_t>(tiles, 1) * 8;
        const int rc = track_alloc(p, (void**)&p->d_rle_tiles, sum_bytes);
        if (rc) return rc;
        BM_CUDA_TRY(cudaMemset(p->d_rle_tiles, 0, sum_bytes));
    }
    // grow the container arena to hold `need` 16-byte units
    auto grow = [&](uint64_t need) -> int {
        if (need <= p->rle_cap) return BM_OK;
        const uint64_t ncap = std::max<uint64_t>({need, p->rle_cap + p->rle_cap / 2, 1u << 16});
        void* nd = nullptr;
        int rc = track_alloc(p, &nd, ncap * 16);
        if (rc) return rc;
        if (p->rle_used)
            BM_CUDA_TRY(cudaMemcpy(nd, p->d_rle_arena, p->rle_used * 16, cudaMemcpyDeviceToDevice));
        track_free(p, p->d_rle_arena, p->rle_cap * 16);
        p->d_rle_arena = static_cast<uint4*>(nd);
        p->rle_cap = ncap;
        return BM_OK;
    };
    // ids in batches: a batch's summaries are one strided copy into the
    // tile-major summary matrix
    constexpr uint32_t kBatch = 64;
    std::vector<uint64_t> host(p->words), runs(kBatch), lits(kBatch), units(kBatch);
    std::vector<uint4> cont;
    std::vector<uint2> sums((size_t)tiles * kBatch);
    for (uint32_t j0 = 0; j0 < count; j0 += kBatch) {
        const uint32_t nb = std::min(kBatch, count - j0);
        for (uint32_t j = 0; j < nb; ++j) {
            const uint32_t id = first_id + j0 + j;
            BM_CUDA_TRY(cudaMemcpy(host.data(), p->d_dense + (uint64_t)id * p->stride_words,
                                   p->words * 8, cudaMemcpyDeviceToHost));
            cont.clear();
            rle_encode(host.data(), p->words, cont, p->rle_used, sums.data() + j, nb, &runs[j],
                       &lits[j]);
            int rc = grow(p->rle_used + cont.size());
            if (rc) return rc;
            if (!cont.empty())
                BM_CUDA_TRY(cudaMemcpy(p->d_rle_arena + p->rle_used, cont.data(),
                                       cont.size() * 16, cudaMemcpyHostToDevice));
            units[j] = cont.size();
            p->rle_used += cont.size();
        }
        const uint32_t id0 = first_id + j0;
        if (tiles)
            BM_CUDA_TRY(cudaMemcpy2D(p->d_rle_tiles + id0, (size_t)p->capacity * 8, sums.data(),
                                     (size_t)nb * 8, (size_t)nb * 8, tiles,
                                     cudaMemcpyHostToDevice));
        for (uint32_t j = 0; j < nb; ++j) {
            p->rle_runs[id0 + j] = runs[j];
            p->rle_lits[id0 + j] = lits[j];
            p->rle_units[id0 + j] = units[j];
            p->rle_present[id0 + j] = 1;
        }
    }
    return BM_OK;
}

int bm_pool_rle_info(const bm_pool* p, uint32_t id, uint64_t* runs, uint64_t* literal_words,
                     uint64_t* device_bytes) {
    if (!p) return BM_EINVAL;
    if (id >= p->capacity || !p->rle_present[id]) return BM_ERANGE;
    if (runs) *runs = p->rle_runs[id];
    if (literal_words) *literal_words = p->rle_lits[id];
    if (device_bytes) *device_bytes = 16 * p->rle_units[id] + 8 * (uint64_t)p->rle_tiles;
    return BM_OK;
}

}  // extern "C"
