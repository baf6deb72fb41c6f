// Column-level pieces of the dense bit-sliced counter shared by the
// single-query kernels and the batch kernel: accumulate one column (64 or
// 128 rows) of n inputs into counter planes, then evaluate the predicate,
// mask rows >= r, store and popcount.
#pragma once

#include "bm_device.cuh"

namespace bm {
namespace dev {

// A thread's column is L 32-bit lanes (L = 4: a 16-byte slice, two 64-bit
// words; L = 2: an 8-byte slice, one word) of every input.
template <int L>
struct Slice;
template <>
struct Slice<4> {
    uint32_t v[4];
};
template <>
struct Slice<2> {
    uint32_t v[2];
};

// Read-only load of one slice: streaming (L1 allocation bypassed: a single
// query reads every input word once), or with Cached through L1 (the batch
// kernel, whose items on one SM read the same slab of the pool for other
// queries).
template <int L, bool Cached = false>
__device__ __forceinline__ Slice<L> ld_slice(const uint64_t* p) {
    Slice<L> s;
    if constexpr (L == 4) {
        if constexpr (Cached)
            asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(s.v[0]), "=r"(s.v[1]), "=r"(s.v[2]), "=r"(s.v[3])
                         : "l"(p));
        else
            asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(s.v[0]), "=r"(s.v[1]), "=r"(s.v[2]), "=r"(s.v[3])
                         : "l"(p));
    } else {
        if constexpr (Cached)
            asm volatile("ld.global.nc.v2.u32 {%0,%1}, [%2];" : "=r"(s.v[0]), "=r"(s.v[1]) : "l"(p));
        else
            asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];"
                         : "=r"(s.v[0]), "=r"(s.v[1])
                         : "l"(p));
    }
    return s;
}

// Per-lane accumulation of a partial group (nb inputs) read by `get(b)`.
template <int K, int L, typename Get>
__device__ __forceinline__ void add_partial(uint32_t (&P)[L][K], uint32_t nb, Get get) {
    uint32_t b = 0;
    for (; b + 2 <= nb; b += 2) {
        const auto u = get(b), v = get(b + 1);
#pragma unroll
        for (int l = 0; l < L; ++l) add2<K>(P[l], u.v[l], v.v[l]);
    }
    if (b < nb) {
        const auto u = get(b);
#pragma unroll
        for (int l = 0; l < L; ++l) add1<K>(P[l], u.v[l]);
    }
}

// One sideways-sum block of G (16 or 8) inputs on every lane.
template <int K, int L, int G>
__device__ __forceinline__ void add_group(uint32_t (&P)[L][K], const Slice<L> (&v)[G]) {
#pragma unroll
    for (int l = 0; l < L; ++l) {
        uint32_t x[G];
#pragma unroll
        for (int b = 0; b < G; ++b) x[b] = v[b].v[l];
        if constexpr (G == 16)
            add16<K>(P[l], x);
        else
            add8<K>(P[l], x);
    }
}

template <int K, int L>
__device__ __forceinline__ void zero_planes(uint32_t (&P)[L][K]) {
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
        for (int j = 0; j < K; ++j) P[l][j] = 0u;
}

// Four ids (16-byte aligned) and one id: read-only global loads, or, with
// Gen, generic loads (ids that may sit in shared memory).
template <bool Gen>
__device__ __forceinline__ uint4 ld_ids4(const uint32_t* p) {
    if constexpr (Gen) return *reinterpret_cast<const uint4*>(p);
    else return __ldg(reinterpret_cast<const uint4*>(p));
}
template <bool Gen>
__device__ __forceinline__ uint32_t ld_id(const uint32_t* p) {
    if constexpr (Gen) return *p;
    else return __ldg(p);
}

// Count one column (L lanes of 32 rows) of the n inputs ids[0..n) with
// direct streaming loads, G (32, 16 or 8) inputs per sideways-sum block.  ids
// must be 16-byte aligned: full blocks read their ids four at a time.  The
// last n mod G inputs go through 8-input blocks padded with zero inputs,
// which costs less than rippling each input through every plane.  Gen: ids
// are read with generic loads (they may be in shared memory).  Cached: input
// words through L1 (ld_slice).
template <int K, int G, int L, bool Gen = false, bool Cached = false>
__device__ __forceinline__ void count_column(uint32_t (&P)[L][K], const uint64_t* colbase,
                                             const uint32_t* ids, uint32_t n,
                                             uint64_t stride_words) {
    uint32_t k = 0;
    if constexpr (G == 32) {
        // two sixteen-input trees per step, joined at plane 4
        for (; k + 32 <= n; k += 32) {
            uint32_t s16[2][L];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t id[16];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint4 q = ld_ids4<Gen>(ids + k + 16 * h + 4 * i);
                    id[4 * i] = q.x;
                    id[4 * i + 1] = q.y;
                    id[4 * i + 2] = q.z;
                    id[4 * i + 3] = q.w;
                }
                Slice<L> v[16];
#pragma unroll
                for (int b = 0; b < 16; ++b)
                    v[b] = ld_slice<L, Cached>(colbase + (uint64_t)id[b] * stride_words);
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    uint32_t x[16];
#pragma unroll
                    for (int b = 0; b < 16; ++b) x[b] = v[b].v[l];
                    s16[h][l] = add16_carry<K>(P[l], x);
                }
            }
#pragma unroll
            for (int l = 0; l < L; ++l) add32_join<K>(P[l], s16[0][l], s16[1][l]);
        }
    }
    constexpr int GB = G == 32 ? 16 : G;  // block size for what is left
    for (; k + GB <= n; k += GB) {
        uint32_t id[GB];
#pragma unroll
        for (int i = 0; i < GB / 4; ++i) {
            const uint4 q = ld_ids4<Gen>(ids + k + 4 * i);
            id[4 * i] = q.x;
            id[4 * i + 1] = q.y;
            id[4 * i + 2] = q.z;
            id[4 * i + 3] = q.w;
        }
        Slice<L> v[GB];
#pragma unroll
        for (int b = 0; b < GB; ++b) v[b] = ld_slice<L, Cached>(colbase + (uint64_t)id[b] * stride_words);
        add_group<K, L, GB>(P, v);
    }
    while (k < n) {
        const uint32_t m = min(8u, n - k);
        Slice<L> v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            if ((uint32_t)b < m) {
                v[b] = ld_slice<L, Cached>(colbase + (uint64_t)ld_id<Gen>(ids + k + b) * stride_words);
            } else {
#pragma unroll
                for (int l = 0; l < L; ++l) v[b].v[l] = 0u;
            }
        }
        add_group<K, L, 8>(P, v);
        k += m;
    }
}

// Predicate, tail mask, store and popcount of one column: output words
// (L/2)*col .. (L/2)*col + L/2 - 1.
template <int K, int L>
__device__ __forceinline__ uint32_t finish_column(const uint32_t (&P)[L][K], const Pred& pred,
                                                  const uint32_t* tab, uint64_t r_bits,
                                                  uint64_t words, uint64_t* out, uint64_t col,
                                                  bool vec_ok) {
    constexpr int W = L / 2;
    uint64_t w[W];
#pragma unroll
    for (int i = 0; i < W; ++i)
        w[i] = (uint64_t)eval_pred<K>(P[2 * i], pred, tab) |
               ((uint64_t)eval_pred<K>(P[2 * i + 1], pred, tab) << 32);
    const uint64_t i0 = (uint64_t)W * col;
    const uint32_t tail = (uint32_t)(r_bits & 63u);
    if (tail) {
        const uint64_t m = (1ull << tail) - 1ull;
#pragma unroll
        for (int i = 0; i < W; ++i)
            if (i0 + i == words - 1) w[i] &= m;
    }
    if constexpr (W == 2) {
        if (i0 + 1 < words) {
            if (vec_ok) {
                asm volatile("st.global.v2.u64 [%0], {%1, %2};" ::"l"(out + i0), "l"(w[0]),
                             "l"(w[1])
                             : "memory");
            } else {
                out[i0] = w[0];
                out[i0 + 1] = w[1];
            }
            return (uint32_t)(__popcll(w[0]) + __popcll(w[1]));
        }
    }
    if (i0 < words) {
        out[i0] = w[0];
        return (uint32_t)__popcll(w[0]);
    }
    return 0;
}

__device__ __forceinline__ void flush_card(unsigned long long card, unsigned long long* out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) card += __shfl_xor_sync(0xFFFFFFFFu, card, o);
    if ((threadIdx.x & 31) == 0 && out && card) atomicAdd(out, card);
}

}  // namespace dev
}  // namespace bm
