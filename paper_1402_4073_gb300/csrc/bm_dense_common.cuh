// Column-level pieces of the dense bit-sliced counter shared by the
// single-query kernels and the batch kernel: accumulate one 128-row column
// of n inputs into counter planes, then evaluate the predicate, mask rows
// >= r, store and popcount.
#pragma once

#include "bm_device.cuh"

namespace bm {
namespace dev {

// Per-lane accumulation of a partial group (nb < group inputs) read by `get(b)`.
template <int K, typename Get>
__device__ __forceinline__ void add_partial(uint32_t (&P)[4][K], uint32_t nb, Get get) {
    uint32_t b = 0;
    for (; b + 2 <= nb; b += 2) {
        uint4 u = get(b), v = get(b + 1);
        add2<K>(P[0], u.x, v.x);
        add2<K>(P[1], u.y, v.y);
        add2<K>(P[2], u.z, v.z);
        add2<K>(P[3], u.w, v.w);
    }
    if (b < nb) {
        uint4 u = get(b);
        add1<K>(P[0], u.x);
        add1<K>(P[1], u.y);
        add1<K>(P[2], u.z);
        add1<K>(P[3], u.w);
    }
}

template <int K>
__device__ __forceinline__ void add_group16(uint32_t (&P)[4][K], const uint4 (&v)[16]) {
    uint32_t x[16];
#pragma unroll
    for (int b = 0; b < 16; ++b) x[b] = v[b].x;
    add16<K>(P[0], x);
#pragma unroll
    for (int b = 0; b < 16; ++b) x[b] = v[b].y;
    add16<K>(P[1], x);
#pragma unroll
    for (int b = 0; b < 16; ++b) x[b] = v[b].z;
    add16<K>(P[2], x);
#pragma unroll
    for (int b = 0; b < 16; ++b) x[b] = v[b].w;
    add16<K>(P[3], x);
}

template <int K>
__device__ __forceinline__ void add_group8(uint32_t (&P)[4][K], const uint4 (&v)[8]) {
    uint32_t x[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) x[b] = v[b].x;
    add8<K>(P[0], x);
#pragma unroll
    for (int b = 0; b < 8; ++b) x[b] = v[b].y;
    add8<K>(P[1], x);
#pragma unroll
    for (int b = 0; b < 8; ++b) x[b] = v[b].z;
    add8<K>(P[2], x);
#pragma unroll
    for (int b = 0; b < 8; ++b) x[b] = v[b].w;
    add8<K>(P[3], x);
}

template <int K>
__device__ __forceinline__ void zero_planes(uint32_t (&P)[4][K]) {
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int j = 0; j < K; ++j) P[l][j] = 0u;
}

// Count one 16-byte column (128 rows) of the n inputs ids[0..n) with direct
// streaming loads, G (16 or 8) inputs per sideways-sum block.
template <int K, int G>
__device__ __forceinline__ void count_column(uint32_t (&P)[4][K], const uint64_t* colbase,
                                             const uint32_t* ids, uint32_t n,
                                             uint64_t stride_words) {
    uint32_t k = 0;
    for (; k + G <= n; k += G) {
        uint4 v[G];
#pragma unroll
        for (int b = 0; b < G; ++b)
            v[b] = ld_stream(colbase + (uint64_t)__ldg(ids + k + b) * stride_words);
        if constexpr (G == 16)
            add_group16<K>(P, v);
        else
            add_group8<K>(P, v);
    }
    if (k < n) {
        const uint32_t* rest = ids + k;
        add_partial<K>(P, n - k, [&](uint32_t b) {
            return ld_stream(colbase + (uint64_t)__ldg(rest + b) * stride_words);
        });
    }
}

// Predicate, tail mask, store and popcount of one 128-row column (words
// 2*col and 2*col+1 of the output).
template <int K>
__device__ __forceinline__ uint32_t finish_column(const uint32_t (&P)[4][K], const Pred& pred,
                                                  const uint32_t* tab, uint64_t r_bits,
                                                  uint64_t words, uint64_t* out, uint64_t col,
                                                  bool vec_ok) {
    uint32_t o0 = eval_pred<K>(P[0], pred, tab);
    uint32_t o1 = eval_pred<K>(P[1], pred, tab);
    uint32_t o2 = eval_pred<K>(P[2], pred, tab);
    uint32_t o3 = eval_pred<K>(P[3], pred, tab);
    uint64_t w0 = (uint64_t)o0 | ((uint64_t)o1 << 32);
    uint64_t w1 = (uint64_t)o2 | ((uint64_t)o3 << 32);
    const uint64_t i0 = 2 * col, i1 = i0 + 1;
    const uint32_t tail = (uint32_t)(r_bits & 63u);
    const uint64_t last = words - 1;
    if (tail) {
        const uint64_t m = (1ull << tail) - 1ull;
        if (i0 == last) w0 &= m;
        if (i1 == last) w1 &= m;
    }
    if (i1 < words) {
        if (vec_ok) {
            asm volatile("st.global.v2.u64 [%0], {%1, %2};" ::"l"(out + i0), "l"(w0), "l"(w1)
                         : "memory");
        } else {
            out[i0] = w0;
            out[i1] = w1;
        }
        return (uint32_t)(__popcll(w0) + __popcll(w1));
    }
    if (i0 < words) {
        out[i0] = w0;
        return (uint32_t)__popcll(w0);
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
