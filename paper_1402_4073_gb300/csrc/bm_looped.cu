// The Looped recurrence (Sec. 4.4) for thresholds with a small T, over the
// dense pool.  After the inputs b_1..b_k, A_t holds the rows where at least t
// of them are set; adding input b updates, for t = T down to 1,
//     A_t <- A_t OR (A_{t-1} AND b),   A_0 = all rows,
// so the threshold costs T three-input logic operations per input word and T
// registers per lane instead of K counter planes and a comparator.
//
// Thresholds near N go through the complement identity in its corrected
// form (Sec. 2.3; NOT theta(T, b) = theta(N - T + 1, NOT b)): with
// T' = N - T + 1 the recurrence runs over the negated inputs and the result
// is negated, so the rows where at least T of N inputs are set cost T'
// operations per input.  A predicate "count < T" is the same with the output
// negated once more.
//
// GPU form: as the direct dense kernel, a thread owns a column of 128 rows
// (one 16-byte slice of every input, four 32-bit lanes) and streams the
// inputs with 16 loads in flight; the T accumulators stay in registers.
#include <algorithm>

#include "bm_dense_common.cuh"

namespace bm {
namespace {

using namespace dev;

// One input word into the T accumulators of a lane (NEG: the input negated).
template <int T, bool NEG>
__device__ __forceinline__ void looped_step(uint32_t (&A)[T], uint32_t x) {
    const uint32_t b = NEG ? ~x : x;
#pragma unroll
    for (int t = T - 1; t >= 1; --t) A[t] |= A[t - 1] & b;
    A[0] |= b;
}

template <int T, bool NEG>
__global__ void __launch_bounds__(256, 2)
    looped_kernel(DenseArgs a, const __grid_constant__ LaunchExtra x, uint32_t flip) {
    constexpr int L = 4;        // 32-bit lanes per thread (two 64-bit words)
    __shared__ __align__(16) uint32_t s_ids[kInlineIds];
    const uint32_t* ids = launch_ids(a.ids, x, s_ids);
    __syncthreads();
    const uint64_t ncols = (a.words + 1) / 2;
    const bool vec_ok = ((reinterpret_cast<uintptr_t>(a.out) & 15u) == 0);
    unsigned long long card = 0;
    for (uint64_t col = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; col < ncols;
         col += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t* colbase = a.base + 2 * col;
        uint32_t A[L][T];
#pragma unroll
        for (int l = 0; l < L; ++l)
#pragma unroll
            for (int t = 0; t < T; ++t) A[l][t] = 0u;
        uint32_t k = 0;
        for (; k + 16 <= a.n; k += 16) {
            uint32_t id[16];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint4 q = ld_ids4<true>(ids + k + 4 * i);
                id[4 * i] = q.x;
                id[4 * i + 1] = q.y;
                id[4 * i + 2] = q.z;
                id[4 * i + 3] = q.w;
            }
            Slice<L> v[16];
#pragma unroll
            for (int b = 0; b < 16; ++b) v[b] = ld_slice<L>(colbase + (uint64_t)id[b] * a.stride_words);
#pragma unroll
            for (int b = 0; b < 16; ++b)
#pragma unroll
                for (int l = 0; l < L; ++l) looped_step<T, NEG>(A[l], v[b].v[l]);
        }
        // the last n mod 16 inputs, eight loads in flight (m is warp-uniform;
        // a missing input cannot be stood in for by a zero word when NEG)
        while (k < a.n) {
            const uint32_t m = min(8u, a.n - k);
            Slice<L> v[8];
#pragma unroll
            for (int b = 0; b < 8; ++b)
                if ((uint32_t)b < m) v[b] = ld_slice<L>(colbase + (uint64_t)ids[k + b] * a.stride_words);
#pragma unroll
            for (int b = 0; b < 8; ++b)
                if ((uint32_t)b < m)
#pragma unroll
                    for (int l = 0; l < L; ++l) looped_step<T, NEG>(A[l], v[b].v[l]);
            k += m;
        }
        // A_T, negated back under the complement identity and for "count < T"
        const uint32_t inv = (NEG ? ~0u : 0u) ^ flip;
        uint64_t w[2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
            w[i] = (uint64_t)(A[2 * i][T - 1] ^ inv) | ((uint64_t)(A[2 * i + 1][T - 1] ^ inv) << 32);
        const uint64_t i0 = 2 * col;
        const uint32_t tail = (uint32_t)(a.r_bits & 63u);
        if (tail) {
            const uint64_t mk = (1ull << tail) - 1ull;
            if (i0 == a.words - 1) w[0] &= mk;
            if (i0 + 1 == a.words - 1) w[1] &= mk;
        }
        if (i0 + 1 < a.words) {
            if (vec_ok) {
                asm volatile("st.global.v2.u64 [%0], {%1, %2};" ::"l"(a.out + i0), "l"(w[0]),
                             "l"(w[1])
                             : "memory");
            } else {
                a.out[i0] = w[0];
                a.out[i0 + 1] = w[1];
            }
            card += (unsigned long long)(__popcll(w[0]) + __popcll(w[1]));
        } else {
            a.out[i0] = w[0];  // i0 == words - 1: the last word alone
            card += (unsigned long long)__popcll(w[0]);
        }
    }
    flush_card_block(card, a.card, x.acc, x.ticket);
}

template <int T, bool NEG>
int launch_t(const DenseArgs& a, const LaunchExtra& x, uint32_t flip, int sm_count, cudaStream_t s) {
    const uint64_t ncols = (a.words + 1) / 2;
    const uint64_t blocks = (ncols + 255) / 256;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(blocks, (uint64_t)sm_count * 2));
    looped_kernel<T, NEG><<<grid, 256, 0, s>>>(a, x, flip);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

}  // namespace

bool looped_form(const Pred& pred, uint32_t n, uint32_t max_t, LoopedForm* form) {
    // a plain threshold: f(c) = v0 XOR [c >= theta], 1 <= theta <= n
    if (max_t == 0 || pred.mode != 1 || pred.ntrans != 1) return false;
    const uint32_t theta = pred.trans[0];
    if (theta < 1 || theta > n) return false;
    const uint32_t t_direct = theta, t_comp = n - theta + 1;
    const uint32_t t = std::min(t_direct, t_comp);
    if (t > max_t || t > kLoopedMaxT) return false;
    form->t = t;
    form->neg = t_comp < t_direct;
    form->flip = pred.v0 ? ~0u : 0u;
    return true;
}

int launch_looped(const DenseArgs& a, const LaunchExtra& x, const LoopedForm& f, int sm_count,
                  cudaStream_t s) {
    if (a.words == 0) return BM_OK;
    if (f.neg) {
        if (f.t == 1) return launch_t<1, true>(a, x, f.flip, sm_count, s);
        if (f.t == 2) return launch_t<2, true>(a, x, f.flip, sm_count, s);
        return launch_t<3, true>(a, x, f.flip, sm_count, s);
    }
    if (f.t == 1) return launch_t<1, false>(a, x, f.flip, sm_count, s);
    if (f.t == 2) return launch_t<2, false>(a, x, f.flip, sm_count, s);
    return launch_t<3, false>(a, x, f.flip, sm_count, s);
}

}  // namespace bm

using namespace bm;

extern "C" int bm_pool_set_looped(bm_pool* p, uint32_t max_t) {
    if (!p || max_t > kLoopedMaxT) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    p->looped_max = max_t;
    return BM_OK;
}

extern "C" int bm_pool_get_looped(bm_pool* p, uint32_t* max_t) {
    if (!p || !max_t) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    *max_t = p->looped_max;
    return BM_OK;
}
