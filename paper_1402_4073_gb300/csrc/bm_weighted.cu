// Weighted threshold queries with an optional combining step, over the dense
// pool: row i is selected iff the sum of weights[k] over the inputs k holding
// row i reaches theta (Sec. 2.3 treats a weight as that many copies of an
// input; here a weight costs one read of the input whatever its size), and
// the result may then be ANDed, ORed or AND-NOTed with one more bitmap of the
// pool in the same pass (the result of a threshold is again a bitmap, Sec. 1).
//
// GPU form: a thread owns a column of one or two 64-bit words and keeps the
// weighted sum of its rows in registers in carry-save form: K sum planes P
// and K carry planes C, the sum being P + C.  Inputs of weight 1 go through
// the sixteen-input sideways-sum blocks of the dense kernel into P.  An input
// x of weight w > 1 is the K-bit number whose plane j is x where bit j of w
// is set; it joins P and C through one full adder per plane (sum to P_j, carry
// to C_{j+1}), so its cost is 3 logic operations per plane, with no carry
// ripple and every plane independent of the others.  One ripple-carry
// addition of C into P ends the column.  When the weights are small (their
// sum at most 8 per input and within BM_N_MAX) they are expanded into copies
// instead, which the sideways-sum blocks add faster.  The predicate is the
// runtime comparator of the dense kernel against theta - 1.
#include <algorithm>
#include <vector>

#include "bm_dense_common.cuh"

namespace bm {
namespace {

using namespace dev;

struct WeightedArgs {
    const uint64_t* base;
    uint64_t stride_words, words, r_bits;
    const uint32_t* ids1;  // inputs of weight 1 (16-byte aligned)
    uint32_t n1;
    uint32_t nw;           // inputs of weight > 1
    const uint32_t* idsw;
    const uint32_t* wts;
    uint64_t theta;        // 1 .. sum of weights (the host settles 0 and larger)
    uint32_t post_op;      // BM_POST_*
    uint32_t all;          // 1: every row is selected before combining (theta = 0)
    const uint64_t* post;  // the combined bitmap's words (post_op != 0)
    uint64_t* out;
    unsigned long long* card;
};

// Add the number whose plane j is x where bit j of w is set to the
// carry-save pair (P, C): a full adder per plane, planes taken from the top
// so that C_{j+1} is read before the carry of plane j replaces it.  The sum
// of the pair stays below 2^K (K holds the largest weighted sum), so no carry
// leaves plane K - 1.
template <int K>
__device__ __forceinline__ void csa_weighted(uint32_t (&P)[K], uint32_t (&C)[K], uint32_t x,
                                             uint32_t w) {
#pragma unroll
    for (int j = K - 1; j >= 0; --j) {
        const uint32_t a = x & (0u - ((w >> j) & 1u));
        const uint32_t carry = maj3(P[j], C[j], a);
        P[j] = xor3(P[j], C[j], a);
        if (j + 1 < K) C[j + 1] = carry;
    }
    C[0] = 0u;
}

// P <- P + C (ripple-carry addition; the sum fits in K planes).
template <int K>
__device__ __forceinline__ void resolve_carries(uint32_t (&P)[K], const uint32_t (&C)[K]) {
    uint32_t cy = 0u;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const uint32_t s = xor3(P[j], C[j], cy);
        cy = maj3(P[j], C[j], cy);
        P[j] = s;
    }
}

// L = 4: a thread owns two 64-bit words (128 rows, 16-byte loads); L = 2: one.
template <int K, int L>
__global__ void __launch_bounds__(256) weighted_kernel(WeightedArgs a) {
    constexpr uint32_t W = L / 2;  // words per thread
    const uint64_t ncols = (a.words + W - 1) / W;
    const bool vec_ok = ((reinterpret_cast<uintptr_t>(a.out) & 15u) == 0);
    unsigned long long card = 0;
    for (uint64_t col = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; col < ncols;
         col += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t w0 = W * col;  // first word of the column
        uint32_t P[L][K];
        zero_planes<K, L>(P);
        count_column<K, 16, L>(P, a.base + w0, a.ids1, a.n1, a.stride_words);
        if (a.nw) {
            uint32_t C[L][K];
            zero_planes<K, L>(C);
            // weighted inputs, the next one's word in flight while this one is added
            Slice<L> x_next = ld_slice<L>(a.base + (uint64_t)__ldg(a.idsw) * a.stride_words + w0);
            for (uint32_t k = 0; k < a.nw; ++k) {
                const Slice<L> x = x_next;
                const uint32_t w = __ldg(a.wts + k);
                if (k + 1 < a.nw)
                    x_next = ld_slice<L>(a.base + (uint64_t)__ldg(a.idsw + k + 1) * a.stride_words + w0);
#pragma unroll
                for (int l = 0; l < L; ++l) csa_weighted<K>(P[l], C[l], x.v[l], w);
            }
#pragma unroll
            for (int l = 0; l < L; ++l) resolve_carries<K>(P[l], C[l]);
        }
        uint64_t word[W];
#pragma unroll
        for (uint32_t i = 0; i < W; ++i)
            word[i] = a.all ? ~0ull
                            : ((uint64_t)greater_than<K>(P[2 * i], (uint32_t)(a.theta - 1)) |
                               ((uint64_t)greater_than<K>(P[2 * i + 1], (uint32_t)(a.theta - 1)) << 32));
#pragma unroll
        for (uint32_t i = 0; i < W; ++i) {
            const uint64_t wi = w0 + i;
            if (wi < a.words) {
                if (a.post_op) {
                    const uint64_t m = __ldg(a.post + wi);
                    word[i] = a.post_op == BM_POST_AND ? (word[i] & m)
                            : a.post_op == BM_POST_OR  ? (word[i] | m)
                                                       : (word[i] & ~m);
                }
                if (wi == a.words - 1 && (a.r_bits & 63u)) word[i] &= (1ull << (a.r_bits & 63u)) - 1ull;
            } else {
                word[i] = 0;
            }
        }
        if (W == 2 && w0 + 1 < a.words && vec_ok) {
            asm volatile("st.global.v2.u64 [%0], {%1, %2};" ::"l"(a.out + w0), "l"(word[0]),
                         "l"(word[W - 1])
                         : "memory");
        } else {
#pragma unroll
            for (uint32_t i = 0; i < W; ++i)
                if (w0 + i < a.words) a.out[w0 + i] = word[i];
        }
#pragma unroll
        for (uint32_t i = 0; i < W; ++i) card += (unsigned long long)__popcll(word[i]);
    }
    flush_card(card, a.card);
}

template <int K, int L>
int launch_k(const WeightedArgs& a, int sm_count, cudaStream_t s) {
    const uint64_t cols = (a.words + L / 2 - 1) / (L / 2);
    const uint64_t blocks = (cols + 255) / 256;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(blocks, (uint64_t)sm_count * 4));
    weighted_kernel<K, L><<<grid, 256, 0, s>>>(a);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" int bm_weighted_threshold(bm_pool* p, const bm_weighted_query* q, uint64_t* out_card,
                                     void* stream) {
    if (!p || !q || !q->out_words || q->reserved || q->n > BM_N_MAX) return BM_EINVAL;
    if (q->n && (!q->ids || !q->weights)) return BM_EINVAL;
    if (q->post_op > BM_POST_ANDNOT) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    int rc = validate_ids(p, q->ids, q->n, BM_PATH_DENSE);
    if (rc) return rc;
    if (q->post_op && (q->post_id >= p->capacity || !p->dense_present[q->post_id])) return BM_ERANGE;
    uint64_t sum = 0;
    std::vector<uint32_t> ids1, idsw, wts;
    for (uint32_t k = 0; k < q->n; ++k) {
        const uint32_t w = q->weights[k];
        if (w > BM_WEIGHT_MAX) return BM_EINVAL;
        sum += w;
        if (w == 1)
            ids1.push_back(q->ids[k]);
        else if (w > 1) {
            idsw.push_back(q->ids[k]);
            wts.push_back(w);
        }
    }
    if (sum > 0xFFFFFFFFull) return BM_EINVAL;
    // small weights: as many copies as the weight (Sec. 2.3's own reading),
    // all through the sideways-sum blocks; the copies of an input sit side by
    // side, so its repeated reads come from the caches
    if (!idsw.empty() && sum <= BM_N_MAX && sum <= 8ull * q->n) {
        ids1.clear();
        for (uint32_t k = 0; k < q->n; ++k) ids1.insert(ids1.end(), q->weights[k], q->ids[k]);
        idsw.clear();
        wts.clear();
    }
    BM_CUDA_TRY(cudaSetDevice(p->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // staging: weight-1 ids (16-byte aligned), weighted ids, weights
    const size_t b1 = (ids1.size() * 4 + 15) & ~(size_t)15;
    const size_t bw = (idsw.size() * 4 + 15) & ~(size_t)15;
    bm_stage_slot* sl = nullptr;
    rc = stage_acquire(p, b1 + 2 * bw + 16, &sl, s);
    if (rc) return rc;
    uint8_t* h = static_cast<uint8_t*>(sl->h);
    if (!ids1.empty()) memcpy(h, ids1.data(), ids1.size() * 4);
    if (!idsw.empty()) {
        memcpy(h + b1, idsw.data(), idsw.size() * 4);
        memcpy(h + b1 + bw, wts.data(), wts.size() * 4);
    }
    rc = stage_commit(sl, b1 + 2 * bw + 16, s);
    if (rc) return rc;
    if (out_card) BM_CUDA_TRY(cudaMemsetAsync(out_card, 0, 8, s));
    const uint8_t* d = static_cast<const uint8_t*>(sl->d);
    WeightedArgs a{};
    a.base = p->d_dense;
    a.stride_words = p->stride_words;
    a.words = p->words;
    a.r_bits = p->r_bits;
    a.ids1 = reinterpret_cast<const uint32_t*>(d);
    a.n1 = (uint32_t)ids1.size();
    a.idsw = reinterpret_cast<const uint32_t*>(d + b1);
    a.wts = reinterpret_cast<const uint32_t*>(d + b1 + bw);
    a.nw = (uint32_t)idsw.size();
    a.post_op = q->post_op;
    a.post = q->post_op ? p->d_dense + (uint64_t)q->post_id * p->stride_words : nullptr;
    a.out = q->out_words;
    a.card = reinterpret_cast<unsigned long long*>(out_card);
    // theta = 0 selects every row; theta > sum selects none (an empty sum of
    // inputs, as no weight is left to reach it)
    a.all = q->theta == 0 ? 1u : 0u;
    a.theta = q->theta;
    int planes = 0;  // bits of the largest sum
    if (q->theta > sum) {
        a.n1 = 0;
        a.nw = 0;
        a.theta = 1;  // the empty sum (0) is below 1: nothing is selected
    } else {
        while (planes < 32 && (sum >> planes) != 0) ++planes;
    }
    if (p->words) {
        // two words per thread while the planes of both fit in registers
        if (planes <= 8)
            rc = launch_k<8, 4>(a, p->sm_count, s);
        else if (planes <= 12)
            rc = launch_k<12, 4>(a, p->sm_count, s);
        else if (planes <= 16)
            rc = launch_k<16, 2>(a, p->sm_count, s);
        else if (planes <= 20)  // a weighted input costs 3 operations per plane
            rc = launch_k<20, 2>(a, p->sm_count, s);
        else if (planes <= 24)
            rc = launch_k<24, 2>(a, p->sm_count, s);
        else if (planes <= 28)
            rc = launch_k<28, 2>(a, p->sm_count, s);
        else
            rc = launch_k<32, 2>(a, p->sm_count, s);
    }
    int rc2 = stage_release(sl, s);
    return rc ? rc : rc2;
}
