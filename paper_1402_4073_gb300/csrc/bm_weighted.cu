// Weighted threshold queries with an optional combining step, over the dense
// pool: row i is selected iff the sum of weights[k] over the inputs k holding
// row i reaches theta (Sec. 2.3 treats a weight as that many copies of an
// input; here a weight costs one read of the input whatever its size), and
// the result may then be ANDed, ORed or AND-NOTed with one more bitmap of the
// pool in the same pass (the result of a threshold is again a bitmap, Sec. 1).
//
// GPU form: a thread owns a column of one or two 64-bit words and keeps K
// counter planes (the bits of the weighted sum of its rows) in registers.  Inputs of
// weight 1 go through the sixteen-input sideways-sum blocks of the dense
// kernel.  An input of weight w > 1 is added once per set bit j of w, at plane
// j, by rippling its word upwards (half adders); the warp stops a ripple as
// soon as no lane carries.  When the weights are small (their sum at most 8
// per input and within BM_N_MAX) they are expanded into copies instead, which
// the sideways-sum blocks add faster than ripples.  The predicate is the
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

// Add word c at plane j (weight 2^j) and ripple the carries upwards; the warp
// leaves as soon as no lane carries.  j is the same in every lane.
template <int K>
__device__ __forceinline__ void add_at(uint32_t (&P)[K], uint32_t c, uint32_t j) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
        if ((uint32_t)i >= j) {
            const uint32_t t = P[i] & c;
            P[i] ^= c;
            c = t;
            if ((i & 1) && !__any_sync(0xFFFFFFFFu, c != 0u)) break;
        }
    }
}

// L = 4: a thread owns two 64-bit words (128 rows, 16-byte loads); L = 2: one.
template <int K, int L>
__global__ void __launch_bounds__(256) weighted_kernel(WeightedArgs a) {
    constexpr uint32_t W = L / 2;  // words per thread
    const uint64_t ncols = (a.words + W - 1) / W;
    for (uint64_t col = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;; col += (uint64_t)gridDim.x * blockDim.x) {
        // the whole warp stays in the loop while any lane has a column (ripples vote)
        if (!__any_sync(0xFFFFFFFFu, col < ncols)) break;
        const bool mine = col < ncols;
        const uint64_t c = mine ? col : ncols - 1;  // idle lanes reread a valid column
        const uint64_t w0 = W * c;                  // first word of the column
        uint32_t P[L][K];
        zero_planes<K, L>(P);
        count_column<K, 16, L>(P, a.base + w0, a.ids1, a.n1, a.stride_words);
        // weighted inputs, the next one's word in flight while this one ripples
        Slice<L> x_next;
        if (a.nw) x_next = ld_slice<L>(a.base + (uint64_t)__ldg(a.idsw) * a.stride_words + w0);
        for (uint32_t k = 0; k < a.nw; ++k) {
            const Slice<L> x = x_next;
            uint32_t w = __ldg(a.wts + k);
            if (k + 1 < a.nw)
                x_next = ld_slice<L>(a.base + (uint64_t)__ldg(a.idsw + k + 1) * a.stride_words + w0);
            while (w) {
                const uint32_t j = __ffs(w) - 1;
                w &= w - 1;
#pragma unroll
                for (int l = 0; l < L; ++l) add_at<K>(P[l], x.v[l], j);
            }
        }
        unsigned long long ones = 0;
#pragma unroll
        for (uint32_t i = 0; i < W; ++i) {
            const uint64_t wi = w0 + i;
            uint64_t word = a.all ? ~0ull
                                  : ((uint64_t)greater_than<K>(P[2 * i], (uint32_t)(a.theta - 1)) |
                                     ((uint64_t)greater_than<K>(P[2 * i + 1], (uint32_t)(a.theta - 1)) << 32));
            if (wi < a.words) {
                if (a.post_op) {
                    const uint64_t m = __ldg(a.post + wi);
                    word = a.post_op == BM_POST_AND ? (word & m)
                         : a.post_op == BM_POST_OR  ? (word | m)
                                                    : (word & ~m);
                }
                if (wi == a.words - 1 && (a.r_bits & 63u)) word &= (1ull << (a.r_bits & 63u)) - 1ull;
                if (mine) {
                    a.out[wi] = word;
                    ones += (unsigned long long)__popcll(word);
                }
            }
        }
        flush_card(ones, a.card);
    }
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
    rc = stage_acquire(p, b1 + 2 * bw + 16, &sl);
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
        else if (planes <= 24)
            rc = launch_k<24, 2>(a, p->sm_count, s);
        else
            rc = launch_k<32, 2>(a, p->sm_count, s);
    }
    int rc2 = stage_release(sl, s);
    return rc ? rc : rc2;
}
