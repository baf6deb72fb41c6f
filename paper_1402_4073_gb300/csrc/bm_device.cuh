// Device building blocks: bit-sliced counter planes, predicates, bounded
// waits and bulk-copy (TMA) primitives, as inline PTX for sm_103a.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bm_internal.cuh"

namespace bm {
namespace dev {

// --- three-input logic in one LOP3 ---------------------------------------
// The immediate is the truth table over inputs (a, b, c) = (0xF0, 0xCC, 0xAA).
__device__ __forceinline__ uint32_t xor3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Full adder over 32 rows at once: a + b + c = lo + 2 * hi, per bit position
// (Sec. 4.3, "Adding": a full adder; here sum and carry are one LOP3 each).
__device__ __forceinline__ void csa(uint32_t& hi, uint32_t& lo, uint32_t a, uint32_t b,
                                    uint32_t c) {
    hi = maj3(a, b, c);
    lo = xor3(a, b, c);
}

// Counter planes P[0..K-1]: the count of a row is sum_j 2^j * bit of P[j].
// Add a carry of weight 2^j0 by ripple (half adders).
template <int K>
__device__ __forceinline__ void ripple(uint32_t (&P)[K], uint32_t c, int j0) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (j >= j0) {
            uint32_t t = P[j] & c;
            P[j] ^= c;
            c = t;
        }
    }
}

// Add one input word (weight 1).
template <int K>
__device__ __forceinline__ void add1(uint32_t (&P)[K], uint32_t x) {
    ripple<K>(P, x, 0);
}

// Add two input words: one full adder into plane 0, carry rippled from 1.
template <int K>
__device__ __forceinline__ void add2(uint32_t (&P)[K], uint32_t x0, uint32_t x1) {
    uint32_t c;
    csa(c, P[0], P[0], x0, x1);
    ripple<K>(P, c, 1);
}

// Add sixteen input words with a sideways-sum tree of full adders
// (Sec. 4.3, "Sideways Sum"): planes 0..3 act as carry-save accumulators,
// 15 full adders per 16 inputs, and the single weight-16 carry is rippled
// into planes 4.. .  Requires K >= 5.
// The sixteen-input tree of add16 without its last ripple: returns the
// weight-16 carry.
template <int K>
__device__ __forceinline__ uint32_t add16_carry(uint32_t (&P)[K], const uint32_t (&x)[16]) {
    uint32_t twosA, twosB, foursA, foursB, eightsA, eightsB, sixteens;
    csa(twosA, P[0], P[0], x[0], x[1]);
    csa(twosB, P[0], P[0], x[2], x[3]);
    csa(foursA, P[1], P[1], twosA, twosB);
    csa(twosA, P[0], P[0], x[4], x[5]);
    csa(twosB, P[0], P[0], x[6], x[7]);
    csa(foursB, P[1], P[1], twosA, twosB);
    csa(eightsA, P[2], P[2], foursA, foursB);
    csa(twosA, P[0], P[0], x[8], x[9]);
    csa(twosB, P[0], P[0], x[10], x[11]);
    csa(foursA, P[1], P[1], twosA, twosB);
    csa(twosA, P[0], P[0], x[12], x[13]);
    csa(twosB, P[0], P[0], x[14], x[15]);
    csa(foursB, P[1], P[1], twosA, twosB);
    csa(eightsB, P[2], P[2], foursA, foursB);
    csa(sixteens, P[3], P[3], eightsA, eightsB);
    return sixteens;
}

// Thirty-two inputs as two sixteen-input trees whose weight-16 carries meet
// plane 4 in one more full adder; only the weight-32 carry ripples, into
// planes 5.. .  Requires K >= 6.
template <int K>
__device__ __forceinline__ void add32_join(uint32_t (&P)[K], uint32_t s16a, uint32_t s16b) {
    uint32_t t32;
    csa(t32, P[4], P[4], s16a, s16b);
    ripple<K>(P, t32, 5);
}

template <int K>
__device__ __forceinline__ void add16(uint32_t (&P)[K], const uint32_t (&x)[16]) {
    uint32_t twosA, twosB, foursA, foursB, eightsA, eightsB, sixteens;
    csa(twosA, P[0], P[0], x[0], x[1]);
    csa(twosB, P[0], P[0], x[2], x[3]);
    csa(foursA, P[1], P[1], twosA, twosB);
    csa(twosA, P[0], P[0], x[4], x[5]);
    csa(twosB, P[0], P[0], x[6], x[7]);
    csa(foursB, P[1], P[1], twosA, twosB);
    csa(eightsA, P[2], P[2], foursA, foursB);
    csa(twosA, P[0], P[0], x[8], x[9]);
    csa(twosB, P[0], P[0], x[10], x[11]);
    csa(foursA, P[1], P[1], twosA, twosB);
    csa(twosA, P[0], P[0], x[12], x[13]);
    csa(twosB, P[0], P[0], x[14], x[15]);
    csa(foursB, P[1], P[1], twosA, twosB);
    csa(eightsB, P[2], P[2], foursA, foursB);
    csa(sixteens, P[3], P[3], eightsA, eightsB);
    ripple<K>(P, sixteens, 4);
}

// Add eight input words: 7 full adders with planes 0..2 as carry-save
// accumulators, the weight-8 carry rippled into planes 3.. .  Requires K >= 4.
template <int K>
__device__ __forceinline__ void add8(uint32_t (&P)[K], const uint32_t (&x)[8]) {
    uint32_t twosA, twosB, foursA, foursB, eights;
    csa(twosA, P[0], P[0], x[0], x[1]);
    csa(twosB, P[0], P[0], x[2], x[3]);
    csa(foursA, P[1], P[1], twosA, twosB);
    csa(twosA, P[0], P[0], x[4], x[5]);
    csa(twosB, P[0], P[0], x[6], x[7]);
    csa(foursB, P[1], P[1], twosA, twosB);
    csa(eights, P[2], P[2], foursA, foursB);
    ripple<K>(P, eights, 3);
}

// [count > a] for each of 32 rows, a < 2^K (Sec. 4.3 comparator against a
// constant, with the constant's bits read at run time; they are the same
// in every thread, so the branches are uniform): scanning bits from the top,
// a 1 in a narrows the prefix match, a 0 in a admits rows whose matched
// prefix carries a 1 there.
template <int K>
__device__ __forceinline__ uint32_t greater_than(const uint32_t (&P)[K], uint32_t a) {
    uint32_t gt = 0u, pm = 0xFFFFFFFFu;
#pragma unroll
    for (int j = K - 1; j >= 0; --j) {
        if ((a >> j) & 1u)
            pm &= P[j];
        else
            gt |= pm & P[j];
    }
    return gt;
}

// Evaluate a compiled predicate on 32 rows.  `tab` is the mode-2 truth table
// in shared memory.
template <int K>
__device__ __forceinline__ uint32_t eval_pred(const uint32_t (&P)[K], const Pred& pr,
                                              const uint32_t* tab) {
    if (pr.mode == 0) return pr.v0 ? 0xFFFFFFFFu : 0u;
    if (pr.mode == 1) {
        uint32_t r = pr.v0 ? 0xFFFFFFFFu : 0u;
#pragma unroll
        for (int i = 0; i < kMaxTransitions; ++i)
            if ((uint32_t)i < pr.ntrans) r ^= greater_than<K>(P, pr.trans[i] - 1u);
        return r;
    }
    // mode 2: rebuild each row's count from the planes and look f up
    uint32_t r = 0;
#pragma unroll 4
    for (int b = 0; b < 32; ++b) {
        uint32_t c = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) c |= ((P[j] >> b) & 1u) << j;
        r |= ((tab[c >> 5] >> (c & 31u)) & 1u) << b;
    }
    return r;
}

// --- ids and cardinality of a single-query launch ---------------------------

// The ids of the launch: a query of at most kInlineIds inputs carries them in
// the parameter block, and each CTA copies them to `s_ids` (the caller
// synchronises the block before reading them); otherwise the staged device
// copy.  Reads through the returned pointer are generic loads.
__device__ __forceinline__ const uint32_t* launch_ids(const uint32_t* ids, const LaunchExtra& x,
                                                      uint32_t* s_ids) {
    if (x.n_inline == 0) return ids;
    for (uint32_t i = threadIdx.x; i < x.n_inline; i += blockDim.x) s_ids[i] = x.inl[i];
    return s_ids;
}

// One contributor's part of the cardinality.  With acc null the part is
// added to *out (zeroed by the caller).  Otherwise the part is added to *acc
// and an arrival counted on *ticket; the last of `contributors` arrivals
// (fences order every part before it) stores the total to *out and returns
// acc and ticket to zero for the next launch that uses them, so *out needs no
// clearing beforehand and the launch needs no separate memset.
__device__ __forceinline__ void card_contribute(unsigned long long part, unsigned long long* out,
                                                unsigned long long* acc, unsigned int* ticket,
                                                uint32_t contributors) {
    if (!acc) {
        if (out && part) atomicAdd(out, part);
        return;
    }
    if (part) atomicAdd(acc, part);
    __threadfence();
    if (atomicAdd(ticket, 1u) == contributors - 1u) {
        __threadfence();
        const unsigned long long total = atomicExch(acc, 0ull);
        atomicExch(ticket, 0u);
        if (out) *out = total;
    }
}

// Block-wide sum of every thread's count, then one contribution per CTA
// (contributors = the grid's CTAs).  Every thread of the block calls it.
__device__ __forceinline__ void flush_card_block(unsigned long long card, unsigned long long* out,
                                                 unsigned long long* acc, unsigned int* ticket) {
    __shared__ unsigned long long s_part[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) card += __shfl_xor_sync(0xFFFFFFFFu, card, o);
    const uint32_t warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) s_part[warp] = card;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (uint32_t w = 0; w < nwarps; ++w) t += s_part[w];
        card_contribute(t, out, acc, ticket, gridDim.x);
    }
}

// --- time, loads ------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bytes of dynamic shared memory this launch was given.
__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
    uint32_t r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

// Streaming 128-bit load that bypasses L1 allocation.
__device__ __forceinline__ uint4 ld_stream(const void* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// --- mbarrier and bulk copies (sm_90+) ---------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of parity `parity` to complete; give up after
// kWaitLimitNs, set the error word and return false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (uint32_t spin = 1;; ++spin) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((spin & 63u) == 0 && globaltimer() - t0 > limit_ns) {
            if (err) atomicOr(err, kErrTimeout);
            return false;
        }
    }
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// Global -> shared bulk copy (TMA, non-tensor form) completing on `bar`.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

// Global -> shared copy of 8 bytes by one thread (cp.async, generic proxy);
// the thread's copies since the last commit form one group.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
// Wait until at most N of the thread's groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Sum of a per-thread value over the warp.
__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
    return __reduce_add_sync(0xFFFFFFFFu, v);
}

}  // namespace dev
}  // namespace bm
