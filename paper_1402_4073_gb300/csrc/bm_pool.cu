// Device-resident bitmap pool: dense storage, position lists with a tile
// index, per-call staging of host arrays, device error word.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "bm_device.cuh"

void bm_note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    static std::atomic<int> reported{0};
    if (getenv("BM_DEBUG") || reported.fetch_add(1) < 8)
        fprintf(stderr, "[bm] CUDA error %s (%d) in %s at %s:%d\n", cudaGetErrorString(e), (int)e,
                what, file, line);
}

namespace bm {

int ensure_smem_limit(const void* fn, size_t bytes) {
    if (bytes <= 48 * 1024) return BM_OK;  // no opt-in needed
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> raised;
    int dev = 0;
    BM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t& have = raised[std::make_pair(fn, dev)];
    if (bytes <= have) return BM_OK;
    BM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    have = bytes;
    return BM_OK;
}

int smem_optin(int* bytes) {
    constexpr int kMaxDevices = 64;
    static std::atomic<int> cached[kMaxDevices];
    int dev = 0;
    BM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < kMaxDevices && (*bytes = cached[dev].load()) > 0) return BM_OK;
    BM_CUDA_TRY(cudaDeviceGetAttribute(bytes, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (dev >= 0 && dev < kMaxDevices) cached[dev].store(*bytes);
    return BM_OK;
}

int track_alloc(bm_pool* p, void** ptr, size_t bytes) {
    if (p->mem_budget && p->device_bytes + bytes > p->mem_budget) return BM_ENOMEM;
    if (cudaMalloc(ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return BM_ENOMEM;
    }
    p->device_bytes += bytes;
    return BM_OK;
}

void track_free(bm_pool* p, void* ptr, size_t bytes) {
    if (!ptr) return;
    cudaFree(ptr);
    p->device_bytes -= std::min<uint64_t>(p->device_bytes, bytes);
}

int stage_acquire(bm_pool* p, size_t bytes, bm_stage_slot** out, cudaStream_t s) {
    bm_stage_slot* sl = &p->slots[p->next_slot];
    p->next_slot = (p->next_slot + 1) % bm_pool::kSlots;
    if (sl->used) BM_CUDA_TRY(cudaEventSynchronize(sl->ev));  // previous call done with it
    sl->used = false;
    if (!sl->ev) BM_CUDA_TRY(cudaEventCreateWithFlags(&sl->ev, cudaEventDisableTiming));
    bytes = std::max<size_t>(bytes, 256);
    if (sl->cap < bytes) {
        size_t cap = std::max(bytes, sl->cap * 2);
        cap = ((cap + kStageHeader + 4095) & ~(size_t)4095) - kStageHeader;
        if (sl->h_base) cudaFreeHost(sl->h_base);
        track_free(p, sl->d_base, sl->cap + kStageHeader);
        sl->h = sl->d = sl->h_base = sl->d_base = nullptr;
        sl->cap = 0;
        if (cudaHostAlloc(&sl->h_base, cap + kStageHeader, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            sl->h_base = nullptr;
            return BM_ENOMEM;
        }
        int rc = track_alloc(p, &sl->d_base, cap + kStageHeader);
        if (rc) {
            cudaFreeHost(sl->h_base);
            sl->h_base = nullptr;
            return rc;
        }
        // the header starts at zero; every kernel that uses it leaves it so
        BM_CUDA_TRY(cudaMemsetAsync(sl->d_base, 0, kStageHeader, s));
        sl->h = static_cast<uint8_t*>(sl->h_base) + kStageHeader;
        sl->d = static_cast<uint8_t*>(sl->d_base) + kStageHeader;
        sl->cap = cap;
    }
    *out = sl;
    return BM_OK;
}

int stage_commit(bm_stage_slot* sl, size_t bytes, cudaStream_t s) {
    BM_CUDA_TRY(cudaMemcpyAsync(sl->d, sl->h, bytes, cudaMemcpyHostToDevice, s));
    return BM_OK;
}

int stage_release(bm_stage_slot* sl, cudaStream_t s) {
    BM_CUDA_TRY(cudaEventRecord(sl->ev, s));
    sl->used = true;
    return BM_OK;
}

namespace {

// Clear rows >= r in the last word of each loaded bitmap.
__global__ void mask_tail_kernel(uint64_t* base, uint64_t stride, uint64_t words, uint32_t first,
                                 uint32_t count, uint32_t tail) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < count) base[(uint64_t)(first + j) * stride + words - 1] &= (1ull << tail) - 1ull;
}

// Cardinality of each of `count` bitmaps, one CTA per bitmap.
__global__ void __launch_bounds__(256) pool_card_kernel(const uint64_t* base, uint64_t stride,
                                                        uint64_t words, uint32_t first,
                                                        unsigned long long* out) {
    const uint64_t* w = base + (uint64_t)(first + blockIdx.x) * stride;
    unsigned long long c = 0;
    for (uint64_t i = threadIdx.x; i < words; i += blockDim.x) c += __popcll(w[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    __shared__ unsigned long long part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < 8; ++i) t += part[i];
        out[blockIdx.x] = t;
    }
}

// Tile index of one list: idx[t] = first entry >= t * kListTileRows, for
// t = 0..tiles (binary search per entry).  One thread per entry.
__global__ void list_index_kernel(const uint32_t* pos, uint64_t len, uint32_t tiles,
                                  uint32_t* idx) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > tiles) return;
    const uint64_t key = (uint64_t)t * kListTileRows;
    uint64_t lo = 0, hi = len;
    while (lo < hi) {
        uint64_t mid = (lo + hi) / 2;
        if ((uint64_t)pos[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    idx[t] = (uint32_t)lo;
}

// Self-test of the bounded-wait path: wait on an mbarrier phase that nothing
// completes; the wait gives up after limit_ns and sets the error word.
__global__ void wait_selftest_kernel(int* err, unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar, 1);
        dev::fence_barrier_init();
        dev::mbar_wait_bounded(&bar, 0, err, limit_ns);  // no thread arrives: expires
    }
}

// Copy list j (src[src_off[j] .. src_off[j+1])) to dst + dst_off[j], a
// multiple of four entries, and fill its padding up to the next multiple of
// four with a value that no row tile holding the list's last position can
// contain (tiles are aligned and at most 65536 rows): all ones when the last
// position is below 65536, else 0.  A 16-byte vector read anywhere inside the
// padded list then holds only positions of that list or such padding.
__global__ void place_lists_kernel(const uint32_t* src, const uint64_t* src_off, uint32_t* dst,
                                   const uint64_t* dst_off, uint32_t count) {
    for (uint32_t j = blockIdx.x; j < count; j += gridDim.x) {
        const uint64_t s0 = src_off[j], len = src_off[j + 1] - s0;
        uint32_t* d = dst + dst_off[j];
        for (uint64_t i = threadIdx.x; i < len; i += blockDim.x) d[i] = src[s0 + i];
        const uint32_t pad = (uint32_t)((4 - (len & 3)) & 3);
        if (len && threadIdx.x < pad) {
            const uint32_t last = src[s0 + len - 1];
            d[len + threadIdx.x] = last < 65536u ? 0xFFFFFFFFu : 0u;
        }
    }
}

// Strict increase and range check of device-resident lists; sets *bad.
__global__ void list_check_kernel(const uint32_t* pos, uint64_t len, uint64_t r_bits, int* bad) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if ((uint64_t)pos[i] >= r_bits || (i > 0 && pos[i - 1] >= pos[i])) *bad = 1;
    }
}

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" {

const char* bm_strerror(int code) {
    switch (code) {
        case BM_OK: return "ok";
        case BM_EINVAL: return "invalid argument";
        case BM_ERANGE: return "id or position out of range, or bitmap not loaded";
        case BM_ENOMEM: return "out of memory or over the memory budget";
        case BM_ECUDA: return "CUDA runtime error";
        case BM_ETIMEOUT: return "a bounded device-side wait expired";
        case BM_EBUSY: return "admission refused";
        case BM_ENOTREADY: return "result not ready";
        default: return "unknown status";
    }
}

int bm_pool_create(int device, uint64_t r_bits, uint32_t capacity, uint64_t mem_budget,
                   bm_pool** out) {
    if (!out || r_bits == 0 || r_bits > (1ull << 32) || capacity == 0) return BM_EINVAL;
    *out = nullptr;
    BM_CUDA_TRY(cudaSetDevice(device));
    bm_pool* p = new bm_pool();
    p->device = device;
    p->r_bits = r_bits;
    p->words = (r_bits + 63) / 64;
    p->stride_words = (p->words + 31) & ~(uint64_t)31;
    p->capacity = capacity;
    p->mem_budget = mem_budget;
    cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, device);
    const size_t dense_bytes = (size_t)capacity * p->stride_words * 8;
    int rc = track_alloc(p, (void**)&p->d_dense, dense_bytes);
    if (!rc) rc = track_alloc(p, (void**)&p->d_err, sizeof(int));
    if (rc) {
        bm_pool_destroy(p);
        return rc;
    }
    if (cudaMemset(p->d_dense, 0, dense_bytes) != cudaSuccess ||
        cudaMemset(p->d_err, 0, sizeof(int)) != cudaSuccess) {
        bm_pool_destroy(p);
        return BM_ECUDA;
    }
    p->dense_present.assign(capacity, 0);
    p->card.assign(capacity, 0);
    p->list_begin.assign(capacity, 0);
    p->list_len.assign(capacity, 0);
    p->list_present.assign(capacity, 0);
    p->list_complement.assign(capacity, 0);
    p->tiles_per_list = (uint32_t)((r_bits + kListTileRows - 1) / kListTileRows);
    p->rle_tiles = (uint32_t)((p->words + kRleTileWords - 1) / kRleTileWords);
    p->rle_present.assign(capacity, 0);
    p->rle_runs.assign(capacity, 0);
    p->rle_lits.assign(capacity, 0);
    p->rle_units.assign(capacity, 0);
    *out = p;
    return BM_OK;
}

int bm_pool_destroy(bm_pool* p) {
    if (!p) return BM_OK;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    batch_state_free(p);
    for (auto& sl : p->slots) {
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.h_base) cudaFreeHost(sl.h_base);
        if (sl.d_base) cudaFree(sl.d_base);
    }
    if (p->d_dense) cudaFree(p->d_dense);
    if (p->d_err) cudaFree(p->d_err);
    if (p->d_pos) cudaFree(p->d_pos);
    if (p->d_tile_index) cudaFree(p->d_tile_index);
    if (p->d_list_begin) cudaFree(p->d_list_begin);
    for (void* q : {(void*)p->d_rle_arena, (void*)p->d_rle_tiles})
        if (q) cudaFree(q);
    delete p;
    return BM_OK;
}

int bm_pool_put_dense(bm_pool* p, uint32_t first_id, uint32_t count, const uint64_t* words,
                      uint64_t src_stride_words, int on_device) {
    if (!p || !words || count == 0) return BM_EINVAL;
    if ((uint64_t)first_id + count > p->capacity) return BM_ERANGE;
    if (src_stride_words < p->words) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    BM_CUDA_TRY(cudaSetDevice(p->device));
    BM_CUDA_TRY(cudaMemcpy2D(p->d_dense + (uint64_t)first_id * p->stride_words,
                             p->stride_words * 8, words, src_stride_words * 8, p->words * 8, count,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    const uint32_t tail = (uint32_t)(p->r_bits & 63u);
    if (tail) {
        mask_tail_kernel<<<(count + 255) / 256, 256>>>(p->d_dense, p->stride_words, p->words,
                                                       first_id, count, tail);
        BM_CUDA_TRY(cudaGetLastError());
    }
    unsigned long long* d_card = nullptr;
    int rc = track_alloc(p, (void**)&d_card, (size_t)count * 8);
    if (rc) return rc;
    pool_card_kernel<<<count, 256>>>(p->d_dense, p->stride_words, p->words, first_id, d_card);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpy(p->card.data() + first_id, d_card, (size_t)count * 8,
                       cudaMemcpyDeviceToHost);
    track_free(p, d_card, (size_t)count * 8);
    if (e != cudaSuccess) {
        bm_note_cuda_error(e, "put_dense cardinality", __FILE__, __LINE__);
        return BM_ECUDA;
    }
    for (uint32_t j = 0; j < count; ++j) p->dense_present[first_id + j] = 1;
    return BM_OK;
}

// Lists of ones (complement = false) or of zeros (complement = true): the
// arena placement, tile index and checks are the same; a list of zeros is
// marked by bit 63 of its device begin offset.
static int put_lists(bm_pool* p, uint32_t first_id, uint32_t count, const uint32_t* positions,
                     const uint64_t* offsets, int on_device, bool complement) {
    if (!p || !offsets || count == 0) return BM_EINVAL;
    if ((uint64_t)first_id + count > p->capacity) return BM_ERANGE;
    const uint64_t total = offsets[count] - offsets[0];
    for (uint32_t j = 0; j < count; ++j)
        if (offsets[j + 1] < offsets[j]) return BM_EINVAL;
    if (total && !positions) return BM_EINVAL;
    if (total > 0xFFFFFFFFull) return BM_EINVAL;  // tile index entries are 32-bit
    // every list starts on a 16-byte boundary and is padded to a multiple of
    // four entries (the sparse kernels read whole 16-byte vectors)
    std::vector<uint64_t> src_off(count + 1), dst_off(count);
    uint64_t padded = 0;
    for (uint32_t j = 0; j < count; ++j) {
        src_off[j] = offsets[j] - offsets[0];
        dst_off[j] = p->pos_used + padded;
        padded += (offsets[j + 1] - offsets[j] + 3) & ~3ull;
    }
    src_off[count] = total;
    // kernels address the arena with 32-bit entry offsets
    if (p->pos_used + padded > 0xFFFFFFFCull) return BM_ENOMEM;
    std::lock_guard<std::mutex> lk(p->mu);
    BM_CUDA_TRY(cudaSetDevice(p->device));
    if (!on_device) {
        for (uint32_t j = 0; j < count; ++j)
            for (uint64_t i = offsets[j]; i < offsets[j + 1]; ++i)
                if ((uint64_t)positions[i] >= p->r_bits ||
                    (i > offsets[j] && positions[i - 1] >= positions[i]))
                    return BM_ERANGE;
    }
    // grow the arena (lists are appended; a replaced list's old space is not reused)
    if (p->pos_used + padded > p->pos_cap) {
        uint64_t cap = std::max<uint64_t>(p->pos_used + padded, p->pos_cap + p->pos_cap / 2);
        cap = std::max<uint64_t>(cap, 1 << 20);
        cap = std::min<uint64_t>(cap, 0x100000000ull);
        uint32_t* nd = nullptr;
        int rc = track_alloc(p, (void**)&nd, cap * 4);
        if (rc) return rc;
        if (p->pos_used)
            BM_CUDA_TRY(cudaMemcpy(nd, p->d_pos, p->pos_used * 4, cudaMemcpyDeviceToDevice));
        track_free(p, p->d_pos, p->pos_cap * 4);
        p->d_pos = nd;
        p->pos_cap = cap;
    }
    if (!p->d_tile_index) {
        int rc = track_alloc(p, (void**)&p->d_tile_index,
                             (size_t)p->capacity * (p->tiles_per_list + 1) * 4);
        if (!rc) rc = track_alloc(p, (void**)&p->d_list_begin, (size_t)p->capacity * 8);
        if (rc) return rc;
        BM_CUDA_TRY(cudaMemset(p->d_tile_index, 0, (size_t)p->capacity * (p->tiles_per_list + 1) * 4));
        BM_CUDA_TRY(cudaMemset(p->d_list_begin, 0, (size_t)p->capacity * 8));
    }
    if (total) {
        // source lists on the device (the caller's, or a temporary copy of
        // the host's), then one placing launch into the arena
        const uint32_t* src = positions + offsets[0];
        uint32_t* tmp = nullptr;
        uint64_t* d_off = nullptr;
        const size_t off_bytes = (size_t)(2 * count + 1) * 8;
        int rc = track_alloc(p, (void**)&d_off, off_bytes);
        if (!rc && !on_device) rc = track_alloc(p, (void**)&tmp, total * 4);
        if (rc) {
            track_free(p, d_off, off_bytes);
            return rc;
        }
        cudaError_t e = cudaSuccess;
        if (!on_device) {
            e = cudaMemcpy(tmp, src, total * 4, cudaMemcpyHostToDevice);
            src = tmp;
        }
        if (e == cudaSuccess)
            e = cudaMemcpy(d_off, src_off.data(), (size_t)(count + 1) * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(d_off + count + 1, dst_off.data(), (size_t)count * 8,
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            place_lists_kernel<<<std::min<uint32_t>(count, 65535u), 256>>>(src, d_off, p->d_pos,
                                                                          d_off + count + 1, count);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        track_free(p, tmp, total * 4);
        track_free(p, d_off, off_bytes);
        if (e != cudaSuccess) {
            bm_note_cuda_error(e, "put_positions placement", __FILE__, __LINE__);
            return BM_ECUDA;
        }
    }
    if (on_device) {
        int* d_bad = nullptr;
        int rc = track_alloc(p, (void**)&d_bad, sizeof(int));
        if (rc) return rc;
        BM_CUDA_TRY(cudaMemset(d_bad, 0, sizeof(int)));
        for (uint32_t j = 0; j < count; ++j) {
            uint64_t len = offsets[j + 1] - offsets[j];
            if (!len) continue;
            uint64_t blocks = std::min<uint64_t>((len + 255) / 256, 4096);
            list_check_kernel<<<(unsigned)blocks, 256>>>(p->d_pos + dst_off[j], len, p->r_bits,
                                                         d_bad);
        }
        int bad = 0;
        cudaError_t e = cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
        track_free(p, d_bad, sizeof(int));
        if (e != cudaSuccess) return BM_ECUDA;
        if (bad) return BM_ERANGE;
    }
    for (uint32_t j = 0; j < count; ++j) {
        const uint64_t len = offsets[j + 1] - offsets[j];
        const uint64_t b = dst_off[j];
        uint32_t* idx = p->d_tile_index + (uint64_t)(first_id + j) * (p->tiles_per_list + 1);
        list_index_kernel<<<(p->tiles_per_list + 1 + 255) / 256, 256>>>(p->d_pos + b, len,
                                                                        p->tiles_per_list, idx);
        BM_CUDA_TRY(cudaGetLastError());
        p->list_begin[first_id + j] = b;
        p->list_len[first_id + j] = len;
        p->list_present[first_id + j] = 1;
        p->list_complement[first_id + j] = complement ? 1 : 0;
        if (!p->dense_present[first_id + j]) p->card[first_id + j] = complement ? p->r_bits - len : len;
        if (complement) dst_off[j] |= kListComplement;
    }
    BM_CUDA_TRY(cudaMemcpy(p->d_list_begin + first_id, dst_off.data(), (size_t)count * 8,
                           cudaMemcpyHostToDevice));
    BM_CUDA_TRY(cudaDeviceSynchronize());
    p->pos_used += padded;
    return BM_OK;
}

int bm_pool_put_positions(bm_pool* p, uint32_t first_id, uint32_t count, const uint32_t* positions,
                          const uint64_t* offsets, int on_device) {
    return put_lists(p, first_id, count, positions, offsets, on_device, false);
}

int bm_pool_put_complement_positions(bm_pool* p, uint32_t first_id, uint32_t count,
                                     const uint32_t* positions, const uint64_t* offsets,
                                     int on_device) {
    return put_lists(p, first_id, count, positions, offsets, on_device, true);
}

int bm_pool_info(const bm_pool* p, bm_pool_info_t* out) {
    if (!p || !out) return BM_EINVAL;
    out->r_bits = p->r_bits;
    out->words = p->words;
    out->stride_words = p->stride_words;
    out->capacity = p->capacity;
    out->dense_loaded = (uint32_t)std::count(p->dense_present.begin(), p->dense_present.end(), 1);
    out->lists_loaded = (uint32_t)std::count(p->list_present.begin(), p->list_present.end(), 1);
    out->rle_loaded = (uint32_t)std::count(p->rle_present.begin(), p->rle_present.end(), 1);
    out->reserved = 0;
    out->sm_count = (uint32_t)p->sm_count;
    out->device_bytes = p->device_bytes;
    out->dense_base = p->d_dense;
    return BM_OK;
}

int bm_pool_set_dense_config(bm_pool* p, const bm_dense_config_t* c) {
    if (!p || !c || c->variant < 0 || c->variant > 1 || c->ctas_per_sm < 1 || c->ctas_per_sm > 8)
        return BM_EINVAL;
    if (c->adder < 0 || c->adder > 2 || (c->variant == 1 && c->adder != 0)) return BM_EINVAL;
    if (c->adder == 2 && c->words_per_thread != 2) return BM_EINVAL;
    if ((c->words_per_thread != 1 && c->words_per_thread != 2) ||
        (c->variant == 1 && c->words_per_thread != 2))
        return BM_EINVAL;
    if (c->variant == 1 && (!(c->threads == 64 || c->threads == 128 || c->threads == 256) ||
                            c->stages < 2 ||
                            c->stages > 8))
        return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    p->dense_cfg = DenseConfig{c->variant, c->variant == 0 ? 256 : c->threads, c->stages,
                               c->ctas_per_sm, c->adder, c->words_per_thread};
    return BM_OK;
}

int bm_pool_get_dense_config(bm_pool* p, bm_dense_config_t* c) {
    if (!p || !c) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    c->variant = p->dense_cfg.variant;
    c->threads = p->dense_cfg.threads;
    c->stages = p->dense_cfg.stages;
    c->ctas_per_sm = p->dense_cfg.ctas_per_sm;
    c->adder = p->dense_cfg.adder;
    c->words_per_thread = p->dense_cfg.words_per_thread;
    return BM_OK;
}

int bm_pool_bitmap_cardinality(const bm_pool* p, uint32_t id, uint64_t* out) {
    if (!p || !out) return BM_EINVAL;
    if (id >= p->capacity || !(p->dense_present[id] || p->list_present[id])) return BM_ERANGE;
    *out = p->card[id];
    return BM_OK;
}

int bm_pool_status(bm_pool* p) {
    if (!p) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    BM_CUDA_TRY(cudaSetDevice(p->device));
    BM_CUDA_TRY(cudaDeviceSynchronize());
    int err = 0;
    BM_CUDA_TRY(cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        BM_CUDA_TRY(cudaMemset(p->d_err, 0, sizeof(int)));
        // a kernel that gave up may have left a cardinality header unfinished
        for (auto& sl : p->slots)
            if (sl.d_base) BM_CUDA_TRY(cudaMemset(sl.d_base, 0, kStageHeader));
        BM_CUDA_TRY(cudaDeviceSynchronize());
        return BM_ETIMEOUT;
    }
    return BM_OK;
}

int bm_pool_selftest_wait(bm_pool* p, uint32_t limit_us, void* stream) {
    if (!p || limit_us == 0 || limit_us > 2000000) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    BM_CUDA_TRY(cudaSetDevice(p->device));
    wait_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(
        p->d_err, (unsigned long long)limit_us * 1000ull);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

int bm_cardinality(const uint64_t* words, uint64_t r_bits, uint64_t* out_card, void* stream) {
    if (!words || !out_card) return BM_EINVAL;
    int dev = 0, sms = 0;
    BM_CUDA_TRY(cudaGetDevice(&dev));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return launch_cardinality(words, r_bits, reinterpret_cast<unsigned long long*>(out_card),
                              sms > 0 ? sms : 1, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
