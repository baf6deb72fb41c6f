// Threshold query for callers that cannot allocate device memory.
//
// The pool-based entry points stage each query's ids in device buffers that
// the pool allocates.  This entry point instead copies the ids into one
// fixed, file-scope device array and launches the same dense kernel on the
// caller's bitmaps, so a call never allocates.
#include <mutex>

#include "bm_device.cuh"

namespace {

// Scratch: the query's ids.  Every GPU that loads the library holds this
// array (64 KiB) until the process exits; all calls on a device share it.
static __device__ __align__(256) uint32_t g_noalloc_ids[BM_NOALLOC_MAX_N];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_ids_addr[kMaxDevices] = {};  // device address of the array, per device
int g_sm_count[kMaxDevices] = {};

// Once per device, with that device current: the array's device address.
// Host code must not use the symbol itself (it names a host-side stand-in).
int noalloc_setup(int dev, uint32_t** ids_addr, int* sm_count) {
    if (dev < 0 || dev >= kMaxDevices) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ids_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_ids);
        if (e != cudaSuccess || !p) {
            bm_note_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_ids)", __FILE__, __LINE__);
            return BM_ECUDA;
        }
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            bm_note_cuda_error(e, "cudaDeviceGetAttribute", __FILE__, __LINE__);
            return BM_ECUDA;
        }
        g_sm_count[dev] = sms > 0 ? sms : 1;
        g_ids_addr[dev] = static_cast<uint32_t*>(p);
    }
    *ids_addr = g_ids_addr[dev];
    *sm_count = g_sm_count[dev];
    return BM_OK;
}

}  // namespace

extern "C" int bm_threshold_noalloc(const uint64_t* words, uint64_t stride_words,
                                    uint32_t n_bitmaps, uint64_t r_bits, const uint32_t* ids,
                                    uint32_t n, uint32_t theta, uint64_t* out_words,
                                    uint64_t* out_card, void* stream) {
    if (!words || !ids || !out_words || n == 0 || r_bits == 0 || r_bits > (1ull << 32))
        return BM_EINVAL;
    if (n > BM_NOALLOC_MAX_N) return BM_EINVAL;  // beyond the fixed scratch array
    const uint64_t nwords = (r_bits + 63) / 64;
    // the kernel reads whole 16-byte slices of each bitmap
    if ((reinterpret_cast<uintptr_t>(words) & 15u) || (stride_words & 1u) ||
        stride_words < ((nwords + 1) & ~(uint64_t)1))
        return BM_EINVAL;
    for (uint32_t k = 0; k < n; ++k)
        if (ids[k] >= n_bitmaps) return BM_ERANGE;

    int dev = 0;
    BM_CUDA_TRY(cudaGetDevice(&dev));
    uint32_t* d_ids = nullptr;
    int sm_count = 1;
    int rc = noalloc_setup(dev, &d_ids, &sm_count);
    if (rc) return rc;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BM_CUDA_TRY(cudaMemcpyAsync(d_ids, ids, (size_t)n * 4, cudaMemcpyHostToDevice, s));
    if (out_card) BM_CUDA_TRY(cudaMemsetAsync(out_card, 0, 8, s));

    // T(theta): constant for theta = 0 (every row) and theta > n (no row),
    // otherwise one comparison count >= theta; built here without any
    // host or device allocation
    bm::Pred pred{};
    if (theta == 0 || theta > n) {
        pred.mode = 0;
        pred.v0 = theta == 0 ? 1u : 0u;
    } else {
        pred.mode = 1;
        pred.v0 = 0;
        pred.ntrans = 1;
        pred.trans[0] = theta;
    }
    bm::DenseArgs a{};
    a.base = words;
    a.stride_words = stride_words;
    a.words = nwords;
    a.r_bits = r_bits;
    a.ids = d_ids;
    a.n = n;
    a.pred = pred;
    a.out = out_words;
    a.card = reinterpret_cast<unsigned long long*>(out_card);
    a.err = nullptr;  // the direct-load kernel has no waits to report
    const bm::DenseConfig cfg{0, 256, 4, 2};
    const bm::LaunchExtra none{};  // ids in the fixed array; out_card zeroed above
    return bm::launch_dense(a, none, cfg, sm_count, s);
}
