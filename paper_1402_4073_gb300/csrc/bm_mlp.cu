// Kernels of the selector network F -> H -> H -> C (ReLU, fp32): forward,
// backward of the mean-squared-error loss, and the Adam update
// (Kingma and Ba 2015).  The network is tiny, so plain tiled CUDA-core
// kernels are used; there is no dense contraction large enough to need the
// tensor cores.
//
// Parameter buffer layout (fp32): W1 [F][H], b1 [H], W2 [H][H], b2 [H],
// W3 [H][C], b3 [C]; weights are [in][out] row-major.
#include <algorithm>

#include "bm_internal.cuh"
#include "bm_select.h"

namespace bm {
namespace {

constexpr int kT = 16;

// C[m][n] = act(sum_k A(m,k) B(k,n) + bias[n]) with A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn], C row-major with leading dimension ldc.
__global__ void __launch_bounds__(kT* kT) gemm_kernel(int M, int N, int K, const float* A, long sam,
                                                      long sak, const float* B, long sbk, long sbn,
                                                      float* C, long ldc, const float* bias,
                                                      int relu) {
    __shared__ float As[kT][kT + 1], Bs[kT][kT + 1];
    const int tx = threadIdx.x % kT, ty = threadIdx.x / kT;
    const int m = blockIdx.y * kT + ty, n = blockIdx.x * kT + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += kT) {
        const int ka = k0 + tx, kb = k0 + ty;
        const int am = blockIdx.y * kT + ty, bn = blockIdx.x * kT + tx;
        As[ty][tx] = (am < M && ka < K) ? A[am * sam + ka * sak] : 0.f;
        Bs[ty][tx] = (kb < K && bn < N) ? B[kb * sbk + bn * sbn] : 0.f;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kT; ++k) acc = fmaf(As[ty][k], Bs[k][tx], acc);
        __syncthreads();
    }
    if (m < M && n < N) {
        if (bias) acc += bias[n];
        if (relu) acc = acc > 0.f ? acc : 0.f;
        C[m * ldc + n] = acc;
    }
}

// dY = 2 (Y - T) / (B C); loss += sum (Y - T)^2 / (B C)
__global__ void mse_grad_kernel(const float* y, const float* t, float* dy, long count, float* loss) {
    const float scale = 1.f / (float)count;
    float part = 0.f;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        dy[i] = 2.f * d * scale;
        part += d * d * scale;
    }
    if (loss) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss, part);
    }
}

// dZ = dH * [H > 0] in place (H = ReLU(Z), so H > 0 exactly where Z > 0)
__global__ void relu_back_kernel(float* d, const float* h, long count) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long)gridDim.x * blockDim.x)
        if (!(h[i] > 0.f)) d[i] = 0.f;
}

// out[j] = sum_b D[b][j], one block per column
__global__ void __launch_bounds__(256) colsum_kernel(const float* D, int rows, int cols, float* out) {
    const int j = blockIdx.x;
    float s = 0.f;
    for (int b = threadIdx.x; b < rows; b += blockDim.x) s += D[(long)b * cols + j];
    __shared__ float part[256];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = part[0];
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, long count, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

int gemm(cudaStream_t s, int M, int N, int K, const float* A, long sam, long sak, const float* B,
         long sbk, long sbn, float* C, long ldc, const float* bias, int relu) {
    dim3 grid((N + kT - 1) / kT, (M + kT - 1) / kT);
    gemm_kernel<<<grid, kT * kT, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, relu);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

unsigned blocks_for(long count) {
    return (unsigned)std::max<long>(1, std::min<long>((count + 255) / 256, 4096));
}

struct Layout {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};
Layout layout(const float* P, int F, int H, int C) {
    Layout L;
    L.W1 = P;
    L.b1 = L.W1 + (long)F * H;
    L.W2 = L.b1 + H;
    L.b2 = L.W2 + (long)H * H;
    L.W3 = L.b2 + H;
    L.b3 = L.W3 + (long)H * C;
    return L;
}

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" {

int bm_mlp_forward(const float* params, uint32_t F, uint32_t H, uint32_t C, const float* x,
                   uint32_t batch, float* h1, float* h2, float* y, void* stream) {
    if (!params || !x || !h1 || !h2 || !y || !F || !H || !C || !batch) return BM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Layout L = layout(params, F, H, C);
    const int B = (int)batch;
    int rc = gemm(s, B, H, F, x, F, 1, L.W1, H, 1, h1, H, L.b1, 1);
    if (!rc) rc = gemm(s, B, H, H, h1, H, 1, L.W2, H, 1, h2, H, L.b2, 1);
    if (!rc) rc = gemm(s, B, C, H, h2, H, 1, L.W3, C, 1, y, C, L.b3, 0);
    return rc;
}

int bm_mlp_backward(const float* params, uint32_t F, uint32_t H, uint32_t C, const float* x,
                    const float* h1, const float* h2, const float* y, const float* target,
                    uint32_t batch, float* grads, float* workspace, float* loss, void* stream) {
    if (!params || !x || !h1 || !h2 || !y || !target || !grads || !workspace || !batch)
        return BM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Layout L = layout(params, F, H, C);
    float* gW1 = grads;
    float* gb1 = gW1 + (long)F * H;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + (long)H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + (long)H * C;
    const int B = (int)batch;
    float* dy = workspace;                    // B x C
    float* d2 = dy + (long)B * C;             // B x H
    float* d1 = d2 + (long)B * H;             // B x H
    if (loss) BM_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), s));
    const long ny = (long)B * C, nh = (long)B * H;
    mse_grad_kernel<<<blocks_for(ny), 256, 0, s>>>(y, target, dy, ny, loss);
    BM_CUDA_TRY(cudaGetLastError());
    // layer 3
    int rc = gemm(s, H, C, B, h2, 1, H, dy, C, 1, gW3, C, nullptr, 0);  // h2^T dy
    if (rc) return rc;
    colsum_kernel<<<C, 256, 0, s>>>(dy, B, C, gb3);
    rc = gemm(s, B, H, C, dy, C, 1, L.W3, 1, C, d2, H, nullptr, 0);  // dy W3^T
    if (rc) return rc;
    relu_back_kernel<<<blocks_for(nh), 256, 0, s>>>(d2, h2, nh);
    // layer 2
    rc = gemm(s, H, H, B, h1, 1, H, d2, H, 1, gW2, H, nullptr, 0);
    if (rc) return rc;
    colsum_kernel<<<H, 256, 0, s>>>(d2, B, H, gb2);
    rc = gemm(s, B, H, H, d2, H, 1, L.W2, 1, H, d1, H, nullptr, 0);
    if (rc) return rc;
    relu_back_kernel<<<blocks_for(nh), 256, 0, s>>>(d1, h1, nh);
    // layer 1
    rc = gemm(s, F, H, B, x, 1, F, d1, H, 1, gW1, H, nullptr, 0);
    if (rc) return rc;
    colsum_kernel<<<H, 256, 0, s>>>(d1, B, H, gb1);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

int bm_mlp_adam(float* params, const float* grads, float* m, float* v, uint64_t count,
                uint32_t step, float lr, float beta1, float beta2, float eps, void* stream) {
    if (!params || !grads || !m || !v || !count || !step) return BM_EINVAL;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<blocks_for((long)count), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        params, grads, m, v, (long)count, lr, beta1, beta2, eps, c1, c2);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

int bm_pool_set_selector(bm_pool* p, const float* params, uint64_t nparams, const float* mean,
                         const float* stdev, uint32_t n_out) {
    if (!p) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    if (!params) {
        p->sel_params.clear();
        p->sel_outputs = 0;
        return BM_OK;
    }
    if (!mean || !stdev || n_out != (uint32_t)kCandidates ||
        nparams != mlp_param_count(kFeatures, kHidden, kCandidates))
        return BM_EINVAL;
    for (int i = 0; i < kFeatures; ++i)
        if (!(stdev[i] > 0.f)) return BM_EINVAL;
    p->sel_params.assign(params, params + nparams);
    for (int i = 0; i < kFeatures; ++i) {
        p->sel_mean[i] = mean[i];
        p->sel_std[i] = stdev[i];
    }
    p->sel_outputs = (int)n_out;
    return BM_OK;
}

int bm_query_features(const bm_pool* p, const bm_query* q, float* out) {
    if (!p || !q || !out || !q->ids || q->n == 0 || q->n > BM_N_MAX) return BM_EINVAL;
    for (uint32_t k = 0; k < q->n; ++k)
        if (q->ids[k] >= p->capacity) return BM_ERANGE;
    std::vector<uint8_t> f;
    int rc = query_truth(q, f);
    if (rc) return rc;
    query_features(p, q->ids, q->n, f, out);
    return BM_OK;
}

int bm_query_select(const bm_pool* p, const bm_query* q, int32_t* path, uint32_t* tile_rows) {
    if (!p || !q || !path || !q->ids || q->n == 0 || q->n > BM_N_MAX) return BM_EINVAL;
    int rc = validate_ids(p, q->ids, q->n, BM_PATH_AUTO);
    if (rc) return rc;
    std::vector<uint8_t> f;
    rc = query_truth(q, f);
    if (rc) return rc;
    Candidate c = single_query_candidate(p, q->ids, q->n, f);
    *path = c.path;
    if (tile_rows)
        *tile_rows = c.path == BM_PATH_SPARSE ? (c.tile_rows ? c.tile_rows : p->sparse_cfg.tile_rows)
                                              : c.dense_words;
    return BM_OK;
}

}  // extern "C"
