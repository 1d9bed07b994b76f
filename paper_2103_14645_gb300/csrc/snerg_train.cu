// snerg_train.cu -- the two element-wise steps of the fine-tuning loop of Sec. 5.5 that
// are not the render: the photometric loss of Eq. 3 with its gradient, and an Adam
// update (the paper fine-tunes the view-dependence network with Adam, learning rate
// 3e-4). Together with snerg_render_rays / snerg_render_backward a whole training step
// runs in this library's kernels.
#include <cmath>

#include "snerg_internal.cuh"

namespace snerg {

// L = sum_i |C_i - C*_i|^2 (Eq. 3): g_i = 2 (C_i - C*_i); the loss is reduced per CTA
// (warp shuffles, then shared memory) and added to *loss with one atomic per CTA.
__global__ void __launch_bounds__(256) l2_loss_kernel(const float* __restrict__ rgb, const float* __restrict__ target,
                                                      int64_t n3, float* __restrict__ grad,
                                                      float* __restrict__ loss) {
    __shared__ float part[8];
    float acc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = rgb[i] - target[i];
        if (grad) grad[i] = 2.0f * d;
        acc = fmaf(d, d, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && loss) atomicAdd(loss, v);
    }
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
__global__ void __launch_bounds__(256) adam_kernel(float* __restrict__ p, float* __restrict__ m,
                                                   float* __restrict__ v, const float* __restrict__ g, int64_t n,
                                                   float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

static unsigned grid_1d(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace snerg

using namespace snerg;

extern "C" snerg_status snerg_l2_loss(const float* d_rgb, const float* d_target, int64_t n, float* d_grad,
                                      float* d_loss, void* stream) {
    if (n < 0 || (n > 0 && (!d_rgb || !d_target))) return SNERG_E_INVAL;
    if (n == 0) return SNERG_OK;
    l2_loss_kernel<<<grid_1d(3 * n), 256, 0, (cudaStream_t)stream>>>(d_rgb, d_target, 3 * n, d_grad, d_loss);
    return cudaGetLastError() == cudaSuccess ? SNERG_OK : SNERG_E_CUDA;
}

extern "C" snerg_status snerg_adam_step(float* d_param, float* d_m, float* d_v, const float* d_grad, int64_t n,
                                        float lr, float beta1, float beta2, float eps, int32_t step, void* stream) {
    if (n < 0 || step < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
        !(eps > 0.0f))
        return SNERG_E_INVAL;
    if (n == 0) return SNERG_OK;
    if (!d_param || !d_m || !d_v || !d_grad) return SNERG_E_INVAL;
    const float c1 = (float)(1.0 - std::pow((double)beta1, (double)step));
    const float c2 = (float)(1.0 - std::pow((double)beta2, (double)step));
    adam_kernel<<<grid_1d(n), 256, 0, (cudaStream_t)stream>>>(d_param, d_m, d_v, d_grad, n, lr, beta1, beta2, eps,
                                                              c1, c2);
    return cudaGetLastError() == cudaSuccess ? SNERG_OK : SNERG_E_CUDA;
}
