// snerg_train.cu -- the two element-wise steps of the fine-tuning loop of Sec. 5.5 that
// are not the render: the photometric loss of Eq. 3 with its gradient, and an Adam
// update (the paper fine-tunes the view-dependence network with Adam, learning rate
// 3e-4). Together with snerg_render_rays / snerg_render_backward a whole training step
// runs in this library's kernels.
#include <cmath>
#include <cstdint>

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

// Data-parallel fine-tuning exchanges the atlas gradient only over the macroblocks some
// rank touched: a per-block "any non-zero" mask, then the touched blocks gathered into a
// packed buffer for the all-reduce and scattered back.
__global__ void __launch_bounds__(256) block_touched_kernel(const float4* __restrict__ g, int64_t nb, int32_t bf4,
                                                            int32_t* __restrict__ mask) {
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        bool nz = false;
        for (int32_t i = threadIdx.x; i < bf4; i += blockDim.x) {
            const float4 v = g[b * bf4 + i];
            nz |= (v.x != 0.0f) | (v.y != 0.0f) | (v.z != 0.0f) | (v.w != 0.0f);
        }
        const int any = __syncthreads_or(nz);
        if (threadIdx.x == 0) mask[b] = any ? 1 : 0;
    }
}

// dst[i] = src[list[i]] (gather) or dst[list[i]] = src[i] (scatter), bf4 float4 per block
template <bool GATHER>
__global__ void __launch_bounds__(256) block_copy_kernel(const float4* __restrict__ src,
                                                         const int32_t* __restrict__ list, int64_t n, int32_t bf4,
                                                         float4* __restrict__ dst) {
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t b = list[i];
        const float4* s = src + (GATHER ? b : i) * bf4;
        float4* d = dst + (GATHER ? i : b) * bf4;
        for (int32_t j = threadIdx.x; j < bf4; j += blockDim.x) d[j] = s[j];
    }
}

// The same update four parameters at a time (16-byte loads and stores) for the bulk of a
// large parameter array.
__global__ void __launch_bounds__(256) adam4_kernel(float4* __restrict__ p, float4* __restrict__ m,
                                                    float4* __restrict__ v, const float4* __restrict__ g, int64_t n4,
                                                    float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 gi = g[i];
        float4 mi = m[i], vi = v[i], pi = p[i];
        const float ga[4] = {gi.x, gi.y, gi.z, gi.w};
        float ma[4] = {mi.x, mi.y, mi.z, mi.w}, va[4] = {vi.x, vi.y, vi.z, vi.w}, pa[4] = {pi.x, pi.y, pi.z, pi.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ma[k] = b1 * ma[k] + (1.0f - b1) * ga[k];
            va[k] = b2 * va[k] + (1.0f - b2) * ga[k] * ga[k];
            pa[k] -= lr * (ma[k] / c1) / (sqrtf(va[k] / c2) + eps);
        }
        m[i] = make_float4(ma[0], ma[1], ma[2], ma[3]);
        v[i] = make_float4(va[0], va[1], va[2], va[3]);
        p[i] = make_float4(pa[0], pa[1], pa[2], pa[3]);
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
    cudaStream_t st = (cudaStream_t)stream;
    const bool aligned = (((uintptr_t)d_param | (uintptr_t)d_m | (uintptr_t)d_v | (uintptr_t)d_grad) & 15u) == 0;
    int64_t done = 0;
    if (aligned && n >= 4096) {
        const int64_t n4 = n / 4;
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t want = (n4 + 255) / 256, cap = (int64_t)sms * 8;
        adam4_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(
            reinterpret_cast<float4*>(d_param), reinterpret_cast<float4*>(d_m), reinterpret_cast<float4*>(d_v),
            reinterpret_cast<const float4*>(d_grad), n4, lr, beta1, beta2, eps, c1, c2);
        done = n4 * 4;
    }
    if (done < n)
        adam_kernel<<<grid_1d(n - done), 256, 0, st>>>(d_param + done, d_m + done, d_v + done, d_grad + done,
                                                       n - done, lr, beta1, beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? SNERG_OK : SNERG_E_CUDA;
}

static bool block_args_ok(const void* a, const void* b, int64_t n, int32_t block_floats) {
    if (n < 0 || block_floats <= 0 || (block_floats & 3)) return false;
    if (n > 0 && (!a || !b || ((uintptr_t)a & 15u) || ((uintptr_t)b & 15u))) return false;
    return true;
}

static unsigned grid_blocks(int64_t n) { return (unsigned)(n < 65535 ? (n > 0 ? n : 1) : 65535); }

extern "C" snerg_status snerg_grad_blocks_touched(const float* d_grad, int64_t num_blocks, int32_t block_floats,
                                                  int32_t* d_mask, void* stream) {
    if (!block_args_ok(d_grad, d_mask, num_blocks, block_floats)) return SNERG_E_INVAL;
    if (num_blocks == 0) return SNERG_OK;
    block_touched_kernel<<<grid_blocks(num_blocks), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(d_grad), num_blocks, block_floats / 4, d_mask);
    return cudaGetLastError() == cudaSuccess ? SNERG_OK : SNERG_E_CUDA;
}

extern "C" snerg_status snerg_grad_blocks_gather(const float* d_grad, const int32_t* d_list, int64_t n,
                                                 int32_t block_floats, float* d_packed, void* stream) {
    if (!block_args_ok(d_grad, d_packed, n, block_floats) || (n > 0 && !d_list)) return SNERG_E_INVAL;
    if (n == 0) return SNERG_OK;
    block_copy_kernel<true><<<grid_blocks(n), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(d_grad), d_list, n, block_floats / 4, reinterpret_cast<float4*>(d_packed));
    return cudaGetLastError() == cudaSuccess ? SNERG_OK : SNERG_E_CUDA;
}

extern "C" snerg_status snerg_grad_blocks_scatter(const float* d_packed, const int32_t* d_list, int64_t n,
                                                  int32_t block_floats, float* d_grad, void* stream) {
    if (!block_args_ok(d_packed, d_grad, n, block_floats) || (n > 0 && !d_list)) return SNERG_E_INVAL;
    if (n == 0) return SNERG_OK;
    block_copy_kernel<false><<<grid_blocks(n), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(d_packed), d_list, n, block_floats / 4, reinterpret_cast<float4*>(d_grad));
    return cudaGetLastError() == cudaSuccess ? SNERG_OK : SNERG_E_CUDA;
}
