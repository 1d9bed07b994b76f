// snerg_bwd.cu -- adjoint of the ray-list render (Sec. 5.5: the per-pixel network is
// fine-tuned against an L2 image loss, Eq. 3; the gradient here also reaches the baked
// colour and feature values, with density frozen).
//
// One thread per ray. Nothing of the forward march is stored: the kernel re-marches
// the ray to get C_d, V, T and the MLP input, runs the MLP adjoint in registers, then
// marches the ray a second time and scatters w_k * (trilinear weight) * dL/d(C_d, V)
// into the FP32 gradient atlas with vector atomics. Because density is frozen the
// composite weights w_k depend only on the samples before k, so the second pass walks
// the ray in forward order and needs no per-sample state. MLP weight gradients are
// summed across the warp with shuffles, across the CTA in shared memory, and reach
// global memory with one atomic per parameter per CTA.
#include "snerg_internal.cuh"

namespace snerg {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void acc_param(float* sG, int idx, float v, int lane) {
    v = warp_sum(v);
    if (lane == 0 && v != 0.0f) atomicAdd(sG + idx, v);
}

__global__ void __launch_bounds__(128) backward_rays_kernel(const DevScene s, const __grid_constant__ CamTable cams,
                                                            int32_t n_cams, const int32_t* __restrict__ pix,
                                                            int64_t n, const float* __restrict__ mlp,
                                                            const float* __restrict__ grad_rgb,
                                                            float* __restrict__ grad_atlas,
                                                            float* __restrict__ grad_mlp) {
    __shared__ float sW[kNParam];
    __shared__ float sG[kNParam];
    load_mlp_smem(sW, mlp);
    for (int p = threadIdx.x; p < kNParam; p += blockDim.x) sG[p] = 0.0f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;

    Ray r;
    r.hit = false;
    r.d[0] = r.d[1] = r.d[2] = 0.0f;
    MarchState st;
    st.active = 0;
    if (i < n) {
        const int ci = __ldg(pix + 3 * i), px = __ldg(pix + 3 * i + 1), py = __ldg(pix + 3 * i + 2);
        if (ci >= 0 && ci < n_cams && px >= 0 && py >= 0 && px < cams.c[ci].W && py < cams.c[ci].H)
            r = make_ray(s, cams.c[ci], px, py);
        else
            atomicCAS(s.status, 0, (int)SNERG_E_INVAL);
        march<false, false>(s, r, st, nullptr, 0, nullptr, nullptr);
        record_status(s, st);
    }
    const bool active = st.active > 0;

    // forward MLP with the activations kept for the adjoint
    float x[kMlpIn];
    MlpAct a;
    float g[3] = {0.0f, 0.0f, 0.0f};
    if (active) {
        const float inv255 = 1.0f / 255.0f;
        float cd[3] = {st.acc[0] * inv255, st.acc[1] * inv255, st.acc[2] * inv255};
        float v[4] = {st.acc[3] * inv255, st.acc[4] * inv255, st.acc[5] * inv255, st.acc[6] * inv255};
        mlp_input(cd, v, r.d, x);
        mlp_forward(sW, x, a);
        g[0] = __ldg(grad_rgb + 3 * i);
        g[1] = __ldg(grad_rgb + 3 * i + 1);
        g[2] = __ldg(grad_rgb + 3 * i + 2);
    } else {
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) x[k] = 0.0f;
#pragma unroll
        for (int k = 0; k < kMlpH; ++k) a.h1[k] = a.h2[k] = 0.0f;
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) a.res[k] = 0.0f;
    }
    // adjoint: sigmoid, layer 3, ReLU, layer 2, ReLU, layer 1
    float gz[kMlpOut], gh2[kMlpH], gh1[kMlpH], gx[kMlpIn];
#pragma unroll
    for (int o = 0; o < kMlpOut; ++o) gz[o] = g[o] * a.res[o] * (1.0f - a.res[o]);
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) {
        float acc = 0.0f;
#pragma unroll
        for (int o = 0; o < kMlpOut; ++o) acc = fmaf(sW[kOffW3 + o * kMlpH + k], gz[o], acc);
        gh2[k] = a.h2[k] > 0.0f ? acc : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) {
        float acc = 0.0f;
#pragma unroll
        for (int o = 0; o < kMlpH; ++o) acc = fmaf(sW[kOffW2 + o * kMlpH + k], gh2[o], acc);
        gh1[k] = a.h1[k] > 0.0f ? acc : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) {
        float acc = 0.0f;
#pragma unroll
        for (int o = 0; o < kMlpH; ++o) acc = fmaf(sW[kOffW1 + o * kMlpIn + k], gh1[o], acc);
        gx[k] = acc;
    }
    if (grad_mlp) {
#pragma unroll
        for (int o = 0; o < kMlpOut; ++o) {
            acc_param(sG, kOffB3 + o, gz[o], lane);
#pragma unroll
            for (int k = 0; k < kMlpH; ++k) acc_param(sG, kOffW3 + o * kMlpH + k, gz[o] * a.h2[k], lane);
        }
#pragma unroll
        for (int o = 0; o < kMlpH; ++o) {
            acc_param(sG, kOffB2 + o, gh2[o], lane);
#pragma unroll
            for (int k = 0; k < kMlpH; ++k) acc_param(sG, kOffW2 + o * kMlpH + k, gh2[o] * a.h1[k], lane);
        }
#pragma unroll
        for (int o = 0; o < kMlpH; ++o) {
            acc_param(sG, kOffB1 + o, gh1[o], lane);
#pragma unroll
            for (int k = 0; k < kMlpIn; ++k) acc_param(sG, kOffW1 + o * kMlpIn + k, gh1[o] * x[k], lane);
        }
    }
    __syncthreads();
    if (grad_mlp)
        for (int p = threadIdx.x; p < kNParam; p += blockDim.x)
            if (sG[p] != 0.0f) atomicAdd(grad_mlp + p, sG[p]);

    if (active && grad_atlas) {
        float gf[7];
#pragma unroll
        for (int c = 0; c < 3; ++c) gf[c] = g[c] + gx[c];     // C = C_d + residual
#pragma unroll
        for (int c = 0; c < 4; ++c) gf[3 + c] = gx[3 + c];
        MarchState st2;
        march<false, true>(s, r, st2, nullptr, 0, gf, grad_atlas);
    }
}

cudaError_t launch_backward_rays(const DevScene& s, const CamTable& cams, int32_t n_cams, const int32_t* pix,
                                 int64_t n, const float* mlp, const float* grad_rgb, float* grad_atlas,
                                 float* grad_mlp, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((n + 127) / 128);
    backward_rays_kernel<<<grid, 128, 0, st>>>(s, cams, n_cams, pix, n, mlp, grad_rgb, grad_atlas, grad_mlp);
    return cudaGetLastError();
}

}  // namespace snerg
