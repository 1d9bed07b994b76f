// snerg_bwd.cu -- adjoint of the ray-list render (Sec. 5.5: the per-pixel network is
// fine-tuned against an L2 image loss, Eq. 3; the gradient here also reaches the baked
// colour and feature values, with density frozen).
//
// One thread per ray. The kernel marches the ray to get C_d, V, T and the MLP input
// (recording the lattice index and weight w_k of its first kRecCap composited samples),
// runs the MLP adjoint in registers, then scatters w_k * (trilinear weight) * dL/d(C_d, V)
// into the FP32 gradient atlas with vector atomics. Because density is frozen the
// composite weights w_k depend only on the samples before k, so the scatter walks the
// recorded samples in forward order and marches on from the last of them only for a
// ray that composited more. MLP weight gradients are
// summed over the CTA's rays from activations staged in shared memory and reach global
// memory with one atomic per parameter per CTA.
#include <atomic>

#include "snerg_internal.cuh"

namespace snerg {

// Per-thread shared-memory row (floats): x[34] | h1[16] | h2[16] | g1[16] | g2[16] | gz[3]
// (MLP input, hidden activations, their adjoints and the output adjoint). 101 is odd,
// so rows of neighbouring threads fall in different banks.
constexpr int kBwdThreads = 128;
constexpr int kRowX = 0, kRowH1 = 34, kRowH2 = 50, kRowG1 = 66, kRowG2 = 82, kRowGZ = 98, kRow = 101;
constexpr int kWFloats = 884;      // transposed weights (883) rounded up to a 16-byte multiple
constexpr int kMaxDevices = 64;     // devices whose shared-memory opt-in is remembered

size_t backward_smem_bytes() { return (size_t)(kWFloats + kBwdThreads * kRow) * sizeof(float); }

// A recorded sample's lattice position, block origin (minus one), block slot and weight.
struct RecSample {
    float u[3], w;
    int o3[3];
    int slot;
};

__device__ __forceinline__ void locate_recorded(const DevScene& s, const Ray& r, const int32_t* ind, float2 e,
                                                int& bprev, int& slot, RecSample& x) {
    const float t = lattice_t(r, e.x);
    int b[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        x.u[i] = lattice_u(r, t, i);
        b[i] = nearest_voxel(x.u[i], s.N) >> s.lgB;
        x.o3[i] = (b[i] << s.lgB) - 1;
    }
    const int bi = (b[2] * s.G + b[1]) * s.G + b[0];
    if (bi != bprev) {
        slot = __ldg(ind + bi);
        bprev = bi;
    }
    x.slot = slot;
    x.w = e.y;
}

// The adjoint scatter (march<..., GRAD>'s) of the n composited samples a march recorded
// (REC: each sample's lattice index and weight w_k), without the block entries and probes
// between them and without reloading their stencils: each sample's block and trilinear
// weights are recomputed from its lattice index as the march computed them, and w_k is
// the march's own. The next sample is located (its record and, on a block change, its
// slot loaded) before the current one's atomics, so that those loads overlap them. T and
// tau after the kRecCap-th sample (rec[kRecCap]) go to st for a march that continues from
// the next lattice index (CONT).
__device__ __forceinline__ void scatter_recorded(const DevScene& s, const Ray& r, const float2* rec, int n,
                                                 const float* gfeat, float* grad_atlas, MarchState& st) {
    if (n > 0) {
        const int oct = (r.d[0] < 0.0f ? 1 : 0) | (r.d[1] < 0.0f ? 2 : 0) | (r.d[2] < 0.0f ? 4 : 0);
        const int32_t* ind = s.ind + oct * s.ind_oct;
        int bprev = -1, slot = -1;
        RecSample cur, nxt;
        locate_recorded(s, r, ind, rec[0], bprev, slot, cur);
        float2 e = n > 1 ? rec[1] : make_float2(0.0f, 0.0f);
        for (int j = 0; j < n; ++j) {
            if (j + 1 < n) {
                locate_recorded(s, r, ind, e, bprev, slot, nxt);
                if (j + 2 < n) e = rec[j + 2];
            }
            // a block without samples is never recorded by a march
            if (cur.slot >= 0) {
                float f[3], g[3], fl[3];
                int fi[3];
                stencil_weights(cur.u, f, g, fl, fi);
                scatter_sample(s, cur.slot, fi, cur.o3, f, g, cur.w, gfeat, grad_atlas);
            }
            cur = nxt;
        }
    }
    if (n == kRecCap) {
        st.T = rec[kRecCap].x;
        st.tau = rec[kRecCap].y;
    }
}

// MLP forward keeping the activations h1, h2 in the row; returns the sigmoid residual.
__device__ __forceinline__ void mlp_forward_rows(const float* sW, float* row, float res[3]) {
    float h[16];
    load16(h, sW + kOffB1);
#pragma unroll 2
    for (int i = 0; i < kMlpIn; ++i) fma16(h, sW + kOffW1 + i * kMlpH, row[kRowX + i]);
#pragma unroll
    for (int o = 0; o < 16; ++o) {
        h[o] = fmaxf(h[o], 0.0f);
        row[kRowH1 + o] = h[o];
    }
    float h2[16];
    load16(h2, sW + kOffB2);
#pragma unroll
    for (int i = 0; i < kMlpH; ++i) fma16(h2, sW + kOffW2 + i * kMlpH, h[i]);
#pragma unroll
    for (int o = 0; o < 16; ++o) {
        h2[o] = fmaxf(h2[o], 0.0f);
        row[kRowH2 + o] = h2[o];
    }
#pragma unroll
    for (int o = 0; o < kMlpOut; ++o) {
        float acc = sW[kOffB3 + o];
#pragma unroll
        for (int i = 0; i < kMlpH; ++i) acc = fmaf(sW[kOffW3 + o * kMlpH + i], h2[i], acc);
        res[o] = 1.0f / (1.0f + expf(-acc));
    }
}

// Adjoint of the MLP for dL/dres = g, from the activations in the row and the residual:
// writes gz, g2, g1 into the row and returns dL/dx for the 7 composited inputs (C_d, V).
__device__ __forceinline__ void mlp_backward_rows(const float* sW, float* row, const float res[3], const float g[3],
                                                  float gx[7]) {
    float gz[3];
#pragma unroll
    for (int o = 0; o < kMlpOut; ++o) {
        gz[o] = g[o] * res[o] * (1.0f - res[o]);       // sigmoid'
        row[kRowGZ + o] = gz[o];
    }
    float g2[16];
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) {
        float acc = 0.0f;
#pragma unroll
        for (int o = 0; o < kMlpOut; ++o) acc = fmaf(sW[kOffW3 + o * kMlpH + k], gz[o], acc);
        g2[k] = row[kRowH2 + k] > 0.0f ? acc : 0.0f;  // ReLU'
        row[kRowG2 + k] = g2[k];
    }
    // g1 = W2^T g2 masked by ReLU', one hidden unit at a time (rolled: keeps the weight
    // loads from being hoisted into registers), written to the row
#pragma unroll 1
    for (int k = 0; k < kMlpH; ++k) {
        const float4* w = reinterpret_cast<const float4*>(sW + kOffW2 + k * kMlpH);   // W2^T[k][o] = W2[o][k]
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = w[q];
            acc = fmaf(v.x, g2[4 * q], acc);
            acc = fmaf(v.y, g2[4 * q + 1], acc);
            acc = fmaf(v.z, g2[4 * q + 2], acc);
            acc = fmaf(v.w, g2[4 * q + 3], acc);
        }
        row[kRowG1 + k] = row[kRowH1 + k] > 0.0f ? acc : 0.0f;
    }
    float g1[16];
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) g1[k] = row[kRowG1 + k];
#pragma unroll 1
    for (int k = 0; k < 7; ++k) {
        const float4* w = reinterpret_cast<const float4*>(sW + kOffW1 + k * kMlpH);   // W1^T[k][o] = W1[o][k]
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = w[q];
            acc = fmaf(v.x, g1[4 * q], acc);
            acc = fmaf(v.y, g1[4 * q + 1], acc);
            acc = fmaf(v.z, g1[4 * q + 2], acc);
            acc = fmaf(v.w, g1[4 * q + 3], acc);
        }
        gx[k] = acc;
    }
}

// MLP forward keeping activations, then its adjoint for dL/dres = g; writes h1, h2, g1,
// g2, gz into the row and returns dL/dx for the 7 composited inputs (C_d, V).
__device__ __forceinline__ void mlp_forward_backward(const float* sW, float* row, const float g[3], float gx[7]) {
    float res[3];
    mlp_forward_rows(sW, row, res);
    mlp_backward_rows(sW, row, res, g, gx);
}

// The MLP weight gradients of one CTA from its rows (after the CTA barrier): each weight
// matrix's gradient is a sum over the 128 rays of an outer product, computed in 4 x 4
// register tiles (8 shared-memory loads per ray for 16 products, against 32 for one
// product at a time): W1 (16 x 34) in 36 tiles, W2 (16 x 16) in 16, W3 (3 x 16) in 4;
// threads 56..90 sum one bias each. Every sum runs over the rays in the same order.
__device__ __forceinline__ void dphi_sums(const float* rows, float* grad_mlp) {
    const int t = threadIdx.x;
    if (t < 56) {
        int a0, b0, out, lda, na, nb;    // rows of the two factors, output offset and stride
        if (t < 36) {
            const int o0 = 4 * (t / 9), i0 = 4 * (t % 9);
            a0 = kRowG1 + o0; b0 = kRowX + i0; out = kOffW1 + o0 * kMlpIn + i0; lda = kMlpIn;
            na = 4; nb = min(4, kMlpIn - i0);
        } else if (t < 52) {
            const int o0 = 4 * ((t - 36) / 4), i0 = 4 * ((t - 36) % 4);
            a0 = kRowG2 + o0; b0 = kRowH1 + i0; out = kOffW2 + o0 * kMlpH + i0; lda = kMlpH;
            na = 4; nb = 4;
        } else {
            const int i0 = 4 * (t - 52);
            a0 = kRowGZ; b0 = kRowH2 + i0; out = kOffW3 + i0; lda = kMlpH;
            na = kMlpOut; nb = 4;
        }
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
#pragma unroll 2
        for (int r = 0; r < kBwdThreads; ++r) {
            const float* row = rows + r * kRow;
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = u < na ? row[a0 + u] : 0.0f;
#pragma unroll
            for (int v = 0; v < 4; ++v) b[v] = v < nb ? row[b0 + v] : 0.0f;
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v)
                if (u < na && v < nb && acc[u][v] != 0.0f) atomicAdd(grad_mlp + out + u * lda + v, acc[u][v]);
    } else if (t < 56 + kMlpH + kMlpH + kMlpOut) {
        const int j = t - 56;
        int a, p;
        if (j < kMlpH) { a = kRowG1 + j; p = kOffB1 + j; }
        else if (j < 2 * kMlpH) { a = kRowG2 + (j - kMlpH); p = kOffB2 + (j - kMlpH); }
        else { a = kRowGZ + (j - 2 * kMlpH); p = kOffB3 + (j - 2 * kMlpH); }
        float acc = 0.0f;
#pragma unroll 4
        for (int r = 0; r < kBwdThreads; ++r) acc += rows[r * kRow + a];
        if (acc != 0.0f) atomicAdd(grad_mlp + p, acc);
    }
}

// STATE: fwd_aux / fwd_counts hold the forward's per-ray outputs (C_d, V, opacity;
// steps, composited samples, indirection reads, first composited lattice index); the
// kernel then skips its own first march and scatters with one march from the first
// composited sample.
// TRAIN: one fine-tuning step for the ray in one pass (Sec. 5.5, Eq. 3): the march and the
// MLP give C, the L2 loss |C - C*|^2 is accumulated into *loss, dL/dC = 2 (C - C*) is taken
// in the kernel, and the adjoint follows as for a given upstream gradient; C goes to
// rgb_out (nullable). grad_rgb, fwd_aux and fwd_counts are not used.
template <bool TRAIN, bool STATE>
__global__ void __launch_bounds__(kBwdThreads, 4) backward_rays_kernel(
    const DevScene s, const __grid_constant__ CamTable cams, int32_t n_cams, const int32_t* __restrict__ pix,
    int64_t n, const float* __restrict__ mlp, const float* __restrict__ grad_rgb,
    const float* __restrict__ fwd_aux, const int32_t* __restrict__ fwd_counts, const float* __restrict__ target,
    float* __restrict__ rgb_out, float* __restrict__ loss, float* __restrict__ grad_atlas,
    float* __restrict__ grad_mlp) {
    extern __shared__ __align__(16) float smem[];
    __shared__ float s_loss[kBwdThreads / 32];
    float* sW = smem;
    float* rows = smem + kWFloats;
    load_mlp_smem_t(sW, mlp);
    __syncthreads();
    float* row = rows + threadIdx.x * kRow;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;

    Ray r;
    r.hit = false;
    r.d[0] = r.d[1] = r.d[2] = 0.0f;
    MarchState st;
    st.active = 0;
    st.T = 1.0f;
    int k_first = 0;
    float2 rec[kRecCap + 1];       // the first march's composited samples (index, w_k), then T, tau
    if (i < n) {
        const int ci = __ldg(pix + 3 * i), px = __ldg(pix + 3 * i + 1), py = __ldg(pix + 3 * i + 2);
        if (ci >= 0 && ci < n_cams && px >= 0 && py >= 0 && px < cams.c[ci].W && py < cams.c[ci].H)
            r = make_ray(s, cams.c[ci], px, py);
        else
            atomicCAS(s.status, 0, (int)SNERG_E_INVAL);
        if (STATE) {
            // the forward's per-ray state: C_d, V (decoded) and the first composited index
            st.active = r.hit ? __ldg(fwd_counts + 4 * i + 1) : 0;
            k_first = __ldg(fwd_counts + 4 * i + 3);
#pragma unroll
            for (int c = 0; c < 7; ++c) st.acc[c] = __ldg(fwd_aux + kAuxCh * i + c) * 255.0f;
        } else {
            march<false, false, false, true, true>(s, r, st, nullptr, 0, nullptr, nullptr, 0, &k_first, nullptr,
                                                   nullptr, rec);
            record_status(s, st);
        }
    }
    const bool active = st.active > 0;
    float g[3] = {0.0f, 0.0f, 0.0f};
    float gx[7];
    float sc = 1.0f;
    float l2 = 0.0f;                 // TRAIN: this ray's |C - C*|^2
    if (active) {
        const float inv255 = 1.0f / 255.0f;
        float cd[3], v[4];
        float T;
        if (STATE) {
#pragma unroll
            for (int c = 0; c < 3; ++c) cd[c] = __ldg(fwd_aux + kAuxCh * i + c);
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = __ldg(fwd_aux + kAuxCh * i + 3 + c);
            T = 1.0f - __ldg(fwd_aux + kAuxCh * i + 7);
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) cd[c] = st.acc[c] * inv255;
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = st.acc[3 + c] * inv255;
            T = st.T;
        }
        // App. C un-premultiply: a density-only (frozen) scale on C_d and V
        sc = unpremultiply_scale(s, T);
#pragma unroll
        for (int c = 0; c < 3; ++c) cd[c] *= sc;
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] *= sc;
        const bool no_mlp = (s.flags & SNERG_FLAG_NO_MLP) != 0;
        float res[3] = {0.0f, 0.0f, 0.0f};
        if (!no_mlp) {
            stage_mlp_input(row + kRowX, cd, v, r.d);
            if (TRAIN) mlp_forward_rows(sW, row, res);
        }
        if (TRAIN) {
            // C = s C_d + residual + T' bg (finish_ray's arithmetic), dL/dC = 2 (C - C*)
            const float Tb = (s.flags & SNERG_FLAG_UNPREMULTIPLY) ? 1.0f - (1.0f - T) * sc : T;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float C = cd[c] + res[c] + Tb * s.bg[c];
                const float d = C - __ldg(target + 3 * i + c);
                if (rgb_out) rgb_out[3 * i + c] = C;
                g[c] = 2.0f * d;
                l2 = fmaf(d, d, l2);
            }
        } else {
            g[0] = __ldg(grad_rgb + 3 * i);
            g[1] = __ldg(grad_rgb + 3 * i + 1);
            g[2] = __ldg(grad_rgb + 3 * i + 2);
        }
        if (no_mlp) {
            // C = s C_d + T bg: nothing reaches the network, and V reaches nothing
#pragma unroll
            for (int c = 0; c < 7; ++c) gx[c] = 0.0f;
            for (int k = 0; k < kRow; ++k) row[k] = 0.0f;
        } else if (TRAIN) {
            mlp_backward_rows(sW, row, res, g, gx);
        } else {
            mlp_forward_backward(sW, row, g, gx);
        }
    } else {
        for (int k = 0; k < kRow; ++k) row[k] = 0.0f;   // contributes nothing to the sums below
        if (TRAIN && i < n) {
            // nothing composited: C = T bg (T = 1 for a ray that composited nothing)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float C = st.T * s.bg[c];
                const float d = C - __ldg(target + 3 * i + c);
                if (rgb_out) rgb_out[3 * i + c] = C;
                l2 = fmaf(d, d, l2);
            }
        }
    }
    // the atlas scatter before the CTA's barrier: each ray's scatter follows its own first
    // march instead of waiting for the CTA's slowest one
    if (active && grad_atlas) {
        float gf[7];
#pragma unroll
        for (int c = 0; c < 3; ++c) gf[c] = sc * (g[c] + gx[c]);     // C = s C_d + residual
#pragma unroll
        for (int c = 0; c < 4; ++c) gf[3 + c] = sc * gx[3 + c];
        MarchState st2;
        if (!STATE) {
            scatter_recorded(s, r, rec, min(st.active, kRecCap), gf, grad_atlas, st2);
            // a ray with more composited samples marches on from the last recorded one
            if (st.active > kRecCap)
                march<false, true, false, true, false, true>(s, r, st2, nullptr, 0, gf, grad_atlas,
                                                             (int)rec[kRecCap - 1].x + 1);
        } else {
            // without a recording (the forward's per-ray state given) a second march starts
            // at the first composited sample: nothing before it contributes (T = 1 and
            // tau = 0 there), so its weights are the first pass's
            march<false, true, false, true>(s, r, st2, nullptr, 0, gf, grad_atlas, k_first);
        }
    }
    if (TRAIN && loss) {
        float v = l2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (TRAIN && loss && threadIdx.x == 0) {
        float v = 0.0f;
        for (int w = 0; w < kBwdThreads / 32; ++w) v += s_loss[w];
        atomicAdd(loss, v);
    }
    // dL/dPhi: sums over the CTA's rays of outer products (one global atomic per parameter
    // per CTA): W1 <- g1 (x) x, W2 <- g2 (x) h1, W3 <- gz (x) h2, biases <- g.
    if (grad_mlp) dphi_sums(rows, grad_mlp);
}

template <bool TRAIN, bool STATE>
static cudaError_t backward_launch(const DevScene& s, const CamTable& cams, int32_t n_cams, const int32_t* pix,
                                   int64_t n, const float* mlp, const float* grad_rgb, const float* fwd_aux,
                                   const int32_t* fwd_counts, const float* target, float* rgb_out, float* loss,
                                   float* grad_atlas, float* grad_mlp, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = backward_smem_bytes();
    // the opt-in for > 48 KB of dynamic shared memory, once per device
    static std::atomic<bool> attr_set[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!attr_set[dev].load()) {
        e = cudaFuncSetAttribute(backward_rays_kernel<TRAIN, STATE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        attr_set[dev].store(true);
    }
    const unsigned grid = (unsigned)((n + kBwdThreads - 1) / kBwdThreads);
    backward_rays_kernel<TRAIN, STATE><<<grid, kBwdThreads, smem, st>>>(s, cams, n_cams, pix, n, mlp, grad_rgb,
                                                                        fwd_aux, fwd_counts, target, rgb_out, loss,
                                                                        grad_atlas, grad_mlp);
    return cudaGetLastError();
}

cudaError_t launch_backward_rays(const DevScene& s, const CamTable& cams, int32_t n_cams, const int32_t* pix,
                                 int64_t n, const float* mlp, const float* grad_rgb, const float* fwd_aux,
                                 const int32_t* fwd_counts, float* grad_atlas, float* grad_mlp, cudaStream_t st) {
    if (fwd_aux)
        return backward_launch<false, true>(s, cams, n_cams, pix, n, mlp, grad_rgb, fwd_aux, fwd_counts, nullptr,
                                            nullptr, nullptr, grad_atlas, grad_mlp, st);
    return backward_launch<false, false>(s, cams, n_cams, pix, n, mlp, grad_rgb, nullptr, nullptr, nullptr, nullptr,
                                         nullptr, grad_atlas, grad_mlp, st);
}

cudaError_t launch_train_rays(const DevScene& s, const CamTable& cams, int32_t n_cams, const int32_t* pix, int64_t n,
                              const float* mlp, const float* target, float* rgb_out, float* loss, float* grad_atlas,
                              float* grad_mlp, cudaStream_t st) {
    return backward_launch<true, false>(s, cams, n_cams, pix, n, mlp, nullptr, nullptr, nullptr, target, rgb_out, loss,
                                 grad_atlas, grad_mlp, st);
}

}  // namespace snerg
