// snerg_bake.cu -- baking an analytic radiance field into the sparse grid on the GPU
// (Sec. 5.3-5.4): alpha at voxel centres, macroblock culling at tau_alpha, packing of the
// kept blocks in raster order, and the anti-aliased content of each kept voxel (the field
// averaged over 16 Gaussian-jittered positions) stored as 8-bit codes.
//
// Three launches and one read-back:
//   alpha pass   persistent CTAs walk the macroblocks; each evaluates its block 256 voxel
//                centres at a time and stops at the first chunk holding alpha >= tau_alpha;
//   scan         one CTA of 1024 threads numbers the flagged blocks (exclusive scan in
//                raster order) into the indirection grid and a slot -> block list;
//   fill pass    persistent CTAs walk the kept voxels (slot-major, so the atlas stores of
//                a warp are one contiguous 256-byte run) and write 8 codes per voxel.
// Each unit of work (a block in the alpha pass, 256 voxels in the fill pass) first keeps
// only the density blobs that can matter over its box (jitter included): blob i is dropped
// where peak_i exp(-|x - c_i|^2 / (2 s_i^2)) < eps over the whole box, with
// eps = 2^-30 min(sigma_max, sigma_tau) and sigma_tau = -ln(1 - tau_alpha) / v the density
// at which alpha reaches tau_alpha. The dropped terms change sigma by less than
// 64 eps = 6e-8 of both the code step and the culling density.
// The colour channels use angle addition: the mean over the 16 samples of
// sin(a + b_s) with a = w . x_centre + phi and b_s = w . j_s v equals
// sin a * mean(cos b_s) + cos a * mean(sin b_s), and the two means depend only on the
// channel, so one sincos per voxel and channel replaces 16 sines.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "snerg.h"

namespace bake_gpu {

constexpr int kMaxBlobs = SNERG_BAKE_MAX_BLOBS;
constexpr int kThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kMaxG = 256;
constexpr size_t kAlign = 256;

struct BakeParams {
    int32_t N, B, lgB, G;
    int32_t n_blob;
    int32_t item_voxels;        // min(256, B^3)
    int32_t lg_items;           // log2(B^3 / item_voxels)
    int32_t alpha_codes;        // channel 0 = 1 - exp(-sigma v) instead of sigma / sigma_max
    float v, tau, inv_sigma_max;
    float bmin[3];
    float jit_lo[3], jit_hi[3]; // per-axis extremes of the jitter offsets (voxel units)
    float blob[kMaxBlobs][5];   // centre xyz, k = log2(e) / (2 s^2), peak
    float cull[kMaxBlobs];      // ln(peak / eps) / ln 2: the blob is dropped beyond this k |x - c|^2
    float color[7][4];          // w xyz, phi
    float cbar[7], sbar[7];     // mean over the samples of cos / sin (w_c . j_s v)
    float jv[16][3];            // jitter offsets times v (world units)
    float jq[16];               // |jv_s|^2
};

struct ItemBox {
    int32_t lo[3], hi[3];       // inclusive global voxel ranges of the item
};

// Voxel ranges covered by voxels [l0, l0 + iv) of block (bx, by, bz), local order
// z-major then y then x: a partial row, whole rows of one slice, or whole slices.
__device__ __forceinline__ ItemBox item_box(const BakeParams& P, int bx, int by, int bz, int l0) {
    const int B = P.B, m = B - 1, l1 = l0 + P.item_voxels - 1;
    const int x0 = l0 & m, y0 = (l0 >> P.lgB) & m, z0 = l0 >> (2 * P.lgB);
    const int x1 = l1 & m, y1 = (l1 >> P.lgB) & m, z1 = l1 >> (2 * P.lgB);
    ItemBox r;
    r.lo[2] = bz * B + z0;
    r.hi[2] = bz * B + z1;
    if (z0 == z1) {
        r.lo[1] = by * B + y0;
        r.hi[1] = by * B + y1;
        r.lo[0] = bx * B + (y0 == y1 ? x0 : 0);
        r.hi[0] = bx * B + (y0 == y1 ? x1 : m);
    } else {
        r.lo[1] = by * B;
        r.hi[1] = by * B + m;
        r.lo[0] = bx * B;
        r.hi[0] = bx * B + m;
    }
    return r;
}

// Threads 0..63 test one blob each against the item's box (voxel centres moved by the
// jitter extremes when `jittered`) and compact the blobs that may contribute into shared
// memory, in blob order. Returns their number after a barrier.
__device__ __forceinline__ int gather_blobs(const BakeParams& P, const ItemBox& box, bool jittered, float4* s_blob,
                                            float* s_peak, int* s_cnt) {
    const int t = threadIdx.x;
    bool rel = false;
    if (t < P.n_blob) {
        float a = 0.0f;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const float lo = P.bmin[ax] + ((float)box.lo[ax] + 0.5f + (jittered ? P.jit_lo[ax] : 0.0f)) * P.v;
            const float hi = P.bmin[ax] + ((float)box.hi[ax] + 0.5f + (jittered ? P.jit_hi[ax] : 0.0f)) * P.v;
            const float c = P.blob[t][ax];
            const float d = fmaxf(fmaxf(lo - c, c - hi), 0.0f);
            a = fmaf(d, d, a);
        }
        rel = a * P.blob[t][3] <= P.cull[t];
    }
    int pos = 0;
    if (t < 64) {
        const unsigned m = __ballot_sync(0xffffffffu, rel);
        pos = __popc(m & ((1u << (t & 31)) - 1u));
        if ((t & 31) == 0) s_cnt[t >> 5] = __popc(m);
    }
    __syncthreads();
    if (rel) {
        const int o = (t >= 32 ? s_cnt[0] : 0) + pos;
        s_blob[o] = make_float4(P.blob[t][0], P.blob[t][1], P.blob[t][2], P.blob[t][3]);
        s_peak[o] = P.blob[t][4];
    }
    __syncthreads();
    return s_cnt[0] + s_cnt[1];
}

// 2^x with the PTX approximate base-2 exponential (relative error about 2^-22 over the
// exponents used here, which are >= -cull > -64).
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float density_at(const float4* s_blob, const float* s_peak, int n, float x, float y,
                                            float z) {
    float acc = 0.0f;
    for (int i = 0; i < n; ++i) {
        const float4 b = s_blob[i];
        const float dx = x - b.x, dy = y - b.y, dz = z - b.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        acc = fmaf(s_peak[i], ex2(-d2 * b.w), acc);
    }
    return acc;
}

__device__ __forceinline__ uint32_t code8(float x) {
    const float q = floorf(fmaf(x, 255.0f, 0.5f));
    return q > 0.0f ? (q < 255.0f ? (uint32_t)q : 255u) : 0u;   // NaN -> 0
}

__global__ void __launch_bounds__(kThreads) bake_alpha_kernel(const __grid_constant__ BakeParams P,
                                                              int32_t* __restrict__ flags, int64_t G3) {
    __shared__ float4 s_blob[kMaxBlobs];
    __shared__ float s_peak[kMaxBlobs];
    __shared__ int s_cnt[2];
    const int t = threadIdx.x, m = P.B - 1;
    const int n_chunks = 1 << P.lg_items;
    for (int64_t b = blockIdx.x; b < G3; b += gridDim.x) {
        const int bx = (int)(b % P.G), by = (int)((b / P.G) % P.G), bz = (int)(b / ((int64_t)P.G * P.G));
        ItemBox box;
        box.lo[0] = bx * P.B;
        box.lo[1] = by * P.B;
        box.lo[2] = bz * P.B;
        box.hi[0] = box.lo[0] + m;
        box.hi[1] = box.lo[1] + m;
        box.hi[2] = box.lo[2] + m;
        __syncthreads();                                   // the previous block's readers are done
        const int n = gather_blobs(P, box, false, s_blob, s_peak, s_cnt);
        if (n == 0) continue;                              // uniform: alpha = 0 < tau everywhere
        for (int ch = 0; ch < n_chunks; ++ch) {
            bool keep = false;
            if (t < P.item_voxels) {
                const int l = ch * P.item_voxels + t;
                const float x = P.bmin[0] + ((float)(box.lo[0] + (l & m)) + 0.5f) * P.v;
                const float y = P.bmin[1] + ((float)(box.lo[1] + ((l >> P.lgB) & m)) + 0.5f) * P.v;
                const float z = P.bmin[2] + ((float)(box.lo[2] + (l >> (2 * P.lgB))) + 0.5f) * P.v;
                const float sigma = density_at(s_blob, s_peak, n, x, y, z);
                keep = -expm1f(-sigma * P.v) >= P.tau;   // alpha = 1 - exp(-sigma v)
            }
            if (__syncthreads_or(keep)) {
                if (t == 0) flags[b] = 1;
                break;                                     // uniform
            }
        }
    }
}

// Exclusive scan of the block flags in raster order (one CTA; thread t owns a contiguous
// chunk): ind[b] = slot or -1, list[slot] = b, *count = number of kept blocks.
__global__ void __launch_bounds__(kScanThreads) bake_scan_kernel(const int32_t* __restrict__ flags, int64_t G3,
                                                                 int32_t* __restrict__ ind,
                                                                 int32_t* __restrict__ list,
                                                                 int64_t* __restrict__ count) {
    __shared__ int s_warp[kScanThreads / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t per = (G3 + kScanThreads - 1) / kScanThreads;
    const int64_t lo = min(G3, (int64_t)t * per), hi = min(G3, lo + per);
    int c = 0;
    for (int64_t i = lo; i < hi; ++i) c += flags[i] != 0;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        int s = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += u;
        }
        s_warp[lane] = s;                                  // inclusive over warps
    }
    __syncthreads();
    int off = incl - c + (w > 0 ? s_warp[w - 1] : 0);
    for (int64_t i = lo; i < hi; ++i) {
        if (flags[i]) {
            ind[i] = off;
            list[off] = (int32_t)i;
            ++off;
        } else {
            ind[i] = -1;
        }
    }
    if (t == kScanThreads - 1) *count = off;
}

__global__ void __launch_bounds__(kThreads) bake_fill_kernel(const __grid_constant__ BakeParams P,
                                                             const int32_t* __restrict__ list,
                                                             const int64_t* __restrict__ count, int64_t max_blocks,
                                                             uint2* __restrict__ atlas) {
    __shared__ float4 s_blob[kMaxBlobs];
    __shared__ float s_peak[kMaxBlobs];
    __shared__ int s_cnt[2];
    const int t = threadIdx.x, m = P.B - 1;
    const int64_t nb = min(*count, max_blocks);
    const int64_t n_items = nb << P.lg_items;
    const int lg3 = 3 * P.lgB;
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int64_t slot = it >> P.lg_items;
        const int l0 = (int)(it & ((1 << P.lg_items) - 1)) * P.item_voxels;
        const int64_t b = list[slot];
        const int bx = (int)(b % P.G), by = (int)((b / P.G) % P.G), bz = (int)(b / ((int64_t)P.G * P.G));
        __syncthreads();
        const int n = gather_blobs(P, item_box(P, bx, by, bz, l0), true, s_blob, s_peak, s_cnt);
        if (t >= P.item_voxels) continue;
        const int l = l0 + t;
        const float fx = (float)(bx * P.B + (l & m)) + 0.5f;
        const float fy = (float)(by * P.B + ((l >> P.lgB) & m)) + 0.5f;
        const float fz = (float)(bz * P.B + (l >> (2 * P.lgB))) + 0.5f;
        const float cx = P.bmin[0] + fx * P.v, cy = P.bmin[1] + fy * P.v, cz = P.bmin[2] + fz * P.v;
        // sum over blobs of peak * sum over samples of 2^(-k |D + jv_s|^2), D = centre - c,
        // expanded as -k |D|^2 - 2k D . jv_s - k |jv_s|^2: four FMAs per blob and sample
        float sigma = 0.0f;
        for (int i = 0; i < n; ++i) {
            const float4 b = s_blob[i];
            const float dx = cx - b.x, dy = cy - b.y, dz = cz - b.z;
            const float a = -b.w * fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float gx = -2.0f * b.w * dx, gy = -2.0f * b.w * dy, gz = -2.0f * b.w * dz;
            float part = 0.0f;
#pragma unroll
            for (int s = 0; s < 16; ++s)
                part += ex2(fmaf(gx, P.jv[s][0], fmaf(gy, P.jv[s][1], fmaf(gz, P.jv[s][2], fmaf(-b.w, P.jq[s], a)))));
            sigma = fmaf(s_peak[i], part, sigma);
        }
        uint32_t q[8];
        q[0] = P.alpha_codes ? code8(-expm1f(-sigma * 0.0625f * P.v)) : code8(sigma * 0.0625f * P.inv_sigma_max);
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            const float a = fmaf(P.color[c][0], cx, fmaf(P.color[c][1], cy, fmaf(P.color[c][2], cz, P.color[c][3])));
            float sa, ca;
            sincosf(a, &sa, &ca);
            q[1 + c] = code8(fmaf(0.5f, fmaf(sa, P.cbar[c], ca * P.sbar[c]), 0.5f));
        }
        atlas[(slot << lg3) + l] = make_uint2(q[0] | q[1] << 8 | q[2] << 16 | q[3] << 24,
                                              q[4] | q[5] << 8 | q[6] << 16 | q[7] << 24);
    }
}

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int ilog2_exact(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return (1 << l) == v ? l : -1;
}

bool desc_ok(const snerg_scene_desc* d) {
    if (!d) return false;
    if (d->N < 1 || d->N > 16384) return false;
    if (d->B < 2 || d->B > 64 || ilog2_exact(d->B) < 0 || d->N % d->B != 0) return false;
    if (d->N / d->B > kMaxG) return false;
    if (!(std::isfinite(d->extent) && d->extent > 0.0f)) return false;
    if (!(std::isfinite(d->sigma_max) && d->sigma_max > 0.0f)) return false;
    return std::isfinite(d->bmin[0]) && std::isfinite(d->bmin[1]) && std::isfinite(d->bmin[2]);
}

bool field_ok(const snerg_bake_field* f) {
    if (!f || f->n_blob < 0 || f->n_blob > kMaxBlobs) return false;
    if (!(f->tau_alpha > 0.0f && f->tau_alpha < 1.0f)) return false;
    for (int i = 0; i < f->n_blob; ++i) {
        for (int k = 0; k < 5; ++k)
            if (!std::isfinite(f->blob[i][k])) return false;
        if (!(f->blob[i][3] > 0.0f) || !(f->blob[i][4] >= 0.0f)) return false;
    }
    for (int c = 0; c < 7; ++c)
        for (int k = 0; k < 4; ++k)
            if (!std::isfinite(f->color[c][k])) return false;
    for (int s = 0; s < 16; ++s)
        for (int k = 0; k < 3; ++k)
            if (!(std::fabs(f->jitter[s][k]) <= 8.0f)) return false;
    return true;
}

struct WsLayout {
    size_t count, flags, list, total;
};

WsLayout ws_layout(int64_t G3) {
    WsLayout L;
    L.count = 0;
    L.flags = kAlign;
    L.list = align_up(L.flags + (size_t)G3 * 4);
    L.total = align_up(L.list + (size_t)G3 * 4);
    return L;
}

int grid_for(const void* fn, int64_t items) {
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kThreads, 0);
    const int64_t g = (int64_t)sms * (per > 0 ? per : 1);
    return (int)(items < g ? (items > 0 ? items : 1) : g);
}

}  // namespace bake_gpu

using namespace bake_gpu;

extern "C" size_t snerg_bake_workspace_bytes(const snerg_scene_desc* desc) {
    if (!desc_ok(desc)) return 0;
    const int64_t G = desc->N / desc->B;
    return ws_layout(G * G * G).total;
}

extern "C" snerg_status snerg_bake(const snerg_scene_desc* desc, const snerg_bake_field* field,
                                   int32_t* d_indirection, uint8_t* d_atlas, int64_t max_blocks, void* d_workspace,
                                   size_t ws_bytes, int64_t* num_blocks, void* stream) {
    if (!desc_ok(desc) || !field_ok(field) || !d_indirection || !num_blocks || max_blocks < 0) return SNERG_E_INVAL;
    if (max_blocks > 0 && (!d_atlas || ((uintptr_t)d_atlas & 7u))) return SNERG_E_INVAL;
    if (!d_workspace || ((uintptr_t)d_workspace & (kAlign - 1))) return SNERG_E_INVAL;
    const int64_t G = desc->N / desc->B, G3 = G * G * G;
    const WsLayout L = ws_layout(G3);
    if (ws_bytes < L.total) return SNERG_E_NOMEM;
    *num_blocks = 0;

    BakeParams P;
    std::memset(&P, 0, sizeof(P));
    P.N = desc->N;
    P.B = desc->B;
    P.lgB = ilog2_exact(desc->B);
    P.G = (int32_t)G;
    P.n_blob = field->n_blob;
    const int B3 = desc->B * desc->B * desc->B;
    P.item_voxels = B3 < kThreads ? B3 : kThreads;
    P.alpha_codes = (desc->flags & SNERG_FLAG_ALPHA_ATLAS) ? 1 : 0;
    P.lg_items = ilog2_exact(B3 / P.item_voxels);
    const double v = (double)desc->extent / (double)desc->N;
    P.v = (float)v;
    P.tau = field->tau_alpha;
    P.inv_sigma_max = (float)(1.0 / (double)desc->sigma_max);
    for (int k = 0; k < 3; ++k) {
        P.bmin[k] = desc->bmin[k];
        float lo = field->jitter[0][k], hi = lo;
        for (int s = 1; s < 16; ++s) {
            lo = std::fmin(lo, field->jitter[s][k]);
            hi = std::fmax(hi, field->jitter[s][k]);
        }
        P.jit_lo[k] = lo;
        P.jit_hi[k] = hi;
    }
    const double sigma_tau = -std::log1p(-(double)field->tau_alpha) / v;
    const double eps = std::ldexp(std::fmin((double)desc->sigma_max, sigma_tau), -30);
    for (int i = 0; i < field->n_blob; ++i) {
        for (int k = 0; k < 3; ++k) P.blob[i][k] = field->blob[i][k];
        const double s = field->blob[i][3], peak = field->blob[i][4];
        P.blob[i][3] = (float)(1.0 / (2.0 * s * s * std::log(2.0)));
        P.blob[i][4] = (float)peak;
        P.cull[i] = peak > eps ? (float)(std::log(peak / eps) / std::log(2.0)) : -1.0f;
    }
    std::memcpy(P.color, field->color, sizeof(P.color));
    for (int j = 0; j < 16; ++j) {
        double q = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double o = (double)field->jitter[j][k] * v;
            P.jv[j][k] = (float)o;
            q += o * o;
        }
        P.jq[j] = (float)q;
    }
    for (int c = 0; c < 7; ++c) {
        double cs = 0.0, sn = 0.0;
        for (int s = 0; s < 16; ++s) {
            const double b = ((double)field->color[c][0] * field->jitter[s][0] +
                              (double)field->color[c][1] * field->jitter[s][1] +
                              (double)field->color[c][2] * field->jitter[s][2]) * v;
            cs += std::cos(b);
            sn += std::sin(b);
        }
        P.cbar[c] = (float)(cs / 16.0);
        P.sbar[c] = (float)(sn / 16.0);
    }

    cudaStream_t st = (cudaStream_t)stream;
    uint8_t* ws = (uint8_t*)d_workspace;
    int64_t* d_count = (int64_t*)(ws + L.count);
    int32_t* d_flags = (int32_t*)(ws + L.flags);
    int32_t* d_list = (int32_t*)(ws + L.list);
    cudaError_t e = cudaMemsetAsync(d_flags, 0, (size_t)G3 * 4, st);
    if (e == cudaSuccess) {
        bake_alpha_kernel<<<grid_for((const void*)bake_alpha_kernel, G3), kThreads, 0, st>>>(P, d_flags, G3);
        bake_scan_kernel<<<1, kScanThreads, 0, st>>>(d_flags, G3, d_indirection, d_list, d_count);
        e = cudaGetLastError();
    }
    int64_t count = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&count, d_count, sizeof(count), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return SNERG_E_CUDA;
    *num_blocks = count;
    if (count > max_blocks) return SNERG_E_NOMEM;
    if (count > 0) {
        bake_fill_kernel<<<grid_for((const void*)bake_fill_kernel, count << P.lg_items), kThreads, 0, st>>>(
            P, d_list, d_count, max_blocks, (uint2*)d_atlas);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return SNERG_E_CUDA;
    }
    return SNERG_OK;
}
