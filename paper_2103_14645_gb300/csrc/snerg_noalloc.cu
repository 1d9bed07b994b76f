// snerg_noalloc.cu -- ray-list render that allocates nothing and needs no workspace.
//
// Some callers cannot allocate device memory: a plug-in living inside a host
// application that owns every byte of the GPU through its own pool (and forbids
// cudaMalloc), a real-time loop where the implicit device synchronisation of
// cudaMalloc/cudaFree would stall the frame, or a sandboxed caller granted only the
// buffers it was handed. snerg_render_rays_noalloc serves them: it renders straight from
// the caller's indirection grid and uint8 atlas (no padded copy, no voxel distance map),
// and keeps its only scratch -- a status word and the block-level empty-space distance
// map with its two transform temporaries -- in one file-scope __device__ array of fixed
// size that every GPU loading the library holds until the process exits.
//
// The array's host-side name is only a stand-in; its device address is fetched with
// cudaGetSymbolAddress once per device (with that device current) on the first call
// made on that device, so that first call should happen before any stream capture. The
// address is kept for the life of the process: a device reset (cudaDeviceReset, or a
// reset of the primary context) reloads the module and may move the array, after which
// the kept address is stale, so this entry point must not be used across a reset.
// Every call shares the array: calls whose work overlaps on the GPU (two streams, or two
// host threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "snerg_internal.cuh"

namespace snerg {
namespace {

constexpr int kNoAllocMaxG = 64;                               // N / B <= 64
constexpr size_t kNoAllocG3 = (size_t)kNoAllocMaxG * kNoAllocMaxG * kNoAllocMaxG;
constexpr size_t kNoAllocHeader = 256;                         // status word at byte 0
constexpr size_t kNoAllocBytes = kNoAllocHeader + 3 * kNoAllocG3;   // 786,688 bytes
constexpr int kNoAllocMaxDevices = 64;

// [0, 256): status word | bdist [G^3] | two G^3 temporaries of the distance transform
__device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mu;
void* g_scratch_dev[kNoAllocMaxDevices] = {};

// device address of g_noalloc_scratch on the current device (set up once per device)
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

// value of channel 0..7 of voxel (x, y, z) of the virtual grid, clamped to the grid;
// 0 in empty blocks (Sec. 5.1)
__device__ __forceinline__ uint2 raw_voxel(const DevScene& s, const uint2* atlas, int64_t nb, int x, int y, int z) {
    x = min(max(x, 0), s.N - 1);
    y = min(max(y, 0), s.N - 1);
    z = min(max(z, 0), s.N - 1);
    const int slot = __ldg(s.ind + (((z >> s.lgB) * s.G + (y >> s.lgB)) * s.G + (x >> s.lgB)));
    if (slot < 0 || slot >= nb) return make_uint2(0u, 0u);
    const int B = s.B;
    const int loc = ((z & (B - 1)) * B + (y & (B - 1))) * B + (x & (B - 1));
    return __ldg(atlas + (size_t)slot * B * B * B + loc);
}

// The march of snerg_internal.cuh on the caller's unpadded atlas: empty blocks are
// skipped through the block distance map, every lattice sample of an occupied block
// probes its nearest voxel's density code, and the 8 trilinear corners are fetched
// through the indirection grid. Same lattice, same binary32 control arithmetic (so the
// same composited samples and the same early exit), and the same colour accumulation
// (accumulate_colour).
__device__ __forceinline__ void march_raw(const DevScene& s, const uint2* atlas, int64_t nb, const Ray& r,
                                          MarchState& st) {
#pragma unroll
    for (int c = 0; c < 7; ++c) st.acc[c] = 0.0f;
    st.T = 1.0f;
    st.tau = 0.0f;
    st.steps = 0;
    st.active = 0;
    st.blocks = 0;
    st.limit = false;
    if (!r.hit) return;
    const int N = s.N, B = s.B;
    float inv_d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) inv_d[i] = __fdividef(1.0f, r.d[i]);
    const float kmax = (float)s.kmax;
    const float exit_m = exit_margin(r, s.fN);
    float k = 0.0f;
    for (;;) {
        if (k >= kmax) { st.limit = true; return; }
        const float t = lattice_t(r, k);
        if (!(t < r.t1)) return;
        int b[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) b[i] = nearest_voxel(lattice_u(r, t, i), N) >> s.lgB;
        const int bi = (b[2] * s.G + b[1]) * s.G + b[0];
        const int slot = __ldg(s.ind + bi);
        st.blocks++;
        if (slot < 0) {
            const int D1 = (int)s.bdist[bi] - 1;
            const int lo[3] = {b[0] - D1, b[1] - D1, b[2] - D1};
            const int hi[3] = {b[0] + D1, b[1] + D1, b[2] + D1};
            k = box_exit(r, inv_d, kmax, k, make_box(s, lo, hi), exit_m);
            continue;
        }
        const float kx = box_exit(r, inv_d, kmax, k, make_box(s, b, b), exit_m);
        if (slot >= nb) {                 // entry outside the atlas: reported, read as empty
            atomicCAS(s.status, 0, (int)SNERG_E_INVAL);
            k = kx;
            continue;
        }
        const uint8_t* blk = reinterpret_cast<const uint8_t*>(atlas + (size_t)slot * B * B * B);
        for (float kk = k; kk < kx; kk += 1.0f) {
            const float tk = lattice_t(r, kk);
            float u[3];
            int j[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                u[i] = lattice_u(r, tk, i);
                j[i] = nearest_voxel(u[i], N);
            }
            const int lx = min(max(j[0] - b[0] * B, 0), B - 1), ly = min(max(j[1] - b[1] * B, 0), B - 1),
                      lz = min(max(j[2] - b[2] * B, 0), B - 1);
            if (__ldg(blk + ((size_t)(lz * B + ly) * B + lx) * 8) == 0) continue;
            st.active++;
            float f[3], g[3], fl[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float x = __fsub_rn(u[i], 0.5f);
                fl[i] = floorf(x);
                f[i] = __fsub_rn(x, fl[i]);
                g[i] = __fsub_rn(1.0f, f[i]);
            }
            uint2 cv[8];   // index = z*4 + y*2 + x
#pragma unroll
            for (int c = 0; c < 8; ++c)
                cv[c] = raw_voxel(s, atlas, nb, (int)fl[0] + (c & 1), (int)fl[1] + ((c >> 1) & 1), (int)fl[2] + (c >> 2));
            const float e00 = __fadd_rn(__fmul_rn(code(cv[0].x, 0), g[0]), __fmul_rn(code(cv[1].x, 0), f[0]));
            const float e10 = __fadd_rn(__fmul_rn(code(cv[2].x, 0), g[0]), __fmul_rn(code(cv[3].x, 0), f[0]));
            const float e01 = __fadd_rn(__fmul_rn(code(cv[4].x, 0), g[0]), __fmul_rn(code(cv[5].x, 0), f[0]));
            const float e11 = __fadd_rn(__fmul_rn(code(cv[6].x, 0), g[0]), __fmul_rn(code(cv[7].x, 0), f[0]));
            const float e0 = __fadd_rn(__fmul_rn(e00, g[1]), __fmul_rn(e10, f[1]));
            const float e1 = __fadd_rn(__fmul_rn(e01, g[1]), __fmul_rn(e11, f[1]));
            const float sq = __fadd_rn(__fmul_rn(e0, g[2]), __fmul_rn(e1, f[2]));
            const float od = __fmul_rn(sq, s.kappa);
            st.tau = __fadd_rn(st.tau, od);
            const float e = expf(-od);
            const float wk = st.T * (1.0f - e);
            st.T *= e;
            accumulate_colour(st, cv, wk, f, g);
            if (st.tau > s.taumax) {
                st.steps += (int)(kk - k) + 1;
                return;
            }
        }
        st.steps += (int)(kx - k);
        k = kx;
    }
}

__global__ void __launch_bounds__(128, 8) render_rays_noalloc_kernel(const DevScene s, const uint2* __restrict__ atlas,
                                                                     int64_t nb,
                                                                     const __grid_constant__ CamTable cams, int32_t n_cams,
                                                                     const int32_t* __restrict__ pix, int64_t n,
                                                                     const float* __restrict__ mlp,
                                                                     float* __restrict__ rgb) {
    __shared__ __align__(16) float sW[kNParam + 1];
    __shared__ float sX[128 * kXStride];
    load_mlp_smem_t(sW, mlp);
    __syncthreads();
    float* xrow = sX + threadIdx.x * kXStride;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ci = __ldg(pix + 3 * i), px = __ldg(pix + 3 * i + 1), py = __ldg(pix + 3 * i + 2);
    Ray r;
    if (ci >= 0 && ci < n_cams && px >= 0 && py >= 0 && px < cams.c[ci].W && py < cams.c[ci].H) {
        r = make_ray(s, cams.c[ci], px, py);
    } else {
        r.hit = false;
        r.d[0] = r.d[1] = r.d[2] = 0.0f;
        atomicCAS(s.status, 0, (int)SNERG_E_INVAL);
    }
    MarchState st;
    march_raw(s, atlas, nb, r, st);
    record_status(s, st);
    float c[3], aux[kAuxCh];
    finish_ray(s, sW, xrow, r, st, c, aux);
    rgb[i * 3 + 0] = c[0];
    rgb[i * 3 + 1] = c[1];
    rgb[i * 3 + 2] = c[2];
}

bool desc_ok_noalloc(const snerg_scene_desc* d) {
    if (!d || d->N < 1 || d->N > 16384 || d->B < 2 || d->B > 64 || (d->B & (d->B - 1)) || d->N % d->B) return false;
    if (d->max_steps < 0 || (d->flags & ~SNERG_FLAG_UNPREMULTIPLY)) return false;   // deferred model only
    if (!(d->extent > 0.0f) || !(d->extent < INFINITY) || !(d->sigma_max >= 0.0f) || !(d->sigma_max < INFINITY))
        return false;
    for (int i = 0; i < 3; ++i)
        if (!(d->bmin[i] > -INFINITY && d->bmin[i] < INFINITY && d->bg[i] > -INFINITY && d->bg[i] < INFINITY))
            return false;
    return true;
}

}  // namespace
}  // namespace snerg

using namespace snerg;

extern "C" snerg_status snerg_render_rays_noalloc(const snerg_scene_desc* desc, const int32_t* d_indirection,
                                                  const uint8_t* d_atlas, int64_t num_blocks,
                                                  const snerg_camera* cams, int32_t n_cams, const int32_t* d_pix,
                                                  int64_t n, const float* d_mlp, float* d_rgb, int32_t* d_status,
                                                  void* stream) {
    if (!desc_ok_noalloc(desc) || num_blocks < 0 || n < 0) return SNERG_E_INVAL;
    const int N = desc->N, B = desc->B, G = N / B;
    if (G > kNoAllocMaxG) return SNERG_E_UNSUPPORTED;
    if (!cams || n_cams < 1 || n_cams > kMaxCams) return SNERG_E_INVAL;
    if (!d_indirection || (num_blocks > 0 && (!d_atlas || ((uintptr_t)d_atlas & 7u)))) return SNERG_E_INVAL;
    CamTable table;                      // on the stack: this entry point allocates nothing
    std::memset(&table, 0, sizeof(table));
    for (int i = 0; i < n_cams; ++i) {
        const snerg_camera& c = cams[i];
        for (int k = 0; k < 12; ++k)
            if (!(c.c2w[k] > -INFINITY && c.c2w[k] < INFINITY)) return SNERG_E_INVAL;
        if (!(c.fx > -INFINITY && c.fx < INFINITY && c.fy > -INFINITY && c.fy < INFINITY) || c.fx == 0.0f ||
            c.fy == 0.0f || !(c.cx > -INFINITY && c.cx < INFINITY && c.cy > -INFINITY && c.cy < INFINITY) ||
            c.W < 0 || c.H < 0)
            return SNERG_E_INVAL;
        table.c[i] = c;
    }
    if (n > 0 && (!d_pix || !d_mlp || !d_rgb)) return SNERG_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return SNERG_E_CUDA;
    uint8_t* scratch = (uint8_t*)base;
    int32_t* status = (int32_t*)scratch;
    uint8_t* bdist = scratch + kNoAllocHeader;
    const size_t G3 = (size_t)G * G * G;
    // the status word must start at zero; the distance map is rewritten in full
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = launch_block_distance(d_indirection, G, 32, bdist + kNoAllocG3, bdist + kNoAllocG3 + G3,
                                                    bdist, st);
    if (e == cudaSuccess && n > 0) {
        DevScene s;
        std::memset(&s, 0, sizeof(s));
        s.ind = d_indirection;
        s.bdist = bdist;
        s.status = status;
        s.N = N;
        s.B = B;
        int lg = 0;
        while ((1 << lg) < B) ++lg;
        s.lgB = lg;
        s.G = G;
        s.P = B + 2;
        s.P3 = s.P * s.P * s.P;
        s.fN = (float)N;
        s.scale = (float)N / desc->extent;
        for (int i = 0; i < 3; ++i) {
            s.bmin[i] = desc->bmin[i];
            s.bg[i] = desc->bg[i];
        }
        s.kappa = (float)((double)desc->sigma_max * ((double)desc->extent / (double)N) / 255.0);
        s.taumax = (float)std::log(1000.0);
        s.tmin = (float)1e-3;
        s.inv255 = (float)(1.0 / 255.0);
        s.flags = desc->flags;
        s.kmax = desc->max_steps > 0 ? (desc->max_steps < 4 * N + 16 ? desc->max_steps : 4 * N + 16) : 4 * N + 16;
        render_rays_noalloc_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
            s, reinterpret_cast<const uint2*>(d_atlas), num_blocks, table, n_cams, d_pix, n, d_mlp, d_rgb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && d_status) e = cudaMemcpyAsync(d_status, status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? SNERG_OK : SNERG_E_CUDA;
}
