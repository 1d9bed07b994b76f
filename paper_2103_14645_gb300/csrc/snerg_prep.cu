// snerg_prep.cu -- scene set-up kernels: validate the indirection grid (Sec. 5.1) and
// build the device layout of the atlas (apron-padded blocks + a split density plane).
//
// The paper's viewer keeps density in its own 8-bit texture so that empty space inside
// occupied blocks costs one byte per sample (App. A); the density plane here plays that
// role. The 1-voxel apron makes every trilinear stencil of a sample a fetch from one
// block: atlas neighbours are not spatial neighbours (Sec. 5.1), so without it a sample
// near a block face would need up to 8 indirection lookups.
#include "snerg_internal.cuh"

namespace snerg {

// err bit 1: entry outside [-1, nb); bit 2: a slot referenced twice.
__global__ void validate_kernel(const int32_t* __restrict__ ind, int64_t n_ind, int64_t nb,
                                int32_t* __restrict__ blk_of_slot, int32_t* __restrict__ err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_ind; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = ind[i];
        if (v < -1 || (int64_t)v >= nb) {
            atomicOr(err, 1);
        } else if (v >= 0) {
            if (atomicCAS(blk_of_slot + v, -1, (int32_t)i) != -1) atomicOr(err, 2);
        }
    }
}

// One thread per padded voxel. Padded coordinate p in [0, B+2) maps to the global voxel
// block_origin + p - 1, clamped to the grid (clamp-to-edge at the border); its owner
// block supplies the value, or 0 if that block is empty.
__global__ void build_padded_kernel(const int32_t* __restrict__ ind, const int32_t* __restrict__ blk_of_slot,
                                    const uint2* __restrict__ atlas, int64_t nb, int N, int B, int lgB,
                                    uint8_t* __restrict__ pdens, uint2* __restrict__ patlas) {
    const int P = B + 2, P3 = P * P * P, G = N >> lgB;
    const int64_t total = nb * (int64_t)P3;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = t / P3;
        const int r = (int)(t - slot * P3);
        const int px = r % P, py = (r / P) % P, pz = r / (P * P);
        const int blk = blk_of_slot[slot];
        uint2 v = make_uint2(0u, 0u);
        if (blk >= 0) {
            const int bx = blk % G, by = (blk / G) % G, bz = blk / (G * G);
            const int gx = min(max(bx * B + px - 1, 0), N - 1);
            const int gy = min(max(by * B + py - 1, 0), N - 1);
            const int gz = min(max(bz * B + pz - 1, 0), N - 1);
            const int owner = ind[((gz >> lgB) * G + (gy >> lgB)) * G + (gx >> lgB)];
            if (owner >= 0) {
                const int loc = ((gz & (B - 1)) * B + (gy & (B - 1))) * B + (gx & (B - 1));
                v = atlas[(int64_t)owner * B * B * B + loc];
            }
        }
        patlas[t] = v;
        pdens[t] = (uint8_t)(v.x & 0xffu);
    }
}

cudaError_t launch_validate(const int32_t* ind, int64_t n_ind, int64_t nb, int32_t* blk_of_slot, int32_t* err,
                            cudaStream_t st) {
    if (n_ind <= 0) return cudaSuccess;
    const int64_t blocks = (n_ind + 255) / 256;
    validate_kernel<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, st>>>(ind, n_ind, nb, blk_of_slot, err);
    return cudaGetLastError();
}

cudaError_t launch_build_padded(const int32_t* ind, const int32_t* blk_of_slot, const uint8_t* atlas, int64_t nb,
                                int N, int B, int lgB, uint8_t* pdens, uint2* patlas, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    const int64_t total = nb * (int64_t)(B + 2) * (B + 2) * (B + 2);
    const int64_t blocks = (total + 255) / 256;
    build_padded_kernel<<<(unsigned)(blocks < 1048576 ? blocks : 1048576), 256, 0, st>>>(
        ind, blk_of_slot, reinterpret_cast<const uint2*>(atlas), nb, N, B, lgB, pdens, patlas);
    return cudaGetLastError();
}

}  // namespace snerg
