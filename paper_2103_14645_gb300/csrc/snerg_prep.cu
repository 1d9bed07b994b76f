// snerg_prep.cu -- scene set-up kernels: validate the indirection grid (Sec. 5.1),
// build the device layout of the atlas (apron-padded blocks) and the two Chebyshev
// distance maps the march uses to skip empty space.
//
// The paper's viewer keeps density in its own 8-bit texture so that empty space inside
// occupied blocks costs one byte per sample (App. A); the voxel distance plane here
// plays that role and, being a distance rather than a code, also says how many of the
// following samples are certainly empty. The 1-voxel apron makes every trilinear
// stencil of a sample a fetch from one block: atlas neighbours are not spatial neighbours (Sec. 5.1), so without it a sample
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
                                    uint2* __restrict__ patlas) {
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
    }
}

// Requantisation of fine-tuned colour/feature values into the padded atlas (Sec. 5.4
// codes): every padded entry whose source voxel is stored takes channels 1..7 from
// floor(255 x + 1/2) of the source's values (binary32, clamped) and keeps its own density
// byte, so the empty-space maps built from the densities stay valid. Interior entries
// also go to atlas_out (nullable) in the unpadded layout.
__device__ __forceinline__ uint32_t quant8(float x) {
    const float q = floorf(__fmaf_rn(x, 255.0f, 0.5f));
    return q > 0.0f ? (q < 255.0f ? (uint32_t)q : 255u) : 0u;   // NaN -> 0
}

__global__ void requantize_padded_kernel(const int32_t* __restrict__ ind, const int32_t* __restrict__ blk_of_slot,
                                         const float4* __restrict__ values, int64_t nb, int N, int B, int lgB,
                                         uint2* __restrict__ patlas, uint2* __restrict__ atlas_out) {
    const int P = B + 2, P3 = P * P * P, G = N >> lgB;
    const int64_t total = nb * (int64_t)P3, B3 = (int64_t)B * B * B;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = t / P3;
        const int r = (int)(t - slot * P3);
        const int px = r % P, py = (r / P) % P, pz = r / (P * P);
        const int blk = blk_of_slot[slot];
        if (blk < 0) continue;
        const int bx = blk % G, by = (blk / G) % G, bz = blk / (G * G);
        const int gx = min(max(bx * B + px - 1, 0), N - 1);
        const int gy = min(max(by * B + py - 1, 0), N - 1);
        const int gz = min(max(bz * B + pz - 1, 0), N - 1);
        const int owner = ind[((gz >> lgB) * G + (gy >> lgB)) * G + (gx >> lgB)];
        if (owner < 0) continue;                               // apron of an empty block: stays 0
        const int loc = ((gz & (B - 1)) * B + (gy & (B - 1))) * B + (gx & (B - 1));
        const int64_t src = (int64_t)owner * B3 + loc;
        const float4 a = values[2 * src], b = values[2 * src + 1];
        const uint2 old = patlas[t];
        uint2 v;
        v.x = (old.x & 0xffu) | quant8(a.y) << 8 | quant8(a.z) << 16 | quant8(a.w) << 24;
        v.y = quant8(b.x) | quant8(b.y) << 8 | quant8(b.z) << 16 | quant8(b.w) << 24;
        patlas[t] = v;
        if (atlas_out && px >= 1 && px <= B && py >= 1 && py <= B && pz >= 1 && pz <= B) atlas_out[src] = v;
    }
}

// ---------------------------------------------------------------------------------
// Chebyshev (L-infinity) distance transform of cubes of side n, in three separable
// passes: along one axis, out(p) = min over q on p's line of max(|q - p|, in(q)),
// capped at `cap`. Starting from in = 0 on occupied cells and cap elsewhere, after the
// x, y and z passes out(p) = min over occupied q of max_i |q_i - p_i| (max distributes
// over min, so the passes compose). The scan walks outwards from p and stops once the
// offset reaches the best value found, so its cost is the distance itself.
//
// `side` restricts q to one half-line (bit 0: q <= p, bit 1: q >= p; 3 = both). With
// one side per axis the result is the distance to the nearest occupied cell in the
// octant cone {q : q_i - p_i of the chosen sign}: the cone is a product of half-lines,
// so the one-sided passes compose the same way.
// ---------------------------------------------------------------------------------
constexpr int kSideLow = 1, kSideHigh = 2, kSideBoth = 3;

__device__ __forceinline__ int dt_line(const uint8_t* __restrict__ in, int64_t base, int64_t stride, int pos, int n,
                                       int cap, int side) {
    int best = min((int)in[base + pos * stride], cap);
    const int a_end = (side & kSideLow) ? -1 : pos, b_end = (side & kSideHigh) ? n : pos;
    for (int d = 1; d < best; ++d) {
        const int a = pos - d, b = pos + d;
        if (a <= a_end && b >= b_end) break;
        if (a > a_end) best = min(best, max(d, (int)in[base + a * stride]));
        if (b < b_end) best = min(best, max(d, (int)in[base + b * stride]));
    }
    return best;
}

// the side of axis i for octant o (bit i of o set: the ray runs towards -i)
__host__ __device__ __forceinline__ int octant_side(int o, int i) { return ((o >> i) & 1) ? kSideLow : kSideHigh; }

// axis: 0 = x (stride 1), 1 = y (stride n), 2 = z (stride n^2); cubes are contiguous
__global__ void dt_pass_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int n, int64_t ncubes,
                               int axis, int cap, int side) {
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t total = ncubes * n3;
    const int64_t stride = axis == 0 ? 1 : (axis == 1 ? n : (int64_t)n * n);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cube = t / n3;
        const int r = (int)(t - cube * n3);
        const int c[3] = {r % n, (r / n) % n, r / (n * n)};
        const int pos = c[axis];
        const int64_t base = t - (int64_t)pos * stride;
        out[t] = (uint8_t)dt_line(in, base, stride, pos, n, cap, side);
    }
}

// 0 where the block is occupied, cap elsewhere
__global__ void block_seed_kernel(const int32_t* __restrict__ ind, int64_t n, int cap, uint8_t* __restrict__ out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = ind[t] >= 0 ? 0 : (uint8_t)cap;
}

// 0 where the voxel's density code is non-zero, cap elsewhere (unpadded [nb][B^3])
__global__ void voxel_seed_kernel(const uint8_t* __restrict__ atlas, int64_t n, int cap, uint8_t* __restrict__ out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = atlas[t * 8] != 0 ? 0 : (uint8_t)cap;
}

// z pass of the voxel transform, written into the padded plane (apron cells = 255)
__global__ void dt_pass_z_padded_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ vskip, int B,
                                        int64_t nb, int cap, int side) {
    const int P = B + 2, P3 = P * P * P;
    const int64_t B3 = (int64_t)B * B * B;
    const int64_t total = nb * P3;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = t / P3;
        const int r = (int)(t - slot * P3);
        const int px = r % P - 1, py = (r / P) % P - 1, pz = r / (P * P) - 1;
        uint8_t v = 255;
        if (px >= 0 && py >= 0 && pz >= 0 && px < B && py < B && pz < B) {
            const int64_t base = slot * B3 + (int64_t)py * B + px;
            v = (uint8_t)dt_line(in, base, (int64_t)B * B, pz, B, cap, side);
        }
        vskip[t] = v;
    }
}

// dst[i] = src[i] for an occupied block, -bdist[i] (>= 1) for an empty one: the march
// reads one word per block. src and dst may be the same array.
__global__ void encode_distance_kernel(const int32_t* src, const uint8_t* __restrict__ bdist, int32_t* dst,
                                       int64_t n) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = src[t];
        dst[t] = v >= 0 ? v : -(int32_t)max((int)bdist[t], 1);
    }
}

// Apron cells of the voxel-distance plane that lie outside the grid get the value of the
// voxel they clamp to (clamp-to-edge, as in the padded atlas). A sample that rounding puts
// a hair outside the grid then finds its clamped nearest voxel's value without a clamp.
// (n_planes planes of [nb][P^3] one after the other; each is filled from itself)
__global__ void fill_vskip_border_kernel(uint8_t* __restrict__ vskip, const int32_t* __restrict__ blk_of_slot,
                                         int64_t nb, int N, int B, int lgB, int n_planes) {
    const int P = B + 2, P3 = P * P * P, G = N >> lgB;
    const int64_t total = n_planes * nb * (int64_t)P3;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ps = t / P3;                       // plane * nb + slot
        const int64_t slot = ps % nb;
        const int r = (int)(t - ps * P3);
        const int p[3] = {r % P, (r / P) % P, r / (P * P)};
        if (p[0] >= 1 && p[0] <= B && p[1] >= 1 && p[1] <= B && p[2] >= 1 && p[2] <= B) continue;   // interior
        const int blk = blk_of_slot[slot];
        if (blk < 0) continue;
        const int b[3] = {blk % G, (blk / G) % G, blk / (G * G)};
        int q[3];
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int g = b[i] * B + p[i] - 1;
            if (p[i] >= 1 && p[i] <= B) { q[i] = p[i]; continue; }
            if (g >= 0 && g < N) { ok = false; break; }      // faces an interior neighbour: never probed
            q[i] = min(max(g, 0), N - 1) - b[i] * B + 1;     // the clamped voxel, inside this block
        }
        if (ok) vskip[t] = vskip[ps * P3 + (q[2] * P + q[1]) * P + q[0]];
    }
}

static unsigned grid_for(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1048576 ? (b > 0 ? b : 1) : 1048576);
}

static void block_distance(const int32_t* ind, int G, int cap, uint8_t* tmp0, uint8_t* tmp1, uint8_t* bdist,
                           const int side[3], cudaStream_t st) {
    const int64_t n = (int64_t)G * G * G;
    block_seed_kernel<<<grid_for(n), 256, 0, st>>>(ind, n, cap, tmp0);
    dt_pass_kernel<<<grid_for(n), 256, 0, st>>>(tmp0, tmp1, G, 1, 0, cap, side[0]);
    dt_pass_kernel<<<grid_for(n), 256, 0, st>>>(tmp1, tmp0, G, 1, 1, cap, side[1]);
    dt_pass_kernel<<<grid_for(n), 256, 0, st>>>(tmp0, bdist, G, 1, 2, cap, side[2]);
}

cudaError_t launch_block_distance(const int32_t* ind, int G, int cap, uint8_t* tmp0, uint8_t* tmp1,
                                  uint8_t* bdist, cudaStream_t st) {
    const int both[3] = {kSideBoth, kSideBoth, kSideBoth};
    block_distance(ind, G, cap, tmp0, tmp1, bdist, both, st);
    return cudaGetLastError();
}

// For each octant o, ind_oct[o] = the indirection grid with every empty entry replaced by
// -D_o, D_o >= 1 the Chebyshev distance (in blocks, capped) to the nearest occupied block
// in o's cone. `ind` may be ind_oct[0].
cudaError_t launch_block_distance_octants(const int32_t* ind, int G, int cap, uint8_t* tmp0, uint8_t* tmp1,
                                          uint8_t* bdist, int32_t* ind_oct, cudaStream_t st) {
    const int64_t n = (int64_t)G * G * G;
    for (int o = 7; o >= 0; --o) {          // octant 0 last: ind may alias its copy
        const int side[3] = {octant_side(o, 0), octant_side(o, 1), octant_side(o, 2)};
        block_distance(ind, G, cap, tmp0, tmp1, bdist, side, st);
        encode_distance_kernel<<<grid_for(n), 256, 0, st>>>(ind, bdist, ind_oct + (size_t)o * n, n);
    }
    return cudaGetLastError();
}

// For each octant o, plane o of vskip ([8][nb][P^3]) holds per interior voxel the
// Chebyshev distance to the nearest voxel of the same block with a non-zero density code
// in o's cone (apron cells 255; the grid-border apron is filled afterwards). The x pass
// depends only on o's x side, the y pass on its x and y sides, so the eight transforms
// share them: 2 x passes, 4 y passes, 8 z passes. `scratch` holds 7 nb B^3 bytes.
cudaError_t launch_voxel_distance_octants(const uint8_t* atlas, int64_t nb, int B, uint8_t* scratch, uint8_t* vskip,
                                          cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    const int64_t n = nb * (int64_t)B * B * B;
    const int64_t plane = nb * (int64_t)(B + 2) * (B + 2) * (B + 2);
    const int cap = 255;
    uint8_t* seed = scratch;
    uint8_t* xs = scratch + n;          // [2][n]: x side (bit 0 of o)
    uint8_t* ys = scratch + 3 * n;      // [4][n]: x and y sides (bits 0, 1 of o)
    voxel_seed_kernel<<<grid_for(n), 256, 0, st>>>(atlas, n, cap, seed);
    for (int a = 0; a < 2; ++a)
        dt_pass_kernel<<<grid_for(n), 256, 0, st>>>(seed, xs + a * n, B, nb, 0, cap, octant_side(a, 0));
    for (int a = 0; a < 4; ++a)
        dt_pass_kernel<<<grid_for(n), 256, 0, st>>>(xs + (a & 1) * n, ys + a * n, B, nb, 1, cap, octant_side(a, 1));
    for (int o = 0; o < 8; ++o)
        dt_pass_z_padded_kernel<<<grid_for(plane), 256, 0, st>>>(ys + (o & 3) * n, vskip + (size_t)o * plane, B, nb,
                                                                 cap, octant_side(o, 2));
    return cudaGetLastError();
}

cudaError_t launch_validate(const int32_t* ind, int64_t n_ind, int64_t nb, int32_t* blk_of_slot, int32_t* err,
                            cudaStream_t st) {
    if (n_ind <= 0) return cudaSuccess;
    const int64_t blocks = (n_ind + 255) / 256;
    validate_kernel<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, st>>>(ind, n_ind, nb, blk_of_slot, err);
    return cudaGetLastError();
}

cudaError_t launch_build_padded(const int32_t* ind, const int32_t* blk_of_slot, const uint8_t* atlas, int64_t nb,
                                int N, int B, int lgB, uint2* patlas, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    const int64_t total = nb * (int64_t)(B + 2) * (B + 2) * (B + 2);
    build_padded_kernel<<<grid_for(total), 256, 0, st>>>(ind, blk_of_slot, reinterpret_cast<const uint2*>(atlas), nb,
                                                          N, B, lgB, patlas);
    return cudaGetLastError();
}

cudaError_t launch_requantize_padded(const int32_t* ind, const int32_t* blk_of_slot, const float* values, int64_t nb,
                                     int N, int B, int lgB, uint2* patlas, uint8_t* atlas_out, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    const int64_t total = nb * (int64_t)(B + 2) * (B + 2) * (B + 2);
    requantize_padded_kernel<<<grid_for(total), 256, 0, st>>>(ind, blk_of_slot, reinterpret_cast<const float4*>(values),
                                                               nb, N, B, lgB, patlas,
                                                               reinterpret_cast<uint2*>(atlas_out));
    return cudaGetLastError();
}

cudaError_t launch_fill_vskip_border(uint8_t* vskip, const int32_t* blk_of_slot, int64_t nb, int N, int B, int lgB,
                                     int n_planes, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    fill_vskip_border_kernel<<<grid_for(n_planes * nb * (int64_t)(B + 2) * (B + 2) * (B + 2)), 256, 0, st>>>(
        vskip, blk_of_slot, nb, N, B, lgB, n_planes);
    return cudaGetLastError();
}
}  // namespace snerg
