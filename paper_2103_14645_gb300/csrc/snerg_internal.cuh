// snerg_internal.cuh -- device-side core of the SNeRG renderer (sm_103a).
//
// Per pixel: pinhole ray (Sec. 4.1), clip to the grid, march the macroblock
// indirection grid skipping empty blocks (Sec. 5.1-5.2, App. A), probe the nearest
// voxel's density and fetch/interpolate all 8 channels only where it is non-zero
// (App. A), alpha-composite diffuse colour and features (Eqs. 2, 5, 6), stop once the
// optical depth exceeds ln(1000) (T < 1e-3; "terminating ray-marching once the opacity
// has saturated", Sec. 5.2), then one evaluation of the view-dependence MLP (Eq. 7).
//
// Integer decisions (sample lattice, nearest voxel, block membership, early exit) use
// IEEE binary32 with one rounding per operation, written with __fadd_rn/__fmul_rn/...
// so nvcc cannot contract them into FMAs; the operation order is part of the renderer's
// arithmetic contract (include/snerg.h) and makes step counts and visited voxels
// reproducible bit for bit. Colour arithmetic is ordinary FP32.
//
// Device layout (built by snerg_prep.cu inside the caller's workspace):
//   ind    int32 [8][G^3]              per octant o of the ray direction (bit i set: d_i
//                                      < 0), the indirection grid (z, y, x): the atlas slot
//                                      of an occupied block, or -D for an empty one, D >= 1
//                                      being the Chebyshev distance (in blocks, capped) to
//                                      the nearest occupied block in o's cone (the blocks
//                                      c with c_i - b_i of d_i's sign) -- one load gives both
//   vskip  uint8 [8][nb][P^3], P = B+2 per octant and interior voxel, Chebyshev distance
//                                      (in voxels) to the nearest voxel of the same block in
//                                      the octant's cone with a non-zero density code; 0 <=>
//                                      the voxel's own code is non-zero (the density probe)
//   patlas uint2 [nb][P^3]             all 8 channels (density, r, g, b | f0..f3)
// A ray's lattice coordinates are monotone in the sample index (each step of the binary32
// lattice arithmetic is a rounded monotone operation), so every later sample's nearest
// voxel and block lie in the cone of the current one: the one-sided distances are the
// ones that bound the empty samples ahead.
// The apron holds the neighbouring blocks' voxels (0 where the neighbour is empty) and
// the clamped edge voxel at the grid border, so every trilinear stencil of a sample
// whose nearest voxel lies in block b reads only block b's padded copy.
//
// The two distance maps only let the march skip samples that provably contribute
// nothing (their nearest voxel is in an empty block, or has a zero density code); the
// lattice, the visited samples and the counts are exactly those of a sample-by-sample
// march.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "snerg.h"

namespace snerg {

constexpr int kMlpIn = 34;
constexpr int kMlpH = 16;
constexpr int kMlpOut = 3;
constexpr int kNParam = 883;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpH * kMlpIn;
constexpr int kOffW2 = kOffB1 + kMlpH;
constexpr int kOffB2 = kOffW2 + kMlpH * kMlpH;
constexpr int kOffW3 = kOffB2 + kMlpH;
constexpr int kOffB3 = kOffW3 + kMlpOut * kMlpH;
static_assert(kOffB3 + kMlpOut == kNParam, "MLP layout");

constexpr int kMaxCams = SNERG_MAX_CAMERAS;
constexpr int kAuxCh = 8;

// device status word bits
constexpr int kStatusStepLimit = SNERG_E_STEP_LIMIT;

struct DevScene {
    const int32_t* ind;    // octant 0's copy; octant o's at ind + o * ind_oct
    const uint8_t* bdist;
    const uint8_t* vskip;  // octant 0's plane; octant o's at vskip + o * vskip_oct
    const uint2* patlas;
    int32_t* status;
    int64_t ind_oct;       // G^3
    int64_t vskip_oct;     // nb * P^3
    int32_t N, B, lgB, G, P, P3;
    float fN;         // (float)N
    float scale;      // binary32(N / extent)
    float bmin[3];
    float kappa;      // binary32(sigma_max * extent / N / 255): optical depth per density code
    float taumax;     // binary32(ln 1000)
    float tmin;       // alpha atlas: binary32(1e-3), the exit threshold on T
    float inv255;     // binary32(1 / 255)
    float bg[3];
    int32_t kmax;     // lattice index cap (4N + 16)
    int32_t flags;    // SNERG_FLAG_*
};

// App. C: the scale min(1, 1.5 a) / a applied after compositing to (C_d, alpha, V) when
// un-premultiply is on and a = 1 - T > 0 (else 1). Depends on density only.
__device__ __forceinline__ float unpremultiply_scale(const DevScene& s, float T) {
    const float a = 1.0f - T;
    if (!(s.flags & SNERG_FLAG_UNPREMULTIPLY) || !(a > 0.0f)) return 1.0f;
    return fminf(1.0f, 1.5f * a) / a;
}

struct CamTable {
    snerg_camera c[kMaxCams];
};

struct Ray {
    float o[3];
    float d[3];
    float t0, t1;
    bool hit;
};

struct MarchState {
    float acc[7];     // sum_k w_k * (sum_corners tw * code) for channels 1..7 (codes, not /255)
    float rgb_ps[3];  // non-deferred comparison model: sum_k w_k (c_d,k + residual_k)
    float T;
    float tau;
    int steps;
    int active;
    int blocks;       // indirection entries read
    bool limit;
};

// ---------------------------------------------------------------------------------
// ray generation and clipping (binary32, fixed order)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ Ray make_ray(const DevScene& s, const snerg_camera& c, int px, int py) {
    Ray r;
    const float xs = __fdiv_rn(__fsub_rn(__fadd_rn((float)px, 0.5f), c.cx), c.fx);
    const float ys = __fdiv_rn(__fsub_rn(__fadd_rn((float)py, 0.5f), c.cy), c.fy);
    const float dc0 = xs, dc1 = -ys, dc2 = -1.0f;
    float d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        d[i] = __fadd_rn(__fadd_rn(__fmul_rn(c.c2w[4 * i], dc0), __fmul_rn(c.c2w[4 * i + 1], dc1)),
                         __fmul_rn(c.c2w[4 * i + 2], dc2));
    const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])), __fmul_rn(d[2], d[2]));
    const float nrm = __fsqrt_rn(n2);
    float tn = -INFINITY, tf = INFINITY;
    r.hit = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        r.d[i] = __fdiv_rn(d[i], nrm);
        r.o[i] = __fmul_rn(__fsub_rn(c.c2w[4 * i + 3], s.bmin[i]), s.scale);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (r.d[i] != 0.0f) {
            const float ta = __fdiv_rn(-r.o[i], r.d[i]);
            const float tb = __fdiv_rn(__fsub_rn(s.fN, r.o[i]), r.d[i]);
            tn = fmaxf(tn, fminf(ta, tb));
            tf = fminf(tf, fmaxf(ta, tb));
        } else if (r.o[i] < 0.0f || r.o[i] > s.fN) {
            r.hit = false;
        }
    }
    r.t0 = fmaxf(tn, 0.0f);
    r.t1 = tf;
    if (!(r.t0 < r.t1)) r.hit = false;
    return r;
}

// Lattice indices are carried as binary32 integers (exact below 2^24; the index cap is
// 4N + 16 <= 65,552), so stepping the lattice needs no integer/float conversions.
__device__ __forceinline__ float lattice_t(const Ray& r, float k) {
    return __fadd_rn(r.t0, __fadd_rn(k, 0.5f));
}

__device__ __forceinline__ float lattice_u(const Ray& r, float t, int i) {
    return __fadd_rn(r.o[i], __fmul_rn(t, r.d[i]));
}

// Floor, ceiling and integer value of a binary32 x with |x| < 2^22, on the FMA and
// integer pipes instead of the conversion unit: x + 1.5 * 2^23 lies in [2^23, 2^24),
// where the spacing of binary32 is 1, so that sum rounded down (up) is 1.5 * 2^23 plus
// floor(x) (ceil(x)) exactly, and its bit pattern is 0x4B400000 plus that integer. The
// results are exactly floorf / ceilf / the conversion of an integral x.
constexpr float kMagic = 12582912.0f;          // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;
__device__ __forceinline__ float floor_small(float x) { return __fsub_rn(__fadd_rd(x, kMagic), kMagic); }
__device__ __forceinline__ float ceil_small(float x) { return __fsub_rn(__fadd_ru(x, kMagic), kMagic); }
__device__ __forceinline__ int floor_int_small(float x) { return __float_as_int(__fadd_rd(x, kMagic)) - kMagicBits; }
__device__ __forceinline__ int int_small(float x) { return __float_as_int(__fadd_rn(x, kMagic)) - kMagicBits; }
// and back: the binary32 value of an integer |v| < 2^22
__device__ __forceinline__ float float_small(int v) { return __fsub_rn(__int_as_float(v + kMagicBits), kMagic); }

// a lattice coordinate lies within the grid up to rounding (|u| <= N + 1 <= 16385)
__device__ __forceinline__ int nearest_voxel(float u, int N) {
    return min(max(floor_int_small(u), 0), N - 1);
}

// A box of blocks lo..hi (inclusive, per axis) as bounds on the sample position: the
// nearest voxel j = clamp(floor(u), 0, N-1) has its block in [lo, hi] iff
// u >= lo*B (no bound if lo*B <= 0, where the clamp applies) and u < (hi+1)*B (no bound
// if (hi+1)*B >= N). floor(u) >= L <=> u >= L and floor(u) <= H <=> u < H + 1 for
// integers L, H, so the test is exact.
struct Box {
    float lo[3], hi[3];
};

__device__ __forceinline__ Box make_box(const DevScene& s, const int lo[3], const int hi[3]) {
    Box bx;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int L = lo[i] * s.B, H = (hi[i] + 1) * s.B;
        bx.lo[i] = L <= 0 ? -INFINITY : float_small(L);       // block corners: 0 < L, H < N <= 16384
        bx.hi[i] = H >= s.N ? INFINITY : float_small(H);
    }
    return bx;
}

// true iff sample k lies before the ray's exit and its nearest voxel's block is in the box
__device__ __forceinline__ bool in_box(const Ray& r, float k, const Box& bx) {
    const float t = lattice_t(r, k);
    if (!(t < r.t1)) return false;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float u = lattice_u(r, t, i);
        if (!(u >= bx.lo[i] && u < bx.hi[i])) return false;
    }
    return true;
}

// The margin (in samples) of box_exit's unconfirmed estimate for ray r in a grid of N
// voxels per axis, with t_m = max(t1, 1) bounding every lattice t the march compares:
//  - the estimate K = fl(fl(te - t0) - 0.5) with te = fl(fl(face - o) * inv_d), inv_d
//    within 2 ulp of 1/d: |K - K*| <= t_m (2^-22 + 2^-23 + 2^-24 + 2 * 2^-24) < t_m 2^-20;
//  - a lattice coordinate u = fl(o + fl(t d)), t = fl(t0 + k + 1/2), lies within
//    (2 t_m |d_i| + |u|) 2^-24 of its exact value, |u| <= N + 1 near a face, and moves by
//    |d_i| per sample: at most (2 t_m + (N + 1) / |d_i|) 2^-24 samples on axis i, and
//    t_m 2^-24 samples for the test t < t1;
// taken four times over. A component of d that is zero makes no face ahead; a tiny one
// makes the margin large and the exact search runs instead.
__device__ __forceinline__ float exit_margin(const Ray& r, float fN) {
    float dmin = INFINITY;
#pragma unroll
    for (int i = 0; i < 3; ++i)
        if (r.d[i] != 0.0f) dmin = fminf(dmin, fabsf(r.d[i]));
    const float tm = fmaxf(r.t1, 1.0f);
    const float lat = (2.0f * tm + (fN + 1.0f) / dmin) * (1.0f / 16777216.0f);
    return 4.0f * (tm * (1.0f / 1048576.0f) + lat + tm * (1.0f / 16777216.0f));
}

// First lattice index k' > k with in_box(k') false, given in_box(k). Each axis's
// nearest voxel is a monotone function of k (every step of the lattice arithmetic is a
// rounded monotone operation), so the samples inside a box form one contiguous run:
// estimate its end from the ray/box exit distance, then confirm or correct it with an
// exact search on the lattice itself.
//
// The estimate needs no confirmation when the real crossing index is at least `margin`
// from every integer, margin bounding (a) the error of the estimate K (rounding of the
// face distances, the approximate reciprocal, the two subtractions) and (b) how far in k
// the binary32 lattice can place a sample across a face or past t1 from where exact
// arithmetic would (see exit_margin). Then every sample before ceil(K) is inside on every
// face still ahead (their crossings are no earlier than K's) and the sample at ceil(K)
// is outside. A margin of 1 or more disables this.
__device__ __forceinline__ float box_exit(const Ray& r, const float inv_d[3], float kmax, float k, const Box& bx,
                                          float margin) {
    float te = r.t1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (r.d[i] > 0.0f) te = fminf(te, (bx.hi[i] - r.o[i]) * inv_d[i]);
        else if (r.d[i] < 0.0f) te = fminf(te, (bx.lo[i] - r.o[i]) * inv_d[i]);
    }
    const float K = te - r.t0 - 0.5f;
    const float n = ceil_small(K);        // |K| <= t1 - t0 + 1 (or NaN, kept)
    // fr in [0, 1). n - K is exact for K >= 1/2 (Sterbenz) and for K <= 0; for K in
    // (0, 1/2), n = 1 and 1 - K rounds by at most 2^-25, far inside the margin (at least
    // 4 * 2^-20, four times the bound on the estimate's own error), so the test below
    // decides the same way.
    const float fr = n - K;
    if (n >= k + 1.0f && n < kmax && fr >= margin && fr < 1.0f - margin) return n;
    // estimate clamped to [k + 1, kmax] (fminf/fmaxf also map a NaN estimate into range)
    const float ke = fmaxf(fminf(n, kmax), k + 1.0f);
    float lo_k = k, hi_k;
    if (ke - 1.0f > k && !in_box(r, ke - 1.0f, bx)) {
        hi_k = ke - 1.0f;
    } else if (ke < kmax && in_box(r, ke, bx)) {
        lo_k = ke;
        float step = 1.0f;
        for (;;) {
            hi_k = lo_k + step;
            if (hi_k >= kmax) { hi_k = kmax; break; }
            if (!in_box(r, hi_k, bx)) break;
            lo_k = hi_k;
            step += step;
        }
    } else {
        return ke;
    }
    while (hi_k - lo_k > 1.0f) {
        const float mid = floorf((lo_k + hi_k) * 0.5f);
        if (in_box(r, mid, bx)) lo_k = mid; else hi_k = mid;
    }
    return hi_k;
}

// Byte `byte` of w as a float, exactly: the byte is placed in the low mantissa bits of
// 2^23 (bit pattern 0x4B0000bb) and 2^23 is subtracted. Two full-rate integer/FP ops
// instead of an integer-to-float conversion.
__device__ __forceinline__ float code(uint32_t w, int byte) {
    return __int_as_float((int)__byte_perm(w, 0x4B000000u, 0x7540u | (unsigned)byte)) - 8388608.0f;
}

// Two bytes as a float pair (one packed subtract for both)
__device__ __forceinline__ float2 code2(uint32_t w0, int b0, uint32_t w1, int b1) {
    const float2 m = make_float2(__int_as_float((int)__byte_perm(w0, 0x4B000000u, 0x7540u | (unsigned)b0)),
                                 __int_as_float((int)__byte_perm(w1, 0x4B000000u, 0x7540u | (unsigned)b1)));
    return __fadd2_rn(m, make_float2(-8388608.0f, -8388608.0f));
}

// colour/feature accumulation of one composited sample: acc += w_k * trilinear(codes),
// corner by corner, channels in packed pairs (each element is the same fused
// multiply-add as the scalar form, in the same order)
__device__ __forceinline__ void accumulate_colour(MarchState& st, const uint2 cv[8], float wk, const float f[3],
                                                  const float g[3]) {
    float2 a01 = make_float2(st.acc[0], st.acc[1]);
    float2 a23 = make_float2(st.acc[2], st.acc[3]);
    float2 a45 = make_float2(st.acc[4], st.acc[5]);
    float a6 = st.acc[6];
    // w_k folded into the z weights: 14 multiplies for the 8 corner weights instead of 20
    const float wz0 = wk * g[2], wz1 = wk * f[2];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float w = ((c & 4) ? wz1 : wz0) * ((c & 2) ? f[1] : g[1]) * ((c & 1) ? f[0] : g[0]);
        const float2 ww = make_float2(w, w);
        a01 = __ffma2_rn(code2(cv[c].x, 1, cv[c].x, 2), ww, a01);
        a23 = __ffma2_rn(code2(cv[c].x, 3, cv[c].y, 0), ww, a23);
        a45 = __ffma2_rn(code2(cv[c].y, 1, cv[c].y, 2), ww, a45);
        a6 = fmaf(code(cv[c].y, 3), w, a6);
    }
    st.acc[0] = a01.x;
    st.acc[1] = a01.y;
    st.acc[2] = a23.x;
    st.acc[3] = a23.y;
    st.acc[4] = a45.x;
    st.acc[5] = a45.y;
    st.acc[6] = a6;
}

// The trilinear stencil of a sample at u in block-padded coordinates (block origin minus
// one at o, integer voxel coordinates): the fractional weights f, g = 1 - f, the lower
// corner (as the float fl and the integer fi, both from one add), and the 8 corners'
// codes (index z*4 + y*2 + x). The lower corner is in [0, B] for a sample of this block
// (the apron holds the neighbours and the clamped border); the index clamp only guards
// the address.
__device__ __forceinline__ void stencil_weights(const float u[3], float f[3], float g[3], float fl[3], int fi[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float x = __fsub_rn(u[i], 0.5f);
        const float m = __fadd_rd(x, kMagic);            // floor_small / floor_int_small of x
        fl[i] = __fsub_rn(m, kMagic);
        fi[i] = __float_as_int(m) - kMagicBits;
        f[i] = __fsub_rn(x, fl[i]);
        g[i] = __fsub_rn(1.0f, f[i]);
    }
}

__device__ __forceinline__ void load_stencil(const float u[3], const int o[3], int P, int P3, const uint2* pa,
                                             float f[3], float g[3], float fl[3], int fi[3], uint2 cv[8]) {
    stencil_weights(u, f, g, fl, fi);
    const int PP = P * P;
    const int i0 = min(max(((fi[2] - o[2]) * P + (fi[1] - o[1])) * P + (fi[0] - o[0]), 0), P3 - 1 - (PP + P + 1));
    const uint2* p0 = pa + i0;
    cv[0] = __ldg(p0);
    cv[1] = __ldg(p0 + 1);
    cv[2] = __ldg(p0 + P);
    cv[3] = __ldg(p0 + P + 1);
    cv[4] = __ldg(p0 + PP);
    cv[5] = __ldg(p0 + PP + 1);
    cv[6] = __ldg(p0 + PP + P);
    cv[7] = __ldg(p0 + PP + P + 1);
}

// Density trilinear of one composited sample (binary32, x then y then z) and its
// compositing (Eqs. 2, 5, 6): returns w_k and advances T (and tau); saturated once the
// ray's remaining transmittance is below the early-exit bound.
__device__ __forceinline__ float composite(const DevScene& s, const uint2 cv[8], const float f[3], const float g[3],
                                           float& T, float& tau, bool& saturated) {
    const float e00 = __fadd_rn(__fmul_rn(code(cv[0].x, 0), g[0]), __fmul_rn(code(cv[1].x, 0), f[0]));
    const float e10 = __fadd_rn(__fmul_rn(code(cv[2].x, 0), g[0]), __fmul_rn(code(cv[3].x, 0), f[0]));
    const float e01 = __fadd_rn(__fmul_rn(code(cv[4].x, 0), g[0]), __fmul_rn(code(cv[5].x, 0), f[0]));
    const float e11 = __fadd_rn(__fmul_rn(code(cv[6].x, 0), g[0]), __fmul_rn(code(cv[7].x, 0), f[0]));
    const float e0 = __fadd_rn(__fmul_rn(e00, g[1]), __fmul_rn(e10, f[1]));
    const float e1 = __fadd_rn(__fmul_rn(e01, g[1]), __fmul_rn(e11, f[1]));
    const float sq = __fadd_rn(__fmul_rn(e0, g[2]), __fmul_rn(e1, f[2]));
    float wk;
    if (s.flags & SNERG_FLAG_ALPHA_ATLAS) {
        // channel 0 holds alpha: a = s * binary32(1/255), T <- T (1 - a) in binary32,
        // stop once T < binary32(1e-3)
        const float a = __fmul_rn(sq, s.inv255);
        wk = T * a;
        T = __fmul_rn(T, __fsub_rn(1.0f, a));
        saturated = T < s.tmin;
    } else {
        const float od = __fmul_rn(sq, s.kappa);
        tau = __fadd_rn(tau, od);
        const float e = expf(-od);
        wk = T * (1.0f - e);
        T *= e;
        saturated = tau > s.taumax;
    }
    return wk;
}

// The adjoint of one composited sample's colour/feature fetch: w_k * (corner weight) *
// gfeat into the eight corners' gradient entries ([slot][B^3][8], channel 0 unused) with
// vector atomics. o: the sample's block origin minus one, fi its stencil's lower corner
// (integer voxel coordinates).
__device__ __forceinline__ void scatter_sample(const DevScene& s, int slot, const int fi[3], const int o[3],
                                               const float f[3], const float g[3], float wk, const float* gfeat,
                                               float* grad_atlas) {
    const int B = s.B, N = s.N;
    float tw[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) tw[c] = ((c & 4) ? f[2] : g[2]) * ((c & 2) ? f[1] : g[1]) * ((c & 1) ? f[0] : g[0]);
    const int B3 = B * B * B;
    // a stencil inside this block (lower corner at padded coordinate 1 .. B-1 on every
    // axis) has all eight corners in its own slot: no indirection reads
    const int ex = fi[0] - o[0], ey = fi[1] - o[1], ez = fi[2] - o[2];
    if (ex >= 1 && ex <= B - 1 && ey >= 1 && ey <= B - 1 && ez >= 1 && ez <= B - 1) {
        float* g0 = grad_atlas + ((size_t)slot * B3 + ((ez - 1) * B + (ey - 1)) * B + (ex - 1)) * 8;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float* gp = g0 + ((((c >> 2) & 1) * B + ((c >> 1) & 1)) * B + (c & 1)) * 8;
            const float w = wk * tw[c];
            atomicAdd(reinterpret_cast<float4*>(gp), make_float4(0.0f, w * gfeat[0], w * gfeat[1], w * gfeat[2]));
            atomicAdd(reinterpret_cast<float4*>(gp + 4),
                      make_float4(w * gfeat[3], w * gfeat[4], w * gfeat[5], w * gfeat[6]));
        }
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int X = min(max(fi[0] + (c & 1), 0), N - 1);
            const int Y = min(max(fi[1] + ((c >> 1) & 1), 0), N - 1);
            const int Z = min(max(fi[2] + ((c >> 2) & 1), 0), N - 1);
            const int cs = __ldg(s.ind + (((Z >> s.lgB) * s.G + (Y >> s.lgB)) * s.G + (X >> s.lgB)));
            if (cs < 0) continue;
            const int loc = (((Z & (B - 1)) * B) + (Y & (B - 1))) * B + (X & (B - 1));
            float* gp = grad_atlas + ((size_t)cs * B3 + loc) * 8;
            const float w = wk * tw[c];
            atomicAdd(reinterpret_cast<float4*>(gp), make_float4(0.0f, w * gfeat[0], w * gfeat[1], w * gfeat[2]));
            atomicAdd(reinterpret_cast<float4*>(gp + 4),
                      make_float4(w * gfeat[3], w * gfeat[4], w * gfeat[5], w * gfeat[6]));
        }
    }
}

// Composited samples a march records (REC) for the adjoint's scatter: (lattice index, w_k)
// of each of the first kRecCap, then (T, tau) after the last of them
constexpr int kRecCap = 32;

// ---------------------------------------------------------------------------------
// the march. TRACE records visited voxels; GRAD scatters w_k * trilinear weight * g
// into the gradient atlas (density frozen, so the weights are the forward ones); REC
// stores the lattice index and weight of the first kRecCap composited samples in rec[j]
// and T, tau after them in rec[kRecCap]; CONT starts from the T and tau already in st (a
// march resumed after recorded samples).
// ---------------------------------------------------------------------------------
// k_begin: first lattice index to consider (0, or a k known to precede every composited
// sample, in which case the result is the same); k_first (nullable) receives the index
// of the first composited sample (kmax if none).
struct MlpWeights;
__device__ __forceinline__ void per_sample_residual(const MlpWeights* pw, const float* sW, const float cd[3],
                                                    const float v[4], const float d[3], float res[3]);

// PS: the non-deferred comparison model (SNERG_FLAG_PER_SAMPLE_MLP): every composited
// sample also evaluates the view-dependence MLP on its own (c_d, v) (weights from pw, else
// from sW) and adds w_k (c_d,k + residual_k) to st.rgb_ps.
template <bool TRACE, bool GRAD, bool PS = false, bool SPEC = false, bool REC = false, bool CONT = false>
__device__ __forceinline__ void march(const DevScene& s, const Ray& r, MarchState& st,
                                      uint64_t* trace, int trace_cap,
                                      const float* gfeat, float* grad_atlas,
                                      int k_begin = 0, int* k_first = nullptr,
                                      const MlpWeights* ps_w = nullptr, const float* ps_sw = nullptr,
                                      float2* rec = nullptr) {
#pragma unroll
    for (int c = 0; c < 7; ++c) st.acc[c] = 0.0f;
    st.rgb_ps[0] = st.rgb_ps[1] = st.rgb_ps[2] = 0.0f;
    if (!CONT) {
        st.T = 1.0f;
        st.tau = 0.0f;
    }
    st.steps = 0;
    st.active = 0;
    st.blocks = 0;
    st.limit = false;
    if (!r.hit) return;
    const int N = s.N, B = s.B, P = s.P;
    float inv_d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) inv_d[i] = __fdividef(1.0f, r.d[i]);
    // Voxel-skip rate: between samples k and k+s every coordinate moves by at most
    // s*m + eps voxels, m = max_i |d_i| and eps bounding the rounding of the binary32
    // lattice arithmetic (a few ulps of the largest t or u the ray meets; max(t1, N) *
    // 2^-19 is well above that). The nearest voxel then moves by at most s*m + eps + 1,
    // so a sample whose nearest voxel is at Chebyshev distance D from every voxel with
    // density is followed by empty samples for every s with s*m + eps < D - 1.
    const float m_max = fmaxf(fmaxf(fabsf(r.d[0]), fabsf(r.d[1])), fabsf(r.d[2]));
    const float skip_inv_m = (1.0f - 1.0f / 1048576.0f) / m_max;   // biased down: never overshoots
    const float skip_eps = fmaxf(r.t1, s.fN) * (1.0f / 524288.0f);
    const float exit_m = exit_margin(r, s.fN);
    const int oct = (r.d[0] < 0.0f ? 1 : 0) | (r.d[1] < 0.0f ? 2 : 0) | (r.d[2] < 0.0f ? 4 : 0);
    const int32_t* ind = s.ind + oct * s.ind_oct;
    const uint8_t* vskip = s.vskip + oct * s.vskip_oct;
    const float kmax = (float)s.kmax;
    float k = (float)k_begin;
    float k_spec = -1.0f;   // the sample after the last composited one
    float steps = 0.0f;
    bool done = false;
    if (k_first) *k_first = s.kmax;
    for (;;) {
        if (k >= kmax) { st.limit = true; break; }
        const float t = lattice_t(r, k);
        if (!(t < r.t1)) break;
        int b[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) b[i] = nearest_voxel(lattice_u(r, t, i), N) >> s.lgB;
        const int bi = (b[2] * s.G + b[1]) * s.G + b[0];
        const int slot = __ldg(ind + bi);
        st.blocks++;
        if (slot < 0) {
            // every block of the ray's cone within Chebyshev distance D-1 of b is empty:
            // leave that one-sided box
            const int D1 = -slot - 1;
            int lo[3], hi[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                lo[i] = ((oct >> i) & 1) ? b[i] - D1 : b[i];
                hi[i] = ((oct >> i) & 1) ? b[i] : b[i] + D1;
            }
            k = box_exit(r, inv_d, kmax, k, make_box(s, lo, hi), exit_m);
            continue;
        }
        const float kx = box_exit(r, inv_d, kmax, k, make_box(s, b, b), exit_m);
        const uint8_t* vs = vskip + (size_t)slot * s.P3;
        const uint2* pa = s.patlas + (size_t)slot * s.P3;
        // block origin minus one, so that the padded local coordinate is floor(u) - o
        const int o3[3] = {(b[0] << s.lgB) - 1, (b[1] << s.lgB) - 1, (b[2] << s.lgB) - 1};
        float kk = k;
        while (kk < kx) {
            const float tk = lattice_t(r, kk);
            float u[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) u[i] = lattice_u(r, tk, i);
            // nearest voxel in padded block coordinates, floor(u) - origin + 1: in [1, B] for
            // a sample of this block, or 0 / B+1 where rounding puts u a hair outside the
            // grid -- apron cells that hold the clamped edge voxel's value (the grid clamp
            // is built into the plane). The index clamp only guards the address.
            const int lx = floor_int_small(u[0]) - o3[0], ly = floor_int_small(u[1]) - o3[1],
                      lz = floor_int_small(u[2]) - o3[2];
            const int pidx = min(max((lz * P + ly) * P + lx, 0), s.P3 - 1);
            // SPEC: the sample's stencil is loaded before the probe's answer when the
            // previous sample was composited (inside a surface the next one usually is
            // too, and one memory latency then serves both), after it otherwise. It pays
            // in latency-bound launches (ray lists, the adjoint); where the launch is
            // issue-bound, lanes that disagree on the guess run the stencil code twice.
            float f[3], g[3], fl[3];
            int fi[3];
            uint2 cv[8];
            const bool spec = SPEC && (kk == k_spec);
            if (spec) load_stencil(u, o3, P, s.P3, pa, f, g, fl, fi, cv);
            const int vd = __ldg(vs + pidx);
            if (vd != 0) {
                // no voxel of this block in the ray's cone within Chebyshev distance vd-1
                // has density: the next s_max samples (s_max*m + eps < vd - 1) are empty,
                // skip them
                const float q = (float_small(vd) - 1.0f - skip_eps) * skip_inv_m;
                kk += fmaxf(1.0f, ceil_small(q));      // = 1 + s_max, s_max = ceil(q) - 1 >= 0
                continue;
            }
            if (TRACE && st.active < trace_cap)
                trace[st.active] = ((uint64_t)nearest_voxel(u[2], N) * N + (uint64_t)nearest_voxel(u[1], N)) * N +
                                   (uint64_t)nearest_voxel(u[0], N);
            if (k_first && st.active == 0) *k_first = (int)kk;
            st.active++;
            // trilinear stencil on the virtual grid, cell-centred
            if (!spec) load_stencil(u, o3, P, s.P3, pa, f, g, fl, fi, cv);
            bool saturated;
            const float wk = composite(s, cv, f, g, st.T, st.tau, saturated);
            if (REC && st.active <= kRecCap) {
                rec[st.active - 1] = make_float2(kk, wk);
                if (st.active == kRecCap) rec[kRecCap] = make_float2(st.T, st.tau);
            }
            accumulate_colour(st, cv, wk, f, g);
            if (PS) {
                // this sample's own decoded colour and features, then its residual
                float ck[7] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float tw = ((c & 4) ? f[2] : g[2]) * ((c & 2) ? f[1] : g[1]) * ((c & 1) ? f[0] : g[0]);
                    ck[0] = fmaf(tw, code(cv[c].x, 1), ck[0]);
                    ck[1] = fmaf(tw, code(cv[c].x, 2), ck[1]);
                    ck[2] = fmaf(tw, code(cv[c].x, 3), ck[2]);
                    ck[3] = fmaf(tw, code(cv[c].y, 0), ck[3]);
                    ck[4] = fmaf(tw, code(cv[c].y, 1), ck[4]);
                    ck[5] = fmaf(tw, code(cv[c].y, 2), ck[5]);
                    ck[6] = fmaf(tw, code(cv[c].y, 3), ck[6]);
                }
                const float inv255 = 1.0f / 255.0f;
                const float cdk[3] = {ck[0] * inv255, ck[1] * inv255, ck[2] * inv255};
                const float vk[4] = {ck[3] * inv255, ck[4] * inv255, ck[5] * inv255, ck[6] * inv255};
                float res[3];
                per_sample_residual(ps_w, ps_sw, cdk, vk, r.d, res);
#pragma unroll
                for (int c = 0; c < 3; ++c) st.rgb_ps[c] = fmaf(wk, cdk[c] + res[c], st.rgb_ps[c]);
            }
            if (GRAD) scatter_sample(s, slot, fi, o3, f, g, wk, gfeat, grad_atlas);
            if (saturated) {
                steps += kk - k + 1.0f;
                done = true;
                break;
            }
            kk += 1.0f;
            if (SPEC) k_spec = kk;
        }
        if (done) break;
        steps += kx - k;
        k = kx;
    }
    st.steps = (int)steps;
}

// ---------------------------------------------------------------------------------
// view-dependence MLP (Eq. 7): x = [C_d, V, d, sin/cos(2^l d), l = 0..3] -> 16 ReLU ->
// 16 ReLU -> 3 -> sigmoid, built to stay small in registers and code:
// weights sit in shared memory with W1 and W2 transposed (rows of 16 outputs, read with
// uniform 128-bit loads), the 34-float input row of each thread is staged in shared
// memory and streamed through a rolled loop, and the direction encoding takes one
// sincosf per axis and the double-angle identities for the higher octaves.
// Layout (floats): W1^T[34][16] | b1[16] | W2^T[16][16] | b2[16] | W3[3][16] | b3[3]
// (the offsets kOff* are those of the flat layout; only W1 and W2 are transposed).
// ---------------------------------------------------------------------------------
constexpr int kXStride = 35;   // per-thread input row stride in shared memory (odd: no bank conflicts)

__device__ __forceinline__ void load_mlp_smem_t(float* sW, const float* mlp) {
    const int nt = blockDim.x * blockDim.y;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    for (int i = tid; i < kNParam; i += nt) {
        int dst = i;
        if (i < kOffB1) {                     // W1[o][k] -> W1^T[k][o]
            const int o = i / kMlpIn, k = i % kMlpIn;
            dst = kOffW1 + k * kMlpH + o;
        } else if (i >= kOffW2 && i < kOffB2) {   // W2[o][k] -> W2^T[k][o]
            const int o = (i - kOffW2) / kMlpH, k = (i - kOffW2) % kMlpH;
            dst = kOffW2 + k * kMlpH + o;
        }
        sW[dst] = __ldg(mlp + i);
    }
}

__device__ __forceinline__ void fma16(float h[16], const float* w, float x) {
    const float4* w4 = reinterpret_cast<const float4*>(w);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 v = w4[q];
        h[4 * q + 0] = fmaf(v.x, x, h[4 * q + 0]);
        h[4 * q + 1] = fmaf(v.y, x, h[4 * q + 1]);
        h[4 * q + 2] = fmaf(v.z, x, h[4 * q + 2]);
        h[4 * q + 3] = fmaf(v.w, x, h[4 * q + 3]);
    }
}

__device__ __forceinline__ void load16(float h[16], const float* w) {
    const float4* w4 = reinterpret_cast<const float4*>(w);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 v = w4[q];
        h[4 * q + 0] = v.x;
        h[4 * q + 1] = v.y;
        h[4 * q + 2] = v.z;
        h[4 * q + 3] = v.w;
    }
}

// x = [C_d, V, d, sin(2^l d), cos(2^l d) for l = 0..3] written to the thread's row
__device__ __forceinline__ void stage_mlp_input(float* xrow, const float cd[3], const float v[4], const float d[3]) {
    xrow[0] = cd[0]; xrow[1] = cd[1]; xrow[2] = cd[2];
    xrow[3] = v[0]; xrow[4] = v[1]; xrow[5] = v[2]; xrow[6] = v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        xrow[7 + i] = d[i];
        float sv, cv;
        sincosf(d[i], &sv, &cv);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            xrow[10 + 6 * l + i] = sv;
            xrow[13 + 6 * l + i] = cv;
            const float s2 = 2.0f * sv * cv;          // sin 2a
            const float c2 = (cv - sv) * (cv + sv);   // cos 2a
            sv = s2;
            cv = c2;
        }
    }
}

__device__ __forceinline__ void mlp_residual(const float* sW, const float* xrow, float res[3]) {
    float h[16];
    load16(h, sW + kOffB1);
#pragma unroll 2
    for (int i = 0; i < kMlpIn; ++i) fma16(h, sW + kOffW1 + i * kMlpH, xrow[i]);
#pragma unroll
    for (int o = 0; o < 16; ++o) h[o] = fmaxf(h[o], 0.0f);
    float h2[16];
    load16(h2, sW + kOffB2);
#pragma unroll
    for (int i = 0; i < kMlpH; ++i) fma16(h2, sW + kOffW2 + i * kMlpH, h[i]);
#pragma unroll
    for (int o = 0; o < kMlpOut; ++o) {
        float w3[16];
        load16(w3, sW + kOffW3 + o * kMlpH);
        float acc = sW[kOffB3 + o];
#pragma unroll
        for (int i = 0; i < kMlpH; ++i) acc = fmaf(w3[i], fmaxf(h2[i], 0.0f), acc);
        res[o] = 1.0f / (1.0f + expf(-acc));
    }
}

// The same MLP with its 34 inputs taken from registers: C_d, V and d directly, the
// direction encoding generated in order (one sincosf per axis, double-angle identities
// for the higher octaves) and consumed as produced. Needs no shared-memory row.
__device__ __forceinline__ void mlp_residual_regs(const float* sW, const float cd[3], const float v[4],
                                                  const float d[3], float res[3]) {
    float h[16];
    load16(h, sW + kOffB1);
#pragma unroll
    for (int i = 0; i < 3; ++i) fma16(h, sW + kOffW1 + i * kMlpH, cd[i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) fma16(h, sW + kOffW1 + (3 + i) * kMlpH, v[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) fma16(h, sW + kOffW1 + (7 + i) * kMlpH, d[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float sv, cv;
        sincosf(d[i], &sv, &cv);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            fma16(h, sW + kOffW1 + (10 + 6 * l + i) * kMlpH, sv);
            fma16(h, sW + kOffW1 + (13 + 6 * l + i) * kMlpH, cv);
            const float s2 = 2.0f * sv * cv;          // sin 2a
            const float c2 = (cv - sv) * (cv + sv);   // cos 2a
            sv = s2;
            cv = c2;
        }
    }
#pragma unroll
    for (int o = 0; o < 16; ++o) h[o] = fmaxf(h[o], 0.0f);
    float h2[16];
    load16(h2, sW + kOffB2);
#pragma unroll
    for (int i = 0; i < kMlpH; ++i) fma16(h2, sW + kOffW2 + i * kMlpH, h[i]);
#pragma unroll
    for (int o = 0; o < kMlpOut; ++o) {
        float w3[16];
        load16(w3, sW + kOffW3 + o * kMlpH);
        float acc = sW[kOffB3 + o];
#pragma unroll
        for (int i = 0; i < kMlpH; ++i) acc = fmaf(w3[i], fmaxf(h2[i], 0.0f), acc);
        res[o] = 1.0f / (1.0f + expf(-acc));
    }
}

// Weights in the same transposed layout, passed by value as a kernel parameter (set with
// snerg_set_mlp). The kernel then reads every weight as a constant-bank operand of its
// FMA: no load, no latency, no registers -- the GPU counterpart of the paper's viewer,
// whose shader has the network biases compiled in (App. A).
struct MlpWeights {
    float w[kNParam + 1];
};

// Packed FP32 pairs (sm_100+ f32x2 FMA): two hidden units per instruction.
__device__ __forceinline__ void fma16_pairs(float2 h[8], const float* w, float x) {
    const float2 xx = make_float2(x, x);
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = __ffma2_rn(make_float2(w[2 * q], w[2 * q + 1]), xx, h[q]);
}

__device__ __forceinline__ void mlp_residual_param(const MlpWeights& W, const float cd[3], const float v[4],
                                                   const float d[3], float res[3]) {
    float2 h[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = make_float2(W.w[kOffB1 + 2 * q], W.w[kOffB1 + 2 * q + 1]);
    const float x[10] = {cd[0], cd[1], cd[2], v[0], v[1], v[2], v[3], d[0], d[1], d[2]};
#pragma unroll
    for (int i = 0; i < 10; ++i) fma16_pairs(h, W.w + kOffW1 + i * kMlpH, x[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float sv, cv;
        sincosf(d[i], &sv, &cv);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            fma16_pairs(h, W.w + kOffW1 + (10 + 6 * l + i) * kMlpH, sv);
            fma16_pairs(h, W.w + kOffW1 + (13 + 6 * l + i) * kMlpH, cv);
            const float s2 = 2.0f * sv * cv;          // sin 2a
            const float c2 = (cv - sv) * (cv + sv);   // cos 2a
            sv = s2;
            cv = c2;
        }
    }
    float2 h2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) h2[q] = make_float2(W.w[kOffB2 + 2 * q], W.w[kOffB2 + 2 * q + 1]);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        fma16_pairs(h2, W.w + kOffW2 + (2 * q) * kMlpH, fmaxf(h[q].x, 0.0f));
        fma16_pairs(h2, W.w + kOffW2 + (2 * q + 1) * kMlpH, fmaxf(h[q].y, 0.0f));
    }
#pragma unroll
    for (int o = 0; o < kMlpOut; ++o) {
        float2 acc = make_float2(W.w[kOffB3 + o], 0.0f);
#pragma unroll
        for (int q = 0; q < 8; ++q)
            acc = __ffma2_rn(make_float2(W.w[kOffW3 + o * kMlpH + 2 * q], W.w[kOffW3 + o * kMlpH + 2 * q + 1]),
                             make_float2(fmaxf(h2[q].x, 0.0f), fmaxf(h2[q].y, 0.0f)), acc);
        res[o] = 1.0f / (1.0f + expf(-(acc.x + acc.y)));
    }
}

__device__ __forceinline__ void per_sample_residual(const MlpWeights* pw, const float* sW, const float cd[3],
                                                    const float v[4], const float d[3], float res[3]) {
    if (pw) mlp_residual_param(*pw, cd, v, d, res);
    else mlp_residual_regs(sW, cd, v, d, res);
}

// Finish one ray: colour = C_d + residual + T bg (residual only if something was
// composited). sW: weights in the transposed layout of load_mlp_smem_t; xrow: this
// thread's kXStride-float row of shared memory to stage the MLP input in, or nullptr to
// evaluate the MLP from registers.
__device__ __forceinline__ void finish_ray(const DevScene& s, const float* sW, float* xrow, const Ray& r,
                                           const MarchState& st, float rgb[3], float aux[kAuxCh],
                                           const MlpWeights* pw = nullptr) {
    const float inv255 = 1.0f / 255.0f;
    float cd[3], v[4];
#pragma unroll
    for (int c = 0; c < 3; ++c) cd[c] = st.acc[c] * inv255;
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = st.acc[3 + c] * inv255;
#pragma unroll
    for (int c = 0; c < 3; ++c) aux[c] = cd[c];
#pragma unroll
    for (int c = 0; c < 4; ++c) aux[3 + c] = v[c];
    aux[7] = 1.0f - st.T;
    float T = st.T;
    if (s.flags & SNERG_FLAG_UNPREMULTIPLY) {
        const float sc = unpremultiply_scale(s, st.T);
#pragma unroll
        for (int c = 0; c < 3; ++c) cd[c] *= sc;
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] *= sc;
        T = 1.0f - (1.0f - st.T) * sc;
    }
    float res[3] = {0.0f, 0.0f, 0.0f};
    if (s.flags & SNERG_FLAG_PER_SAMPLE_MLP) {
#pragma unroll
        for (int c = 0; c < 3; ++c) res[c] = st.rgb_ps[c];
    } else if (st.active > 0 && (s.flags & SNERG_FLAG_NO_MLP)) {
#pragma unroll
        for (int c = 0; c < 3; ++c) res[c] = cd[c];
    } else if (st.active > 0) {
        float m[3];
        if (pw) {
            mlp_residual_param(*pw, cd, v, r.d, m);
        } else if (xrow) {
            stage_mlp_input(xrow, cd, v, r.d);
            mlp_residual(sW, xrow, m);
        } else {
            mlp_residual_regs(sW, cd, v, r.d, m);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) res[c] = cd[c] + m[c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) rgb[c] = res[c] + T * s.bg[c];
}

__device__ __forceinline__ void record_status(const DevScene& s, const MarchState& st) {
    if (st.limit) atomicCAS(s.status, 0, kStatusStepLimit);
}

// ---------------------------------------------------------------------------------
// host-side launchers (defined in the .cu files)
// ---------------------------------------------------------------------------------
struct DebugOut {
    float* aux;
    int32_t* counts;
    uint64_t* trace;
    int32_t trace_cap;
};

// Tile schedule from the previous frame (snerg_render_opts.schedule): the image's 16x8
// tiles in cost buckets, bucket = 3 log2(the tile's CTA duration / 250 ns) clamped to
// [0, 32). Bucket b's tiles are list[b * cap + 0 .. count[b]). A set's header (int32
// words) holds the 32 counts, the launch's first CTA start (uint64 %globaltimer, stored
// complemented so that an atomic max over a zeroed word finds the minimum) and its last CTA
// end, then per sparse slot the slowest quarter's duration and the quarters done.
constexpr int kSchedBuckets = 32;
constexpr int kSchedMaxTiles = SNERG_SCHEDULE_MAX_TILES;
constexpr int kSchedMaxSparse = 256;      // tiles one launch may render sparsely
constexpr float kSchedSparseFrac = 0.7f;  // ... those that took >= this fraction of the frame
constexpr float kSchedSparseGain = 1.5f;  // a sparse tile's cost is recorded as its slowest quarter x this
constexpr int kSchedHdrTimes = kSchedBuckets;                 // word offsets in a set's header
constexpr int kSchedHdrSlotMax = kSchedHdrTimes + 4;
constexpr int kSchedHdrSlotCnt = kSchedHdrSlotMax + kSchedMaxSparse;
constexpr int kSchedHdrInfo = kSchedHdrSlotCnt + kSchedMaxSparse;   // tiles rendered sparsely + 1, and
                                                                    // 1 if the previous order was used
constexpr int kSchedHdrWords = kSchedHdrInfo + 2;
struct SchedArgs {
    const int32_t* rd_count;   // the previous frame's buckets and times (nullptr: raster order)
    const int32_t* rd_list;
    int32_t* wr_count;         // this frame's (header zeroed before the launch)
    int32_t* wr_list;
    int32_t cap;               // list capacity per bucket (>= the image's tiles)
    int32_t nt;                // the image's tiles
    int32_t tiles_x;
    int32_t smax;              // sparse slots of this launch (0 without previous buckets)
};

// pw: weights as a kernel parameter (nullptr: read them from `mlp` in device memory)
// sch: nullable; with it the launch takes its tile order from the previous frame's
// buckets and records its own tile costs (deferred model, all rows, no debug outputs)
cudaError_t launch_render_image(const DevScene& s, const snerg_camera& cam, const float* mlp, const MlpWeights* pw,
                                float* rgb, const DebugOut& dbg, cudaStream_t st, int row0, int row1,
                                const SchedArgs* sch = nullptr);
cudaError_t launch_render_rays(const DevScene& s, const CamTable& cams, int32_t n_cams, const int32_t* pix,
                               int64_t n, const float* mlp, const MlpWeights* pw, float* rgb, const DebugOut& dbg,
                               int num_sms, cudaStream_t st);
cudaError_t launch_backward_rays(const DevScene& s, const CamTable& cams, int32_t n_cams, const int32_t* pix, int64_t n,
                                 const float* mlp, const float* grad_rgb, const float* fwd_aux,
                                 const int32_t* fwd_counts, float* grad_atlas, float* grad_mlp, cudaStream_t st);
cudaError_t launch_validate(const int32_t* ind, int64_t n_ind, int64_t nb, int32_t* blk_of_slot, int32_t* err,
                            cudaStream_t st);
cudaError_t launch_build_padded(const int32_t* ind, const int32_t* blk_of_slot, const uint8_t* atlas, int64_t nb,
                                int N, int B, int lgB, uint2* patlas, cudaStream_t st);
// Chebyshev distance maps (three separable passes, distances capped at `cap`):
// block level over the G^3 indirection grid, voxel level inside each stored block.
// The render maps are per octant of the ray direction (distances inside its cone).
cudaError_t launch_block_distance(const int32_t* ind, int G, int cap, uint8_t* tmp0, uint8_t* tmp1,
                                  uint8_t* bdist, cudaStream_t st);
cudaError_t launch_block_distance_octants(const int32_t* ind, int G, int cap, uint8_t* tmp0, uint8_t* tmp1,
                                          uint8_t* bdist, int32_t* ind_oct, cudaStream_t st);
cudaError_t launch_voxel_distance_octants(const uint8_t* atlas, int64_t nb, int B, uint8_t* scratch, uint8_t* vskip,
                                          cudaStream_t st);
cudaError_t launch_fill_vskip_border(uint8_t* vskip, const int32_t* blk_of_slot, int64_t nb, int N, int B, int lgB,
                                     int n_planes, cudaStream_t st);

struct PersistentParams {
    snerg_camera cams[kMaxCams];
    int32_t tile_start[kMaxCams + 1];   // prefix sum of work items per camera
    int32_t tiles_x[kMaxCams];
    int32_t n_cams;
    int32_t total_items;
    int32_t tile_w, tile_h;             // pixels per work item (tile_w * tile_h % 32 == 0)
    int32_t warp_w, warp_h;             // pixels per warp pass (warp_w * warp_h == 32)
};

cudaError_t launch_render_persistent(const DevScene& s, const PersistentParams& p, const float* mlp,
                                     const MlpWeights* pw, float* rgb, int32_t* queue, int grid, int block,
                                     cudaStream_t st);
// the persistent kernel for weights as parameters or in device memory, and for work items
// of one warp pass or several (multi)
const void* persistent_kernel_fn(bool param_weights, bool multi);

}  // namespace snerg
