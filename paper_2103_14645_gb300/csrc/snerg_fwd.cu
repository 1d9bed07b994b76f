// snerg_fwd.cu -- forward render kernels: one camera per launch, ray lists, and the
// persistent multi-camera kernel that drains a (camera, tile) work queue.
// The per-ray arithmetic is in snerg_internal.cuh (Sec. 5.2, App. A; Eqs. 2, 5-7).
//
// Every kernel comes in two flavours for the view-dependence MLP (Eq. 7): PW = true
// reads the weights from the kernel parameter `pw` (constant-bank operands; set with
// snerg_set_mlp), PW = false stages them from device memory into shared memory (the
// form the autograd path uses, where the weights live in a tensor).
#include "snerg_internal.cuh"

namespace snerg {

// Each warp covers an 8x4 pixel packet, so its 32 rays are neighbours on screen and walk
// neighbouring voxels together. A CTA holds NW warps (1: 8x4, 2: 16x4, 4: 16x8 pixels);
// small CTAs free their SM slot as soon as their own packets are done, which matters
// because packets on the object take several times longer than background packets.
template <int NW>
struct ImageTile {
    static constexpr int WX = NW >= 2 ? 2 : 1;      // warps across
    static constexpr int WY = NW >= 4 ? 2 : 1;      // warps down
    static constexpr int TW = 8 * WX, TH = 4 * WY;  // CTA tile in pixels
};

// SCHED: the launch's CTAs take the image's tiles in the order of the previous frame's
// cost buckets (slowest first). The slowest tiles -- those whose recorded cost is at least
// kSchedSparseFrac of the previous frame's time, at most smax of them -- are rendered
// sparsely: four CTAs per tile, each CTA two of its eight rows, 8 rays per warp, so that
// their long chains of dependent loads run with less divergence beside them. Launch index
// c < 4 smax: quarter c % 4 of sparse tile c / 4 (idle if there are fewer); c >= 4 smax:
// the next tile in order, rendered as usual. The pixels of every tile are rendered once,
// whatever the order and mapping. Each CTA records its duration when all its warps are
// done (a sparse tile by its last quarter to finish, as its slowest quarter times
// kSchedSparseGain: about its dense cost, so that it stays sparse while it stays slow) and
// the launch's start and end. The grid is nt + 4 smax CTAs: 4 smax sparse slots (S <= smax
// used), then nt dense slots for the tiles S .. nt - 1 of the order (the last S idle).
struct SchedSlot {
    int tile;       // -1: idle
    int quarter;    // -1: dense
};

__device__ __forceinline__ SchedSlot sched_map(const SchedArgs& sch, int c, unsigned long long* t0) {
    __shared__ SchedSlot s_slot;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (lane == 0) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            *t0 = t;
        }
        int incl = 0, c_b = 0, S = 0;
        bool use = false;
        const int b = kSchedBuckets - 1 - lane;          // lane 0: the slowest bucket
        if (sch.rd_count) {
            c_b = __ldg(sch.rd_count + b);
            incl = c_b;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            // the buckets are used only when they hold exactly this launch's tiles
            use = __shfl_sync(0xffffffffu, incl, 31) == sch.nt;
            if (use && sch.smax > 0) {
                const unsigned long long* tw = reinterpret_cast<const unsigned long long*>(sch.rd_count + kSchedHdrTimes);
                const float T = (float)(__ldg(tw + 1) - ~__ldg(tw));        // the previous frame's time
                const int bthr = (int)ceilf(3.0f * __log2f(fmaxf(kSchedSparseFrac * T, 250.0f) * (1.0f / 250.0f)));
                if (bthr < kSchedBuckets)
                    S = min(sch.smax, __shfl_sync(0xffffffffu, incl, kSchedBuckets - 1 - max(bthr, 0)));
            }
        }
        int item = -1, q = -1;
        if (c < 4 * sch.smax) {
            if ((c >> 2) < S) {
                item = c >> 2;
                q = c & 3;
            }
        } else {
            item = S + (c - 4 * sch.smax);
            if (item >= sch.nt) item = -1;
        }
        if (lane == 0) {
            s_slot = SchedSlot{use ? -1 : item, q};
            if (c == 0) {           // what this launch did, for snerg_schedule_stats
                sch.wr_count[kSchedHdrInfo] = S + 1;
                sch.wr_count[kSchedHdrInfo + 1] = use ? 1 : 0;
            }
        }
        __syncwarp();
        const int excl = incl - c_b;
        if (use && item >= 0 && item >= excl && item < incl && item - excl < sch.cap)
            s_slot.tile = __ldg(sch.rd_list + (size_t)b * sch.cap + (item - excl));
    }
    __syncthreads();
    return s_slot;
}

__device__ __forceinline__ void sched_record(const SchedArgs& sch, const SchedSlot& sl, const unsigned long long* t0) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        unsigned long long* tw = reinterpret_cast<unsigned long long*>(sch.wr_count + kSchedHdrTimes);
        atomicMax(tw, ~*t0);
        atomicMax(tw + 1, t1);
        float ns = (float)(t1 - *t0);
        bool rec = sl.tile >= 0 && sl.quarter < 0;
        if (sl.tile >= 0 && sl.quarter >= 0) {
            // sparse: the last of the tile's four quarters records the slowest one
            const int j = (int)(blockIdx.x >> 2);
            unsigned int* qmax = reinterpret_cast<unsigned int*>(sch.wr_count + kSchedHdrSlotMax);
            int* qcnt = sch.wr_count + kSchedHdrSlotCnt;
            atomicMax(qmax + j, (unsigned int)min(t1 - *t0, 0xffffffffull));
            __threadfence();
            if (atomicAdd(qcnt + j, 1) == 3) {
                ns = (float)atomicMax(qmax + j, 0u) * kSchedSparseGain;
                rec = true;
            }
        }
        if (rec) {
            const int b = min(max((int)(3.0f * __log2f(fmaxf(ns, 1.0f) * (1.0f / 250.0f))), 0), kSchedBuckets - 1);
            const int pos = atomicAdd(sch.wr_count + b, 1);
            if (pos < sch.cap) sch.wr_list[(size_t)b * sch.cap + pos] = sl.tile;
        }
    }
}

// one pixel of render_image_kernel: march, MLP, store (and the debug outputs)
template <bool DBG, bool PS>
__device__ __forceinline__ void image_pixel(const DevScene& s, const snerg_camera& cam, const float* sW,
                                            const MlpWeights* pwp, float* __restrict__ rgb, const DebugOut& dbg,
                                            int px, int py) {
    const Ray r = make_ray(s, cam, px, py);
    const int64_t pix = cam.out_offset + (int64_t)py * cam.W + px;
    MarchState st;
    int k_first = 0;
    if (DBG && dbg.trace)
        march<true, false, PS>(s, r, st, dbg.trace + pix * dbg.trace_cap, dbg.trace_cap, nullptr, nullptr, 0,
                               &k_first, pwp, sW);
    else
        march<false, false, PS>(s, r, st, nullptr, 0, nullptr, nullptr, 0, DBG ? &k_first : nullptr, pwp, sW);
    record_status(s, st);
    float c[3], aux[kAuxCh];
    finish_ray(s, sW, nullptr, r, st, c, aux, pwp);
    rgb[pix * 3 + 0] = c[0];
    rgb[pix * 3 + 1] = c[1];
    rgb[pix * 3 + 2] = c[2];
    if (DBG) {
        if (dbg.aux)
            for (int k = 0; k < kAuxCh; ++k) dbg.aux[pix * kAuxCh + k] = aux[k];
        if (dbg.counts) {
            dbg.counts[pix * 4] = st.steps;
            dbg.counts[pix * 4 + 1] = st.active;
            dbg.counts[pix * 4 + 2] = st.blocks;
            dbg.counts[pix * 4 + 3] = st.active > 0 ? k_first : -1;
        }
    }
}

template <bool DBG, bool PW, int NW, bool PS, bool SCHED = false>
__global__ void __launch_bounds__(32 * NW, 32 / NW) render_image_kernel(const DevScene s, const snerg_camera cam,
                                                                        const float* __restrict__ mlp,
                                                                        const __grid_constant__ MlpWeights pw,
                                                                        float* __restrict__ rgb, const DebugOut dbg,
                                                                        int row0, int row1, const SchedArgs sch) {
    __shared__ __align__(16) float sW[PW ? 4 : kNParam + 1];
    if (!PW) {
        load_mlp_smem_t(sW, mlp);
        __syncthreads();
    }
    const MlpWeights* pwp = PW ? &pw : nullptr;
    using T = ImageTile<NW>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (SCHED) {
        static_assert(NW == 4, "the sparse mapping assumes 16x8 tiles of four 8x4 warps");
        __shared__ unsigned long long s_t0;
        const SchedSlot sl = sched_map(sch, (int)blockIdx.x, &s_t0);
        if (sl.tile >= 0) {
            const int tx = sl.tile % sch.tiles_x, ty = sl.tile / sch.tiles_x;
            int px, py;
            bool on = true;
            if (sl.quarter < 0) {
                px = tx * T::TW + (warp % T::WX) * 8 + (lane & 7);
                py = ty * T::TH + (warp / T::WX) * 4 + (lane >> 3);
            } else {
                const int idx = warp * 8 + (lane & 7);            // 0..31: rows 2q, 2q + 1
                on = lane < 8;
                px = tx * T::TW + (idx & 15);
                py = ty * T::TH + 2 * sl.quarter + (idx >> 4);
            }
            if (on && px < cam.W && py < row1) image_pixel<DBG, PS>(s, cam, sW, pwp, rgb, dbg, px, py);
        }
        sched_record(sch, sl, &s_t0);
    } else {
        const int px = blockIdx.x * T::TW + (warp % T::WX) * 8 + (lane & 7);
        const int py = row0 + blockIdx.y * T::TH + (warp / T::WX) * 4 + (lane >> 3);
        if (px >= cam.W || py >= row1) return;
        image_pixel<DBG, PS>(s, cam, sW, pwp, rgb, dbg, px, py);
    }
}

// MINB: resident CTAs per SM the build is limited to (8: 64 registers; 4: up to 128)
template <bool DBG, bool PW, int MINB>
__global__ void __launch_bounds__(128, MINB) render_rays_kernel(const DevScene s, const __grid_constant__ CamTable cams,
                                                                int32_t n_cams, const int32_t* __restrict__ pix,
                                                                int64_t n, const float* __restrict__ mlp,
                                                                const __grid_constant__ MlpWeights pw,
                                                                float* __restrict__ rgb, const DebugOut dbg) {
    __shared__ __align__(16) float sW[PW ? 4 : kNParam + 1];
    if (!PW) {
        load_mlp_smem_t(sW, mlp);
        __syncthreads();
    }
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
    int k_first = 0;
    if (DBG && dbg.trace)
        march<true, false>(s, r, st, dbg.trace + i * dbg.trace_cap, dbg.trace_cap, nullptr, nullptr, 0, &k_first);
    else
        march<false, false, false, true>(s, r, st, nullptr, 0, nullptr, nullptr, 0, DBG ? &k_first : nullptr);
    record_status(s, st);
    float c[3], aux[kAuxCh];
    finish_ray(s, sW, nullptr, r, st, c, aux, PW ? &pw : nullptr);
    rgb[i * 3 + 0] = c[0];
    rgb[i * 3 + 1] = c[1];
    rgb[i * 3 + 2] = c[2];
    if (DBG) {
        if (dbg.aux)
            for (int k = 0; k < kAuxCh; ++k) dbg.aux[i * kAuxCh + k] = aux[k];
        if (dbg.counts) {
            dbg.counts[i * 4] = st.steps;
            dbg.counts[i * 4 + 1] = st.active;
            dbg.counts[i * 4 + 2] = st.blocks;
            dbg.counts[i * 4 + 3] = st.active > 0 ? k_first : -1;
        }
    }
}

// Persistent multi-camera render: gridDim = SMs x CTAs/SM. Each warp pulls work items
// (tile_w x tile_h pixels of one camera) from a global counter until the queue is empty,
// and renders each item in warp_w x warp_h packets of 32 rays. The counter is zeroed by
// the launch sequence (a memset node of the captured graph) before every launch.
// One pixel of the persistent launch: march, shade and store.
template <bool PW>
__device__ __forceinline__ void persistent_pixel(const DevScene& s, const snerg_camera& cam, const float* sW,
                                                 const MlpWeights& pw, float* rgb, int px, int py) {
    // the output row before the march, so that only it stays live across it
    float* out = rgb + (cam.out_offset + (int64_t)py * cam.W + px) * 3;
    const Ray r = make_ray(s, cam, px, py);
    MarchState st;
    march<false, false>(s, r, st, nullptr, 0, nullptr, nullptr);
    record_status(s, st);
    float c[3], aux[kAuxCh];
    finish_ray(s, sW, nullptr, r, st, c, aux, PW ? &pw : nullptr);
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
}

// MULTI: a work item is several warp passes (tile_w x tile_h larger than warp_w x
// warp_h); without it an item is exactly one warp pass and no pass loop stays live across
// the march.
template <bool PW, bool MULTI>
__global__ void __launch_bounds__(128, 8) render_persistent_kernel(const DevScene s,
                                                                   const __grid_constant__ PersistentParams p,
                                                                   const float* __restrict__ mlp,
                                                                   const __grid_constant__ MlpWeights pw,
                                                                   float* __restrict__ rgb,
                                                                   int32_t* __restrict__ queue) {
    __shared__ __align__(16) float sW[PW ? 4 : kNParam + 1];
    if (!PW) {
        load_mlp_smem_t(sW, mlp);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(queue, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= p.total_items) break;
        int lo = 0, hi = p.n_cams;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (p.tile_start[mid] <= item) lo = mid; else hi = mid;
        }
        const snerg_camera& cam = p.cams[lo];
        const int rem = item - p.tile_start[lo];
        const int tx = rem % p.tiles_x[lo], ty = rem / p.tiles_x[lo];
        const int lx = lane % p.warp_w, ly = lane / p.warp_w;
        if (MULTI) {
            const int passes_x = p.tile_w / p.warp_w;
            const int passes = passes_x * (p.tile_h / p.warp_h);
            for (int ps = 0; ps < passes; ++ps) {
                const int px = tx * p.tile_w + (ps % passes_x) * p.warp_w + lx;
                const int py = ty * p.tile_h + (ps / passes_x) * p.warp_h + ly;
                if (px < cam.W && py < cam.H) persistent_pixel<PW>(s, cam, sW, pw, rgb, px, py);
            }
        } else {
            const int px = tx * p.warp_w + lx;
            const int py = ty * p.warp_h + ly;
            if (px < cam.W && py < cam.H) persistent_pixel<PW>(s, cam, sW, pw, rgb, px, py);
        }
    }
}

constexpr int kImageWarps = 4;     // warps per CTA of the one-camera launch

static const MlpWeights& no_weights() {
    static const MlpWeights z = {};
    return z;
}

template <bool PS>
static void image_launch(const DevScene& s, const snerg_camera& cam, const float* mlp, const MlpWeights* pw,
                         float* rgb, const DebugOut& dbg, cudaStream_t st, int row0, int row1, const SchedArgs* sch) {
    using T = ImageTile<kImageWarps>;
    dim3 grid((cam.W + T::TW - 1) / T::TW, (row1 - row0 + T::TH - 1) / T::TH);
    const int nt = 32 * kImageWarps;
    const bool d = dbg.aux || dbg.counts || dbg.trace;
    const MlpWeights& w = pw ? *pw : no_weights();
    const SchedArgs none{nullptr, nullptr, nullptr, nullptr, 0};
    if (!PS && !d && sch) {
        const dim3 g1((unsigned)(sch->nt + 4 * sch->smax));   // 4 smax sparse slots, then nt dense ones
        if (pw) render_image_kernel<false, true, kImageWarps, false, true><<<g1, nt, 0, st>>>(s, cam, mlp, w, rgb, dbg,
                                                                                            row0, row1, *sch);
        else render_image_kernel<false, false, kImageWarps, false, true><<<g1, nt, 0, st>>>(s, cam, mlp, w, rgb, dbg,
                                                                                              row0, row1, *sch);
        return;
    }
    if (pw) {
        if (d) render_image_kernel<true, true, kImageWarps, PS><<<grid, nt, 0, st>>>(s, cam, mlp, w, rgb, dbg, row0, row1, none);
        else render_image_kernel<false, true, kImageWarps, PS><<<grid, nt, 0, st>>>(s, cam, mlp, w, rgb, dbg, row0, row1, none);
    } else {
        if (d) render_image_kernel<true, false, kImageWarps, PS><<<grid, nt, 0, st>>>(s, cam, mlp, w, rgb, dbg, row0, row1, none);
        else render_image_kernel<false, false, kImageWarps, PS><<<grid, nt, 0, st>>>(s, cam, mlp, w, rgb, dbg, row0, row1, none);
    }
}

// rows [row0, row1) of the camera (clamped to [0, H]); all rows when row1 <= row0 after clamping
cudaError_t launch_render_image(const DevScene& s, const snerg_camera& cam, const float* mlp, const MlpWeights* pw,
                                float* rgb, const DebugOut& dbg, cudaStream_t st, int row0, int row1,
                                const SchedArgs* sch) {
    row0 = max(row0, 0);
    row1 = min(row1, cam.H);
    if (cam.W <= 0 || row1 <= row0) return cudaSuccess;
    if (s.flags & SNERG_FLAG_PER_SAMPLE_MLP) image_launch<true>(s, cam, mlp, pw, rgb, dbg, st, row0, row1, nullptr);
    else image_launch<false>(s, cam, mlp, pw, rgb, dbg, st, row0, row1, sch);
    return cudaGetLastError();
}

template <int MINB>
static void rays_launch(const DevScene& s, const CamTable& cams, int32_t n_cams, const int32_t* pix, int64_t n,
                        const float* mlp, const MlpWeights* pw, float* rgb, const DebugOut& dbg, cudaStream_t st) {
    const unsigned grid = (unsigned)((n + 127) / 128);
    const bool d = dbg.aux || dbg.counts || dbg.trace;
    const MlpWeights& w = pw ? *pw : no_weights();
    if (pw) {
        if (d) render_rays_kernel<true, true, MINB><<<grid, 128, 0, st>>>(s, cams, n_cams, pix, n, mlp, w, rgb, dbg);
        else render_rays_kernel<false, true, MINB><<<grid, 128, 0, st>>>(s, cams, n_cams, pix, n, mlp, w, rgb, dbg);
    } else {
        if (d) render_rays_kernel<true, false, MINB><<<grid, 128, 0, st>>>(s, cams, n_cams, pix, n, mlp, w, rgb, dbg);
        else render_rays_kernel<false, false, MINB><<<grid, 128, 0, st>>>(s, cams, n_cams, pix, n, mlp, w, rgb, dbg);
    }
}

// A ray list that fits one wave of 4 CTAs per SM runs the build limited to 4 (the march
// keeps its state in registers, and a single wave gains nothing from the 8-CTA
// occupancy); longer lists keep 8 CTAs per SM to hide the march's latencies.
cudaError_t launch_render_rays(const DevScene& s, const CamTable& cams, int32_t n_cams, const int32_t* pix,
                               int64_t n, const float* mlp, const MlpWeights* pw, float* rgb, const DebugOut& dbg,
                               int num_sms, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if ((n + 127) / 128 <= 4 * (int64_t)num_sms) rays_launch<4>(s, cams, n_cams, pix, n, mlp, pw, rgb, dbg, st);
    else rays_launch<8>(s, cams, n_cams, pix, n, mlp, pw, rgb, dbg, st);
    return cudaGetLastError();
}

static bool persistent_multi(const PersistentParams& p) { return p.tile_w != p.warp_w || p.tile_h != p.warp_h; }

cudaError_t launch_render_persistent(const DevScene& s, const PersistentParams& p, const float* mlp,
                                     const MlpWeights* pw, float* rgb, int32_t* queue, int grid, int block,
                                     cudaStream_t st) {
    const void* fn = persistent_kernel_fn(pw != nullptr, persistent_multi(p));
    const MlpWeights& w = pw ? *pw : no_weights();
    void* args[] = {(void*)&s, (void*)&p, (void*)&mlp, (void*)&w, (void*)&rgb, (void*)&queue};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, 0, st);
}

const void* persistent_kernel_fn(bool param_weights, bool multi) {
    if (param_weights)
        return multi ? (const void*)render_persistent_kernel<true, true> : (const void*)render_persistent_kernel<true, false>;
    return multi ? (const void*)render_persistent_kernel<false, true> : (const void*)render_persistent_kernel<false, false>;
}

}  // namespace snerg
