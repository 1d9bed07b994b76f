// snerg_api.cu -- host side of the C ABI declared in include/snerg.h.
//
// Validates arguments, lays out the caller's workspace, launches the kernels of
// snerg_prep.cu / snerg_fwd.cu / snerg_bwd.cu on the caller's stream, and owns the
// host state of the persistent multi-camera path: the autotuned launch shape and the
// CUDA graphs (work-queue reset + persistent kernel) that are captured once per shape
// and replayed with updated kernel parameters.
#include <cuda_runtime.h>

#include <chrono>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "snerg_internal.cuh"

using namespace snerg;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

struct Layout {
    size_t ind, bdist, btmp, blk, vskip, patlas, sched, total;
};

// tile schedule (snerg_render_opts.schedule): two sets (the previous frame's and this
// frame's) of kSchedBuckets counts and kSchedBuckets x kSchedMaxTiles tile lists
constexpr size_t kSchedCountBytes = 4096;            // a set's header: kSchedHdrWords int32 words
static_assert(kSchedHdrWords * 4 <= kSchedCountBytes, "schedule header");
constexpr size_t kSchedSetBytes = kSchedCountBytes + (size_t)kSchedBuckets * kSchedMaxTiles * 4;

constexpr int kBlockDistCap = 32;   // block-level distances are capped (a smaller box is still empty)

int ilog2_exact(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return (1 << l) == v ? l : -1;
}

bool finite3(const float* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

bool desc_ok(const snerg_scene_desc* d) {
    if (!d) return false;
    if (d->N < 1 || d->N > 16384) return false;
    if (d->B < 2 || d->B > 64 || ilog2_exact(d->B) < 0 || d->N % d->B != 0) return false;
    if (d->N / d->B > 1024) return false;
    if (!(std::isfinite(d->extent) && d->extent > 0.0f)) return false;
    if (!(std::isfinite(d->sigma_max) && d->sigma_max >= 0.0f)) return false;
    if (d->max_steps < 0) return false;
    if (d->flags & ~(SNERG_FLAG_UNPREMULTIPLY | SNERG_FLAG_PER_SAMPLE_MLP | SNERG_FLAG_ALPHA_ATLAS |
                     SNERG_FLAG_NO_MLP))
        return false;
    if ((d->flags & SNERG_FLAG_UNPREMULTIPLY) && (d->flags & SNERG_FLAG_PER_SAMPLE_MLP)) return false;
    if ((d->flags & SNERG_FLAG_NO_MLP) && (d->flags & SNERG_FLAG_PER_SAMPLE_MLP)) return false;
    return finite3(d->bmin) && finite3(d->bg);
}

bool make_layout(const snerg_scene_desc* d, int64_t nb, Layout* L) {
    if (!desc_ok(d) || nb < 0 || nb > (int64_t)1 << 31) return false;
    const int64_t G = d->N / d->B;
    const int64_t P = d->B + 2;
    const size_t P3 = (size_t)(P * P * P);
    const size_t G3 = (size_t)(G * G * G);
    L->ind = kAlign;                                          // [0, 256): header words
    L->bdist = align_up(L->ind + 8 * G3 * 4);                 // one indirection copy per octant
    L->btmp = align_up(L->bdist + G3);                        // 2 G^3 scratch (set-up only)
    L->blk = align_up(L->btmp + 2 * G3);
    L->vskip = align_up(L->blk + (size_t)nb * 4);
    L->patlas = align_up(L->vskip + 8 * (size_t)nb * P3);    // one voxel plane per octant
    L->sched = align_up(L->patlas + (size_t)nb * P3 * 8);
    L->total = align_up(L->sched + 2 * kSchedSetBytes);
    return true;
}

// header word indices (int32)
constexpr int kHdrStatus = 0;
constexpr int kHdrCreateErr = 1;
constexpr int kHdrQueue = 16;    // own 64-byte line

bool camera_ok(const snerg_camera& c) {
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(c.c2w[i])) return false;
    if (!(std::isfinite(c.fx) && std::isfinite(c.fy) && std::isfinite(c.cx) && std::isfinite(c.cy))) return false;
    if (c.fx == 0.0f || c.fy == 0.0f) return false;
    if (c.W < 0 || c.H < 0 || c.out_offset < 0) return false;
    return true;
}

struct PersistentConfig {
    int warp_w, warp_h, passes, block, ctas_per_sm;
    int tile_w() const { return warp_w; }
    int tile_h() const { return warp_h * passes; }
    bool operator<(const PersistentConfig& o) const {
        return std::tie(warp_w, warp_h, passes, block, ctas_per_sm) <
               std::tie(o.warp_w, o.warp_h, o.passes, o.block, o.ctas_per_sm);
    }
};

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t knode = nullptr;
};

}  // namespace

struct snerg_scene {
    snerg_scene_desc desc;
    int64_t nb = 0;
    DevScene ds;
    uint8_t* ws = nullptr;
    int32_t* hdr = nullptr;
    int64_t launches = 0;
    int num_sms = 1;
    cudaStream_t cap_stream = nullptr;
    std::map<std::vector<int32_t>, PersistentConfig> tuned;   // key: camera sizes
    std::map<std::pair<PersistentConfig, bool>, GraphEntry> graphs;   // key: shape, weights-as-parameters
    PersistentConfig last{0, 0, 0, 0, 0};
    MlpWeights host_w;        // snerg_set_mlp: weights in the transposed kernel layout
    bool has_w = false;
    // tile schedule: the image size whose tile costs set `sched_set` holds (valid after the
    // first schedule = 1 render of that size)
    int32_t sched_w = 0, sched_h = 0;
    int sched_set = 0;
    bool sched_valid = false;
    std::vector<cudaStream_t> band_streams;   // snerg_render_to_host: one per band
    std::vector<cudaEvent_t> band_done;
    cudaEvent_t band_fork = nullptr;
};

extern "C" size_t snerg_workspace_bytes(const snerg_scene_desc* desc, int64_t num_blocks) {
    Layout L;
    if (!make_layout(desc, num_blocks, &L)) return 0;
    return L.total;
}

extern "C" snerg_status snerg_create(const snerg_scene_desc* desc, const int32_t* d_indirection,
                                     const uint8_t* d_atlas, int64_t num_blocks, void* d_workspace,
                                     size_t ws_bytes, void* stream, snerg_handle* out) {
    if (!out) return SNERG_E_INVAL;
    *out = nullptr;
    Layout L;
    if (!make_layout(desc, num_blocks, &L)) return SNERG_E_INVAL;
    if (!d_indirection || !d_workspace) return SNERG_E_INVAL;
    if (num_blocks > 0 && (!d_atlas || ((uintptr_t)d_atlas & 7u))) return SNERG_E_INVAL;
    if ((uintptr_t)d_workspace & (kAlign - 1)) return SNERG_E_INVAL;
    if (ws_bytes < L.total) return SNERG_E_NOMEM;
    cudaStream_t st = (cudaStream_t)stream;

    snerg_scene* h = new (std::nothrow) snerg_scene();
    if (!h) return SNERG_E_NOMEM;
    h->desc = *desc;
    h->nb = num_blocks;
    h->ws = (uint8_t*)d_workspace;
    h->hdr = (int32_t*)d_workspace;
    const int N = desc->N, B = desc->B, G = N / B, P = B + 2;
    const int64_t G3 = (int64_t)G * G * G;
    int32_t* ws_ind = (int32_t*)(h->ws + L.ind);
    uint8_t* bdist = h->ws + L.bdist;
    uint8_t* btmp = h->ws + L.btmp;
    int32_t* blk = (int32_t*)(h->ws + L.blk);
    uint8_t* vskip = h->ws + L.vskip;
    uint2* patlas = (uint2*)(h->ws + L.patlas);
    // the voxel distance transform runs before the padded atlas exists and borrows its
    // region (8 (B+2)^3 >= 7 B^3 bytes per block) as scratch
    uint8_t* vscratch = (uint8_t*)patlas;

    cudaError_t e = cudaMemsetAsync(h->hdr, 0, kAlign, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ws_ind, d_indirection, (size_t)G3 * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && num_blocks > 0) e = cudaMemsetAsync(blk, 0xff, (size_t)num_blocks * 4, st);
    if (e == cudaSuccess) e = launch_validate(ws_ind, G3, num_blocks, blk, h->hdr + kHdrCreateErr, st);
    int32_t err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, h->hdr + kHdrCreateErr, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { delete h; return SNERG_E_CUDA; }
    if (err != 0) { delete h; return SNERG_E_INVAL; }
    // the padded atlas reads occupancy from ws_ind, whose sign every octant copy keeps
    e = launch_block_distance_octants(ws_ind, G, kBlockDistCap, btmp, btmp + G3, bdist, ws_ind, st);
    if (e == cudaSuccess) e = launch_voxel_distance_octants(d_atlas, num_blocks, B, vscratch, vskip, st);
    if (e == cudaSuccess)
        e = launch_build_padded(ws_ind, blk, d_atlas, num_blocks, N, B, ilog2_exact(B), patlas, st);
    if (e == cudaSuccess) e = launch_fill_vskip_border(vskip, blk, num_blocks, N, B, ilog2_exact(B), 8, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { delete h; return SNERG_E_CUDA; }
    h->launches = 2 + 8 * 5 + (num_blocks > 0 ? 15 + 1 + 1 : 0);

    DevScene& s = h->ds;
    s.ind = ws_ind;
    s.bdist = bdist;
    s.vskip = vskip;
    s.ind_oct = G3;
    s.vskip_oct = num_blocks * (int64_t)P * P * P;
    s.patlas = patlas;
    s.status = h->hdr + kHdrStatus;
    s.N = N;
    s.B = B;
    s.lgB = ilog2_exact(B);
    s.G = G;
    s.P = P;
    s.P3 = P * P * P;
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
    s.kmax = desc->max_steps > 0 ? std::min(desc->max_steps, 4 * N + 16) : 4 * N + 16;
    s.flags = desc->flags;

    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (h->num_sms < 1) h->num_sms = 1;
    *out = h;
    return SNERG_OK;
}

namespace snerg {
// snerg_bwd.cu: one fine-tuning step per ray (render, L2 loss and adjoint in one launch)
cudaError_t launch_train_rays(const DevScene& s, const CamTable& cams, int32_t n_cams, const int32_t* pix, int64_t n,
                              const float* mlp, const float* target, float* rgb_out, float* loss, float* grad_atlas,
                              float* grad_mlp, cudaStream_t st);
// snerg_prep.cu
cudaError_t launch_requantize_padded(const int32_t* ind, const int32_t* blk_of_slot, const float* values, int64_t nb,
                                     int N, int B, int lgB, uint2* patlas, uint8_t* atlas_out, cudaStream_t st);
}  // namespace snerg

extern "C" snerg_status snerg_requantize_atlas(snerg_handle h, const float* d_values, uint8_t* d_atlas_out,
                                             void* stream) {
    if (!h) return SNERG_E_INVAL;
    if (h->nb == 0) return SNERG_OK;
    if (!d_values || ((uintptr_t)d_values & 15u) || ((uintptr_t)d_atlas_out & 7u)) return SNERG_E_INVAL;
    Layout L;
    make_layout(&h->desc, h->nb, &L);
    const cudaError_t e = launch_requantize_padded(h->ds.ind, (const int32_t*)(h->ws + L.blk), d_values, h->nb,
                                                   h->ds.N, h->ds.B, h->ds.lgB, (uint2*)(h->ws + L.patlas), d_atlas_out,
                                                   (cudaStream_t)stream);
    if (e != cudaSuccess) return SNERG_E_CUDA;
    ++h->launches;
    return SNERG_OK;
}

static bool opts_debug(const snerg_render_opts* o) {
    return o && (o->d_aux || o->d_counts || (o->d_trace && o->trace_cap > 0));
}

static DebugOut make_dbg(const snerg_render_opts* o) {
    DebugOut d{nullptr, nullptr, nullptr, 0};
    if (o) {
        d.aux = o->d_aux;
        d.counts = o->d_counts;
        if (o->d_trace && o->trace_cap > 0) {
            d.trace = o->d_trace;
            d.trace_cap = o->trace_cap;
        }
    }
    return d;
}

// ---------------------------------------------------------------------------------
// persistent multi-camera path
// ---------------------------------------------------------------------------------
static void fill_params(PersistentParams& p, const snerg_camera* cams, int32_t n, const PersistentConfig& c) {
    std::memset(&p, 0, sizeof(p));
    p.n_cams = n;
    p.tile_w = c.tile_w();
    p.tile_h = c.tile_h();
    p.warp_w = c.warp_w;
    p.warp_h = c.warp_h;
    int32_t acc = 0;
    for (int i = 0; i < n; ++i) {
        p.cams[i] = cams[i];
        const int tx = (cams[i].W + p.tile_w - 1) / p.tile_w;
        const int ty = (cams[i].H + p.tile_h - 1) / p.tile_h;
        p.tiles_x[i] = tx > 0 ? tx : 1;
        p.tile_start[i] = acc;
        acc += (cams[i].W > 0 && cams[i].H > 0) ? tx * ty : 0;
    }
    p.tile_start[n] = acc;
    p.total_items = acc;
}

static cudaError_t launch_persistent_direct(snerg_scene* h, const PersistentParams& p, const PersistentConfig& c,
                                            const float* mlp, const MlpWeights* pw, float* rgb, cudaStream_t st) {
    int32_t* queue = h->hdr + kHdrQueue;
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    h->launches++;
    return launch_render_persistent(h->ds, p, mlp, pw, rgb, queue, h->num_sms * c.ctas_per_sm, c.block, st);
}

// Work items of one warp pass only: items of several passes (the kernel build with a pass
// loop) took about twice as long on every workload measured. Each candidate is timed twice
// after a warm-up launch and scored by the faster of the two.
static PersistentConfig autotune(snerg_scene* h, const snerg_camera* cams, int32_t n, const float* mlp,
                                 const MlpWeights* pw, float* rgb, cudaStream_t st) {
    static const int shapes[4][2] = {{8, 4}, {4, 8}, {16, 2}, {32, 1}};
    static const int ctas[2] = {4, 8};
    std::vector<PersistentConfig> cand;
    for (auto& s : shapes)
        for (int c : ctas) cand.push_back(PersistentConfig{s[0], s[1], 1, 128, c});
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    PersistentConfig best = cand[0];
    float best_ms = 1e30f;
    PersistentParams* p = new PersistentParams;
    for (const auto& c : cand) {
        fill_params(*p, cams, n, c);
        if (launch_persistent_direct(h, *p, c, mlp, pw, rgb, st) != cudaSuccess) continue;   // warm-up
        float ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, st);
            if (launch_persistent_direct(h, *p, c, mlp, pw, rgb, st) != cudaSuccess) break;
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = fminf(ms, t);
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    delete p;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

static snerg_status render_persistent(snerg_scene* h, const snerg_camera* cams, int32_t n, const float* mlp,
                                      const MlpWeights* pw, float* rgb, const snerg_render_opts* o, cudaStream_t st) {
    PersistentConfig cfg{0, 0, 0, 128, 0};
    const bool manual = o && o->tile_w > 0 && o->tile_h > 0 && o->ctas_per_sm > 0;
    if (manual) {
        // tile_w x tile_h with tile_w dividing 32 (a warp pass is tile_w x (32 / tile_w))
        if (32 % o->tile_w != 0 || o->tile_h % (32 / o->tile_w) != 0 || o->ctas_per_sm > 16)
            return SNERG_E_INVAL;
        cfg.warp_w = o->tile_w;
        cfg.warp_h = 32 / o->tile_w;
        cfg.passes = o->tile_h / cfg.warp_h;
        cfg.ctas_per_sm = o->ctas_per_sm;
    } else {
        std::vector<int32_t> key;
        for (int i = 0; i < n; ++i) {
            key.push_back(cams[i].W);
            key.push_back(cams[i].H);
        }
        auto it = h->tuned.find(key);
        if (it == h->tuned.end()) it = h->tuned.emplace(key, autotune(h, cams, n, mlp, pw, rgb, st)).first;
        cfg = it->second;
    }
    h->last = cfg;
    PersistentParams* p = new (std::nothrow) PersistentParams;
    if (!p) return SNERG_E_NOMEM;
    fill_params(*p, cams, n, cfg);
    const int grid = h->num_sms * cfg.ctas_per_sm;
    int32_t* queue = h->hdr + kHdrQueue;
    const auto gkey = std::make_pair(cfg, pw != nullptr);
    GraphEntry& ge = h->graphs[gkey];
    cudaError_t e = cudaSuccess;
    if (!ge.exec) {
        if (!h->cap_stream) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(queue, 0, sizeof(int32_t), h->cap_stream);
            launch_render_persistent(h->ds, *p, mlp, pw, rgb, queue, grid, cfg.block, h->cap_stream);
            e = cudaStreamEndCapture(h->cap_stream, &ge.graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge.exec, ge.graph, 0);
        if (e == cudaSuccess) {
            size_t cnt = 0;
            cudaGraphGetNodes(ge.graph, nullptr, &cnt);
            std::vector<cudaGraphNode_t> nodes(cnt);
            cudaGraphGetNodes(ge.graph, nodes.data(), &cnt);
            for (auto nd : nodes) {
                cudaGraphNodeType t;
                cudaGraphNodeGetType(nd, &t);
                if (t == cudaGraphNodeTypeKernel) ge.knode = nd;
            }
            if (!ge.knode) e = cudaErrorUnknown;
        }
        if (e != cudaSuccess) {
            if (ge.exec) cudaGraphExecDestroy(ge.exec);
            if (ge.graph) cudaGraphDestroy(ge.graph);
            h->graphs.erase(gkey);
            delete p;
            return SNERG_E_CUDA;
        }
    }
    // refresh the kernel node with this call's cameras and buffers, then replay
    DevScene ds = h->ds;
    const float* mlp_arg = mlp;
    float* rgb_arg = rgb;
    static const MlpWeights zero_w = {};
    const MlpWeights* w_arg = pw ? pw : &zero_w;
    void* args[] = {(void*)&ds, (void*)p, (void*)&mlp_arg, (void*)w_arg, (void*)&rgb_arg, (void*)&queue};
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void*>(persistent_kernel_fn(pw != nullptr, cfg.passes > 1));
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(cfg.block);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    e = cudaGraphExecKernelNodeSetParams(ge.exec, ge.knode, &kp);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge.exec, st);
    delete p;
    if (e != cudaSuccess) return SNERG_E_CUDA;
    h->launches++;
    return SNERG_OK;
}

extern "C" snerg_status snerg_render(snerg_handle h, const snerg_camera* cams, int32_t n_cams, const float* d_mlp,
                                     float* d_rgb, const snerg_render_opts* opts, void* stream) {
    if (!h || !cams || n_cams < 1) return SNERG_E_INVAL;
    int64_t pixels = 0;
    for (int i = 0; i < n_cams; ++i) {
        if (!camera_ok(cams[i])) return SNERG_E_INVAL;
        pixels += (int64_t)cams[i].W * cams[i].H;
    }
    if (pixels == 0) return SNERG_OK;
    if (!d_rgb || (!d_mlp && !h->has_w)) return SNERG_E_INVAL;
    const MlpWeights* pw = d_mlp ? nullptr : &h->host_w;
    cudaStream_t st = (cudaStream_t)stream;
    const bool rows = opts && (opts->row_begin != 0 || opts->row_end != 0);
    if (rows && (opts->row_begin < 0 || opts->row_end < opts->row_begin)) return SNERG_E_INVAL;
    if (opts && opts->persistent && !opts_debug(opts)) {
        if (h->desc.flags & SNERG_FLAG_PER_SAMPLE_MLP) return SNERG_E_UNSUPPORTED;
        if (rows) return SNERG_E_UNSUPPORTED;
        // the camera table of one persistent launch holds kMaxCams cameras; a larger batch
        // runs as consecutive launches (each camera's pixels go to its own out_offset)
        for (int c0 = 0; c0 < n_cams; c0 += kMaxCams) {
            const snerg_status e = render_persistent(h, cams + c0, std::min(kMaxCams, n_cams - c0), d_mlp, pw, d_rgb,
                                                     opts, st);
            if (e != SNERG_OK) return e;
        }
        return SNERG_OK;
    }
    if (opts && (opts->schedule < 0 || opts->schedule > 1)) return SNERG_E_INVAL;
    const DebugOut dbg = make_dbg(opts);
    const int tiles = ((cams[0].W + 15) / 16) * ((cams[0].H + 7) / 8);
    if (opts && opts->schedule == 1 && n_cams == 1 && !rows && !opts_debug(opts) &&
        !(h->desc.flags & SNERG_FLAG_PER_SAMPLE_MLP) && tiles <= kSchedMaxTiles) {
        // the previous frame's buckets (if they describe an image of this size) give the
        // order; this frame's go to the other set, whose counts start at zero
        Layout L;
        make_layout(&h->desc, h->nb, &L);
        uint8_t* set[2] = {h->ws + L.sched, h->ws + L.sched + kSchedSetBytes};
        const bool use = h->sched_valid && h->sched_w == cams[0].W && h->sched_h == cams[0].H;
        uint8_t* rd = set[h->sched_set];
        uint8_t* wr = set[h->sched_set ^ 1];
        SchedArgs sa;
        sa.rd_count = use ? (const int32_t*)rd : nullptr;
        sa.rd_list = (const int32_t*)(rd + kSchedCountBytes);
        sa.wr_count = (int32_t*)wr;
        sa.wr_list = (int32_t*)(wr + kSchedCountBytes);
        sa.cap = kSchedMaxTiles;
        sa.nt = tiles;
        sa.tiles_x = (cams[0].W + 15) / 16;
        // sparse slots only with a previous frame to choose the slow tiles from
        sa.smax = use ? std::min(kSchedMaxSparse, std::max(1, tiles / 8)) : 0;
        cudaError_t e = cudaMemsetAsync(wr, 0, kSchedCountBytes, st);
        if (e == cudaSuccess) e = launch_render_image(h->ds, cams[0], d_mlp, pw, d_rgb, dbg, st, 0, cams[0].H, &sa);
        if (e != cudaSuccess) return SNERG_E_CUDA;
        h->launches++;
        h->sched_set ^= 1;
        h->sched_w = cams[0].W;
        h->sched_h = cams[0].H;
        h->sched_valid = true;
        return SNERG_OK;
    }
    for (int i = 0; i < n_cams; ++i) {
        if (cams[i].W == 0 || cams[i].H == 0) continue;
        const int r0 = rows ? opts->row_begin : 0, r1 = rows ? opts->row_end : cams[i].H;
        if (std::min(r1, cams[i].H) <= r0) continue;
        cudaError_t e = launch_render_image(h->ds, cams[i], d_mlp, pw, d_rgb, dbg, st, r0, r1);
        if (e != cudaSuccess) return SNERG_E_CUDA;
        h->launches++;
    }
    return SNERG_OK;
}

constexpr int kMaxBands = 16;

extern "C" snerg_status snerg_render_to_host(snerg_handle h, const snerg_camera* cams, int32_t n_cams,
                                             const float* d_mlp, float* d_rgb, float* h_rgb, int32_t n_bands,
                                             void* stream) {
    if (!h || !cams || n_cams < 1 || n_bands < 1 || n_bands > kMaxBands) return SNERG_E_INVAL;
    int64_t pixels = 0;
    int Hmax = 0;
    for (int i = 0; i < n_cams; ++i) {
        if (!camera_ok(cams[i])) return SNERG_E_INVAL;
        pixels += (int64_t)cams[i].W * cams[i].H;
        Hmax = std::max(Hmax, cams[i].H);
    }
    if (pixels == 0) return SNERG_OK;
    if (!h_rgb || (!d_mlp && !h->has_w)) return SNERG_E_INVAL;
    const MlpWeights* pw = d_mlp ? nullptr : &h->host_w;
    cudaStream_t st = (cudaStream_t)stream;
    const DebugOut dbg{nullptr, nullptr, nullptr, 0};
    // page-locked host memory mapped for the device: the kernels store the pixels straight
    // into it (over NVLink-C2C on a Grace host), so the frame needs no separate copy
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, h_rgb) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer) {
        float* mapped = (float*)pa.devicePointer;
        for (int i = 0; i < n_cams; ++i) {
            if (cams[i].W == 0 || cams[i].H == 0) continue;
            if (launch_render_image(h->ds, cams[i], d_mlp, pw, mapped, dbg, st, 0, cams[i].H) != cudaSuccess)
                return SNERG_E_CUDA;
            h->launches++;
        }
        return SNERG_OK;
    }
    cudaGetLastError();                  // an unregistered pointer is not an error here
    if (!d_rgb) return SNERG_E_INVAL;
    cudaError_t e = cudaSuccess;
    if (!h->band_fork) e = cudaEventCreateWithFlags(&h->band_fork, cudaEventDisableTiming);
    while (e == cudaSuccess && (int)h->band_streams.size() < n_bands) {
        cudaStream_t b = nullptr;
        cudaEvent_t d = nullptr;
        e = cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking);
        if (e == cudaSuccess) h->band_streams.push_back(b);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d, cudaEventDisableTiming);
        if (e == cudaSuccess) h->band_done.push_back(d);
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->band_fork, st);
    n_bands = std::min(n_bands, Hmax);
    for (int b = 0; b < n_bands && e == cudaSuccess; ++b) {
        const int y0 = (int)((int64_t)Hmax * b / n_bands), y1 = (int)((int64_t)Hmax * (b + 1) / n_bands);
        cudaStream_t bs = h->band_streams[b];
        e = cudaStreamWaitEvent(bs, h->band_fork, 0);
        for (int i = 0; i < n_cams && e == cudaSuccess; ++i) {
            const snerg_camera& c = cams[i];
            const int r0 = std::min(y0, c.H), r1 = std::min(y1, c.H);
            if (c.W == 0 || r1 <= r0) continue;
            e = launch_render_image(h->ds, c, d_mlp, pw, d_rgb, dbg, bs, r0, r1);
            if (e != cudaSuccess) break;
            h->launches++;
            const size_t first = (size_t)(c.out_offset + (int64_t)r0 * c.W) * 3;
            const size_t count = (size_t)(r1 - r0) * c.W * 3;
            e = cudaMemcpyAsync(h_rgb + first, d_rgb + first, count * sizeof(float), cudaMemcpyDeviceToHost, bs);
        }
        if (e == cudaSuccess) e = cudaEventRecord(h->band_done[b], bs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->band_done[b], 0);
    }
    return e == cudaSuccess ? SNERG_OK : SNERG_E_CUDA;
}

static bool make_table(const snerg_camera* cams, int32_t n_cams, CamTable* t) {
    if (!cams || n_cams < 1 || n_cams > kMaxCams) return false;
    std::memset(t, 0, sizeof(*t));
    for (int i = 0; i < n_cams; ++i) {
        if (!camera_ok(cams[i])) return false;
        t->c[i] = cams[i];
    }
    return true;
}

extern "C" snerg_status snerg_render_rays(snerg_handle h, const snerg_camera* cams, int32_t n_cams,
                                          const int32_t* d_pix, int64_t n, const float* d_mlp, float* d_rgb,
                                          const snerg_render_opts* opts, void* stream) {
    if (!h || n < 0) return SNERG_E_INVAL;
    if (h->desc.flags & SNERG_FLAG_PER_SAMPLE_MLP) return SNERG_E_UNSUPPORTED;
    CamTable* t = new (std::nothrow) CamTable;
    if (!t) return SNERG_E_NOMEM;
    if (!make_table(cams, n_cams, t)) { delete t; return SNERG_E_INVAL; }
    if (n == 0) { delete t; return SNERG_OK; }
    if (!d_pix || !d_rgb || (!d_mlp && !h->has_w)) { delete t; return SNERG_E_INVAL; }
    cudaError_t e = launch_render_rays(h->ds, *t, n_cams, d_pix, n, d_mlp, d_mlp ? nullptr : &h->host_w, d_rgb,
                                       make_dbg(opts), h->num_sms, (cudaStream_t)stream);
    delete t;
    if (e != cudaSuccess) return SNERG_E_CUDA;
    h->launches++;
    return SNERG_OK;
}

extern "C" snerg_status snerg_render_backward(snerg_handle h, const snerg_camera* cams, int32_t n_cams,
                                              const int32_t* d_pix, int64_t n, const float* d_mlp,
                                              const float* d_grad_rgb, const float* d_fwd_aux,
                                              const int32_t* d_fwd_counts, float* d_grad_atlas, float* d_grad_mlp,
                                              void* stream) {
    if (!h || n < 0) return SNERG_E_INVAL;
    if (h->desc.flags & SNERG_FLAG_PER_SAMPLE_MLP) return SNERG_E_UNSUPPORTED;
    CamTable* t = new (std::nothrow) CamTable;
    if (!t) return SNERG_E_NOMEM;
    if (!make_table(cams, n_cams, t)) { delete t; return SNERG_E_INVAL; }
    if (n == 0 || (!d_grad_atlas && !d_grad_mlp)) { delete t; return SNERG_OK; }
    if (!d_pix || !d_mlp || !d_grad_rgb) { delete t; return SNERG_E_INVAL; }
    if (d_grad_atlas && ((uintptr_t)d_grad_atlas & 15u)) { delete t; return SNERG_E_INVAL; }
    if ((d_fwd_aux == nullptr) != (d_fwd_counts == nullptr)) { delete t; return SNERG_E_INVAL; }
    cudaError_t e = launch_backward_rays(h->ds, *t, n_cams, d_pix, n, d_mlp, d_grad_rgb, d_fwd_aux, d_fwd_counts,
                                         d_grad_atlas, d_grad_mlp, (cudaStream_t)stream);
    delete t;
    if (e != cudaSuccess) return SNERG_E_CUDA;
    h->launches++;
    return SNERG_OK;
}

extern "C" snerg_status snerg_train_rays(snerg_handle h, const snerg_camera* cams, int32_t n_cams,
                                         const int32_t* d_pix, int64_t n, const float* d_mlp, const float* d_target,
                                         float* d_rgb, float* d_loss, float* d_grad_atlas, float* d_grad_mlp,
                                         void* stream) {
    if (!h || n < 0) return SNERG_E_INVAL;
    if (h->desc.flags & SNERG_FLAG_PER_SAMPLE_MLP) return SNERG_E_UNSUPPORTED;
    CamTable* t = new (std::nothrow) CamTable;
    if (!t) return SNERG_E_NOMEM;
    if (!make_table(cams, n_cams, t)) { delete t; return SNERG_E_INVAL; }
    if (n == 0) { delete t; return SNERG_OK; }
    if (!d_pix || !d_mlp || !d_target) { delete t; return SNERG_E_INVAL; }
    if (d_grad_atlas && ((uintptr_t)d_grad_atlas & 15u)) { delete t; return SNERG_E_INVAL; }
    cudaError_t e = launch_train_rays(h->ds, *t, n_cams, d_pix, n, d_mlp, d_target, d_rgb, d_loss, d_grad_atlas,
                                      d_grad_mlp, (cudaStream_t)stream);
    delete t;
    if (e != cudaSuccess) return SNERG_E_CUDA;
    h->launches++;
    return SNERG_OK;
}

// the CUDA errors that leave the context unusable (a fault in a kernel)
static bool sticky_fault(cudaError_t e) {
    switch (e) {
        case cudaErrorIllegalAddress:
        case cudaErrorIllegalInstruction:
        case cudaErrorMisalignedAddress:
        case cudaErrorInvalidAddressSpace:
        case cudaErrorInvalidPc:
        case cudaErrorHardwareStackError:
        case cudaErrorLaunchFailure:
        case cudaErrorAssert:
        case cudaErrorLaunchTimeout:
            return true;
        default:
            return false;
    }
}

extern "C" snerg_status snerg_last_status(snerg_handle h, void* stream) {
    if (!h) return SNERG_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t v = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (sticky_fault(e)) return SNERG_E_DEVICE_FAULT;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, h->hdr + kHdrStatus, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->hdr + kHdrStatus, 0, 4, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return SNERG_E_CUDA;
    return (snerg_status)v;
}

extern "C" snerg_status snerg_set_mlp(snerg_handle h, const float* mlp) {
    if (!h || !mlp) return SNERG_E_INVAL;
    MlpWeights w;
    std::memset(&w, 0, sizeof(w));
    for (int i = 0; i < kNParam; ++i) {
        if (!std::isfinite(mlp[i])) return SNERG_E_INVAL;
        int dst = i;
        if (i < kOffB1) {                              // W1[o][k] -> W1^T[k][o]
            dst = kOffW1 + (i % kMlpIn) * kMlpH + i / kMlpIn;
        } else if (i >= kOffW2 && i < kOffB2) {        // W2[o][k] -> W2^T[k][o]
            dst = kOffW2 + ((i - kOffW2) % kMlpH) * kMlpH + (i - kOffW2) / kMlpH;
        }
        w.w[dst] = mlp[i];
    }
    h->host_w = w;
    h->has_w = true;
    return SNERG_OK;
}

extern "C" int64_t snerg_launch_count(snerg_handle h) { return h ? h->launches : 0; }

extern "C" snerg_status snerg_schedule_stats(snerg_handle h, void* stream, int32_t* sparse_tiles, int32_t* ordered) {
    if (!h || !sparse_tiles || !ordered) return SNERG_E_INVAL;
    *sparse_tiles = 0;
    *ordered = 0;
    if (!h->sched_valid) return SNERG_OK;
    Layout L;
    make_layout(&h->desc, h->nb, &L);
    // the set the last scheduled launch wrote is the one the next launch will read
    const int32_t* hdr = (const int32_t*)(h->ws + L.sched + (size_t)h->sched_set * kSchedSetBytes);
    int32_t info[2] = {0, 0};
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(info, hdr + kSchedHdrInfo, sizeof(info), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return SNERG_E_CUDA;
    *sparse_tiles = info[0] > 0 ? info[0] - 1 : 0;
    *ordered = info[1];
    return SNERG_OK;
}

extern "C" snerg_status snerg_persistent_config(snerg_handle h, int32_t* tile_w, int32_t* tile_h,
                                                int32_t* ctas_per_sm) {
    if (!h || !tile_w || !tile_h || !ctas_per_sm) return SNERG_E_INVAL;
    *tile_w = h->last.warp_w ? h->last.tile_w() : 0;
    *tile_h = h->last.warp_w ? h->last.tile_h() : 0;
    *ctas_per_sm = h->last.ctas_per_sm;
    return SNERG_OK;
}

extern "C" void snerg_destroy(snerg_handle h) {
    if (!h) return;
    for (auto& kv : h->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (cudaStream_t b : h->band_streams) cudaStreamDestroy(b);
    for (cudaEvent_t e : h->band_done) cudaEventDestroy(e);
    if (h->band_fork) cudaEventDestroy(h->band_fork);
    delete h;
}

extern "C" const char* snerg_status_str(snerg_status s) {
    switch (s) {
        case SNERG_OK: return "ok";
        case SNERG_E_INVAL: return "invalid argument";
        case SNERG_E_NOMEM: return "buffer too small";
        case SNERG_E_CUDA: return "CUDA error";
        case SNERG_E_STEP_LIMIT: return "a ray exceeded its iteration cap";
        case SNERG_E_UNSUPPORTED: return "unsupported";
        case SNERG_E_DEVICE_FAULT: return "device fault";
    }
    return "unknown status";
}
