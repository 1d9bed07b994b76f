/*
 * snerg.h -- C ABI of the GB300 renderer for baked Sparse Neural Radiance Grids
 * (SNeRG, "Baking Neural Radiance Fields for Real-Time View Synthesis").
 *
 * The library renders the paper's baked representation (Sec. 5.1): an N^3 virtual
 * voxel grid stored as an (N/B)^3 indirection grid whose entries are -1 (empty
 * macroblock) or the slot of a B^3 macroblock in a uint8 atlas holding, per voxel,
 * density, diffuse RGB and a 4-channel feature (Sec. 4.2, 8 bits each, Sec. 5.4).
 * Each pixel's ray is marched through the grid (Sec. 5.2, App. A), composited with
 * Eqs. 2, 5, 6, stopped once T < 1e-3, and finished with one evaluation of the
 * view-dependence MLP (Eq. 7). A hand-written adjoint gives the gradients used to
 * fine-tune the baked grid's view-dependent appearance (Sec. 5.5).
 *
 * Conventions for every entry point:
 *   * Pointers prefixed d_ are DEVICE memory owned by the caller; h_ / unprefixed
 *     struct pointers are HOST memory read during the call only. The library never
 *     allocates device memory and never frees caller memory; its only device state is
 *     the caller-provided workspace.
 *   * Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) unless the entry point says it synchronises.
 *   * Errors are return codes; nothing is thrown across the ABI. Errors found on the
 *     device (a ray exceeding its iteration cap) are recorded in a status word in the
 *     workspace and reported by snerg_last_status().
 *   * A handle may be used from one host thread at a time.
 *
 * Arithmetic contract (what is bit-exact and what is not):
 *   * integer decisions -- the sample lattice, the nearest voxel of each sample, the
 *     block lookup, the density probe and the early-exit test -- are taken in IEEE
 *     binary32 with one rounding per operation in a fixed order, so step counts and
 *     visited voxels are reproducible bit for bit by an independent implementation;
 *   * colours are accumulated in FP32 (max abs error vs FP64 well under 1e-4).
 */
#ifndef SNERG_H
#define SNERG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SNERG_OK = 0,
    SNERG_E_INVAL = 1,        /* invalid argument (sizes, pointers, indirection entries) */
    SNERG_E_NOMEM = 2,        /* caller-provided buffer smaller than required */
    SNERG_E_CUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    SNERG_E_STEP_LIMIT = 4,   /* device: a ray reached its lattice cap (desc.max_steps) */
    SNERG_E_UNSUPPORTED = 5,  /* request outside the compiled limits */
    SNERG_E_DEVICE_FAULT = 6  /* snerg_last_status: the stream's context took a sticky device
                                 fault (illegal address or instruction, misaligned access,
                                 failed launch); the CUDA context must be recreated */
} snerg_status;

typedef struct snerg_scene* snerg_handle;

/* Scene description (Sec. 5.1). World-space grid = axis-aligned cube
 * [bmin, bmin + extent]^3; voxel width delta = extent / N. */
typedef struct {
    int32_t N;          /* virtual grid resolution per axis; 1 <= N <= 16384, N % B == 0 */
    int32_t B;          /* macroblock edge; power of two in [2, 64] */
    float bmin[3];      /* world-space minimum corner */
    float extent;       /* world-space edge length, > 0 */
    float sigma_max;    /* density of code 255 (1/world units): sigma = q / 255 * sigma_max */
    float bg[3];        /* background colour, added with weight T_final */
    int32_t max_steps;  /* cap on the lattice index of a ray; 0 = 4N + 16 (never reached by a
                           valid ray). A ray reaching the cap stops, keeps what it composited
                           and records SNERG_E_STEP_LIMIT in the device status word. */
    int32_t flags;      /* SNERG_FLAG_* */
} snerg_scene_desc;

/* Partial un-premultiply after compositing (the paper's forward-facing scenes, App. C):
 * when alpha = 1 - T_final > 0, (C_d, alpha, V) *= min(1, 1.5 alpha) / alpha, so the MLP
 * sees the scaled C_d and V and the background weight is 1 - min(1, 1.5 alpha). The aux
 * output keeps the composites before scaling. */
#define SNERG_FLAG_UNPREMULTIPLY 1
/* The non-deferred comparison model (the paper's per-sample ablation, Sec. 6): the
 * view-dependence MLP is evaluated at every composited sample on that sample's own
 * (c_d, v) and the sample colours c_d + residual are composited; there is no per-pixel
 * residual. Forward only, one-camera launches only (snerg_render without persistent;
 * other entry points return SNERG_E_UNSUPPORTED); not combinable with UNPREMULTIPLY. */
#define SNERG_FLAG_PER_SAMPLE_MLP 2
/* Alpha atlas (App. A keeps alpha in its own 8-bit texture): channel 0 of the atlas holds
 * alpha codes instead of density codes. A sample's alpha is a = s * binary32(1/255), s the
 * binary32 trilinear of the codes (the same arithmetic as the density path), composited as
 * w = T a, T <- T (1 - a) with the product rounded in binary32, and the ray stops after the
 * sample that brings T below binary32(1e-3); sigma_max is not used. The empty-space maps,
 * the probe (code 0 = empty) and all entry points but snerg_render_rays_noalloc work
 * unchanged. snerg_bake with this flag stores alpha = 1 - exp(-sigma v) in channel 0. */
#define SNERG_FLAG_ALPHA_ATLAS 4
/* The paper's performance ablation without the view-dependence network (Sec. 6): the
 * pixel is C_d + T bg; the MLP weights are not read, and the adjoint gives no dL/dPhi and
 * no gradient for the feature channels. Not combinable with SNERG_FLAG_PER_SAMPLE_MLP. */
#define SNERG_FLAG_NO_MLP 8

/* Pinhole camera (Sec. 4.1 r(t) = o + t d). 80 bytes, host memory.
 * Pixel (x, y) looks along R (x + 0.5 - cx) / fx, -(y + 0.5 - cy) / fy, -1) normalised,
 * i.e. the camera looks down its -z axis with +y up and image rows growing downwards.
 * Its RGB is written at out[(out_offset + y * W + x) * 3 + c]. */
typedef struct {
    float c2w[12];      /* row-major 3x4 camera-to-world [R | t] */
    float fx, fy, cx, cy;
    int32_t W, H;
    int64_t out_offset; /* first output pixel of this camera */
} snerg_camera;

/* Optional per-call outputs and launch choices. All pointers nullable (device). */
typedef struct {
    float* d_aux;          /* [pixels][8]: C_d (3), V (4), accumulated opacity 1 - T */
    int32_t* d_counts;     /* [pixels][4]: steps (lattice samples in occupied blocks), active
                              (composited) samples, indirection entries read, lattice index
                              of the first composited sample (-1 if none) */
    uint64_t* d_trace;     /* [pixels][trace_cap]: z*N*N + y*N + x of each composited sample */
    int32_t trace_cap;
    int32_t persistent;    /* snerg_render only: 1 = all cameras in one persistent launch,
                              captured into a CUDA graph on first use and replayed */
    int32_t tile_w, tile_h;/* persistent only: pixel tile per work item; 0 = autotune */
    int32_t ctas_per_sm;   /* persistent only: 0 = autotune */
    int32_t row_begin;     /* snerg_render without persistent: render only image rows
                              [row_begin, row_end) of every camera (clamped to its H), with
                              exactly the rays of the full render; other pixels of d_rgb
                              are not written. 0, 0 = all rows. Lets a caller split a frame
                              into bands on several streams and copy each band out as soon
                              as it is done. */
    int32_t row_end;
    int32_t schedule;      /* snerg_render only. 1 = a viewer's tile schedule: this call's
                              16x8-pixel tiles are launched in the order of the tile costs
                              (CTA durations) the handle recorded on its last schedule = 1
                              render of a camera of the same W x H, slowest first, and this
                              call records its own tile costs for the next one; the first such
                              call, or a new size, launches in raster order. Consecutive
                              frames of a moving camera have their slow tiles (rays grazing
                              surfaces) in nearly the same places, so those start first
                              instead of at their raster position. The pixels are exactly
                              those of a raster-order launch. Applies to one camera, all
                              rows, no debug outputs, not persistent, the deferred model and
                              at most SNERG_SCHEDULE_MAX_TILES tiles; other calls launch in
                              raster order. Calls that overlap on the GPU must not both use
                              it. 0 = raster order. */
} snerg_render_opts;

/* Largest image (in 16x8-pixel tiles) whose tile costs a handle records (4096 x 2048
 * pixels). */
#define SNERG_SCHEDULE_MAX_TILES 65536

/* Largest number of cameras in one ray-list call (snerg_render_rays, snerg_render_backward,
 * snerg_train_rays, snerg_render_rays_noalloc: a ray may name any of them) and in one
 * persistent launch. snerg_render and snerg_render_to_host take any number; a persistent
 * render of more cameras runs as consecutive persistent launches of up to this many. */
#define SNERG_MAX_CAMERAS 256
/* Number of MLP parameters: W1[16][34], b1[16], W2[16][16], b2[16], W3[3][16], b3[3]
 * (row-major, out x in), float32 (Eq. 7; "2 layers with 16 channels", Sec. 4.2). */
#define SNERG_MLP_PARAMS 883

/* Bytes of device workspace snerg_create needs for `num_blocks` occupied macroblocks;
 * 0 if the description is invalid. The workspace holds the apron-padded device copy of
 * the atlas, the indirection grid, the empty-space distance maps (per octant of the ray
 * direction: one per block, one per stored voxel), the status word and the tile costs of
 * the viewer's schedule (snerg_render_opts.schedule): about 16 (B+2)^3 bytes per block
 * + 35 (N/B)^3 bytes + 16 MiB. */
size_t snerg_workspace_bytes(const snerg_scene_desc* desc, int64_t num_blocks);

/* Build a scene handle (Sec. 5.1 data structure).
 *   d_indirection : int32 [G][G][G] (z, y, x), G = N / B; each entry -1 or a slot in
 *                   [0, num_blocks); no slot may be referenced twice.
 *   d_atlas       : uint8 [num_blocks][B][B][B][8] (z, y, x, channel); channels
 *                   density, r, g, b, f0, f1, f2, f3.
 *   d_workspace   : >= snerg_workspace_bytes(desc, num_blocks) bytes, 256-byte
 *                   aligned, owned by the caller and kept alive until snerg_destroy.
 * Both inputs are copied into the workspace; the caller may free them afterwards.
 * SYNCHRONISES `stream` (to validate the indirection grid). Returns SNERG_E_INVAL for
 * a bad description, an out-of-range or repeated slot; SNERG_E_NOMEM if ws_bytes is
 * too small. On error *out is NULL. */
snerg_status snerg_create(const snerg_scene_desc* desc, const int32_t* d_indirection,
                          const uint8_t* d_atlas, int64_t num_blocks, void* d_workspace,
                          size_t ws_bytes, void* stream, snerg_handle* out);

/* Store view-dependence MLP weights (HOST float32 [SNERG_MLP_PARAMS], flat layout above)
 * in the handle. Render calls made with d_mlp == NULL then take these weights as a
 * kernel parameter, so every weight is a constant operand of the kernel's FMAs (the
 * paper's viewer likewise compiles the network's biases into its shader and keeps the
 * weights in uniform textures, App. A). Returns SNERG_E_INVAL for non-finite weights. */
snerg_status snerg_set_mlp(snerg_handle h, const float* mlp);

/* Render every pixel of n_cams cameras (Sec. 5.2 and App. A; Eqs. 2, 5-7).
 *   cams   : HOST array of n_cams >= 1 cameras, W, H >= 0.
 *   d_mlp  : float32 [SNERG_MLP_PARAMS] view-dependence MLP weights in device memory,
 *            or NULL to use the weights stored with snerg_set_mlp (SNERG_E_INVAL if
 *            none were stored).
 *   d_rgb  : float32 output [total pixels][3] addressed through out_offset; device memory,
 *            or page-locked host memory mapped for the device (the kernels then store the
 *            pixels into host memory directly, see snerg_render_to_host).
 *   opts   : nullable. Debug outputs (aux, counts, trace) use the plain launch.
 * The colour is C = C_d + sigmoid(MLP(C_d, V, PE(d))) + T bg if any sample was
 * composited, else T bg (App. A evaluates the MLP only where alpha > 0). */
snerg_status snerg_render(snerg_handle h, const snerg_camera* cams, int32_t n_cams,
                          const float* d_mlp, float* d_rgb, const snerg_render_opts* opts,
                          void* stream);

/* Render every pixel of n_cams cameras and deliver the image to host memory h_rgb
 * (float32 [pixels][3] through out_offset), with the rays and colours of snerg_render
 * (plain launch), asynchronously on `stream`; h_rgb is complete once `stream` is
 * synchronised.
 *   * h_rgb page-locked and mapped for the device (memory from cudaHostAlloc /
 *     cudaMallocHost under unified addressing, e.g. PyTorch's pinned tensors): the kernels
 *     store the pixels straight into it through the device's mapping (NVLink-C2C on a Grace
 *     host), so no copy follows the render; d_rgb and n_bands are not used (d_rgb may be
 *     NULL).
 *   * otherwise: the rows are split into n_bands bands (1..16, by the tallest camera), each
 *     rendered into d_rgb (float32 device image, required) on one of the handle's side
 *     streams (created by the first call) after the work already queued on `stream`, and
 *     copied to h_rgb as soon as it is done; `stream` waits for every band.
 * d_mlp as for snerg_render (NULL = the snerg_set_mlp weights). Call it with the handle's
 * device current (the side streams belong to that device). */
snerg_status snerg_render_to_host(snerg_handle h, const snerg_camera* cams, int32_t n_cams, const float* d_mlp,
                                  float* d_rgb, float* h_rgb, int32_t n_bands, void* stream);

/* Render a list of rays: d_pix int32 [n][3] = (camera index, x, y). Output row i of
 * d_rgb (and of the optional opts outputs) belongs to ray i; out_offset is ignored.
 * d_mlp as for snerg_render (NULL = the snerg_set_mlp weights). */
snerg_status snerg_render_rays(snerg_handle h, const snerg_camera* cams, int32_t n_cams,
                               const int32_t* d_pix, int64_t n, const float* d_mlp,
                               float* d_rgb, const snerg_render_opts* opts, void* stream);

/* Adjoint of snerg_render_rays for an upstream gradient d_grad_rgb [n][3] = dL/dC
 * (Sec. 5.5 fine-tunes against an L2 image loss, Eq. 3). Density is frozen. No
 * per-sample state passes between calls: the kernel marches each ray itself (keeping its
 * first 32 composited samples' lattice indices and weights for its own scatter).
 * ACCUMULATES (caller zeroes):
 *   d_grad_atlas : float32 [num_blocks][B][B][B][8], dL/d(q/255) of channels 1..7 of
 *                  every stored voxel; channel 0 (density) receives exactly zero;
 *   d_grad_mlp   : float32 [SNERG_MLP_PARAMS].
 * Either gradient pointer may be NULL to skip it. d_mlp must be device weights.
 * d_fwd_aux / d_fwd_counts (both or neither, nullable): the opts.d_aux and
 * opts.d_counts outputs of the snerg_render_rays call that produced C for these rays with
 * the same cameras, rays and weights. Given them, the kernel takes C_d, V and the first
 * composited lattice index from them (per-ray state, 9 words) instead of its own first
 * march, and scatters with one march from that index; the gradients are the same. */
snerg_status snerg_render_backward(snerg_handle h, const snerg_camera* cams, int32_t n_cams,
                                   const int32_t* d_pix, int64_t n, const float* d_mlp,
                                   const float* d_grad_rgb, const float* d_fwd_aux,
                                   const int32_t* d_fwd_counts, float* d_grad_atlas,
                                   float* d_grad_mlp, void* stream);

/* Data-parallel fine-tuning (one exchange step per training step, Sec. 5.5 run on several
 * GPUs): every rank sums dL/dPhi and the atlas gradient of its own rays, and the ranks
 * all-reduce them before the optimiser step. The atlas gradient is exchanged only over the
 * macroblocks some rank touched; these three calls prepare that exchange (the all-reduce
 * itself is the caller's, e.g. NCCL). block_floats = floats per block (B^3 * 8), a
 * multiple of 4; device pointers 16-byte aligned; asynchronous on `stream`.
 *   snerg_grad_blocks_touched : d_mask[b] = 1 if any of block b's floats is non-zero, else 0
 *                               (d_grad [num_blocks][block_floats], d_mask int32 [num_blocks]);
 *   snerg_grad_blocks_gather  : d_packed[i] = d_grad[d_list[i]] for i < n (whole blocks);
 *   snerg_grad_blocks_scatter : d_grad[d_list[i]] = d_packed[i] for i < n.
 * List entries must lie in [0, num_blocks) of the gradient they index and, for the
 * scatter, be distinct. */
snerg_status snerg_grad_blocks_touched(const float* d_grad, int64_t num_blocks, int32_t block_floats,
                                       int32_t* d_mask, void* stream);
snerg_status snerg_grad_blocks_gather(const float* d_grad, const int32_t* d_list, int64_t n, int32_t block_floats,
                                      float* d_packed, void* stream);
snerg_status snerg_grad_blocks_scatter(const float* d_packed, const int32_t* d_list, int64_t n,
                                       int32_t block_floats, float* d_grad, void* stream);

/* Requantise fine-tuned colour and feature values into the scene. The paper fine-tunes the
 * view-dependence MLP against the training images (Sec. 5.5); the baked colours and
 * features can be fine-tuned the same way through an FP32 shadow copy that takes the
 * optimiser's steps on the d_grad_atlas of snerg_render_backward, and this call turns the
 * shadow back into the 8-bit codes the renderer reads (Sec. 5.4).
 *   d_values    : float32 [num_blocks][B][B][B][8] (16-byte aligned), the atlas layout;
 *                 channels 1..7 (diffuse RGB, features) are read as values x and stored as
 *                 floor(255 x + 1/2) clamped to [0, 255], decided in binary32 (NaN -> 0);
 *                 channel 0 is ignored: densities stay frozen, and with them the
 *                 empty-space maps built by snerg_create.
 *   d_atlas_out : nullable uint8 [num_blocks][B][B][B][8] (8-byte aligned); receives the
 *                 new codes with the scene's density codes in channel 0.
 * Rewrites every stored voxel of the handle's padded atlas and its copies in the
 * neighbouring blocks' aprons. Asynchronous on `stream`; later calls on the same stream
 * render the new codes. */
snerg_status snerg_requantize_atlas(snerg_handle h, const float* d_values, uint8_t* d_atlas_out, void* stream);

/* One fine-tuning step's render, loss and adjoint for a ray list in a single launch (Sec.
 * 5.5, Eq. 3): each ray is marched and shaded as by snerg_render_rays, its L2 loss
 * |C - C*|^2 is ADDED to *d_loss (caller zeroes; nullable), dL/dC = 2 (C - C*) is taken in
 * the kernel, and the adjoint ACCUMULATES into d_grad_atlas / d_grad_mlp exactly as
 * snerg_render_backward does for that upstream gradient (either nullable).
 *   d_target : float32 [n][3], the observed colours C*;
 *   d_rgb    : nullable float32 [n][3], receives C.
 * The same result as snerg_render_rays + snerg_l2_loss + snerg_render_backward, without
 * the per-ray state between them. d_mlp must be device weights. */
snerg_status snerg_train_rays(snerg_handle h, const snerg_camera* cams, int32_t n_cams, const int32_t* d_pix,
                              int64_t n, const float* d_mlp, const float* d_target, float* d_rgb, float* d_loss,
                              float* d_grad_atlas, float* d_grad_mlp, void* stream);

/* Photometric loss of Eq. 3 over n rays: *d_loss += sum |C - C*|^2 (ACCUMULATED, caller
 * zeroes; nullable), d_grad [n][3] = 2 (C - C*) (nullable). d_rgb, d_target: [n][3]. */
snerg_status snerg_l2_loss(const float* d_rgb, const float* d_target, int64_t n, float* d_grad,
                           float* d_loss, void* stream);

/* One Adam step (the optimiser of the paper's fine-tuning, Sec. 5.5; learning rate 3e-4
 * there) on n float32 parameters in place: m and v are the caller's moment buffers
 * (zero before step 1), step counts from 1 (bias correction 1 - beta^step). */
snerg_status snerg_adam_step(float* d_param, float* d_m, float* d_v, const float* d_grad, int64_t n,
                             float lr, float beta1, float beta2, float eps, int32_t step, void* stream);

/* Ray-list render for callers that cannot allocate device memory. The paper has no
 * counterpart: this entry point exists for callers such as a plug-in inside a host
 * application that owns all GPU memory through its own pool and forbids cudaMalloc, a
 * real-time loop that cannot afford the implicit device synchronisation of
 * cudaMalloc/cudaFree, or a sandboxed caller that is only handed its input and output
 * buffers. It needs no handle and no workspace, and calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *   desc, d_indirection, d_atlas, num_blocks : the scene, laid out as for snerg_create;
 *       read in place during the call (not copied, not validated: entries must lie in
 *       [-1, num_blocks); an entry >= num_blocks is reported and read as empty).
 *   cams, n_cams, d_pix, n, d_mlp, d_rgb : as for snerg_render_rays (same colours up to
 *       floating-point rounding; it renders from the unpadded atlas without the voxel
 *       distance map).
 *   d_status : nullable device int32; receives SNERG_OK or the first device-side error
 *       of this call (SNERG_E_INVAL for a bad pixel or atlas entry).
 * Limit: N / B <= 64; larger grids return SNERG_E_UNSUPPORTED. Of the scene flags only
 * SNERG_FLAG_UNPREMULTIPLY is accepted (others return SNERG_E_INVAL).
 * Scratch: a status word and the block-level empty-space distance map live in one static
 * device array of 786,688 bytes that every GPU loading this library holds until the
 * process exits. The first call on each device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current): make that first call before any
 * stream capture. The address is kept for the life of the process, so do not use this
 * entry point after a device reset (cudaDeviceReset or a primary-context reset may move
 * the array). All calls share the array and each call rewrites it, so calls whose
 * work overlaps on the GPU (different streams or host threads) race; serialise them.
 * Asynchronous on `stream`. */
snerg_status snerg_render_rays_noalloc(const snerg_scene_desc* desc, const int32_t* d_indirection,
                                       const uint8_t* d_atlas, int64_t num_blocks,
                                       const snerg_camera* cams, int32_t n_cams,
                                       const int32_t* d_pix, int64_t n, const float* d_mlp,
                                       float* d_rgb, int32_t* d_status, void* stream);

/* Largest number of density blobs of an analytic bake field. */
#define SNERG_BAKE_MAX_BLOBS 64

/* An analytic radiance field that stands in for the trained network when baking
 * (Sec. 5.3). HOST memory, read during the call only. World units throughout.
 *   density sigma(x) = sum_i peak_i exp(-|x - c_i|^2 / (2 s_i^2)),
 *                      blob[i] = {c_x, c_y, c_z, s_i > 0, peak_i >= 0};
 *   channel c of (diffuse r, g, b, f0..f3) = 0.5 + 0.5 sin(w_c . x + phi_c),
 *                      color[c] = {w_x, w_y, w_z, phi}. */
typedef struct {
    int32_t n_blob;                            /* 0..SNERG_BAKE_MAX_BLOBS */
    float tau_alpha;                           /* culling threshold, in (0, 1); paper: 0.005 */
    float blob[SNERG_BAKE_MAX_BLOBS][5];
    float color[7][4];
    float jitter[16][3];                       /* offsets of the 16 anti-aliasing samples in
                                                  voxel units (the paper draws them from a
                                                  Gaussian of std 1/sqrt(12) voxels), same for
                                                  every voxel; |offset| <= 8 */
} snerg_bake_field;

/* Bytes of device workspace snerg_bake needs (G^3 flags, G^3 block list, counters); 0 if
 * the description is invalid or G = N / B > 256. */
size_t snerg_bake_workspace_bytes(const snerg_scene_desc* desc);

/* Bake an analytic field into the Sec. 5.1 representation on the GPU (Sec. 5.3-5.4):
 *   1. alpha = 1 - exp(-sigma v) at every voxel centre of the N^3 grid (v = extent / N);
 *      a macroblock is kept iff its largest alpha is >= tau_alpha (the paper also culls by
 *      visibility from the training views; there are no training views here);
 *   2. kept macroblocks get atlas slots 0, 1, ... in raster order of the indirection grid
 *      (x fastest), culled ones -1;
 *   3. each voxel of a kept block stores the average of the field over its 16 jittered
 *      positions (voxel centre + jitter * v), as 8-bit codes round(255 x) clamped to
 *      [0, 255]: density as sigma / desc->sigma_max, then the 7 channels.
 * Outputs (device, caller-owned): d_indirection int32 [G][G][G] (z, y, x); d_atlas uint8
 * [max_blocks][B][B][B][8] laid out as snerg_create reads it. *num_blocks (host) receives
 * the number of kept blocks. If that exceeds max_blocks the atlas is not written and
 * SNERG_E_NOMEM is returned (retry with max_blocks = *num_blocks). desc->bg and max_steps
 * are not used; of desc->flags only SNERG_FLAG_ALPHA_ATLAS matters (channel 0 then stores
 * alpha = 1 - exp(-sigma v) of the averaged density). Floating point: binary32 (PTX ex2.approx, sincosf); over each unit of work a
 * blob is left out where its term stays below 2^-30 min(sigma_max, sigma_tau), sigma_tau =
 * -ln(1 - tau_alpha) / v. Codes agree with an exact evaluation except where the exact value
 * lies within about 1e-5 of a rounding boundary (and likewise for the tau_alpha decision).
 * SYNCHRONISES `stream`. */
snerg_status snerg_bake(const snerg_scene_desc* desc, const snerg_bake_field* field,
                        int32_t* d_indirection, uint8_t* d_atlas, int64_t max_blocks,
                        void* d_workspace, size_t ws_bytes, int64_t* num_blocks, void* stream);

/* SYNCHRONISES `stream`, returns and clears the device status word (SNERG_OK or the
 * first device error recorded since the last call); SNERG_E_DEVICE_FAULT if the stream
 * reports a sticky device fault (the context is unusable afterwards), SNERG_E_CUDA for
 * any other asynchronous CUDA error. */
snerg_status snerg_last_status(snerg_handle h, void* stream);

/* Number of kernels the library launched through this handle since creation. */
int64_t snerg_launch_count(snerg_handle h);

/* SYNCHRONISES `stream`. What the handle's last snerg_render with schedule = 1 did:
 * *ordered = 1 if it launched its tiles in the order recorded on the render before (0:
 * raster order), *sparse_tiles = how many of its slowest tiles it rendered sparsely (0 and 0
 * if there was no such render). For tests and tuning; the render does not need it. */
snerg_status snerg_schedule_stats(snerg_handle h, void* stream, int32_t* sparse_tiles, int32_t* ordered);

/* Tile shape and CTAs/SM chosen by the last persistent launch (or 0s). */
snerg_status snerg_persistent_config(snerg_handle h, int32_t* tile_w, int32_t* tile_h,
                                     int32_t* ctas_per_sm);

/* Release host state (cached graphs). Device memory is the caller's. NULL is allowed. */
void snerg_destroy(snerg_handle h);

/* Static string for a status code. */
const char* snerg_status_str(snerg_status s);

#ifdef __cplusplus
}
#endif

#endif /* SNERG_H */
