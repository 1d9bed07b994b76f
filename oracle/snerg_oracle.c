/*
 * snerg_oracle.c -- plain, slow FP64 CPU renderer for baked SNeRG grids.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call this file: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg use it. It shares no
 * code, header, table or constant with the CUDA renderer.
 *
 * What it computes (paper: Sec. 4.2 Eqs. 2, 5-7; Sec. 5.1-5.2; App. A):
 *   * one ray per pixel of a pinhole camera, r(t) = o + t d (Sec. 4.1);
 *   * the ray is clipped to the N^3 virtual grid and sampled once per voxel width
 *     (Sec. 5.2), on the lattice t_k = t_start + (k + 1/2) voxel widths;
 *   * a sample whose nearest voxel lies in an empty macroblock (indirection entry -1,
 *     Sec. 5.1), or whose nearest-voxel density is zero (App. A), contributes nothing;
 *   * otherwise density, diffuse colour and the 4 features are trilinearly
 *     interpolated on the virtual dense grid (Sec. 5.2) and alpha-composited
 *     (Eqs. 2, 5, 6): w_k = T_k (1 - exp(-sigma_k delta)), T_k = exp(-sum_{k'<k} sigma delta);
 *   * marching stops once the opacity saturates (Sec. 5.2), read as T < 1e-3;
 *   * if any sample was composited, the tiny MLP (2 hidden layers of 16, Sec. 4.2)
 *     adds a view-dependent residual (Eq. 7): C = C_d + sigmoid(MLP(C_d, V, PE(d))),
 *     plus T_final * background (App. A evaluates the MLP only where alpha > 0);
 *   * optional non-deferred comparison model (the per-sample ablation of Sec. 6): the same
 *     MLP evaluated at every composited sample on that sample's own (c_d, v), the sample
 *     colour c_d + sigmoid(MLP(c_d, v, PE(d))) composited with the same weights, no
 *     per-pixel residual;
 *   * optional partial un-premultiply (App. C, forward-facing scenes): after compositing,
 *     (C_d, alpha, V) *= min(1, 1.5 alpha) / alpha where alpha = 1 - T_final > 0, so the
 *     MLP sees the scaled C_d and V and the background weight becomes 1 - min(1, 1.5 alpha);
 *   * optional alpha atlas (App. A keeps alpha in its own texture): channel 0 holds alpha
 *     codes, the sample's alpha is the trilinear code / 255, T <- T (1 - alpha), and the
 *     exit test is T < 1e-3 on a binary32 running product;
 *   * optional ablation without the view-dependence network (the paper's performance
 *     ablation, Sec. 6): C = C_d + T_final * background;
 *   * the backward pass is the exact adjoint of the above w.r.t. the decoded colour and
 *     feature values and the MLP weights, with density frozen (Sec. 5.5 fine-tunes the
 *     per-pixel network against an L2 image loss, Eq. 3);
 *   * baking (Sec. 5.3) of an analytic field that stands in for the trained network:
 *     alpha = 1 - exp(-sigma v) at voxel centres, blocks with max alpha < tau_alpha
 *     culled, 16 Gaussian-jittered samples per kept voxel averaged, 8-bit codes
 *     (Sec. 5.4), kept blocks packed in raster order.
 *
 * Method decisions that the paper leaves open are taken as follows and are part of the
 * definition this oracle states (they fix which integer decisions are made):
 *   * integer decisions (sample lattice, nearest voxel, block lookup, the early-exit
 *     test) are taken in IEEE binary32 with one rounding per operation, in the exact
 *     operation order written below (compile with -ffp-contract=off);
 *   * the early-exit test accumulates the binary32 optical depth tau += s * kappa,
 *     s = binary32 trilinear of the density codes, kappa = binary32(sigma_max * delta / 255),
 *     and stops after the sample with tau > binary32(ln 1000);
 *   * all colour arithmetic (trilinear weights, alpha, transmittance, MLP) is FP64.
 *
 * Atlas layout consumed: atlas[nb][B][B][B][8] uint8 (z, y, x, channel), channels
 * sigma, r, g, b, f0..f3; indirection ind[G][G][G] int32 (z, y, x), -1 = empty.
 * Camera record: float[16] = c2w row-major 3x4 (12), fx, fy, cx, cy.
 */
#pragma STDC FP_CONTRACT OFF
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_E_INVAL 1
#define OR_E_STEP_LIMIT 4

#define MLP_IN 34
#define MLP_H 16
#define MLP_OUT 3
#define NPARAM 883
/* flat MLP layout: W1[16][34], b1[16], W2[16][16], b2[16], W3[3][16], b3[3] */
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + MLP_H * MLP_IN)
#define OFF_W2 (OFF_B1 + MLP_H)
#define OFF_B2 (OFF_W2 + MLP_H * MLP_H)
#define OFF_W3 (OFF_B2 + MLP_H)
#define OFF_B3 (OFF_W3 + MLP_OUT * MLP_H)

typedef struct {
    int32_t N, B, G;
    float bmin[3];
    float extent;
    double sigma_max;
    double bg[3];
    const int32_t* ind;
    const uint8_t* atlas;
    const double* val;     /* decoded colour/feature values [nb][B^3][8] (channel 0 unused) */
    int64_t nb;
    float kappa32;         /* binary32(sigma_max * delta / 255) */
    float taumax32;        /* binary32(ln 1000) */
    double delta;          /* voxel width in world units, extent / N */
    int64_t max_iter;
    int unpremultiply;     /* App. C partial un-premultiply */
    int per_sample_mlp;    /* non-deferred comparison model */
    int alpha_atlas;       /* channel 0 holds alpha codes (App. A's alpha texture) */
    int no_mlp;            /* the performance ablation without the view-dependence network */
    float tmin32;          /* binary32(1e-3): the alpha-atlas exit threshold on T */
    float inv255_32;       /* binary32(1 / 255) */
    const double* mlp;     /* weights, for the per-sample model */
} OScene;

/* ------------------------------------------------------------------------- */
/* virtual dense grid: voxel (x,y,z) clamped to the grid; empty blocks read 0 */

static int64_t voxel_slot(const OScene* S, int32_t x, int32_t y, int32_t z, int64_t* local) {
    int32_t bx = x / S->B, by = y / S->B, bz = z / S->B;
    int64_t slot = S->ind[((int64_t)bz * S->G + by) * S->G + bx];
    int32_t lx = x - bx * S->B, ly = y - by * S->B, lz = z - bz * S->B;
    *local = ((int64_t)lz * S->B + ly) * S->B + lx;
    return slot;
}

static int32_t clampi(int32_t v, int32_t lo, int32_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

static uint8_t density_code(const OScene* S, int32_t x, int32_t y, int32_t z) {
    int64_t local;
    int64_t slot = voxel_slot(S, x, y, z, &local);
    if (slot < 0) return 0;
    return S->atlas[(slot * S->B * S->B * S->B + local) * 8];
}

static double channel_value(const OScene* S, int32_t x, int32_t y, int32_t z, int c) {
    int64_t local;
    int64_t slot = voxel_slot(S, x, y, z, &local);
    if (slot < 0) return 0.0;
    int64_t idx = (slot * S->B * S->B * S->B + local) * 8 + c;
    if (S->val) return S->val[idx];
    return (double)S->atlas[idx] / 255.0;
}

/* ------------------------------------------------------------------------- */
/* ray generation and clipping (binary32, fixed operation order) */

typedef struct {
    float o[3];      /* origin in voxel units of the virtual grid */
    float d[3];      /* unit direction (world = voxel frame up to scale) */
    float t_start, t_end;
    int hit;
} ORay;

static ORay ray_setup(const OScene* S, const float* cam, int32_t px, int32_t py) {
    ORay r;
    const float* m = cam;    /* c2w row-major 3x4 */
    float fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    float xs = ((float)px + 0.5f - cx) / fx;
    float ys = ((float)py + 0.5f - cy) / fy;
    float dc0 = xs, dc1 = -ys, dc2 = -1.0f;            /* camera looks along -z, +y up */
    float d0 = m[0] * dc0 + m[1] * dc1 + m[2] * dc2;
    float d1 = m[4] * dc0 + m[5] * dc1 + m[6] * dc2;
    float d2 = m[8] * dc0 + m[9] * dc1 + m[10] * dc2;
    float n2 = d0 * d0 + d1 * d1 + d2 * d2;
    float nrm = sqrtf(n2);
    r.d[0] = d0 / nrm;
    r.d[1] = d1 / nrm;
    r.d[2] = d2 / nrm;
    float s = (float)S->N / S->extent;
    r.o[0] = (m[3] - S->bmin[0]) * s;
    r.o[1] = (m[7] - S->bmin[1]) * s;
    r.o[2] = (m[11] - S->bmin[2]) * s;
    /* slab clip against [0, N]^3 */
    float tn = -INFINITY, tf = INFINITY;
    float fN = (float)S->N;
    r.hit = 1;
    for (int i = 0; i < 3; ++i) {
        if (r.d[i] != 0.0f) {
            float ta = (-r.o[i]) / r.d[i];
            float tb = (fN - r.o[i]) / r.d[i];
            float lo = fminf(ta, tb), hi = fmaxf(ta, tb);
            tn = fmaxf(tn, lo);
            tf = fminf(tf, hi);
        } else if (r.o[i] < 0.0f || r.o[i] > fN) {
            r.hit = 0;
        }
    }
    r.t_start = fmaxf(tn, 0.0f);
    r.t_end = tf;
    if (!(r.t_start < r.t_end)) r.hit = 0;
    return r;
}

/* ------------------------------------------------------------------------- */
/* one ray: forward march (and optional adjoint scatter into grad)            */

typedef struct {
    double cd[3], v[4];
    double T;
    double rgb_ps[3];      /* per-sample model: sum_k w_k (c_d,k + residual_k) */
    int32_t steps, active;
    int status;
} OMarch;

static void mlp_input(const double cd[3], const double v[4], const float d[3], double x[]);
static double sample_residual(const double* w, const double x[], int c);

static void march(const OScene* S, const ORay* r, uint64_t* trace, int32_t trace_cap,
                  const double* g_feat /* 7 adjoint values or NULL */, double* grad, OMarch* out) {
    memset(out, 0, sizeof(*out));
    out->T = 1.0;
    if (!r->hit) return;
    const int32_t N = S->N;
    const int64_t vox = (int64_t)S->B * S->B * S->B;
    float tau = 0.0f;
    float Tc = 1.0f;        /* alpha atlas: binary32 transmittance of the exit test */
    for (int64_t k = 0;; ++k) {
        if (k >= S->max_iter) { out->status = OR_E_STEP_LIMIT; return; }
        float tk = r->t_start + ((float)k + 0.5f);
        if (!(tk < r->t_end)) break;
        float u[3];
        int32_t j[3];
        for (int i = 0; i < 3; ++i) {
            u[i] = r->o[i] + tk * r->d[i];
            j[i] = clampi((int32_t)floorf(u[i]), 0, N - 1);
        }
        int64_t local;
        int64_t slot = voxel_slot(S, j[0], j[1], j[2], &local);
        if (slot < 0) continue;                       /* empty macroblock: skipped */
        out->steps++;
        uint8_t qn = S->atlas[(slot * vox + local) * 8];
        if (qn == 0) continue;                        /* nearest-voxel density probe */
        if (out->active < trace_cap)
            trace[out->active] = ((uint64_t)j[2] * N + (uint64_t)j[1]) * N + (uint64_t)j[0];
        out->active++;

        /* corners of the cell-centred trilinear stencil */
        float xs[3], fl[3], f32[3], g32[3];
        int32_t c0[3], c1[3];
        double f64[3];
        for (int i = 0; i < 3; ++i) {
            xs[i] = u[i] - 0.5f;
            fl[i] = floorf(xs[i]);
            f32[i] = xs[i] - fl[i];
            g32[i] = 1.0f - f32[i];
            c0[i] = clampi((int32_t)fl[i], 0, N - 1);
            c1[i] = clampi((int32_t)fl[i] + 1, 0, N - 1);
            f64[i] = ((double)u[i] - 0.5) - (double)fl[i];
        }
        float q[2][2][2];       /* q[cz][cy][cx] */
        double w64[2][2][2];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int c = 0; c < 2; ++c) {
                    int32_t X = c ? c1[0] : c0[0], Y = b ? c1[1] : c0[1], Z = a ? c1[2] : c0[2];
                    q[a][b][c] = (float)density_code(S, X, Y, Z);
                    w64[a][b][c] = (c ? f64[0] : 1.0 - f64[0]) * (b ? f64[1] : 1.0 - f64[1]) *
                                   (a ? f64[2] : 1.0 - f64[2]);
                }
        /* binary32 control: x, then y, then z */
        float e00 = q[0][0][0] * g32[0] + q[0][0][1] * f32[0];
        float e10 = q[0][1][0] * g32[0] + q[0][1][1] * f32[0];
        float e01 = q[1][0][0] * g32[0] + q[1][0][1] * f32[0];
        float e11 = q[1][1][0] * g32[0] + q[1][1][1] * f32[0];
        float e0 = e00 * g32[1] + e10 * f32[1];
        float e1 = e01 * g32[1] + e11 * f32[1];
        float s32 = e0 * g32[2] + e1 * f32[2];
        int saturated;
        if (S->alpha_atlas) {
            /* channel 0 is alpha itself: a = s * binary32(1/255), T <- T (1 - a), stop once
             * T < binary32(1e-3) */
            float a32 = s32 * S->inv255_32;
            Tc = Tc * (1.0f - a32);
            saturated = Tc < S->tmin32;
        } else {
            float od32 = s32 * S->kappa32;
            tau = tau + od32;
            saturated = tau > S->taumax32;
        }

        /* FP64 compositing, Eqs. 2, 5, 6 */
        double qi = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int c = 0; c < 2; ++c) qi += w64[a][b][c] * (double)q[a][b][c];
        double sigma = qi / 255.0 * S->sigma_max;
        double x = sigma * S->delta;
        double alpha = S->alpha_atlas ? qi / 255.0 : -expm1(-x);
        double wk = out->T * alpha;
        if (S->per_sample_mlp) {
            double cdk[3] = {0, 0, 0}, vk[4] = {0, 0, 0, 0}, x[34];
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int c = 0; c < 2; ++c) {
                        int32_t X = c ? c1[0] : c0[0], Y = b ? c1[1] : c0[1], Z = a ? c1[2] : c0[2];
                        for (int ch = 0; ch < 3; ++ch) cdk[ch] += w64[a][b][c] * channel_value(S, X, Y, Z, 1 + ch);
                        for (int ch = 0; ch < 4; ++ch) vk[ch] += w64[a][b][c] * channel_value(S, X, Y, Z, 4 + ch);
                    }
            mlp_input(cdk, vk, r->d, x);
            for (int ch = 0; ch < 3; ++ch) out->rgb_ps[ch] += wk * (cdk[ch] + sample_residual(S->mlp, x, ch));
        }
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int c = 0; c < 2; ++c) {
                    int32_t X = c ? c1[0] : c0[0], Y = b ? c1[1] : c0[1], Z = a ? c1[2] : c0[2];
                    double cw = wk * w64[a][b][c];
                    if (g_feat) {
                        int64_t lc;
                        int64_t sc = voxel_slot(S, X, Y, Z, &lc);
                        if (sc >= 0) {
                            double* gp = grad + (sc * vox + lc) * 8;
                            for (int ch = 0; ch < 7; ++ch) {
                                double gv = cw * g_feat[ch];
                                #pragma omp atomic
                                gp[1 + ch] += gv;
                            }
                        }
                    }
                    for (int ch = 0; ch < 3; ++ch) out->cd[ch] += cw * channel_value(S, X, Y, Z, 1 + ch);
                    for (int ch = 0; ch < 4; ++ch) out->v[ch] += cw * channel_value(S, X, Y, Z, 4 + ch);
                }
        out->T *= S->alpha_atlas ? 1.0 - alpha : exp(-x);
        if (saturated) break;                          /* opacity saturated */
    }
}

/* App. C: (C_d, alpha, V) *= min(1, 1.5 alpha) / alpha when alpha = 1 - T > 0. Returns the
 * scale (1 when not applied) and rewrites m->cd, m->v and m->T accordingly. */
static double unpremultiply(const OScene* S, OMarch* m) {
    double a = 1.0 - m->T;
    if (!S->unpremultiply || !(a > 0.0)) return 1.0;
    double a2 = 1.5 * a < 1.0 ? 1.5 * a : 1.0;
    double sc = a2 / a;
    for (int c = 0; c < 3; ++c) m->cd[c] *= sc;
    for (int c = 0; c < 4; ++c) m->v[c] *= sc;
    m->T = 1.0 - a2;
    return sc;
}

/* ------------------------------------------------------------------------- */
/* view-dependence MLP, Eq. 7: 34 -> 16 ReLU -> 16 ReLU -> 3 -> sigmoid       */

static void mlp_input(const double cd[3], const double v[4], const float d[3], double x[MLP_IN]) {
    x[0] = cd[0]; x[1] = cd[1]; x[2] = cd[2];
    x[3] = v[0]; x[4] = v[1]; x[5] = v[2]; x[6] = v[3];
    x[7] = d[0]; x[8] = d[1]; x[9] = d[2];
    for (int l = 0; l < 4; ++l) {
        double sc = (double)(1 << l);
        for (int i = 0; i < 3; ++i) {
            x[10 + 6 * l + i] = sin(sc * (double)d[i]);
            x[13 + 6 * l + i] = cos(sc * (double)d[i]);
        }
    }
}

typedef struct { double p1[MLP_H], h1[MLP_H], p2[MLP_H], h2[MLP_H], z[MLP_OUT], res[MLP_OUT]; } OMlp;

static void mlp_forward(const double* w, const double x[MLP_IN], OMlp* m) {
    for (int o = 0; o < MLP_H; ++o) {
        double a = w[OFF_B1 + o];
        for (int i = 0; i < MLP_IN; ++i) a += w[OFF_W1 + o * MLP_IN + i] * x[i];
        m->p1[o] = a;
        m->h1[o] = a > 0.0 ? a : 0.0;
    }
    for (int o = 0; o < MLP_H; ++o) {
        double a = w[OFF_B2 + o];
        for (int i = 0; i < MLP_H; ++i) a += w[OFF_W2 + o * MLP_H + i] * m->h1[i];
        m->p2[o] = a;
        m->h2[o] = a > 0.0 ? a : 0.0;
    }
    for (int o = 0; o < MLP_OUT; ++o) {
        double a = w[OFF_B3 + o];
        for (int i = 0; i < MLP_H; ++i) a += w[OFF_W3 + o * MLP_H + i] * m->h2[i];
        m->z[o] = a;
        m->res[o] = 1.0 / (1.0 + exp(-a));
    }
}

/* residual channel c of the MLP at input x (per-sample model) */
static double sample_residual(const double* w, const double x[], int c) {
    OMlp m;
    mlp_forward(w, x, &m);
    return m.res[c];
}

/* adjoint of mlp_forward: g_res -> grads of the weights (accumulated) and of the input */
static void mlp_backward(const double* w, const double x[MLP_IN], const OMlp* m, const double g_res[MLP_OUT],
                         double* gw, double gx[MLP_IN]) {
    double gz[MLP_OUT], gh2[MLP_H], gh1[MLP_H];
    for (int o = 0; o < MLP_OUT; ++o) gz[o] = g_res[o] * m->res[o] * (1.0 - m->res[o]);
    for (int i = 0; i < MLP_H; ++i) gh2[i] = 0.0;
    for (int o = 0; o < MLP_OUT; ++o) {
        gw[OFF_B3 + o] += gz[o];
        for (int i = 0; i < MLP_H; ++i) {
            gw[OFF_W3 + o * MLP_H + i] += gz[o] * m->h2[i];
            gh2[i] += w[OFF_W3 + o * MLP_H + i] * gz[o];
        }
    }
    for (int i = 0; i < MLP_H; ++i) gh2[i] = m->p2[i] > 0.0 ? gh2[i] : 0.0;
    for (int i = 0; i < MLP_H; ++i) gh1[i] = 0.0;
    for (int o = 0; o < MLP_H; ++o) {
        gw[OFF_B2 + o] += gh2[o];
        for (int i = 0; i < MLP_H; ++i) {
            gw[OFF_W2 + o * MLP_H + i] += gh2[o] * m->h1[i];
            gh1[i] += w[OFF_W2 + o * MLP_H + i] * gh2[o];
        }
    }
    for (int i = 0; i < MLP_H; ++i) gh1[i] = m->p1[i] > 0.0 ? gh1[i] : 0.0;
    for (int i = 0; i < MLP_IN; ++i) gx[i] = 0.0;
    for (int o = 0; o < MLP_H; ++o) {
        gw[OFF_B1 + o] += gh1[o];
        for (int i = 0; i < MLP_IN; ++i) {
            gw[OFF_W1 + o * MLP_IN + i] += gh1[o] * x[i];
            gx[i] += w[OFF_W1 + o * MLP_IN + i] * gh1[o];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* exported entry points                                                      */

static int scene_init(OScene* S, int32_t N, int32_t B, const float* bmin, float extent, double sigma_max,
                      const double* bg, const int32_t* ind, const uint8_t* atlas, const double* val, int64_t nb,
                      int32_t flags) {
    if (N <= 0 || B <= 0 || N % B != 0 || !(extent > 0.0f)) return OR_E_INVAL;
    S->N = N; S->B = B; S->G = N / B;
    for (int i = 0; i < 3; ++i) { S->bmin[i] = bmin[i]; S->bg[i] = bg[i]; }
    S->extent = extent;
    S->sigma_max = sigma_max;
    S->ind = ind; S->atlas = atlas; S->val = val; S->nb = nb;
    S->delta = (double)extent / (double)N;
    S->kappa32 = (float)(sigma_max * ((double)extent / (double)N) / 255.0);
    S->taumax32 = (float)log(1000.0);
    S->max_iter = 4 * (int64_t)N + 16;
    if ((flags & ~15) || (flags & 3) == 3 || (flags & 10) == 10) return OR_E_INVAL;   /* 1 and 8 are deferred-model options */
    S->unpremultiply = (flags & 1) != 0;
    S->per_sample_mlp = (flags & 2) != 0;
    S->alpha_atlas = (flags & 4) != 0;
    S->no_mlp = (flags & 8) != 0;
    S->tmin32 = (float)1e-3;
    S->inv255_32 = (float)(1.0 / 255.0);
    S->mlp = NULL;
    for (int64_t i = 0; i < (int64_t)S->G * S->G * S->G; ++i)
        if (ind[i] < -1 || ind[i] >= nb) return OR_E_INVAL;
    return OR_OK;
}

/* Render a list of rays. pix[n][3] = (camera, x, y). Outputs (nullable except rgb):
 *   rgb[n][3]; aux[n][8] = C_d(3), V(4), 1 - T_final; counts[n][2] = steps, active;
 *   trace[n][trace_cap] = linear indices z*N*N + y*N + x of composited samples.
 * Returns 0, or the first nonzero ray status. */
int oracle_render_rays(int32_t N, int32_t B, const float* bmin, float extent, double sigma_max, const double* bg,
                       const int32_t* ind, const uint8_t* atlas, const double* val, int64_t nb, int32_t flags,
                       const double* mlp, const float* cams, int32_t n_cams, const int32_t* pix, int64_t n,
                       double* rgb, double* aux, int32_t* counts, uint64_t* trace, int32_t trace_cap) {
    OScene S;
    int st = scene_init(&S, N, B, bmin, extent, sigma_max, bg, ind, atlas, val, nb, flags);
    if (st) return st;
    S.mlp = mlp;
    int err = 0;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int32_t ci = pix[3 * i];
        if (ci < 0 || ci >= n_cams) {
            #pragma omp atomic write
            err = OR_E_INVAL;
            continue;
        }
        ORay r = ray_setup(&S, cams + 16 * ci, pix[3 * i + 1], pix[3 * i + 2]);
        OMarch m;
        march(&S, &r, trace ? trace + i * trace_cap : NULL, trace ? trace_cap : 0, NULL, NULL, &m);
        if (m.status) {
            #pragma omp atomic write
            err = m.status;
        }
        const double raw_T = m.T;
        double raw_cd[3], raw_v[4];
        for (int c = 0; c < 3; ++c) raw_cd[c] = m.cd[c];
        for (int c = 0; c < 4; ++c) raw_v[c] = m.v[c];
        unpremultiply(&S, &m);
        double res[3] = {0.0, 0.0, 0.0};
        if (m.active > 0 && !S.no_mlp) {
            double x[MLP_IN];
            OMlp mm;
            mlp_input(m.cd, m.v, r.d, x);
            mlp_forward(mlp, x, &mm);
            for (int c = 0; c < 3; ++c) res[c] = mm.res[c];
        }
        for (int c = 0; c < 3; ++c) {
            if (S.per_sample_mlp)
                rgb[3 * i + c] = m.rgb_ps[c] + m.T * S.bg[c];
            else
                rgb[3 * i + c] = (m.active > 0 ? m.cd[c] + res[c] : 0.0) + m.T * S.bg[c];
        }
        if (aux) {       /* the composites before any un-premultiply */
            for (int c = 0; c < 3; ++c) aux[8 * i + c] = raw_cd[c];
            for (int c = 0; c < 4; ++c) aux[8 * i + 3 + c] = raw_v[c];
            aux[8 * i + 7] = 1.0 - raw_T;
        }
        if (counts) { counts[2 * i] = m.steps; counts[2 * i + 1] = m.active; }
    }
    return err;
}

/* Adjoint of oracle_render_rays for an upstream gradient g_rgb[n][3] (dL/dC).
 * Accumulates dL/d(decoded value) of channels 1..7 into grad[nb][B^3][8] (channel 0,
 * density, is frozen and left untouched; grad may be NULL to skip it) and dL/d(MLP
 * weights) into gmlp[883]. */
int oracle_backward_rays(int32_t N, int32_t B, const float* bmin, float extent, double sigma_max, const double* bg,
                         const int32_t* ind, const uint8_t* atlas, const double* val, int64_t nb, int32_t flags,
                         const double* mlp, const float* cams, int32_t n_cams, const int32_t* pix, int64_t n,
                         const double* g_rgb, double* grad, double* gmlp) {
    OScene S;
    int st = scene_init(&S, N, B, bmin, extent, sigma_max, bg, ind, atlas, val, nb, flags);
    if (st) return st;
    if (S.per_sample_mlp) return OR_E_INVAL;   /* comparison model: forward only */
    int err = 0;
    #pragma omp parallel
    {
        double* gl = (double*)calloc(NPARAM, sizeof(double));
        #pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            int32_t ci = pix[3 * i];
            if (ci < 0 || ci >= n_cams) {
                #pragma omp atomic write
                err = OR_E_INVAL;
                continue;
            }
            ORay r = ray_setup(&S, cams + 16 * ci, pix[3 * i + 1], pix[3 * i + 2]);
            OMarch m;
            march(&S, &r, NULL, 0, NULL, NULL, &m);
            if (m.status) {
                #pragma omp atomic write
                err = m.status;
            }
            if (m.active == 0) continue;          /* C = T bg: no parameter reaches the output */
            /* the un-premultiply scale depends on density only (frozen): a constant factor */
            const double sc = unpremultiply(&S, &m);
            double x[MLP_IN], gx[MLP_IN];
            const double* g = g_rgb + 3 * i;
            if (S.no_mlp) {
                for (int c = 0; c < MLP_IN; ++c) gx[c] = 0.0;   /* C = s C_d + T bg */
            } else {
                OMlp mm;
                mlp_input(m.cd, m.v, r.d, x);
                mlp_forward(mlp, x, &mm);
                mlp_backward(mlp, x, &mm, g, gl, gx);
            }
            if (!grad) continue;                  /* only dL/dPhi requested */
            double gf[7];
            for (int c = 0; c < 3; ++c) gf[c] = sc * (g[c] + gx[c]);      /* C = s C_d + residual */
            for (int c = 0; c < 4; ++c) gf[3 + c] = sc * gx[3 + c];
            OMarch m2;
            march(&S, &r, NULL, 0, gf, grad, &m2);
        }
        #pragma omp critical
        for (int p = 0; p < NPARAM; ++p) gmlp[p] += gl[p];
        free(gl);
    }
    return err;
}

/* MLP alone on explicit inputs x[n][34] -> out[n][3] (sigmoid residual). */
void oracle_mlp_eval(const double* mlp, const double* x, int64_t n, double* out) {
    for (int64_t i = 0; i < n; ++i) {
        OMlp m;
        mlp_forward(mlp, x + MLP_IN * i, &m);
        for (int c = 0; c < 3; ++c) out[3 * i + c] = m.res[c];
    }
}

/* MLP input vector for a composited C_d, V and a direction d. */
void oracle_mlp_input(const double* cd, const double* v, const float* d, double* x) { mlp_input(cd, v, d, x); }

/* Ray set-up for one pixel: out_f[8] = o(3), d(3), t_start, t_end; returns hit flag. */
int oracle_ray(int32_t N, float extent, const float* bmin, const float* cam, int32_t px, int32_t py, float* out_f) {
    OScene S;
    memset(&S, 0, sizeof(S));
    S.N = N; S.extent = extent;
    for (int i = 0; i < 3; ++i) S.bmin[i] = bmin[i];
    ORay r = ray_setup(&S, cam, px, py);
    for (int i = 0; i < 3; ++i) { out_f[i] = r.o[i]; out_f[3 + i] = r.d[i]; }
    out_f[6] = r.t_start;
    out_f[7] = r.t_end;
    return r.hit;
}


/* ------------------------------------------------------------------------- */
/* Baking (Sec. 5.3) of an analytic field standing in for the trained network:  */
/* dense evaluation at voxel centres, alpha = 1 - exp(-sigma v), macroblock      */
/* culling at max alpha < tau_alpha, 16 Gaussian-jittered samples per voxel      */
/* (std v / sqrt 12, offsets given by the caller) averaged, 8-bit quantisation   */
/* (Sec. 5.4), packing in raster order of the kept blocks.                       */
/* Field: sigma(x) = sum_i peak_i exp(-|x - c_i|^2 / (2 s_i^2)) (blob[i] = c, s,  */
/* peak; world units); channel c (1..7) = 0.5 + 0.5 sin(w_c . x + phi_c).         */

static double field_sigma(const float* blob, int nb, double x, double y, double z) {
    double acc = 0.0;
    for (int i = 0; i < nb; ++i) {
        const float* b = blob + 5 * i;
        double dx = x - b[0], dy = y - b[1], dz = z - b[2];
        acc += (double)b[4] * exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * (double)b[3] * (double)b[3]));
    }
    return acc;
}

static double field_channel(const float* col, int c, double x, double y, double z) {
    const float* w = col + 4 * c;
    return 0.5 + 0.5 * sin((double)w[0] * x + (double)w[1] * y + (double)w[2] * z + (double)w[3]);
}

static uint8_t quant8(double v) {
    if (!(v > 0.0)) return 0;
    if (v >= 1.0) return 255;
    return (uint8_t)floor(v * 255.0 + 0.5);
}

/* Largest alpha = 1 - exp(-sigma v) over the voxel centres of macroblock (bx, by, bz). */
static double bake_block_alpha(int32_t B, const float* bmin, double v, int32_t n_blob, const float* blob,
                               int32_t bx, int32_t by, int32_t bz) {
    double amax = 0.0;
    for (int32_t z = 0; z < B; ++z)
        for (int32_t y = 0; y < B; ++y)
            for (int32_t x = 0; x < B; ++x) {
                double px = bmin[0] + ((bx * B + x) + 0.5) * v;
                double py = bmin[1] + ((by * B + y) + 0.5) * v;
                double pz = bmin[2] + ((bz * B + z) + 0.5) * v;
                double a = -expm1(-field_sigma(blob, n_blob, px, py, pz) * v);
                if (a > amax) amax = a;
            }
    return amax;
}

/* The 8 codes of every voxel of macroblock (bx, by, bz): the field averaged over the 16
 * jittered positions (voxel centre + jitter * v), density divided by sigma_max. */
static void bake_block_fill(int32_t B, const float* bmin, double v, float sigma_max, int32_t n_blob,
                            const float* blob, const float* color, const float* jitter, int32_t bx, int32_t by,
                            int32_t bz, uint8_t* out_block, double* raw_block /* nullable: 255 x before rounding */,
                            int32_t alpha_codes /* channel 0 = 1 - exp(-sigma v) instead of sigma / sigma_max */) {
    for (int32_t z = 0; z < B; ++z)
        for (int32_t y = 0; y < B; ++y)
            for (int32_t x = 0; x < B; ++x) {
                double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                for (int sidx = 0; sidx < 16; ++sidx) {
                    double px = bmin[0] + ((bx * B + x) + 0.5 + jitter[3 * sidx]) * v;
                    double py = bmin[1] + ((by * B + y) + 0.5 + jitter[3 * sidx + 1]) * v;
                    double pz = bmin[2] + ((bz * B + z) + 0.5 + jitter[3 * sidx + 2]) * v;
                    acc[0] += field_sigma(blob, n_blob, px, py, pz);
                    for (int c = 0; c < 7; ++c) acc[1 + c] += field_channel(color, c, px, py, pz);
                }
                const int64_t o = (((int64_t)z * B + y) * B + x) * 8;
                uint8_t* out = out_block + o;
                const double d0 = alpha_codes ? -expm1(-acc[0] / 16.0 * v) : acc[0] / 16.0 / (double)sigma_max;
                out[0] = quant8(d0);
                for (int c = 0; c < 7; ++c) out[1 + c] = quant8(acc[1 + c] / 16.0);
                if (raw_block) {
                    raw_block[o] = d0 * 255.0;
                    for (int c = 0; c < 7; ++c) raw_block[o + 1 + c] = acc[1 + c] / 16.0 * 255.0;
                }
            }
}

/* Outputs: ind[G^3] (-1 or slot), atlas[max_blocks][B^3][8]; returns the number of
 * kept blocks (or -1 if more than max_blocks), and per-block maximum alpha in
 * block_alpha[G^3] (for diagnosing threshold ties). */
int64_t oracle_bake(int32_t N, int32_t B, const float* bmin, float extent, float sigma_max, float tau_alpha,
                    int32_t n_blob, const float* blob, const float* color, const float* jitter /*[16][3]*/,
                    int32_t* ind, uint8_t* atlas, int64_t max_blocks, double* block_alpha, int32_t alpha_codes) {
    const int32_t G = N / B;
    const double v = (double)extent / (double)N;
    const int64_t G3 = (int64_t)G * G * G;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < G3; ++b)
        block_alpha[b] = bake_block_alpha(B, bmin, v, n_blob, blob, (int32_t)(b % G), (int32_t)((b / G) % G),
                                          (int32_t)(b / ((int64_t)G * G)));
    int64_t nb = 0;
    for (int64_t b = 0; b < G3; ++b) {
        if (block_alpha[b] >= (double)tau_alpha) {
            if (nb >= max_blocks) return -1;
            ind[b] = (int32_t)nb++;
        } else {
            ind[b] = -1;
        }
    }
    const int64_t vox = (int64_t)B * B * B;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < G3; ++b) {
        if (ind[b] < 0) continue;
        bake_block_fill(B, bmin, v, sigma_max, n_blob, blob, color, jitter, (int32_t)(b % G),
                        (int32_t)((b / G) % G), (int32_t)(b / ((int64_t)G * G)), atlas + (int64_t)ind[b] * vox * 8,
                        NULL, alpha_codes);
    }
    return nb;
}

/* The same quantities for a list of macroblocks (raster indices), whether kept or not:
 * their maximum alpha and their 8-bit content, and optionally the values before rounding
 * (255 x), which tell how close each code is to a rounding boundary. For sampled checks
 * of large bakes. */
void oracle_bake_blocks(int32_t N, int32_t B, const float* bmin, float extent, float sigma_max, int32_t n_blob,
                        const float* blob, const float* color, const float* jitter, int64_t n,
                        const int64_t* blocks, double* block_alpha, uint8_t* content, double* raw,
                        int32_t alpha_codes) {
    const int32_t G = N / B;
    const double v = (double)extent / (double)N;
    const int64_t vox = (int64_t)B * B * B;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) {
        const int64_t b = blocks[i];
        const int32_t bx = (int32_t)(b % G), by = (int32_t)((b / G) % G), bz = (int32_t)(b / ((int64_t)G * G));
        block_alpha[i] = bake_block_alpha(B, bmin, v, n_blob, blob, bx, by, bz);
        bake_block_fill(B, bmin, v, sigma_max, n_blob, blob, color, jitter, bx, by, bz, content + i * vox * 8,
                        raw ? raw + i * vox * 8 : NULL, alpha_codes);
    }
}


/* ------------------------------------------------------------------------- */
/* 8-bit requantisation (Sec. 5.4) of fine-tuned values: code = floor(255 x + 1/2) clamped
 * to [0, 255], the rounding decision taken in binary32 (one fused multiply-add, correctly
 * rounded, then floor), the precision the kernels decide it in. NaN -> 0. */
void oracle_requantize(const float* x, int64_t n, uint8_t* out) {
    for (int64_t i = 0; i < n; ++i) {
        const float q = floorf(fmaf(x[i], 255.0f, 0.5f));
        out[i] = q > 0.0f ? (q < 255.0f ? (uint8_t)q : 255) : 0;
    }
}


/* Threads the parallel loops use (the timing of the CPU baseline reports it), and a way to
 * change it for the calling thread's later loops. */
int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
