/*
 * Seeded synthetic volume filler for SNeRG test and benchmark scenes.
 *
 * This is an INPUT GENERATOR. It holds none of the renderer's arithmetic: it only
 * writes uint8 voxel values (density plus seven colour/feature channels) for a list
 * of macroblocks, from analytic fields whose parameters the Python side draws from a
 * seeded generator. Both the CUDA renderer and the CPU oracle consume its output.
 *
 * Layout written (one macroblock = B^3 voxels, z slowest, then y, then x):
 *   out[blk][z][y][x][8]  channel 0 = density code, 1..3 = diffuse RGB, 4..7 = features
 * Voxel centres are at integer + 0.5 in voxel units of the virtual N^3 grid.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

static inline uint8_t quant01(double v) {
    if (!(v > 0.0)) return 0;
    if (v >= 1.0) return 255;
    return (uint8_t)floor(v * 255.0 + 0.5);
}

/* Sum of isotropic Gaussian blobs. g[i] = {cx, cy, cz, std, amp} in unit-cube units.
 * Field values below `cut` are set to zero before scaling by `scale`. */
static double gauss_field(const double* g, int ng, double px, double py, double pz) {
    double acc = 0.0;
    for (int i = 0; i < ng; ++i) {
        const double* p = g + 5 * i;
        double dx = px - p[0], dy = py - p[1], dz = pz - p[2];
        double r2 = dx * dx + dy * dy + dz * dz;
        acc += p[4] * exp(-0.5 * r2 / (p[3] * p[3]));
    }
    return acc;
}

/* Union of thin shells around closed surfaces. s[i] = {kind, cx, cy, cz, rx, ry, rz}
 * in voxel units; kind 0 = sphere (rx), kind 1 = axis-aligned ellipsoid.
 * Returns exp(-(d/width)^2) for the closest surface distance d. */
static double shell_field(const double* s, int ns, double width, double px, double py, double pz) {
    double best = 0.0;
    for (int i = 0; i < ns; ++i) {
        const double* p = s + 7 * i;
        double dx = px - p[1], dy = py - p[2], dz = pz - p[3];
        double d;
        if (p[0] == 0.0) {
            d = sqrt(dx * dx + dy * dy + dz * dz) - p[4];
        } else {
            double ax = dx / p[4], ay = dy / p[5], az = dz / p[6];
            double bx = ax / p[4], by = ay / p[5], bz = az / p[6];
            double k0 = sqrt(ax * ax + ay * ay + az * az);
            double k1 = sqrt(bx * bx + by * by + bz * bz);
            d = (k1 > 0.0) ? k0 * (k0 - 1.0) / k1 : -p[4];
        }
        double e = d / width;
        if (e * e < 30.0) {
            double v = exp(-e * e);
            if (v > best) best = v;
        }
    }
    return best;
}

/* Density channel for a list of blocks.
 * mode 0: Gaussian sum (params = gauss list, coordinates in unit-cube units),
 * mode 1: shells (params = shell list, coordinates in voxel units).
 * q = quant01(scale * field) with field < cut forced to 0. Returns nothing; writes
 * channel 0 of out and the per-block maximum code into blk_max. */
void synth_density(int32_t N, int32_t B, int64_t nblk, const int32_t* blk_xyz,
                   int32_t mode, int32_t nparam, const double* params, double width,
                   double cut, double scale, uint8_t* out, uint8_t* blk_max) {
    const int64_t vox = (int64_t)B * B * B;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < nblk; ++b) {
        uint8_t mx = 0;
        const int32_t bx = blk_xyz[3 * b], by = blk_xyz[3 * b + 1], bz = blk_xyz[3 * b + 2];
        for (int32_t z = 0; z < B; ++z)
            for (int32_t y = 0; y < B; ++y)
                for (int32_t x = 0; x < B; ++x) {
                    double vx = (double)(bx * B + x) + 0.5;
                    double vy = (double)(by * B + y) + 0.5;
                    double vz = (double)(bz * B + z) + 0.5;
                    double f;
                    if (mode == 0)
                        f = gauss_field(params, nparam, vx / N, vy / N, vz / N);
                    else
                        f = shell_field(params, nparam, width, vx, vy, vz);
                    if (f < cut) f = 0.0;
                    uint8_t q = quant01(scale * f);
                    int64_t idx = b * vox + ((int64_t)z * B + y) * B + x;
                    out[idx * 8] = q;
                    if (q > mx) mx = q;
                }
        blk_max[b] = mx;
    }
}

/* Seven smooth colour/feature channels: v_c = 0.5 + 0.5 sin(w_c . p + phi_c) with p
 * in unit-cube units. freq[c] = {wx, wy, wz, phi} for c = 0..6 (channels 1..7). */
void synth_colors(int32_t N, int32_t B, int64_t nblk, const int32_t* blk_xyz,
                  const double* freq, uint8_t* out) {
    const int64_t vox = (int64_t)B * B * B;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < nblk; ++b) {
        const int32_t bx = blk_xyz[3 * b], by = blk_xyz[3 * b + 1], bz = blk_xyz[3 * b + 2];
        for (int32_t z = 0; z < B; ++z)
            for (int32_t y = 0; y < B; ++y)
                for (int32_t x = 0; x < B; ++x) {
                    double px = ((double)(bx * B + x) + 0.5) / N;
                    double py = ((double)(by * B + y) + 0.5) / N;
                    double pz = ((double)(bz * B + z) + 0.5) / N;
                    int64_t idx = b * vox + ((int64_t)z * B + y) * B + x;
                    for (int c = 0; c < 7; ++c) {
                        const double* w = freq + 4 * c;
                        double v = 0.5 + 0.5 * sin(w[0] * px + w[1] * py + w[2] * pz + w[3]);
                        out[idx * 8 + 1 + c] = quant01(v);
                    }
                }
    }
}
