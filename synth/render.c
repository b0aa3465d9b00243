/*
 * Seeded synthetic ultrasound phantom renderer.
 *
 * Input generation only: this file renders uint8 B-mode-like frames of a
 * synthetic phantom at given probe poses.  It contains none of the DARE
 * reconstruction or reslicing arithmetic; both the CUDA library and the CPU
 * oracle consume its output.
 *
 * Phantom model (stand-in for the paper's gelatin/tubing phantoms and the
 * freehand human dataset of Sec. 2.2, which are not available):
 *   - speckle: Rayleigh(sigma) values on a world-space lattice of cell
 *     `cell_mm`, drawn from a counter-based hash of (seed, node index), so the
 *     same tissue point looks the same in every frame; a pixel takes the
 *     trilinear blend of the 8 surrounding lattice nodes;
 *   - specular ellipsoid shells: echo 200*|cos(beam . surface normal)|^4 times
 *     a Gaussian profile (sigma_t) of the distance to the surface -- the
 *     orientation-dependent reflectivity the paper's Sec. 1 motivates;
 *   - tubular vessels along polylines: anechoic lumen (speckle x 0.1) and a
 *     specular wall, same echo law as the shells.
 *
 * Pixel geometry: pixel (u, v) of a W x H frame with spacing (sx, sy) sits at
 * image point ((u - (W-1)/2) sx, v sy, 0); image x = lateral, y = beam/depth.
 * Poses are row-major 4x4 image->world transforms in mm.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define RAYLEIGH_LUT 4096

/* splitmix64 finaliser (S. Vigna's published mixing function). */
static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t node_hash(uint64_t seed, int64_t ix, int64_t iy, int64_t iz) {
    uint64_t h = mix64(seed ^ 0xD1B54A32D192ED03ULL);
    h = mix64(h ^ (uint64_t)ix);
    h = mix64(h ^ (uint64_t)iy);
    h = mix64(h ^ (uint64_t)iz);
    return h;
}

typedef struct {
    double c[3];     /* centre, world mm */
    double inv_s[3]; /* 1 / semi-axes */
    double R[9];     /* row-major rotation: local->world columns */
    double reach;    /* bounding radius + margin, for early rejection */
} shell_t;

static inline double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* distance from p to segment [a, b]; also returns the closest point */
static inline double seg_dist(const double* p, const double* a, const double* b, double* q) {
    double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    double L2 = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
    double t = L2 > 0 ? (ap[0] * ab[0] + ap[1] * ab[1] + ap[2] * ab[2]) / L2 : 0.0;
    t = clampd(t, 0.0, 1.0);
    q[0] = a[0] + t * ab[0]; q[1] = a[1] + t * ab[1]; q[2] = a[2] + t * ab[2];
    double d[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
    return sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

/*
 * Render n frames.  shells: n_shells x 15 doubles (centre 3, semi-axes 3,
 * rotation 9 row-major, local->world).  vessels: n_vessels x (1 + 3 n_pts)
 * doubles (radius, then polyline points).  out: n x H x W uint8, row-major.
 * Returns 0 on success.
 */
int synth_render(int32_t n, int32_t W, int32_t H, double sx, double sy,
                 const double* poses, uint64_t seed, double sigma, double cell_mm,
                 double sigma_t, double echo_gain,
                 int32_t n_shells, const double* shells,
                 int32_t n_vessels, int32_t n_pts, const double* vessels,
                 uint8_t* out) {
    if (n < 0 || W <= 0 || H <= 0 || (n_vessels > 0 && n_pts < 2)) return 1;
    double lut[RAYLEIGH_LUT];
    for (int i = 0; i < RAYLEIGH_LUT; ++i) {
        double U = (i + 0.5) / RAYLEIGH_LUT;
        lut[i] = sigma * sqrt(-2.0 * log(U));
    }
    shell_t sh[64];
    if (n_shells > 64) return 2;
    for (int k = 0; k < n_shells; ++k) {
        const double* s = shells + 15 * k;
        double smax = 0;
        for (int a = 0; a < 3; ++a) {
            sh[k].c[a] = s[a];
            sh[k].inv_s[a] = 1.0 / s[3 + a];
            if (s[3 + a] > smax) smax = s[3 + a];
        }
        for (int a = 0; a < 9; ++a) sh[k].R[a] = s[6 + a];
        sh[k].reach = smax + 4.0 * sigma_t + 1e-3;
    }
    const int vstride = 1 + 3 * n_pts;
    const double inv_cell = 1.0 / cell_mm;
    const double inv2s2 = 1.0 / (2.0 * sigma_t * sigma_t);

#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int64_t f = 0; f < n; ++f) {
        for (int32_t v = 0; v < H; ++v) {
            const double* T = poses + 16 * f;
            /* beam direction = image y axis in world */
            double beam[3] = {T[1], T[5], T[9]};
            uint8_t* row = out + ((size_t)f * H + v) * (size_t)W;
            for (int32_t u = 0; u < W; ++u) {
                double x = (u - 0.5 * (W - 1)) * sx, y = v * sy;
                double p[3];
                for (int a = 0; a < 3; ++a) p[a] = T[4 * a + 0] * x + T[4 * a + 1] * y + T[4 * a + 3];
                /* speckle: trilinear blend of lattice nodes */
                double g[3], fr[3];
                int64_t i0[3];
                for (int a = 0; a < 3; ++a) {
                    g[a] = p[a] * inv_cell;
                    double fl = floor(g[a]);
                    i0[a] = (int64_t)fl;
                    fr[a] = g[a] - fl;
                }
                double spk = 0.0;
                for (int c = 0; c < 8; ++c) {
                    int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
                    double wgt = (dx ? fr[0] : 1 - fr[0]) * (dy ? fr[1] : 1 - fr[1]) * (dz ? fr[2] : 1 - fr[2]);
                    uint64_t h = node_hash(seed, i0[0] + dx, i0[1] + dy, i0[2] + dz);
                    spk += wgt * lut[h & (RAYLEIGH_LUT - 1)];
                }
                double echo = 0.0, lumen = 1.0;
                for (int k = 0; k < n_shells; ++k) {
                    double d0 = p[0] - sh[k].c[0], d1 = p[1] - sh[k].c[1], d2 = p[2] - sh[k].c[2];
                    if (fabs(d0) > sh[k].reach || fabs(d1) > sh[k].reach || fabs(d2) > sh[k].reach) continue;
                    const double* R = sh[k].R;
                    /* local = R^T d */
                    double l[3];
                    for (int a = 0; a < 3; ++a) l[a] = R[0 + a] * d0 + R[3 + a] * d1 + R[6 + a] * d2;
                    double q[3], F = 0.0;
                    for (int a = 0; a < 3; ++a) { q[a] = l[a] * sh[k].inv_s[a]; F += q[a] * q[a]; }
                    /* gradient of F in local coordinates: 2 l / s^2 */
                    double gl[3], gn = 0.0;
                    for (int a = 0; a < 3; ++a) { gl[a] = 2.0 * q[a] * sh[k].inv_s[a]; gn += gl[a] * gl[a]; }
                    gn = sqrt(gn);
                    if (gn <= 0) continue;
                    double dist = (F - 1.0) / gn; /* first-order distance to F = 1 */
                    if (fabs(dist) > 4.0 * sigma_t) continue;
                    double nw[3];
                    for (int a = 0; a < 3; ++a) nw[a] = (R[3 * a + 0] * gl[0] + R[3 * a + 1] * gl[1] + R[3 * a + 2] * gl[2]) / gn;
                    double cosb = beam[0] * nw[0] + beam[1] * nw[1] + beam[2] * nw[2];
                    double c2 = cosb * cosb;
                    echo += echo_gain * c2 * c2 * exp(-dist * dist * inv2s2);
                }
                for (int k = 0; k < n_vessels; ++k) {
                    const double* V = vessels + (size_t)vstride * k;
                    double r = V[0];
                    double best = 1e300, bq[3] = {0, 0, 0};
                    for (int s = 0; s + 1 < n_pts; ++s) {
                        double q[3];
                        double d = seg_dist(p, V + 1 + 3 * s, V + 1 + 3 * (s + 1), q);
                        if (d < best) { best = d; bq[0] = q[0]; bq[1] = q[1]; bq[2] = q[2]; }
                    }
                    if (best < r - sigma_t) lumen = 0.1;
                    double dw = best - r;
                    if (fabs(dw) < 4.0 * sigma_t && best > 0) {
                        double nw[3] = {(p[0] - bq[0]) / best, (p[1] - bq[1]) / best, (p[2] - bq[2]) / best};
                        double cosb = beam[0] * nw[0] + beam[1] * nw[1] + beam[2] * nw[2];
                        double c2 = cosb * cosb;
                        echo += echo_gain * c2 * c2 * exp(-dw * dw * inv2s2);
                    }
                }
                double val = spk * lumen + echo;
                val = clampd(floor(val + 0.5), 0.0, 255.0);
                row[u] = (uint8_t)val;
            }
        }
    }
    return 0;
}
