/*
 * DARE CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 restatement of the paper's method (Jaeggi, Black,
 * Salcudean, "Real-time, Directionality Aware 3D Ultrasound Reconstruction and
 * Re-Slicing"), used to check the CUDA library.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load this file.  It
 * shares no code with the CUDA path and the CUDA path never calls it.
 *
 * Steps follow the paper's order:
 *   reconstruction (Sec. 2.1 "Volume reconstruction", Fig. 1):
 *     frames are placed at their tracked poses, voxelised into a grid, and
 *     every grid cell keeps a flat list of samples, each an intensity with the
 *     acquisition orientation as a quaternion;
 *   reslicing (Sec. 2.1 "Reslicing", Eq. 1, Eq. 2, Fig. 2):
 *     every pixel of a virtual plane is mapped into the volume, the samples of
 *     a cubic neighbourhood are gathered, each sample's alignment with the
 *     plane is measured by the two dot products of Eq. 1, samples beyond the
 *     angular thresholds are dropped, the rest are averaged with the
 *     exponential weights of Eq. 2 (times a distance weight, Fig. 2); a pixel
 *     with no valid sample is left unassigned.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - pixel geometry: pixel (u,v) at image point ((u-(W-1)/2) sx, v sy, 0);
 *     image x = lateral (the in-plane direction of Eq. 1), y = beam;
 *   - "acquisition normal" of Eq. 1 = beam direction R*y (normal_axis 0), or
 *     the image-plane normal R*z (normal_axis 1);
 *   - a sample passes iff d_normal >= cos(thr_normal) and
 *     d_inplane >= cos(thr_inplane) (inclusive); a threshold >= 180 deg is off;
 *   - distance weight: TENT prod_a (1 - |g_a - c_a| / R) over the 2R-wide
 *     support (trilinear at R = 1), BOX = 1 over the (2R+1)^3 cube around the
 *     nearest voxel, EXP = exp(-k_d |g - c| / R) over the 2R-wide support;
 *   - voxelisation: nearest voxel, floor(g + 1/2) per axis; one sample per
 *     (voxel, frame), the mean of that frame's pixels in the voxel;
 *   - geometry in fixed point: the pixel->voxel affine is rounded to
 *     multiples of 2^-20 voxel (round-half-even of x * 2^20, FP64, the
 *     canonical evaluation order documented in include/dare.h), after which
 *     every pixel coordinate is exact in int64;
 *   - stored value: RN_fp32(sum/npix), then rounded to the storage type
 *     (u8: round-half-even, clamped to [0,255]; f16 and bf16: RN-even);
 *   - capacity: when a voxel holds more than kmax samples, keep the kmax with
 *     the largest npix (ties: lower frame id), ordered by frame id;
 *   - curvilinear probes (an extension: the paper's probe is a linear array,
 *     Sec. 2.2, whose beam is the image y axis everywhere): the beams fan out
 *     from an apex a = (a_x, a_y) of the image plane.  The beam through image
 *     point p runs along (p - a) / |p - a|, i.e. the image axes turned about
 *     image z by alpha = atan2(-(p_x - a_x), p_y - a_y) (alpha = 0 at p = a).
 *     A sample's acquisition orientation, the quaternion the paper stores per
 *     sample, is its frame's quaternion times that turn, taken at the centre
 *     of the sample's voxel expressed in the frame's image coordinates (the
 *     in-plane part; the voxel centre lies within half a voxel diagonal of
 *     the plane).  A curvilinear virtual plane turns its own axes the same
 *     way at every output pixel, about its own apex.  Eq. 1 and Eq. 2 are
 *     unchanged, applied to the turned axes;
 *   - pixel mask: a build may exclude pixels (the dark corners outside a fan
 *     image); an excluded pixel is never voxelised;
 *   - per-pixel samples (the other reading of Sec. 2.1's storage, where every
 *     pixel is kept as its own sample with its frame's orientation): all of a
 *     frame's pixels in a voxel share the orientation weight, so their sum
 *     w * sum(I) equals the merged sample's w * npix * mean; sample_weight 1
 *     weights each merged sample by its npix, which is that reading exactly.
 *
 * Arithmetic is FP64 throughout except the storage rounding, which is the
 * storage type's own.  Compile with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_U8 0
#define ORA_F16 1
#define ORA_BF16 2
#define ORA_F32 3

#define ORA_TENT 0
#define ORA_BOX 1
#define ORA_EXP 2

#define ORA_LINEAR 0
#define ORA_CURVILINEAR 1

#define FIX_BITS 20
#define FIX_ONE ((int64_t)1 << FIX_BITS)

typedef struct {
    double k_normal, k_inplane;        /* Eq. 2 sensitivities */
    double thr_normal_deg, thr_inplane_deg;
    double k_dist;                     /* EXP distance kernel rate */
    double unassigned;                 /* value written to unassigned pixels */
    int32_t radius;                    /* R, interpolation distance in voxels */
    int32_t kernel;                    /* ORA_TENT / ORA_BOX / ORA_EXP */
    int32_t normal_axis;               /* 0 = beam (R y), 1 = plane normal (R z) */
    int32_t use_exact;                 /* 1: FP64 means instead of stored values */
    int32_t probe;                     /* virtual probe: ORA_LINEAR / ORA_CURVILINEAR */
    int32_t pad;
    double apex_x, apex_y;             /* curvilinear virtual probe: fan apex, image point (mm) */
    int32_t sample_weight;             /* 0: one sample per (voxel, frame); 1: per pixel (see below) */
    int32_t pad2;
} ora_params;

typedef struct {
    int32_t dims[3];
    double h;
    double vol_to_world[16];
    int32_t dtype, kmax;
    int64_t n_vox;
    int64_t n_samples;
    int64_t* offsets;     /* n_vox + 1 */
    int32_t* frame_id;    /* per sample */
    int64_t* npix;
    int64_t* sum;
    double* mean_exact;
    double* stored;
    double* quat;         /* 4 per sample: w, x, y, z (volume frame) */
    int64_t n_overflow;   /* voxels that held more than kmax samples */
    int64_t n_dropped;    /* samples removed by the capacity rule */
    /* mean-compounding totals over every sample (before the capacity rule) */
    int64_t* tot_sum;
    int64_t* tot_npix;
} ora_volume;

/* ------------------------------------------------------------ geometry */

/* floor(a / 2^FIX_BITS) for signed a */
static int64_t fix_floor(int64_t a) {
    int64_t q = a / FIX_ONE;
    if (a % FIX_ONE != 0 && a < 0) q -= 1;
    return q;
}

/* x * 2^20 rounded half-to-even (default FP environment) */
static int64_t fix_round(double x) { return (int64_t)nearbyint(x * (double)FIX_ONE); }

/*
 * Pixel -> voxel affine of a plane, quantised to 2^-20 voxel.
 * out = [G0 (3), A (3), B (3)]: voxel coordinate of pixel (u, v) is
 * (G0 + u A + v B) * 2^-20.  The rigid volume pose is inverted as
 * (R_v^T, -R_v^T t_v); the order of every FP64 operation is the canonical one.
 */
int ora_pixel_affine(const double* V, double h, const double* T, int32_t W, double sx, double sy,
                     int64_t* out) {
    if (!(h > 0)) return 1;
    double d[3], c0[3], c1[3], tm[3];
    for (int k = 0; k < 3; ++k) d[k] = T[4 * k + 3] - V[4 * k + 3];
    for (int r = 0; r < 3; ++r) {
        /* (R_v^T R_i)[r][0], (R_v^T R_i)[r][1], R_v^T (t_i - t_v) [r] */
        c0[r] = V[0 * 4 + r] * T[0 * 4 + 0] + V[1 * 4 + r] * T[1 * 4 + 0] + V[2 * 4 + r] * T[2 * 4 + 0];
        c1[r] = V[0 * 4 + r] * T[0 * 4 + 1] + V[1 * 4 + r] * T[1 * 4 + 1] + V[2 * 4 + r] * T[2 * 4 + 1];
        tm[r] = V[0 * 4 + r] * d[0] + V[1 * 4 + r] * d[1] + V[2 * 4 + r] * d[2];
    }
    double half_w = 0.5 * (double)(W - 1) * sx;
    for (int r = 0; r < 3; ++r) {
        out[r] = fix_round((tm[r] - half_w * c0[r]) / h);
        out[3 + r] = fix_round((c0[r] * sx) / h);
        out[6 + r] = fix_round((c1[r] * sy) / h);
    }
    return 0;
}

/* rotation of the image frame expressed in the volume frame: R_v^T R_i */
static void rel_rotation(const double* V, const double* T, double R[9]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            R[3 * r + c] = V[0 * 4 + r] * T[0 * 4 + c] + V[1 * 4 + r] * T[1 * 4 + c] + V[2 * 4 + r] * T[2 * 4 + c];
}

/* unit quaternion (w, x, y, z) of a rotation matrix, Shepperd's method, w >= 0 */
static void mat_to_quat(const double R[9], double q[4]) {
    double tr = R[0] + R[4] + R[8];
    double w, x, y, z;
    if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
        double s = sqrt(1.0 + tr) * 2.0;
        w = 0.25 * s; x = (R[7] - R[5]) / s; y = (R[2] - R[6]) / s; z = (R[3] - R[1]) / s;
    } else if (R[0] >= R[4] && R[0] >= R[8]) {
        double s = sqrt(1.0 + R[0] - R[4] - R[8]) * 2.0;
        w = (R[7] - R[5]) / s; x = 0.25 * s; y = (R[1] + R[3]) / s; z = (R[2] + R[6]) / s;
    } else if (R[4] >= R[8]) {
        double s = sqrt(1.0 + R[4] - R[0] - R[8]) * 2.0;
        w = (R[2] - R[6]) / s; x = (R[1] + R[3]) / s; y = 0.25 * s; z = (R[5] + R[7]) / s;
    } else {
        double s = sqrt(1.0 + R[8] - R[0] - R[4]) * 2.0;
        w = (R[3] - R[1]) / s; x = (R[2] + R[6]) / s; y = (R[5] + R[7]) / s; z = 0.25 * s;
    }
    double n = sqrt(w * w + x * x + y * y + z * z);
    if (w < 0) n = -n;
    q[0] = w / n; q[1] = x / n; q[2] = y / n; q[3] = z / n;
}

/* column `axis` (0 = image x, 1 = image y, 2 = image z) of the rotation of q */
static void quat_axis(const double q[4], int axis, double v[3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    if (axis == 0) {
        v[0] = 1 - 2 * (y * y + z * z); v[1] = 2 * (x * y + w * z); v[2] = 2 * (x * z - w * y);
    } else if (axis == 1) {
        v[0] = 2 * (x * y - w * z); v[1] = 1 - 2 * (x * x + z * z); v[2] = 2 * (y * z + w * x);
    } else {
        v[0] = 2 * (x * z + w * y); v[1] = 2 * (y * z - w * x); v[2] = 1 - 2 * (x * x + y * y);
    }
}

/* Hamilton product a * b: the rotation b followed by a */
static void quat_mul(const double a[4], const double b[4], double out[4]) {
    out[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    out[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    out[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    out[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

/*
 * Orientation of the beam of a curvilinear probe through image point
 * (px, py): q turned about its image z axis by the steering angle from the
 * apex (ax, ay).
 */
static void steer(const double q[4], double px, double py, double ax, double ay, double out[4]) {
    double dx = px - ax, dy = py - ay;
    double alpha = (dx == 0.0 && dy == 0.0) ? 0.0 : atan2(-dx, dy);
    double turn[4] = {cos(0.5 * alpha), 0.0, 0.0, sin(0.5 * alpha)};
    quat_mul(q, turn, out);
}

/* ------------------------------------------------------------ storage rounding */

static float rn_f32_quotient(int64_t s, int64_t n) { return (float)s / (float)n; }

static double to_stored(float m, int dtype) {
    switch (dtype) {
    case ORA_F32: return (double)m;
    case ORA_F16: return (double)(_Float16)m;
    case ORA_BF16: {
        uint32_t b;
        memcpy(&b, &m, 4);
        uint32_t lsb = (b >> 16) & 1u;
        b = (b + 0x7FFFu + lsb) & 0xFFFF0000u;
        float r;
        memcpy(&r, &b, 4);
        return (double)r;
    }
    case ORA_U8: {
        float r = nearbyintf(m);
        if (r < 0.f) r = 0.f;
        if (r > 255.f) r = 255.f;
        return (double)r;
    }
    }
    return NAN;
}

double ora_round_stored(double sum, double npix, int32_t dtype) {
    return to_stored(rn_f32_quotient((int64_t)sum, (int64_t)npix), dtype);
}

/* ------------------------------------------------------------ volume */

void ora_volume_free(ora_volume* v) {
    if (!v) return;
    free(v->offsets); free(v->frame_id); free(v->npix); free(v->sum);
    free(v->mean_exact); free(v->stored); free(v->quat);
    free(v->tot_sum); free(v->tot_npix);
    free(v);
}

static ora_volume* vol_alloc(const int32_t* dims, double h, const double* V, int32_t dtype, int32_t kmax) {
    ora_volume* v = (ora_volume*)calloc(1, sizeof(ora_volume));
    if (!v) return NULL;
    memcpy(v->dims, dims, 3 * sizeof(int32_t));
    v->h = h;
    memcpy(v->vol_to_world, V, 16 * sizeof(double));
    v->dtype = dtype;
    v->kmax = kmax;
    v->n_vox = (int64_t)dims[0] * dims[1] * dims[2];
    v->offsets = (int64_t*)calloc((size_t)v->n_vox + 1, sizeof(int64_t));
    v->tot_sum = (int64_t*)calloc((size_t)v->n_vox, sizeof(int64_t));
    v->tot_npix = (int64_t*)calloc((size_t)v->n_vox, sizeof(int64_t));
    if (!v->offsets || !v->tot_sum || !v->tot_npix) { ora_volume_free(v); return NULL; }
    return v;
}

typedef struct { int32_t frame; int64_t npix; } keyed_t;

/* capacity ordering: larger npix first, then lower frame id */
static int cmp_keep(const void* a, const void* b) {
    const keyed_t* x = (const keyed_t*)a;
    const keyed_t* y = (const keyed_t*)b;
    if (x->npix != y->npix) return x->npix > y->npix ? -1 : 1;
    return x->frame < y->frame ? -1 : (x->frame > y->frame);
}

static int cmp_int32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return x < y ? -1 : (x > y);
}

/*
 * Reconstruction (Sec. 2.1, Fig. 1).  frames: n x H x W uint8 row-major;
 * poses: n x 16 row-major image->world.  Frame k gets id k.  voxel_filter,
 * when non-NULL, keeps only voxels whose byte is non-zero (used to build the
 * neighbourhood of a few sampled pixels of a large workload).  probe, when
 * non-NULL, gives each frame's probe (ORA_LINEAR / ORA_CURVILINEAR) and apex
 * holds its fan apex (n x 2, image mm); pixel_mask, when non-NULL, is H x W
 * and a zero byte excludes that pixel of every frame.
 */
ora_volume* ora_build_probe(const int32_t* dims, double h, const double* V, int32_t n, int32_t W, int32_t H,
                            double sx, double sy, const uint8_t* frames, const double* poses,
                            int32_t dtype, int32_t kmax, const uint8_t* voxel_filter, const int32_t* probe,
                            const double* apex, const uint8_t* pixel_mask) {
    if (dims[0] <= 0 || dims[1] <= 0 || dims[2] <= 0 || n < 0 || W <= 0 || H <= 0 || kmax <= 0) return NULL;
    if (probe && !apex) return NULL;
    ora_volume* v = vol_alloc(dims, h, V, dtype, kmax);
    if (!v) return NULL;
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    int64_t* aff = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * 9 * sizeof(int64_t));
    double* fq = (double*)malloc((size_t)(n > 0 ? n : 1) * 4 * sizeof(double));
    int64_t* count = (int64_t*)calloc((size_t)v->n_vox, sizeof(int64_t));
    if (!aff || !fq || !count) { free(aff); free(fq); free(count); ora_volume_free(v); return NULL; }
    for (int32_t f = 0; f < n; ++f) {
        ora_pixel_affine(V, h, poses + 16 * (size_t)f, W, sx, sy, aff + 9 * (size_t)f);
        double R[9];
        rel_rotation(V, poses + 16 * (size_t)f, R);
        mat_to_quat(R, fq + 4 * (size_t)f);
    }
    /* pass 1: count pixels per voxel */
    for (int pass = 0; pass < 2; ++pass) {
        int32_t* ent_frame = NULL;
        uint8_t* ent_val = NULL;
        int64_t* fill = NULL;
        int64_t* start = NULL;
        if (pass == 1) {
            start = (int64_t*)malloc(((size_t)v->n_vox + 1) * sizeof(int64_t));
            start[0] = 0;
            for (int64_t i = 0; i < v->n_vox; ++i) start[i + 1] = start[i] + count[i];
            ent_frame = (int32_t*)malloc((size_t)(start[v->n_vox] > 0 ? start[v->n_vox] : 1) * sizeof(int32_t));
            ent_val = (uint8_t*)malloc((size_t)(start[v->n_vox] > 0 ? start[v->n_vox] : 1));
            fill = (int64_t*)calloc((size_t)v->n_vox, sizeof(int64_t));
        }
        for (int32_t f = 0; f < n; ++f) {
            const int64_t* G0 = aff + 9 * (size_t)f;
            const int64_t* A = G0 + 3;
            const int64_t* B = G0 + 6;
            const uint8_t* img = frames + (size_t)f * W * H;
            for (int32_t y = 0; y < H; ++y) {
                for (int32_t x = 0; x < W; ++x) {
                    if (pixel_mask && !pixel_mask[(size_t)y * W + x]) continue;
                    int64_t c[3];
                    for (int a = 0; a < 3; ++a) {
                        int64_t G = G0[a] + (int64_t)x * A[a] + (int64_t)y * B[a];
                        c[a] = fix_floor(G + FIX_ONE / 2); /* nearest voxel, ties up */
                    }
                    if (c[0] < 0 || c[0] >= nx || c[1] < 0 || c[1] >= ny || c[2] < 0 || c[2] >= nz) continue;
                    int64_t vi = c[0] + nx * (c[1] + ny * c[2]);
                    if (voxel_filter && !voxel_filter[vi]) continue;
                    if (pass == 0) {
                        count[vi] += 1;
                    } else {
                        int64_t at = start[vi] + fill[vi]++;
                        ent_frame[at] = f;
                        ent_val[at] = img[(size_t)y * W + x];
                    }
                }
            }
        }
        if (pass == 1) {
            /* entries of each voxel are in frame order; group them into samples */
            int64_t cap = 0;
            for (int64_t i = 0; i < v->n_vox; ++i) {
                int64_t m = 0;
                for (int64_t e = start[i]; e < start[i + 1]; ++e)
                    if (e == start[i] || ent_frame[e] != ent_frame[e - 1]) ++m;
                cap += m < kmax ? m : kmax;
            }
            size_t cs = (size_t)(cap > 0 ? cap : 1);
            v->frame_id = (int32_t*)malloc(cs * sizeof(int32_t));
            v->npix = (int64_t*)malloc(cs * sizeof(int64_t));
            v->sum = (int64_t*)malloc(cs * sizeof(int64_t));
            v->mean_exact = (double*)malloc(cs * sizeof(double));
            v->stored = (double*)malloc(cs * sizeof(double));
            v->quat = (double*)malloc(cs * 4 * sizeof(double));
            keyed_t* tmp = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)(n > 0 ? n : 1));
            int64_t* tmp_sum = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
            int32_t* keep = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
            int64_t out = 0;
            for (int64_t i = 0; i < v->n_vox; ++i) {
                v->offsets[i] = out;
                int m = 0;
                for (int64_t e = start[i]; e < start[i + 1]; ++e) {
                    if (e == start[i] || ent_frame[e] != ent_frame[e - 1]) {
                        tmp[m].frame = ent_frame[e];
                        tmp[m].npix = 0;
                        tmp_sum[m] = 0;
                        ++m;
                    }
                    tmp[m - 1].npix += 1;
                    tmp_sum[m - 1] += ent_val[e];
                    v->tot_sum[i] += ent_val[e];
                    v->tot_npix[i] += 1;
                }
                /* frame -> sum lookup survives the capacity sort */
                int m_keep = m;
                if (m > kmax) {
                    v->n_overflow += 1;
                    v->n_dropped += m - kmax;
                    keyed_t* sorted = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)m);
                    memcpy(sorted, tmp, sizeof(keyed_t) * (size_t)m);
                    qsort(sorted, (size_t)m, sizeof(keyed_t), cmp_keep);
                    for (int k = 0; k < kmax; ++k) keep[k] = sorted[k].frame;
                    free(sorted);
                    qsort(keep, (size_t)kmax, sizeof(int32_t), cmp_int32);
                    m_keep = kmax;
                } else {
                    for (int k = 0; k < m; ++k) keep[k] = tmp[k].frame;
                }
                for (int k = 0; k < m_keep; ++k) {
                    int j = 0;
                    while (tmp[j].frame != keep[k]) ++j;
                    v->frame_id[out] = tmp[j].frame;
                    v->npix[out] = tmp[j].npix;
                    v->sum[out] = tmp_sum[j];
                    v->mean_exact[out] = (double)tmp_sum[j] / (double)tmp[j].npix;
                    v->stored[out] = to_stored(rn_f32_quotient(tmp_sum[j], tmp[j].npix), dtype);
                    const int32_t fr = tmp[j].frame;
                    if (probe && probe[fr] == ORA_CURVILINEAR) {
                        /* voxel centre in world, then in the frame's image coordinates */
                        const double* T = poses + 16 * (size_t)fr;
                        double c[3] = {(double)(i % nx), (double)((i / nx) % ny), (double)(i / (nx * ny))};
                        double w[3], p[2];
                        for (int r = 0; r < 3; ++r)
                            w[r] = V[4 * r + 0] * (h * c[0]) + V[4 * r + 1] * (h * c[1]) + V[4 * r + 2] * (h * c[2]) +
                                   V[4 * r + 3];
                        for (int k = 0; k < 2; ++k)
                            p[k] = T[0 * 4 + k] * (w[0] - T[3]) + T[1 * 4 + k] * (w[1] - T[7]) +
                                   T[2 * 4 + k] * (w[2] - T[11]);
                        steer(fq + 4 * (size_t)fr, p[0], p[1], apex[2 * fr], apex[2 * fr + 1], v->quat + 4 * out);
                    } else {
                        memcpy(v->quat + 4 * out, fq + 4 * (size_t)fr, 4 * sizeof(double));
                    }
                    ++out;
                }
            }
            v->offsets[v->n_vox] = out;
            v->n_samples = out;
            free(tmp); free(tmp_sum); free(keep);
            free(start); free(ent_frame); free(ent_val); free(fill);
        }
    }
    free(aff); free(fq); free(count);
    return v;
}

/* Reconstruction from linear-array frames, every pixel used. */
ora_volume* ora_build(const int32_t* dims, double h, const double* V, int32_t n, int32_t W, int32_t H,
                      double sx, double sy, const uint8_t* frames, const double* poses,
                      int32_t dtype, int32_t kmax, const uint8_t* voxel_filter) {
    return ora_build_probe(dims, h, V, n, W, H, sx, sy, frames, poses, dtype, kmax, voxel_filter, NULL, NULL, NULL);
}

/*
 * A volume given sample by sample (for hand-made test cases).  Samples must
 * be listed in (voxel, frame) order; quat is 4 per sample.
 */
ora_volume* ora_volume_manual(const int32_t* dims, double h, const double* V, int64_t n_samples,
                              const int64_t* voxel, const int32_t* frame, const double* value,
                              const double* quat) {
    ora_volume* v = vol_alloc(dims, h, V, ORA_F32, 1 << 30);
    if (!v) return NULL;
    size_t cs = (size_t)(n_samples > 0 ? n_samples : 1);
    v->frame_id = (int32_t*)malloc(cs * sizeof(int32_t));
    v->npix = (int64_t*)malloc(cs * sizeof(int64_t));
    v->sum = (int64_t*)malloc(cs * sizeof(int64_t));
    v->mean_exact = (double*)malloc(cs * sizeof(double));
    v->stored = (double*)malloc(cs * sizeof(double));
    v->quat = (double*)malloc(cs * 4 * sizeof(double));
    for (int64_t s = 0; s < n_samples; ++s) {
        if (voxel[s] < 0 || voxel[s] >= v->n_vox || (s > 0 && voxel[s] < voxel[s - 1])) {
            ora_volume_free(v);
            return NULL;
        }
        v->offsets[voxel[s] + 1] += 1;
        v->frame_id[s] = frame[s];
        v->npix[s] = 1;
        v->sum[s] = 0;
        v->mean_exact[s] = value[s];
        v->stored[s] = value[s];
        double n = sqrt(quat[4 * s] * quat[4 * s] + quat[4 * s + 1] * quat[4 * s + 1] +
                        quat[4 * s + 2] * quat[4 * s + 2] + quat[4 * s + 3] * quat[4 * s + 3]);
        for (int k = 0; k < 4; ++k) v->quat[4 * s + k] = quat[4 * s + k] / n;
    }
    for (int64_t i = 0; i < v->n_vox; ++i) v->offsets[i + 1] += v->offsets[i];
    v->n_samples = n_samples;
    return v;
}

int64_t ora_volume_nsamples(const ora_volume* v) { return v->n_samples; }
int64_t ora_volume_noverflow(const ora_volume* v) { return v->n_overflow; }
int64_t ora_volume_ndropped(const ora_volume* v) { return v->n_dropped; }

void ora_volume_export(const ora_volume* v, int64_t* offsets, int32_t* frame_id, int64_t* npix, int64_t* sum,
                       double* mean_exact, double* stored, double* quat, int64_t* tot_sum, int64_t* tot_npix) {
    if (offsets) memcpy(offsets, v->offsets, ((size_t)v->n_vox + 1) * sizeof(int64_t));
    size_t n = (size_t)v->n_samples;
    if (frame_id) memcpy(frame_id, v->frame_id, n * sizeof(int32_t));
    if (npix) memcpy(npix, v->npix, n * sizeof(int64_t));
    if (sum) memcpy(sum, v->sum, n * sizeof(int64_t));
    if (mean_exact) memcpy(mean_exact, v->mean_exact, n * sizeof(double));
    if (stored) memcpy(stored, v->stored, n * sizeof(double));
    if (quat) memcpy(quat, v->quat, n * 4 * sizeof(double));
    if (tot_sum) memcpy(tot_sum, v->tot_sum, (size_t)v->n_vox * sizeof(int64_t));
    if (tot_npix) memcpy(tot_npix, v->tot_npix, (size_t)v->n_vox * sizeof(int64_t));
}

/* ------------------------------------------------------------ reslicing */

typedef struct {
    int64_t aff[9];
    double n_r[3], x_r[3];
    double cos_n, cos_i;
    int use_thr_n, use_thr_i;
    double q[4];             /* plane orientation in the volume frame */
    double half_w, sx, sy;   /* pixel (u, v) sits at image point ((u - (W-1)/2) sx, v sy) */
} plane_ctx;

static void plane_setup(const ora_volume* v, const double* P, int32_t W, double sx, double sy,
                        const ora_params* p, plane_ctx* c) {
    ora_pixel_affine(v->vol_to_world, v->h, P, W, sx, sy, c->aff);
    double R[9], q[4];
    rel_rotation(v->vol_to_world, P, R);
    mat_to_quat(R, q);
    memcpy(c->q, q, sizeof(q));
    c->half_w = 0.5 * (double)(W - 1);
    c->sx = sx;
    c->sy = sy;
    quat_axis(q, p->normal_axis == 1 ? 2 : 1, c->n_r);
    quat_axis(q, 0, c->x_r);
    c->use_thr_n = p->thr_normal_deg < 180.0;
    c->use_thr_i = p->thr_inplane_deg < 180.0;
    c->cos_n = cos(p->thr_normal_deg * (M_PI / 180.0));
    c->cos_i = cos(p->thr_inplane_deg * (M_PI / 180.0));
}

/*
 * Eq. 1 and Eq. 2 for one stored sample against the plane: returns the
 * orientation weight, or 0 when a threshold discards the sample.
 */
static double orientation_weight(const double* q, const plane_ctx* c, const ora_params* p) {
    double n_s[3], x_s[3];
    quat_axis(q, p->normal_axis == 1 ? 2 : 1, n_s);
    quat_axis(q, 0, x_s);
    double d_normal = n_s[0] * c->n_r[0] + n_s[1] * c->n_r[1] + n_s[2] * c->n_r[2];
    double d_inplane = fabs(x_s[0] * c->x_r[0] + x_s[1] * c->x_r[1] + x_s[2] * c->x_r[2]);
    if (c->use_thr_n && d_normal < c->cos_n) return 0.0;
    if (c->use_thr_i && d_inplane < c->cos_i) return 0.0;
    return exp(p->k_normal * (d_normal - 1.0) + p->k_inplane * (d_inplane - 1.0));
}

static void reslice_pixel(const ora_volume* v, const plane_ctx* c0, const ora_params* p, int32_t x, int32_t y,
                          double* out, uint8_t* mask) {
    plane_ctx cp = *c0;
    const plane_ctx* c = &cp;
    if (p->probe == ORA_CURVILINEAR) {
        /* a curvilinear virtual plane: this pixel's beam and lateral axes */
        double qp[4];
        steer(c0->q, ((double)x - c0->half_w) * c0->sx, (double)y * c0->sy, p->apex_x, p->apex_y, qp);
        quat_axis(qp, p->normal_axis == 1 ? 2 : 1, cp.n_r);
        quat_axis(qp, 0, cp.x_r);
    }
    double g[3];
    for (int a = 0; a < 3; ++a) {
        int64_t G = c->aff[a] + (int64_t)x * c->aff[3 + a] + (int64_t)y * c->aff[6 + a];
        g[a] = (double)G / (double)FIX_ONE; /* exact: |G| < 2^53 */
    }
    const int R = p->radius;
    int64_t lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        if (p->kernel == ORA_BOX) {
            int64_t r = (int64_t)floor(g[a] + 0.5);
            lo[a] = r - R; hi[a] = r + R;
        } else {
            int64_t f = (int64_t)floor(g[a]);
            lo[a] = f - R + 1; hi[a] = f + R;
        }
    }
    double num = 0.0, den = 0.0;
    for (int64_t cz = lo[2]; cz <= hi[2]; ++cz)
        for (int64_t cy = lo[1]; cy <= hi[1]; ++cy)
            for (int64_t cx = lo[0]; cx <= hi[0]; ++cx) {
                if (cx < 0 || cy < 0 || cz < 0 || cx >= v->dims[0] || cy >= v->dims[1] || cz >= v->dims[2]) continue;
                double dx = g[0] - (double)cx, dy = g[1] - (double)cy, dz = g[2] - (double)cz;
                double t;
                if (p->kernel == ORA_TENT) {
                    t = (1.0 - fabs(dx) / R) * (1.0 - fabs(dy) / R) * (1.0 - fabs(dz) / R);
                } else if (p->kernel == ORA_BOX) {
                    t = 1.0;
                } else {
                    t = exp(-p->k_dist * sqrt(dx * dx + dy * dy + dz * dz) / R);
                }
                int64_t vi = cx + (int64_t)v->dims[0] * (cy + (int64_t)v->dims[1] * cz);
                for (int64_t s = v->offsets[vi]; s < v->offsets[vi + 1]; ++s) {
                    double w = orientation_weight(v->quat + 4 * s, c, p);
                    double I = p->use_exact ? v->mean_exact[s] : v->stored[s];
                    double m = p->sample_weight ? (double)v->npix[s] : 1.0;
                    num += t * w * m * I;
                    den += t * w * m;
                }
            }
    if (den > 0) {
        *out = num / den;
        *mask = 1;
    } else {
        *out = p->unassigned;
        *mask = 0;
    }
}

/* Reslice a whole W x H plane; out (FP64) and mask (u8) are row-major H x W. */
int ora_reslice(const ora_volume* v, const double* P, int32_t W, int32_t H, double sx, double sy,
                const ora_params* p, double* out, uint8_t* mask) {
    if (p->radius < 1 || W <= 0 || H <= 0) return 1;
    plane_ctx c;
    plane_setup(v, P, W, sx, sy, p, &c);
#pragma omp parallel for schedule(dynamic, 4)
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x)
            reslice_pixel(v, &c, p, x, y, out + (size_t)y * W + x, mask + (size_t)y * W + x);
    return 0;
}

/* Reslice selected pixels: uv holds n (u, v) pairs. */
int ora_reslice_pixels(const ora_volume* v, const double* P, int32_t W, double sx, double sy,
                       const ora_params* p, int64_t n, const int32_t* uv, double* out, uint8_t* mask) {
    if (p->radius < 1 || W <= 0) return 1;
    plane_ctx c;
    plane_setup(v, P, W, sx, sy, p, &c);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) reslice_pixel(v, &c, p, uv[2 * i], uv[2 * i + 1], out + i, mask + i);
    return 0;
}

/*
 * Compounded value of every voxel: RN_fp32(total sum / total npix) of all its
 * pixels, NaN where no pixel landed (the mean compounding of Sec. 2.2's PLUS
 * baseline).
 */
void ora_compounded(const ora_volume* v, double* values) {
    for (int64_t i = 0; i < v->n_vox; ++i)
        values[i] = v->tot_npix[i] > 0 ? (double)rn_f32_quotient(v->tot_sum[i], v->tot_npix[i]) : NAN;
}

/*
 * Hole filling of the compounded volume (the PLUS baseline of Sec. 2.2 runs
 * mean compounding "with hole-filling"; this reading: one pass, inverse
 * distance weights).  An empty voxel takes the mean of the occupied voxels of
 * the (2r+1)^3 cube around it, each weighted by 1 / its Euclidean distance in
 * voxels, when at least min_neighbours of them are occupied; otherwise it
 * stays empty (NaN).  Occupied voxels keep their value.  Reads `values`
 * (ora_compounded), writes `filled`.
 */
void ora_fill_holes(const ora_volume* v, const double* values, int32_t r, int32_t min_neighbours, double* filled) {
    const int64_t nx = v->dims[0], ny = v->dims[1], nz = v->dims[2];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < v->n_vox; ++i) {
        if (!isnan(values[i])) {
            filled[i] = values[i];
            continue;
        }
        const int64_t x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
        double num = 0.0, den = 0.0;
        int64_t n = 0;
        for (int64_t dz = -r; dz <= r; ++dz)
            for (int64_t dy = -r; dy <= r; ++dy)
                for (int64_t dx = -r; dx <= r; ++dx) {
                    const int64_t cx = x + dx, cy = y + dy, cz = z + dz;
                    if (cx < 0 || cy < 0 || cz < 0 || cx >= nx || cy >= ny || cz >= nz) continue;
                    const double S = values[cx + nx * (cy + ny * cz)];
                    if (isnan(S)) continue;  /* also skips the voxel itself */
                    const double w = 1.0 / sqrt((double)(dx * dx + dy * dy + dz * dz));
                    num += w * S;
                    den += w;
                    n += 1;
                }
        filled[i] = (n >= min_neighbours && n > 0) ? num / den : NAN;
    }
}

/*
 * Trilinear reslice of a scalar volume (NaN = empty voxel): a pixel is the
 * trilinear blend of the non-empty corners, renormalised by their weights,
 * and unassigned when none is.
 */
int ora_reslice_values(const int32_t* dims, double h, const double* V, const double* values, const double* P,
                       int32_t W, int32_t H, double sx, double sy, double unassigned, double* out, uint8_t* mask) {
    int64_t aff[9];
    ora_pixel_affine(V, h, P, W, sx, sy, aff);
#pragma omp parallel for schedule(dynamic, 4)
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x) {
            double g[3];
            int64_t f[3];
            for (int a = 0; a < 3; ++a) {
                int64_t G = aff[a] + (int64_t)x * aff[3 + a] + (int64_t)y * aff[6 + a];
                g[a] = (double)G / (double)FIX_ONE;
                f[a] = (int64_t)floor(g[a]);
            }
            double num = 0, den = 0;
            for (int k = 0; k < 8; ++k) {
                int64_t cx = f[0] + (k & 1), cy = f[1] + ((k >> 1) & 1), cz = f[2] + (k >> 2);
                if (cx < 0 || cy < 0 || cz < 0 || cx >= dims[0] || cy >= dims[1] || cz >= dims[2]) continue;
                const double S = values[cx + (int64_t)dims[0] * (cy + (int64_t)dims[1] * cz)];
                if (isnan(S)) continue;
                double t = (1.0 - fabs(g[0] - cx)) * (1.0 - fabs(g[1] - cy)) * (1.0 - fabs(g[2] - cz));
                num += t * S;
                den += t;
            }
            size_t o = (size_t)y * W + x;
            if (den > 0) { out[o] = num / den; mask[o] = 1; }
            else { out[o] = unassigned; mask[o] = 0; }
        }
    return 0;
}

/*
 * Mean-compounding comparator (the scalar reading of the PLUS baseline of
 * Sec. 2.2): every voxel holds RN_fp32(total sum / total npix) over all of
 * its pixels; a pixel is the trilinear blend of the occupied corners,
 * renormalised by their weights, and unassigned when none is occupied.
 */
int ora_reslice_scalar(const ora_volume* v, const double* P, int32_t W, int32_t H, double sx, double sy,
                       double unassigned, double* out, uint8_t* mask) {
    int64_t aff[9];
    ora_pixel_affine(v->vol_to_world, v->h, P, W, sx, sy, aff);
#pragma omp parallel for schedule(dynamic, 4)
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x) {
            double g[3];
            int64_t f[3];
            for (int a = 0; a < 3; ++a) {
                int64_t G = aff[a] + (int64_t)x * aff[3 + a] + (int64_t)y * aff[6 + a];
                g[a] = (double)G / (double)FIX_ONE;
                f[a] = (int64_t)floor(g[a]);
            }
            double num = 0, den = 0;
            for (int k = 0; k < 8; ++k) {
                int64_t cx = f[0] + (k & 1), cy = f[1] + ((k >> 1) & 1), cz = f[2] + (k >> 2);
                if (cx < 0 || cy < 0 || cz < 0 || cx >= v->dims[0] || cy >= v->dims[1] || cz >= v->dims[2]) continue;
                int64_t vi = cx + (int64_t)v->dims[0] * (cy + (int64_t)v->dims[1] * cz);
                if (v->tot_npix[vi] == 0) continue;
                double t = (1.0 - fabs(g[0] - cx)) * (1.0 - fabs(g[1] - cy)) * (1.0 - fabs(g[2] - cz));
                double S = (double)rn_f32_quotient(v->tot_sum[vi], v->tot_npix[vi]);
                num += t * S;
                den += t;
            }
            size_t o = (size_t)y * W + x;
            if (den > 0) { out[o] = num / den; mask[o] = 1; }
            else { out[o] = unassigned; mask[o] = 0; }
        }
    return 0;
}

/*
 * Footprint: number of distinct in-grid voxels in the neighbourhood window of
 * any pixel of the plane (TENT/EXP: 2R per axis; BOX: 2R+1 around the
 * nearest voxel).  This is the count of voxel records a single reslice must
 * read at least once.
 */
int64_t ora_footprint(const int32_t* dims, double h, const double* V, const double* P, int32_t W, int32_t H,
                      double sx, double sy, int32_t radius, int32_t kernel) {
    int64_t aff[9];
    ora_pixel_affine(V, h, P, W, sx, sy, aff);
    int64_t nvox = (int64_t)dims[0] * dims[1] * dims[2];
    uint8_t* seen = (uint8_t*)calloc((size_t)nvox, 1);
    if (!seen) return -1;
    int64_t count = 0;
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x) {
            int64_t lo[3], hi[3];
            for (int a = 0; a < 3; ++a) {
                int64_t G = aff[a] + (int64_t)x * aff[3 + a] + (int64_t)y * aff[6 + a];
                if (kernel == ORA_BOX) {
                    int64_t r = fix_floor(G + FIX_ONE / 2);
                    lo[a] = r - radius; hi[a] = r + radius;
                } else {
                    int64_t f = fix_floor(G);
                    lo[a] = f - radius + 1; hi[a] = f + radius;
                }
            }
            for (int64_t cz = lo[2]; cz <= hi[2]; ++cz)
                for (int64_t cy = lo[1]; cy <= hi[1]; ++cy)
                    for (int64_t cx = lo[0]; cx <= hi[0]; ++cx) {
                        if (cx < 0 || cy < 0 || cz < 0 || cx >= dims[0] || cy >= dims[1] || cz >= dims[2]) continue;
                        int64_t vi = cx + (int64_t)dims[0] * (cy + (int64_t)dims[1] * cz);
                        if (!seen[vi]) { seen[vi] = 1; ++count; }
                    }
        }
    free(seen);
    return count;
}
