// DARE reslicing (Sec. 2.1 "Reslicing", Eq. 1, Eq. 2) for curvilinear
// probes on sm_103a.
//
// The paper's probe is a linear array: a frame's beam is its image y axis
// everywhere, so Eq. 1 depends only on (plane, frame) and the other kernels
// read it from a per-frame weight table.  A curvilinear probe's beams fan out
// from an apex: the beam through image point p runs along (p - a) / |p - a|,
// the frame's image axes turned about image z.  A stored sample's axes are
// its frame's turned toward the centre of its voxel (projected into the
// frame); a curvilinear virtual plane turns its own axes at every output
// pixel.  The weight then depends on (pixel, voxel, frame) and no longer
// factors through a per-voxel sum, so this kernel gathers per pixel and
// evaluates Eq. 1 and Eq. 2 for every sample it reads:
//   u_s = (p_s - a_s) / |p_s - a_s|, b_s = R_f (u_s,x, u_s,y, 0), x_s = R_f (u_s,y, -u_s,x, 0)
//   d_normal = n_s . n_p (n = b, or the elevation axis R z), d_inplane = |x_s . x_p|
//   w = exp(-k_normal |n_s - n_p|^2 / 2 - k_inplane |x_s -+ x_p|^2 / 2)
// (1 - n_s . n_p = |n_s - n_p|^2 / 2 for unit vectors: the form that keeps its
// accuracy where the weight is large).
//
// Thresholds: a sample passes iff d >= cos(threshold), decided exactly.  The
// FP32 dot products carry an error of at most
//   E = 4 (k1_s / |p_s| + k1_p / |p_p|) + 96 eps
// (k1 = 17 eps S, S a bound on the FP32 point computation's operands, from the
// host); a decision with |d - cos| <= E is re-taken in FP64 from the FP64
// geometry (a filtered predicate: FP32 speed, FP64 decisions).
#include <cfloat>

#include "dare_internal.h"
#include "device_common.cuh"

namespace dare {
namespace {

using namespace dev;

constexpr float kEps = 5.9604645e-8f;  // 2^-24, FP32 unit roundoff

__device__ __forceinline__ float tent_factor(float d, float R) { return 1.0f - __fdiv_rn(fabsf(d), R); }
__device__ __forceinline__ float exp_weight(float d2, float kr) { return expf(-kr * sqrtf(d2)); }

struct V3 {
    float x, y, z;
};

// a p + b q
__device__ __forceinline__ V3 comb(float a, V3 p, float b, V3 q) {
    return {fmaf(a, p.x, b * q.x), fmaf(a, p.y, b * q.y), fmaf(a, p.z, b * q.z)};
}
__device__ __forceinline__ float dot(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
// |a - s b|^2 / 2
__device__ __forceinline__ float half_gap2(V3 a, V3 b, float s) {
    const float dx = fmaf(-s, b.x, a.x), dy = fmaf(-s, b.y, a.y), dz = fmaf(-s, b.z, a.z);
    return 0.5f * fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// The output pixel's axes (volume frame) and its part of the error bound.
struct PixelAxes {
    V3 n, x;   // Eq. 1 normal (beam or elevation) and lateral axis
    float e;   // k1_p / |p_p|; infinite at the apex (every decision in FP64)
};

__device__ __forceinline__ PixelAxes pixel_axes(const CurvJob& C, int u, int v) {
    float ux = 0.0f, uy = 1.0f, e = 0.0f;
    if (C.curv_out) {
        const float px = fmaf(static_cast<float>(u), C.sxf, C.oxf);
        const float py = fmaf(static_cast<float>(v), C.syf, C.oyf);
        const float r2 = fmaf(px, px, py * py);
        if (r2 > 0.0f) {
            const float inv = rsqrtf(r2);
            ux = px * inv;
            uy = py * inv;
            e = C.k1p * inv;
        } else {
            e = INFINITY;
        }
    }
    const V3 c0 = {C.Rf[0], C.Rf[3], C.Rf[6]}, c1 = {C.Rf[1], C.Rf[4], C.Rf[7]};
    PixelAxes P;
    P.x = comb(uy, c0, -ux, c1);
    P.n = C.elevation ? V3{C.Rf[2], C.Rf[5], C.Rf[8]} : comb(ux, c0, uy, c1);
    P.e = e;
    return P;
}

// d >= c for d = L / sqrt(N) (N > 0), decided without the square root:
// FP64 divisions and square roots are slow on this part.
__device__ __forceinline__ bool at_least(double L, double N, double c) {
    if (c >= 0.0) return L >= 0.0 && L * L >= c * c * N;
    return L >= 0.0 || L * L <= c * c * N;
}

// Threshold decisions of one (pixel, sample) pair in FP64: bit 0 normal
// passes, bit 1 in-plane passes.  Off the hot path.  The fan directions stay
// unnormalised (apex-relative points p_s, p_p; (0, 1) for a linear probe or at
// the apex): with M = (R_f^T R_p) restricted to image x, y,
//   d_normal  = p_s^T M p_p / (|p_s| |p_p|)       (beam)
//   d_inplane = |q_s^T M q_p| / (|p_s| |p_p|),  q = (p_y, -p_x)
// and each comparison with a cosine is taken on squares.
__device__ __noinline__ int decide64(const CurvJob& C, int f, float ci, float cj, float ck, int u, int v) {
    const double* R = C.rot64 + 9 * static_cast<int64_t>(f);
    double sx = 0.0, sy = 1.0;
    if (__ldg(&C.geom[5 * f + 4].z) != 0.0f) {
        const double* o = C.off64 + 2 * static_cast<int64_t>(f);
        const double hi = C.h * ci, hj = C.h * cj, hk = C.h * ck;
        const double px = R[0] * hi + R[3] * hj + R[6] * hk + o[0], py = R[1] * hi + R[4] * hj + R[7] * hk + o[1];
        if (px != 0.0 || py != 0.0) {
            sx = px;
            sy = py;
        }
    }
    double qx = 0.0, qy = 1.0;
    if (C.curv_out) {
        const double px = (static_cast<double>(u) - C.half_w) * C.sx - C.ax, py = static_cast<double>(v) * C.sy - C.ay;
        if (px != 0.0 || py != 0.0) {
            qx = px;
            qy = py;
        }
    }
    // M[a][b] = column a of R_f . column b of R_p (a, b: image x, y)
    double M00 = 0.0, M01 = 0.0, M10 = 0.0, M11 = 0.0, Mzz = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        M00 += R[3 * r] * C.R[3 * r];
        M01 += R[3 * r] * C.R[3 * r + 1];
        M10 += R[3 * r + 1] * C.R[3 * r];
        M11 += R[3 * r + 1] * C.R[3 * r + 1];
        Mzz += R[3 * r + 2] * C.R[3 * r + 2];
    }
    const double N = (sx * sx + sy * sy) * (qx * qx + qy * qy);
    // beam: (sx, sy) M (qx, qy); lateral: (sy, -sx) M (qy, -qx)
    const double Ln = sx * (M00 * qx + M01 * qy) + sy * (M10 * qx + M11 * qy);
    const double Li = sy * (M00 * qy - M01 * qx) - sx * (M10 * qy - M11 * qx);
    const bool pn = C.elevation ? Mzz >= C.cos_n64 : at_least(Ln, N, C.cos_n64);
    const bool pi = at_least(fabs(Li), N, C.cos_i64);
    return (pn ? 1 : 0) | (pi ? 2 : 0);
}

// Eq. 1 / Eq. 2 weight of frame f's sample in voxel (ci, cj, ck) for this
// pixel, 0 when a threshold discards it.
__device__ __forceinline__ float sample_weight(const CurvJob& C, const PixelAxes& P, int f, float ci, float cj,
                                               float ck, int u, int v) {
    const float4* G = C.geom + 5 * static_cast<int64_t>(f);
    const float4 g2 = __ldg(G + 2), g3 = __ldg(G + 3), g4 = __ldg(G + 4);
    float ux = 0.0f, uy = 1.0f, es = 0.0f;
    if (g4.z != 0.0f) {  // curvilinear frame: turn toward the voxel centre
        const float4 g0 = __ldg(G), g1 = __ldg(G + 1);
        const float px = fmaf(g0.x, ci, fmaf(g0.y, cj, fmaf(g0.z, ck, g0.w)));
        const float py = fmaf(g1.x, ci, fmaf(g1.y, cj, fmaf(g1.z, ck, g1.w)));
        const float r2 = fmaf(px, px, py * py);
        if (r2 > 0.0f) {
            const float inv = rsqrtf(r2);
            ux = px * inv;
            uy = py * inv;
            es = g4.y * inv;
        } else {
            es = INFINITY;
        }
    }
    const V3 c0 = {g2.x, g2.y, g2.z}, c1 = {g2.w, g3.x, g3.y};
    const V3 xs = comb(uy, c0, -ux, c1);
    const V3 ns = C.elevation ? V3{g3.z, g3.w, g4.x} : comb(ux, c0, uy, c1);
    const float dn = dot(ns, P.n), dx = dot(xs, P.x), di = fabsf(dx);
    bool pass_n = !C.use_n || dn >= C.cos_n;
    bool pass_i = !C.use_i || di >= C.cos_i;
    const float E = fmaf(4.0f, es + P.e, 96.0f * kEps);
    if ((C.use_n && fabsf(dn - C.cos_n) <= E) || (C.use_i && fabsf(di - C.cos_i) <= E)) {
        const int d = decide64(C, f, ci, cj, ck, u, v);
        pass_n = !C.use_n || (d & 1);
        pass_i = !C.use_i || (d & 2);
    }
    if (!(pass_n && pass_i)) return 0.0f;
    const float en = half_gap2(ns, P.n, 1.0f), ei = half_gap2(xs, P.x, dx < 0.0f ? -1.0f : 1.0f);
    return expf(-fmaf(C.k_n, en, C.k_i * ei));
}

// One voxel's (A, B) = (sum w I, sum w) for this pixel.
template <int K, typename VT>
__device__ __forceinline__ float2 curv_voxel(const CurvJob& C, const PixelAxes& P, int64_t vi, float ci, float cj,
                                             float ck, int u, int v) {
    using S = RecShape<K, VT>;
    uint4 r[S::kVec];
    load_record<K, VT>(C.j.rec + vi * S::kBytes, r);
    // per-pixel samples: each merged sample counts npix times (its pixels share the weight)
    uint2 n[K / 4];
    if (C.j.npix) {
        const uint2* q = reinterpret_cast<const uint2*>(C.j.npix + vi * K);
#pragma unroll
        for (int i = 0; i < K / 4; ++i) n[i] = __ldg(q + i);
    }
    float A = 0.0f, B = 0.0f;
#pragma unroll
    for (int s = 0; s < K; ++s) {
        const uint32_t id = slot_id<K, VT>(r, s);
        if (id == DARE_EMPTY_FRAME) break;  // empty slots come last
        float w = sample_weight(C, P, static_cast<int>(id), ci, cj, ck, u, v);
        if (C.j.npix) {
            const uint32_t word = (s & 2) ? n[s >> 2].y : n[s >> 2].x;
            w *= static_cast<float>((word >> (16 * (s & 1))) & 0xFFFFu);
        }
        A = fmaf(w, slot_value<K, VT>(r, s), A);
        B += w;
    }
    return make_float2(A, B);
}

// The pixel's support (as in the linear-probe kernels) with per-sample weights.
template <int K, typename VT>
__device__ __noinline__ float2 gather_pixel_curv(const CurvJob& C, int u, int v) {
    float num = 0.0f, den = 0.0f;
    const ResliceJob& J = C.j;
    const int R = J.radius;
    const bool box = J.kernel == DARE_BOX;
    const int S = box ? 2 * R + 1 : 2 * R;
    int64_t lo[3];
    float fr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int64_t G = J.g0[a] + static_cast<int64_t>(u) * J.a[a] + static_cast<int64_t>(v) * J.b[a];
        const int64_t f = G >> kFixBits;
        fr[a] = static_cast<float>(static_cast<int32_t>(G & (kFixOne - 1))) * (1.0f / static_cast<float>(kFixOne));
        lo[a] = box ? f + (fr[a] >= 0.5f ? 1 : 0) - R : f - R + 1;
        if (lo[a] + S - 1 < 0 || lo[a] > J.dims[a] - 1) return make_float2(num, den);  // the support misses the grid
        fr[a] -= static_cast<float>(static_cast<int>(lo[a] - f));  // g - lo, exact (int32: a fast conversion)
    }
    const PixelAxes P = pixel_axes(C, u, v);
    const float Rf = static_cast<float>(R), kr = J.k_dist / Rf;
    for (int jz = 0; jz < S; ++jz) {
        const int64_t cz = lo[2] + jz;
        if (cz < 0 || cz >= J.dims[2]) continue;
        const float dz = fr[2] - static_cast<float>(jz);
        const float tz = J.kernel == DARE_TENT ? tent_factor(dz, Rf) : 1.0f;
        for (int jy = 0; jy < S; ++jy) {
            const int64_t cy = lo[1] + jy;
            if (cy < 0 || cy >= J.dims[1]) continue;
            const float dy = fr[1] - static_cast<float>(jy);
            const float tyz = J.kernel == DARE_TENT ? tent_factor(dy, Rf) * tz : 1.0f;
            for (int jx = 0; jx < S; ++jx) {
                const int64_t cx = lo[0] + jx;
                if (cx < 0 || cx >= J.dims[0]) continue;
                const float dx = fr[0] - static_cast<float>(jx);
                float t;
                if (J.kernel == DARE_TENT)
                    t = tent_factor(dx, Rf) * tyz;
                else if (box)
                    t = 1.0f;
                else
                    t = exp_weight(dx * dx + dy * dy + dz * dz, kr);
                const int64_t vi = cx + static_cast<int64_t>(J.dims[0]) * (cy + static_cast<int64_t>(J.dims[1]) * cz);
                // voxel coordinates < 2^31: converted from int32 (int64 conversions are slow here)
                const float2 ab = curv_voxel<K, VT>(C, P, vi, static_cast<float>(static_cast<int>(cx)),
                                                    static_cast<float>(static_cast<int>(cy)),
                                                    static_cast<float>(static_cast<int>(cz)), u, v);
                num = fmaf(t, ab.x, num);
                den = fmaf(t, ab.y, den);
            }
        }
    }
    return make_float2(num, den);
}

// 32 x 8 pixels per CTA, one per thread; a warp writes one mask word.
template <int K, typename VT>
__device__ __forceinline__ void curv_body(const CurvJob& C) {
    const ResliceJob& J = C.j;
    const int lane = threadIdx.x;
    const int u = blockIdx.x * 32 + lane;
    const int v = blockIdx.y * 8 + threadIdx.y;
    if (v >= J.height || static_cast<int>(blockIdx.x) * 32 >= J.width) return;  // warp-uniform
    const bool active = u < J.width;
    float num = 0.0f, den = 0.0f;
    if (active) {
        const float2 nd = gather_pixel_curv<K, VT>(C, u, v);
        num = nd.x;
        den = nd.y;
        J.out[static_cast<int64_t>(v) * J.width + u] = den > 0.0f ? num / den : J.unassigned;
    }
    const unsigned bits = __ballot_sync(0xFFFFFFFFu, active && den > 0.0f);
    if (lane == 0) J.mask[static_cast<int64_t>(v) * J.mask_stride + blockIdx.x] = bits;
}

// 4 CTAs per SM (64 registers): measured on 1000 512^2 planes, 47 ms against
// 51 / 58 / 55 ms at 3 / 2 / 6 CTAs per SM (the extra warps hide the record and
// geometry-row loads better than registers save spills)
template <int K, typename VT>
__global__ void __launch_bounds__(256, 4) k_reslice_curv_one(const __grid_constant__ CurvJob C) {
    curv_body<K, VT>(C);
}

template <int K, typename VT>
__global__ void __launch_bounds__(256, 4) k_reslice_curv_batch(const CurvJob* __restrict__ jobs) {
    curv_body<K, VT>(jobs[blockIdx.z]);
}

template <int K, typename VT>
cudaError_t launch_c(const CurvJob* jobs_dev, const CurvJob* one, int n_jobs, int max_w, int max_h, cudaStream_t st) {
    const dim3 block(32, 8);
    const dim3 grid((max_w + 31) / 32, (max_h + 7) / 8, one ? 1 : n_jobs);
    if (one)
        k_reslice_curv_one<K, VT><<<grid, block, 0, st>>>(*one);
    else
        k_reslice_curv_batch<K, VT><<<grid, block, 0, st>>>(jobs_dev);
    return cudaPeekAtLastError();
}

template <int K>
cudaError_t launch_c_k(const CurvJob* jobs_dev, const CurvJob* one, int n_jobs, int max_w, int max_h, int dtype,
                       cudaStream_t st) {
    switch (dtype) {
    case DARE_U8: return launch_c<K, uint8_t>(jobs_dev, one, n_jobs, max_w, max_h, st);
    case DARE_F16: return launch_c<K, __half>(jobs_dev, one, n_jobs, max_w, max_h, st);
    case DARE_BF16: return launch_c<K, __nv_bfloat16>(jobs_dev, one, n_jobs, max_w, max_h, st);
    case DARE_F32: return launch_c<K, float>(jobs_dev, one, n_jobs, max_w, max_h, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_reslice_curv(const CurvJob* jobs_dev, const CurvJob* one_job, int n_jobs, int max_w, int max_h,
                                int K, int dtype, cudaStream_t st) {
    if (n_jobs <= 0 || max_w <= 0 || max_h <= 0) return cudaSuccess;
    if (!one_job && n_jobs > 65535) return cudaErrorInvalidValue;
    switch (K) {
    case 4: return launch_c_k<4>(jobs_dev, one_job, n_jobs, max_w, max_h, dtype, st);
    case 8: return launch_c_k<8>(jobs_dev, one_job, n_jobs, max_w, max_h, dtype, st);
    case 12: return launch_c_k<12>(jobs_dev, one_job, n_jobs, max_w, max_h, dtype, st);
    case 16: return launch_c_k<16>(jobs_dev, one_job, n_jobs, max_w, max_h, dtype, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dare
