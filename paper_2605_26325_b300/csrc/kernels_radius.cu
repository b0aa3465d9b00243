// DARE reslicing (Sec. 2.1 "Reslicing", Eq. 1, Eq. 2) for any interpolation
// radius and distance kernel -- the paper's timing axis (Sec. 3: radii of
// 0.125, 0.25 and 0.5 mm, i.e. 3^3 to 9^3 voxel neighbourhoods) -- on sm_103a.
//
// A pixel at fixed-point position g (floor f, exact 20-bit fraction) reads,
// per axis:
//   TENT: voxels f - R + 1 .. f + R,        t = prod_a (1 - |g_a - c_a| / R)
//   BOX:  voxels round(g) - R .. round(g) + R, t = 1  (round = floor(g + 1/2))
//   EXP:  voxels f - R + 1 .. f + R,        t = exp(-k_d |g - c| / R)
// and averages t w_f I / t w_f over the valid samples of those voxels.
//
// Two kernels: a per-pixel gather (one thread per pixel; also the fallback of
// the tiled kernel for planes whose tiles do not fit shared memory), and the
// tiled kernel of kernels_tiled.cu widened to a radius: a tile reduces every
// voxel its pixels can reach once to (A_c = sum w I, B_c = sum w) -- exact
// for any distance kernel, which depends only on the voxel's offset from the
// pixel -- then blends the whole support of each pixel from shared memory.
#include <cfloat>

#include "dare_internal.h"
#include "device_common.cuh"

namespace dare {
namespace {

using namespace dev;

constexpr int kThreads = 256;
constexpr int kTH = 32;          // tile rows of the general tiled kernel (tile 32 x 32)

// tiles that gathered per pixel because their column box did not fit shared memory
__device__ unsigned long long g_fallback_tiles_r;
constexpr float kMargin = 0.02f; // voxel; > FP32 error of the plane height for |g| < 2^14

// distance weights: TENT factor of one axis, EXP of the squared distance
__device__ __forceinline__ float tent_factor(float d, float R) { return 1.0f - __fdiv_rn(fabsf(d), R); }
__device__ __forceinline__ float exp_weight(float d2, float kr) { return expf(-kr * sqrtf(d2)); }

// npix of slot s from a voxel's npix row held as K/4 uint2
template <int K>
__device__ __forceinline__ float slot_npix(const uint2 (&n)[K / 4], int s) {
    const uint2 q = n[s >> 2];
    const uint32_t w = (s & 2) ? q.y : q.x;
    return static_cast<float>((w >> (16 * (s & 1))) & 0xFFFFu);
}

// (A_c, B_c) of one voxel with every sample weighted by its pixel count: the
// per-pixel reading of the storage (each pixel a sample with its frame's
// orientation), exactly, since a frame's pixels in a voxel share one weight.
template <int K, typename VT, typename WT>
__device__ __forceinline__ float2 collapse_voxel_px(const uint8_t* rec, const uint16_t* npix, int64_t vi,
                                                    const WT* wt) {
    using S = RecShape<K, VT>;
    uint4 r[S::kVec];
    load_record<K, VT>(rec + vi * S::kBytes, r);
    uint2 n[K / 4];
    const uint2* q = reinterpret_cast<const uint2*>(npix + vi * K);
#pragma unroll
    for (int i = 0; i < K / 4; ++i) n[i] = __ldg(q + i);
    float A = 0.0f, B = 0.0f;
    constexpr int G = SlotGroup<K>::G;  // table lookups in groups, as in collapse_voxel
#pragma unroll
    for (int g = 0; g < K; g += G) {
        uint32_t id[G];
        float wf[G];
#pragma unroll
        for (int j = 0; j < G; ++j) id[j] = g + j < K ? slot_id<K, VT>(r, g + j) : DARE_EMPTY_FRAME;
        if (id[0] == DARE_EMPTY_FRAME) break;
#pragma unroll
        for (int j = 0; j < G; ++j) wf[j] = id[j] != DARE_EMPTY_FRAME ? weight_of(wt, static_cast<int>(id[j])) : 0.0f;
#pragma unroll
        for (int j = 0; j < G; ++j)
            if (id[j] != DARE_EMPTY_FRAME) {
                const float w = wf[j] * slot_npix<K>(n, g + j);
                A = fmaf(w, slot_value<K, VT>(r, g + j), A);
                B += w;
            }
        if (id[G - 1] == DARE_EMPTY_FRAME) break;
    }
    return make_float2(A, B);
}

// Per-pixel gather over the kernel's support (records read from global memory).
template <int K, typename VT, typename WT>
__device__ __noinline__ float2 gather_pixel_r(const ResliceJob& J, int u, int v) {
    float num = 0.0f, den = 0.0f;
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
    const WT* wt = static_cast<const WT*>(J.wtab);
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
                const float2 ab = J.npix ? collapse_voxel_px<K, VT, WT>(J.rec, J.npix, vi, wt)
                                         : collapse_voxel<K, VT, WT>(J.rec, vi, wt);
                num = fmaf(t, ab.x, num);
                den = fmaf(t, ab.y, den);
            }
        }
    }
    return make_float2(num, den);
}

template <int K, typename VT, typename WT>
__device__ __forceinline__ void plain_r_body(const ResliceJob& J) {
    const int lane = threadIdx.x;
    const int u = blockIdx.x * 32 + lane;
    const int v = blockIdx.y * 8 + threadIdx.y;
    if (v >= J.height || static_cast<int>(blockIdx.x) * 32 >= J.width) return;  // warp-uniform
    const bool active = u < J.width;
    float num = 0.0f, den = 0.0f;
    if (active) {
        const float2 nd = gather_pixel_r<K, VT, WT>(J, u, v);
        num = nd.x;
        den = nd.y;
        J.out[static_cast<int64_t>(v) * J.width + u] = den > 0.0f ? num / den : J.unassigned;
    }
    const unsigned bits = __ballot_sync(0xFFFFFFFFu, active && den > 0.0f);
    if (lane == 0) J.mask[static_cast<int64_t>(v) * J.mask_stride + blockIdx.x] = bits;
}

template <int K, typename VT, typename WT>
__global__ void __launch_bounds__(256) k_reslice_plain_r_one(const __grid_constant__ ResliceJob J) {
    plain_r_body<K, VT, WT>(J);
}

template <int K, typename VT, typename WT>
__global__ void __launch_bounds__(256) k_reslice_plain_r_batch(const ResliceJob* __restrict__ jobs) {
    plain_r_body<K, VT, WT>(jobs[blockIdx.z]);
}

// ------------------------------------------------------------------ tiled

template <int D>
struct Axes {
    static constexpr int E1 = D == 0 ? 1 : 0;
    static constexpr int E2 = D == 2 ? 1 : 2;
};

__device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t lmax(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ int64_t axis_fix(const ResliceJob& J, int a, int u, int v) {
    return J.g0[a] + static_cast<int64_t>(u) * J.a[a] + static_cast<int64_t>(v) * J.b[a];
}

__device__ __forceinline__ int find_job(const ResliceJob* jobs, int n_jobs, int tile) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&jobs[mid].tile_base) <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

struct TileSetupR {
    int u0, v0, u1, v1;      // pixel range of the tile
    int b1, b2, n1, n2;      // column box (its first columns and sizes along e1, e2)
    int direct, empty;
    int R1, R2, Rd;          // 20-bit remainders of the tile origin's coordinates
    int O1, O2, Od;          // floors of the origin, relative to the box (Od absolute)
};

// The box holds every column a pixel of the tile reads: floors of the tile's
// corners (convexity) widened by the support's reach ext_lo / ext_hi.
template <int D>
__device__ void tile_setup_r(const ResliceJob& J, int u0, int v0, int u1, int v1, int col_cap, int slot_cap,
                             TileSetupR& T) {
    constexpr int E1 = Axes<D>::E1, E2 = Axes<D>::E2;
    int64_t lo1 = INT64_MAX, hi1 = INT64_MIN, lo2 = INT64_MAX, hi2 = INT64_MIN, lod = INT64_MAX, hid = INT64_MIN;
    for (int k = 0; k < 4; ++k) {
        const int u = (k & 1) ? u1 : u0, v = (k & 2) ? v1 : v0;
        const int64_t f1 = axis_fix(J, E1, u, v) >> kFixBits, f2 = axis_fix(J, E2, u, v) >> kFixBits;
        const int64_t fd = axis_fix(J, D, u, v) >> kFixBits;
        lo1 = lmin(lo1, f1); hi1 = lmax(hi1, f1);
        lo2 = lmin(lo2, f2); hi2 = lmax(hi2, f2);
        lod = lmin(lod, fd); hid = lmax(hid, fd);
    }
    const int el = J.ext_lo, eh = J.ext_hi;
    T.empty = hi1 + eh < 0 || lo1 - el > J.dims[E1] - 1 || hi2 + eh < 0 || lo2 - el > J.dims[E2] - 1 ||
              hid + eh < 0 || lod - el > J.dims[D] - 1;
    const int64_t n1 = hi1 - lo1 + el + eh + 1, n2 = hi2 - lo2 + el + eh + 1;
    const int S = J.kernel == DARE_BOX ? 2 * J.radius + 1 : 2 * J.radius;  // support per axis
    T.direct = !T.empty && (J.direct || S > kMaxSupport || n1 > col_cap || n2 > col_cap || n1 * n2 > col_cap ||
                            n1 * n2 * J.levels > slot_cap || lo1 < -(1 << 30) || lo2 < -(1 << 30) ||
                            hi1 > (1 << 30) || hi2 > (1 << 30));
    T.b1 = static_cast<int>(lmax(lmin(lo1 - el, 1 << 30), -(1 << 30)));
    T.b2 = static_cast<int>(lmax(lmin(lo2 - el, 1 << 30), -(1 << 30)));
    T.n1 = T.direct || T.empty ? 0 : static_cast<int>(n1);
    T.n2 = T.direct || T.empty ? 0 : static_cast<int>(n2);
    const int64_t G1 = axis_fix(J, E1, u0, v0), G2 = axis_fix(J, E2, u0, v0), Gd = axis_fix(J, D, u0, v0);
    T.R1 = static_cast<int>(G1 & (kFixOne - 1));
    T.R2 = static_cast<int>(G2 & (kFixOne - 1));
    T.Rd = static_cast<int>(Gd & (kFixOne - 1));
    T.O1 = static_cast<int>(lmax(lmin((G1 >> kFixBits) - T.b1, 1 << 24), -(1 << 24)));
    T.O2 = static_cast<int>(lmax(lmin((G2 >> kFixBits) - T.b2, 1 << 24), -(1 << 24)));
    T.Od = static_cast<int>(lmax(lmin(Gd >> kFixBits, 1 << 24), -(1 << 24)));
}

template <int K, typename VT, typename WT, int D>
__device__ __forceinline__ void tile_body_r(const ResliceJob& J, const TileSetupR& T, float2* sAB, int* sCol) {
    constexpr int E1 = Axes<D>::E1, E2 = Axes<D>::E2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WT* wt = static_cast<const WT*>(J.wtab);
    const int u0 = T.u0, v0 = T.v0, u1 = T.u1, v1 = T.v1;
    const int b1 = T.b1, b2 = T.b2, n1 = T.n1, n2 = T.n2, ncol = n1 * n2, L = J.levels;
    const bool direct = T.direct != 0, empty = T.empty != 0;
    const int R = J.radius, el = J.ext_lo, eh = J.ext_hi;
    const bool box = J.kernel == DARE_BOX, tent = J.kernel == DARE_TENT;

    if (!direct && !empty) {
        // (A) per column: lowest level, then L slots (A_c, B_c) of levels lo .. lo + L - 1;
        // slots outside the grid, past the column's range or of unreached columns hold zeros
        const float inv_n1 = 1.0f / static_cast<float>(n1);
        const float reach = static_cast<float>(max(eh, el + 1));
        const float sm = (J.spread + kMargin) * reach;
        const int dd = J.dims[D], d1 = J.dims[E1], d2 = J.dims[E2];
        const float ou = J.ou, ov = J.ov, m00 = J.m00, m01 = J.m01, m10 = J.m10, m11 = J.m11, hu = J.hu, hv = J.hv;
        const float alpha = J.alpha, beta1 = J.beta1, beta2 = J.beta2;
        const float fu0 = static_cast<float>(u0), fu1 = static_cast<float>(u1);
        const float fv0 = static_cast<float>(v0), fv1 = static_cast<float>(v1);
        const uint8_t* const rec = J.rec;
        const uint16_t* const npx = J.npix;
        const int64_t sx = 1, sy = J.dims[0], sz = static_cast<int64_t>(J.dims[0]) * J.dims[1];
        const int64_t st1 = E1 == 0 ? sx : sy, st2 = E2 == 1 ? sy : sz, std_ = D == 0 ? sx : (D == 1 ? sy : sz);
        for (int c = threadIdx.x; c < ncol; c += kThreads) {
            const int k2 = static_cast<int>((static_cast<float>(c) + 0.5f) * inv_n1);
            const int k1 = c - k2 * n1;
            const int c1 = b1 + k1, c2 = b2 + k2;
            const float uc = ou + m00 * c1 + m01 * c2;
            const float vc = ov + m10 * c1 + m11 * c2;
            const bool near = fabsf(uc - fminf(fmaxf(uc, fu0), fu1)) <= hu && fabsf(vc - fminf(fmaxf(vc, fv0), fv1)) <= hv;
            const float gd = alpha + beta1 * c1 + beta2 * c2;
            int lo = 0, top = -1;  // levels lo .. top may be read
            if (near && fabsf(gd) < 16384.0f && static_cast<unsigned>(c1) < static_cast<unsigned>(d1) &&
                static_cast<unsigned>(c2) < static_cast<unsigned>(d2)) {
                lo = static_cast<int>(floorf(gd - sm)) - el;
                top = min(static_cast<int>(floorf(gd + sm)) + eh, dd - 1);
            }
            sCol[c] = lo;
            const int64_t base = c1 * st1 + c2 * st2;
            for (int lev = 0; lev < L; ++lev) {
                const int g = lo + lev;
                sAB[c * L + lev] = (g >= 0 && g <= top)
                                       ? (npx ? collapse_voxel_px<K, VT, WT>(rec, npx, base + g * std_, wt)
                                              : collapse_voxel<K, VT, WT>(rec, base + g * std_, wt))
                                       : make_float2(0.0f, 0.0f);
            }
        }
        __syncthreads();
    }
    // (B) pixels: a warp walks the 32 pixels of a tile row and blends each pixel's support
    const int A1 = static_cast<int>(J.a[E1]), B1 = static_cast<int>(J.b[E1]);
    const int A2 = static_cast<int>(J.a[E2]), B2 = static_cast<int>(J.b[E2]);
    const int Ad = static_cast<int>(J.a[D]), Bd = static_cast<int>(J.b[D]);
    const int Rr1 = T.R1 + lane * A1, Rr2 = T.R2 + lane * A2, Rrd = T.Rd + lane * Ad;
    const int O1 = T.O1, O2 = T.O2, Od = T.Od;
    float* const out = J.out;
    uint32_t* const mask = J.mask;
    const int64_t width = J.width, mstride = J.mask_stride;
    const float unassigned = J.unassigned;
    const int Sp = box ? 2 * R + 1 : 2 * R;  // support per axis
    const float Rf = static_cast<float>(R), kr = J.k_dist / Rf;
    const int u = u0 + lane;
    const bool active = u <= u1;
    for (int r = warp; r < kTH; r += kThreads / 32) {
        const int v = v0 + r;
        if (v > v1) break;  // warp-uniform
        float num = 0.0f, den = 0.0f;
        if (active) {
            if (direct) {
                const float2 nd = gather_pixel_r<K, VT, WT>(J, u, v);
                num = nd.x;
                den = nd.y;
            } else if (!empty) {
                const int r1 = Rr1 + r * B1, r2 = Rr2 + r * B2, rd = Rrd + r * Bd;
                const float p1 = static_cast<float>(r1 & (kFixOne - 1)) * (1.0f / static_cast<float>(kFixOne));
                const float p2 = static_cast<float>(r2 & (kFixOne - 1)) * (1.0f / static_cast<float>(kFixOne));
                const float pd = static_cast<float>(rd & (kFixOne - 1)) * (1.0f / static_cast<float>(kFixOne));
                // first voxel of the support per axis, relative to the floor
                const int s1 = box ? (p1 >= 0.5f ? 1 : 0) - R : 1 - R;
                const int s2 = box ? (p2 >= 0.5f ? 1 : 0) - R : 1 - R;
                const int sd = box ? (pd >= 0.5f ? 1 : 0) - R : 1 - R;
                // k1 + s1 in [0, n1 - Sp], k2 + s2 in [0, n2 - Sp] by construction of the box
                const int k1 = (r1 >> kFixBits) + O1 + s1, k2 = (r2 >> kFixBits) + O2 + s2;
                const int fd = (rd >> kFixBits) + Od + sd;
                // along d: the TENT factors, or the offsets for EXP
                float wd[kMaxSupport];
#pragma unroll
                for (int jd = 0; jd < kMaxSupport; ++jd) {
                    const float dd = pd - static_cast<float>(sd + jd);
                    wd[jd] = tent ? (jd < Sp ? tent_factor(dd, Rf) : 0.0f) : dd * dd;
                }
                for (int j2 = 0; j2 < Sp; ++j2) {
                    const float d2 = p2 - static_cast<float>(s2 + j2);
                    const float f2 = tent ? tent_factor(d2, Rf) : d2 * d2;
                    for (int j1 = 0; j1 < Sp; ++j1) {
                        const float d1 = p1 - static_cast<float>(s1 + j1);
                        const float f12 = tent ? tent_factor(d1, Rf) * f2 : d1 * d1 + f2;
                        const int c = k1 + j1 + n1 * (k2 + j2);
                        // the levels fd .. fd + Sp - 1 lie in the column's range; the clamp only keeps reads in bounds
                        const int lb = min(max(fd - sCol[c], 0), L - Sp);
                        const float2* col = sAB + c * L + lb;
#pragma unroll
                        for (int jd = 0; jd < kMaxSupport; ++jd) {
                            if (jd < Sp) {
                                const float t = tent ? f12 * wd[jd] : (box ? 1.0f : exp_weight(f12 + wd[jd], kr));
                                const float2 ab = col[jd];
                                num = fmaf(t, ab.x, num);
                                den = fmaf(t, ab.y, den);
                            }
                        }
                    }
                }
            }
            out[v * width + u] = den > 0.0f ? num / den : unassigned;
        }
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, active && den > 0.0f);
        if (lane == 0) mask[v * mstride + u0 / 32] = bits;
    }
}

template <int K, typename VT, typename WT>
__global__ void __launch_bounds__(kThreads, 3) k_reslice_tiled_r(const ResliceJob* __restrict__ jobs, int n_jobs,
                                                              int tile_offset, int uniform, int col_cap,
                                                              int slot_cap, const __grid_constant__ ResliceJob one) {
    extern __shared__ __align__(16) unsigned char smem_r[];
    float2* sAB = reinterpret_cast<float2*>(smem_r);
    int* sCol = reinterpret_cast<int*>(sAB + slot_cap);
    __shared__ TileSetupR T;
    __shared__ ResliceJob sJob;
    static_assert(sizeof(ResliceJob) % 4 == 0, "job copied as 32-bit words");
    if (threadIdx.x < 32) {
        int job = 0, lt = static_cast<int>(blockIdx.x);
        if (jobs && uniform) {
            job = static_cast<int>(blockIdx.y);
        } else if (jobs) {
            const int tile = tile_offset + static_cast<int>(blockIdx.x);
            job = find_job(jobs, n_jobs, tile);
            lt = tile - __ldg(&jobs[job].tile_base);
        }
        const uint32_t* src = reinterpret_cast<const uint32_t*>(jobs ? jobs + job : &one);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&sJob);
        for (int i = threadIdx.x; i < static_cast<int>(sizeof(ResliceJob) / 4); i += 32) dst[i] = src[i];
        __syncwarp();
        if (threadIdx.x == 0) {
            const ResliceJob& J0 = sJob;
            const int ty = lt / J0.tiles_x, tx = lt - ty * J0.tiles_x;
            T.u0 = tx * kTileW;
            T.v0 = ty * kTH;
            T.u1 = min(T.u0 + kTileW, J0.width) - 1;
            T.v1 = min(T.v0 + kTH, J0.height) - 1;
            if (J0.d == 0) tile_setup_r<0>(J0, T.u0, T.v0, T.u1, T.v1, col_cap, slot_cap, T);
            else if (J0.d == 1) tile_setup_r<1>(J0, T.u0, T.v0, T.u1, T.v1, col_cap, slot_cap, T);
            else tile_setup_r<2>(J0, T.u0, T.v0, T.u1, T.v1, col_cap, slot_cap, T);
            if (T.direct && !J0.direct) atomicAdd(&g_fallback_tiles_r, 1ull);
        }
    }
    __syncthreads();
    const ResliceJob& J = sJob;
    switch (J.d) {
    case 0: tile_body_r<K, VT, WT, 0>(J, T, sAB, sCol); break;
    case 1: tile_body_r<K, VT, WT, 1>(J, T, sAB, sCol); break;
    default: tile_body_r<K, VT, WT, 2>(J, T, sAB, sCol); break;
    }
}

template <int K, typename VT, typename WT>
cudaError_t launch_r(const ResliceJob* jobs_dev, const ResliceJob* one, int n_jobs, int tile_offset, int n_tiles,
                     int uniform, int col_cap, int slot_cap, int max_w, int max_h, bool tiled, cudaStream_t st) {
    if (!tiled) {
        dim3 block(32, 8);
        dim3 grid((max_w + 31) / 32, (max_h + 7) / 8, one ? 1 : n_jobs);
        if (one)
            k_reslice_plain_r_one<K, VT, WT><<<grid, block, 0, st>>>(*one);
        else
            k_reslice_plain_r_batch<K, VT, WT><<<grid, block, 0, st>>>(jobs_dev);
        return cudaPeekAtLastError();
    }
    const size_t smem = size_t(slot_cap) * sizeof(float2) + size_t(col_cap) * sizeof(int);
    if (smem > size_t(kGeneralSmemCap)) return cudaErrorInvalidValue;
    static int configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !configured[dev]) {
        e = cudaFuncSetAttribute(k_reslice_tiled_r<K, VT, WT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kGeneralSmemCap);
        if (e != cudaSuccess) return e;
        configured[dev] = 1;
    }
    ResliceJob dummy{};
    const dim3 grid(n_tiles, (one || !uniform) ? 1 : n_jobs);
    k_reslice_tiled_r<K, VT, WT><<<grid, kThreads, smem, st>>>(one ? nullptr : jobs_dev, n_jobs, tile_offset,
                                                               uniform, col_cap, slot_cap, one ? *one : dummy);
    return cudaPeekAtLastError();
}

template <int K, typename VT>
cudaError_t launch_r_w(const ResliceJob* jobs_dev, const ResliceJob* one, int n_jobs, int tile_offset, int n_tiles,
                       int uniform, int col_cap, int slot_cap, int max_w, int max_h, bool tiled, int half_w,
                       cudaStream_t st) {
    return half_w ? launch_r<K, VT, __half>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, col_cap, slot_cap,
                                            max_w, max_h, tiled, st)
                  : launch_r<K, VT, float>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, col_cap, slot_cap,
                                           max_w, max_h, tiled, st);
}

template <int K>
cudaError_t launch_r_k(const ResliceJob* jobs_dev, const ResliceJob* one, int n_jobs, int tile_offset, int n_tiles,
                       int uniform, int col_cap, int slot_cap, int max_w, int max_h, bool tiled, int dtype, int half_w,
                       cudaStream_t st) {
    switch (dtype) {
    case DARE_U8:
        return launch_r_w<K, uint8_t>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, col_cap, slot_cap, max_w,
                                      max_h, tiled, half_w, st);
    case DARE_F16:
        return launch_r_w<K, __half>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, col_cap, slot_cap, max_w,
                                     max_h, tiled, half_w, st);
    case DARE_BF16:
        return launch_r_w<K, __nv_bfloat16>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, col_cap, slot_cap,
                                            max_w, max_h, tiled, half_w, st);
    case DARE_F32:
        return launch_r_w<K, float>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, col_cap, slot_cap, max_w,
                                    max_h, tiled, half_w, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_r_any(const ResliceJob* jobs_dev, const ResliceJob* one, int n_jobs, int tile_offset, int n_tiles,
                         int uniform, int col_cap, int slot_cap, int max_w, int max_h, bool tiled, int K, int dtype,
                         int half_w, cudaStream_t st) {
    switch (K) {
    case 4: return launch_r_k<4>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, col_cap, slot_cap, max_w, max_h, tiled, dtype, half_w, st);
    case 8: return launch_r_k<8>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, col_cap, slot_cap, max_w, max_h, tiled, dtype, half_w, st);
    case 12: return launch_r_k<12>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, col_cap, slot_cap, max_w, max_h, tiled, dtype, half_w, st);
    case 16: return launch_r_k<16>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, col_cap, slot_cap, max_w, max_h, tiled, dtype, half_w, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_reslice_plain_r(const ResliceJob* jobs_dev, const ResliceJob* one_job, int n_jobs, int max_w,
                                   int max_h, int K, int dtype, int half_weights, cudaStream_t st) {
    if (n_jobs <= 0 || max_w <= 0 || max_h <= 0) return cudaSuccess;
    return launch_r_any(jobs_dev, one_job, n_jobs, 0, 0, 0, 0, 0, max_w, max_h, false, K, dtype, half_weights, st);
}

cudaError_t launch_reslice_tiled_r(const ResliceJob* jobs_dev, const ResliceJob* one_job, int n_jobs,
                                   int tile_offset, int n_tiles, int uniform, int col_cap, int slot_cap, int K,
                                   int dtype, int half_weights, cudaStream_t st) {
    if (n_jobs <= 0 || n_tiles <= 0) return cudaSuccess;
    return launch_r_any(jobs_dev, one_job, n_jobs, tile_offset, n_tiles, uniform, max(col_cap, 1), max(slot_cap, 1),
                        0, 0, true, K, dtype, half_weights, st);
}

cudaError_t read_fallback_tiles_general(unsigned long long* out, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_fallback_tiles_r, sizeof(*out));
    if (e != cudaSuccess || !reset) return e;
    const unsigned long long zero = 0;
    return cudaMemcpyToSymbol(g_fallback_tiles_r, &zero, sizeof(zero));
}

}  // namespace dare
