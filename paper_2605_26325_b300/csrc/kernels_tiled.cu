// Tiled DARE reslice (sm_103a): one CTA per 32 x 16 pixel tile.
//
// For a plane r the orientation weight w_f of Eq. 2 depends only on the
// sample's frame f, so the weighted average of Sec. 2.1 with TENT weights t_c
// regroups exactly per voxel c:
//     out = sum_c t_c A_c / sum_c t_c B_c,   A_c = sum_s w_f(s) I_s,  B_c = sum_s w_f(s)
// A tile therefore (A) reduces each voxel its pixels can touch once to
// (A_c, B_c) in shared memory -- one record read per voxel instead of one per
// (pixel, corner) -- and (B) blends 8 corners per pixel from shared memory.
//
// Support enumeration.  Let d be the axis of the plane normal's largest
// component in voxel space and e1 < e2 the other two.  On the plane
// g_d = alpha + beta1 g_e1 + beta2 g_e2 with |beta| <= 1.  A pixel touches
// voxel column (c1, c2) only if g_e1 in [c1-1, c1+1) and g_e2 in
// [c2-1, c2+1), and then reads levels floor(g_d) and floor(g_d)+1; over that
// square g_d stays within spread = |beta1|+|beta2| of its value at the column,
// which bounds the column's levels.  Columns come from the tile's exact
// fixed-point bounding box, pruned by a conservative test against the tile's
// pixel rectangle.  The plane coefficients come from the host (FP64) as FP32
// with margins far above FP32 rounding, so any error only adds work.  Every
// shared-memory read is range-checked.  A tile whose box does not fit in
// shared memory gathers per pixel instead, with the same result.
#include <cfloat>

#include "dare_internal.h"
#include "device_common.cuh"

namespace dare {
namespace {

using namespace dev;

constexpr int kThreads = 256;
constexpr int kColMax = 1024;
constexpr int kSlotMax = 4096;   // (A, B) float2 slots: 32 KB
constexpr float kMargin = 0.02f; // voxel; > FP32 error of the plane height for |g| < 2^14

template <int D>
struct Axes {
    static constexpr int E1 = D == 0 ? 1 : 0;
    static constexpr int E2 = D == 2 ? 1 : 2;
};

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

// (A_c, B_c) of one voxel: reads only the 16-byte chunks that hold its
// occupied slots (ids first, values after; empty ids sort last).
template <int K, typename VT, typename WT>
__device__ __forceinline__ float2 collapse_voxel(const uint8_t* rec, int64_t vi, const WT* wt) {
    using S = RecShape<K, VT>;
    constexpr int kIdChunks = (2 * K + 15) / 16;
    const uint4* q = reinterpret_cast<const uint4*>(rec + vi * S::kBytes);
    uint4 r[S::kVec];
#pragma unroll
    for (int i = 0; i < kIdChunks; ++i) r[i] = __ldg(q + i);
    int count = 0;
#pragma unroll
    for (int w = 0; w < K / 2; ++w) count += __popc(__vcmpne2(word_of(r, w), 0xFFFFFFFFu)) >> 4;
#pragma unroll
    for (int i = kIdChunks; i < S::kVec; ++i) {
        constexpr int vb = static_cast<int>(sizeof(VT));
        const int first = (16 * i - 2 * K + vb - 1) / vb;  // first slot whose value starts in chunk i
        r[i] = first < count ? __ldg(q + i) : make_uint4(0, 0, 0, 0);
    }
    float A = 0.0f, B = 0.0f;
#pragma unroll
    for (int s = 0; s < K; ++s) {
        if (s < count) {
            const float w = weight_of(wt, static_cast<int>(slot_id<K, VT>(r, s)));
            A = fmaf(w, slot_value<K, VT>(r, s), A);
            B += w;
        }
    }
    return make_float2(A, B);
}

template <int K, typename VT, typename WT>
__device__ __noinline__ void direct_pixel(const ResliceJob& J, int u, int v, float& num, float& den) {
    const PixelCoord pc = pixel_coord(J, u, v);
    if (!pc.any) return;
    const WT* wt = static_cast<const WT*>(J.wtab);
    for (int corner = 0; corner < 8; ++corner) {
        const int dx = corner & 1, dy = (corner >> 1) & 1, dz = corner >> 2;
        const int cx = pc.c0[0] + dx, cy = pc.c0[1] + dy, cz = pc.c0[2] + dz;
        if (cx < 0 || cy < 0 || cz < 0 || cx >= J.dims[0] || cy >= J.dims[1] || cz >= J.dims[2]) continue;
        const float t = (dx ? pc.fr[0] : 1.0f - pc.fr[0]) * (dy ? pc.fr[1] : 1.0f - pc.fr[1]) *
                        (dz ? pc.fr[2] : 1.0f - pc.fr[2]);
        const int64_t vi = cx + static_cast<int64_t>(J.dims[0]) * (cy + static_cast<int64_t>(J.dims[1]) * cz);
        const float2 ab = collapse_voxel<K, VT, WT>(J.rec, vi, wt);
        num = fmaf(t, ab.x, num);
        den = fmaf(t, ab.y, den);
    }
}

__device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t lmax(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ int64_t axis_fix(const ResliceJob& J, int a, int u, int v) {
    return J.g0[a] + static_cast<int64_t>(u) * J.a[a] + static_cast<int64_t>(v) * J.b[a];
}

__device__ __forceinline__ float fix_frac(int64_t G) {
    return static_cast<float>(static_cast<int32_t>(G & (kFixOne - 1))) * (1.0f / static_cast<float>(kFixOne));
}

template <int K, typename VT, typename WT, int D>
__device__ __forceinline__ void tile_body(const ResliceJob& J, int u0, int v0, int u1, int v1, float2* sAB,
                                          int* sCol) {
    constexpr int E1 = Axes<D>::E1, E2 = Axes<D>::E2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WT* wt = static_cast<const WT*>(J.wtab);

    // exact bounding box of the tile's corner pixels in (e1, e2), grown by the TENT support
    int64_t lo1 = INT64_MAX, hi1 = INT64_MIN, lo2 = INT64_MAX, hi2 = INT64_MIN;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int u = (k & 1) ? u1 : u0, v = (k & 2) ? v1 : v0;
        const int64_t f1 = axis_fix(J, E1, u, v) >> kFixBits, f2 = axis_fix(J, E2, u, v) >> kFixBits;
        lo1 = lmin(lo1, f1); hi1 = lmax(hi1, f1);
        lo2 = lmin(lo2, f2); hi2 = lmax(hi2, f2);
    }
    const int b1 = static_cast<int>(lmax(lmin(lo1, J.dims[E1]), 0));
    const int b2 = static_cast<int>(lmax(lmin(lo2, J.dims[E2]), 0));
    const int n1 = static_cast<int>(lmax(0, lmin(hi1 + 1, J.dims[E1] - 1) - b1 + 1));
    const int n2 = static_cast<int>(lmax(0, lmin(hi2 + 1, J.dims[E2] - 1) - b2 + 1));
    const int ncol = n1 * n2;
    const int L = J.levels;
    const bool direct = J.direct || ncol > kColMax || ncol * L > kSlotMax;

    if (!direct) {
        // (A) per column: level range, then one collapse per candidate voxel
        const float inv_n1 = 1.0f / static_cast<float>(max(n1, 1));
        const float sm = J.spread + kMargin;
        const int dd = J.dims[D];
        for (int c = threadIdx.x; c < ncol; c += kThreads) {
            const int k2 = static_cast<int>((static_cast<float>(c) + 0.5f) * inv_n1);
            const int k1 = c - k2 * n1;
            const int c1 = b1 + k1, c2 = b2 + k2;
            const float uc = J.ou + J.m00 * c1 + J.m01 * c2;
            const float vc = J.ov + J.m10 * c1 + J.m11 * c2;
            const bool near = fabsf(uc - fminf(fmaxf(uc, static_cast<float>(u0)), static_cast<float>(u1))) <= J.hu &&
                              fabsf(vc - fminf(fmaxf(vc, static_cast<float>(v0)), static_cast<float>(v1))) <= J.hv;
            const float gd = J.alpha + J.beta1 * c1 + J.beta2 * c2;
            int lo = 0, cnt = 0;
            if (near && fabsf(gd) < 16384.0f) {
                lo = max(static_cast<int>(floorf(gd - sm)), 0);
                const int hi = min(static_cast<int>(floorf(gd + sm)) + 1, dd - 1);
                cnt = max(0, min(hi - lo + 1, L));
            }
            sCol[c] = (lo & 0xFFFF) | (cnt << 16);
            for (int lev = 0; lev < cnt; ++lev) {
                const int cd = lo + lev;
                const int x = D == 0 ? cd : c1;
                const int y = D == 1 ? cd : (E1 == 1 ? c1 : c2);
                const int z = D == 2 ? cd : c2;
                const int64_t vi = x + static_cast<int64_t>(J.dims[0]) * (y + static_cast<int64_t>(J.dims[1]) * z);
                sAB[c * L + lev] = collapse_voxel<K, VT, WT>(J.rec, vi, wt);
            }
        }
        __syncthreads();
    }
    // (B) pixels: a warp walks the 32 pixels of a tile row
    for (int r = warp; r < kTileH; r += kThreads / 32) {
        const int v = v0 + r;
        if (v > v1) break;  // warp-uniform
        const int u = u0 + lane;
        const bool active = u <= u1;
        float num = 0.0f, den = 0.0f;
        if (active) {
            if (direct) {
                direct_pixel<K, VT, WT>(J, u, v, num, den);
            } else {
                const int64_t G1 = axis_fix(J, E1, u, v), G2 = axis_fix(J, E2, u, v), Gd = axis_fix(J, D, u, v);
                const int64_t k1 = (G1 >> kFixBits) - b1, k2 = (G2 >> kFixBits) - b2, fd = Gd >> kFixBits;
                const float p1 = fix_frac(G1), p2 = fix_frac(G2), pd = fix_frac(Gd);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        if (k1 + i < 0 || k1 + i >= n1 || k2 + j < 0 || k2 + j >= n2) continue;
                        const int c = static_cast<int>(k1 + i) + n1 * static_cast<int>(k2 + j);
                        const int info = sCol[c];
                        const int64_t lev = fd - (info & 0xFFFF);
                        const int cnt = info >> 16;
                        const float wc = (i ? p1 : 1.0f - p1) * (j ? p2 : 1.0f - p2);
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            if (lev + k < 0 || lev + k >= cnt) continue;
                            const float2 ab = sAB[c * L + static_cast<int>(lev) + k];
                            const float t = wc * (k ? pd : 1.0f - pd);
                            num = fmaf(t, ab.x, num);
                            den = fmaf(t, ab.y, den);
                        }
                    }
                }
            }
            J.out[static_cast<int64_t>(v) * J.width + u] = den > 0.0f ? num / den : J.unassigned;
        }
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, active && den > 0.0f);
        if (lane == 0) J.mask[static_cast<int64_t>(v) * J.mask_stride + u0 / 32] = bits;
    }
}

template <int K, typename VT, typename WT>
__global__ void __launch_bounds__(kThreads, 4) k_reslice_tiled(const ResliceJob* __restrict__ jobs, int n_jobs,
                                                               int tile_offset,
                                                               const __grid_constant__ ResliceJob one) {
    __shared__ float2 sAB[kSlotMax];
    __shared__ int sCol[kColMax];  // per column: lowest level | (level count << 16)
    const int tile = tile_offset + static_cast<int>(blockIdx.x);
    const ResliceJob& J = jobs ? jobs[find_job(jobs, n_jobs, tile)] : one;
    const int lt = tile - J.tile_base;
    const int ty = lt / J.tiles_x, tx = lt - ty * J.tiles_x;
    const int u0 = tx * kTileW, v0 = ty * kTileH;
    const int u1 = min(u0 + kTileW, J.width) - 1, v1 = min(v0 + kTileH, J.height) - 1;
    switch (J.d) {
    case 0: tile_body<K, VT, WT, 0>(J, u0, v0, u1, v1, sAB, sCol); break;
    case 1: tile_body<K, VT, WT, 1>(J, u0, v0, u1, v1, sAB, sCol); break;
    default: tile_body<K, VT, WT, 2>(J, u0, v0, u1, v1, sAB, sCol); break;
    }
}

template <int K, typename VT, typename WT>
cudaError_t tiled_launch(const ResliceJob* jobs_dev, const ResliceJob* one, int n_jobs, int tile_offset,
                         int n_tiles, cudaStream_t st) {
    ResliceJob dummy{};
    k_reslice_tiled<K, VT, WT><<<n_tiles, kThreads, 0, st>>>(one ? nullptr : jobs_dev, n_jobs, tile_offset,
                                                            one ? *one : dummy);
    return cudaPeekAtLastError();
}

template <int K, typename VT>
cudaError_t tiled_launch_w(const ResliceJob* jobs_dev, const ResliceJob* one, int n_jobs, int tile_offset,
                           int n_tiles, int half_w, cudaStream_t st) {
    return half_w ? tiled_launch<K, VT, __half>(jobs_dev, one, n_jobs, tile_offset, n_tiles, st)
                  : tiled_launch<K, VT, float>(jobs_dev, one, n_jobs, tile_offset, n_tiles, st);
}

template <int K>
cudaError_t tiled_launch_k(const ResliceJob* jobs_dev, const ResliceJob* one, int n_jobs, int tile_offset,
                           int n_tiles, int dtype, int half_w, cudaStream_t st) {
    switch (dtype) {
    case DARE_U8: return tiled_launch_w<K, uint8_t>(jobs_dev, one, n_jobs, tile_offset, n_tiles, half_w, st);
    case DARE_F16: return tiled_launch_w<K, __half>(jobs_dev, one, n_jobs, tile_offset, n_tiles, half_w, st);
    case DARE_BF16: return tiled_launch_w<K, __nv_bfloat16>(jobs_dev, one, n_jobs, tile_offset, n_tiles, half_w, st);
    case DARE_F32: return tiled_launch_w<K, float>(jobs_dev, one, n_jobs, tile_offset, n_tiles, half_w, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_reslice_tiled(const ResliceJob* jobs_dev, const ResliceJob* one_job, int n_jobs, int tile_offset,
                                 int n_tiles, int K, int dtype, int half_weights, cudaStream_t st) {
    if (n_jobs <= 0 || n_tiles <= 0) return cudaSuccess;
    switch (K) {
    case 4: return tiled_launch_k<4>(jobs_dev, one_job, n_jobs, tile_offset, n_tiles, dtype, half_weights, st);
    case 8: return tiled_launch_k<8>(jobs_dev, one_job, n_jobs, tile_offset, n_tiles, dtype, half_weights, st);
    case 12: return tiled_launch_k<12>(jobs_dev, one_job, n_jobs, tile_offset, n_tiles, dtype, half_weights, st);
    case 16: return tiled_launch_k<16>(jobs_dev, one_job, n_jobs, tile_offset, n_tiles, dtype, half_weights, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dare
