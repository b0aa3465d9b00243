// Tiled DARE reslice (sm_103a): one CTA per 32 x 16 pixel tile.
//
// For a plane r the orientation weight w_f of Eq. 2 depends only on the
// sample's frame f, so the weighted average of Sec. 2.1 with TENT weights t_c
// regroups exactly per voxel c:
//     out = sum_c t_c A_c / sum_c t_c B_c,   A_c = sum_s w_f(s) I_s,  B_c = sum_s w_f(s)
// A tile therefore (1) enumerates the voxels its pixels can touch, (2) reduces
// each of them once to (A_c, B_c) in shared memory -- one record read per
// voxel instead of one per (pixel, corner) -- and (3) blends 8 corners per
// pixel from shared memory.
//
// Support enumeration.  Let d be the axis of the plane normal's largest
// component in voxel space and e1 < e2 the other two.  The plane is the
// graph g_d = alpha + beta1 g_e1 + beta2 g_e2 with |beta| <= 1.  A pixel
// touches voxel column (c1, c2) only if g_e1 in [c1-1, c1+1) and
// g_e2 in [c2-1, c2+1), and then reads c_d in {floor(g_d), floor(g_d)+1};
// over that square g_d moves by at most |beta1|+|beta2| from its centre value,
// which bounds the column's levels.  The column box is the tile's bounding
// box in (e1, e2), pruned by a conservative test against the tile's
// parallelogram.  Any over-approximation only costs work; every corner a
// pixel reads lies inside (checked before every shared-memory read).
// Tiles whose box does not fit in shared memory take the direct path (each
// pixel gathers its 8 records), which gives the same result.
#include <cfloat>

#include "dare_internal.h"
#include "device_common.cuh"

namespace dare {
namespace {

using namespace dev;

constexpr int kThreads = 256;
constexpr int kColMax = 2048;
constexpr int kSlotMax = 6144;  // (A, B) float2 slots: 48 KB

struct TileGeom {
    int e1, e2, d;
    int b1, b2;          // column box origin
    int n1, n2;          // column box size
    int levels;          // level slots per column
    int direct;          // 1: tile takes the direct path
    double alpha, beta1, beta2, spread;
    double m00, m01, m10, m11;  // (g_e1, g_e2) -> (u, v), per voxel
    double ou, ov;              // (u, v) of (g_e1, g_e2) = 0
    double hu, hv;              // |du|, |dv| for a unit move per axis
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

__device__ void tile_geometry(const ResliceJob& J, int u0, int v0, int u1, int v1, TileGeom& T) {
    const double s = 1.0 / static_cast<double>(kFixOne);
    double A[3], B[3], G0[3];
    for (int a = 0; a < 3; ++a) {
        A[a] = static_cast<double>(J.a[a]) * s;
        B[a] = static_cast<double>(J.b[a]) * s;
        G0[a] = static_cast<double>(J.g0[a]) * s;
    }
    const double n[3] = {A[1] * B[2] - A[2] * B[1], A[2] * B[0] - A[0] * B[2], A[0] * B[1] - A[1] * B[0]};
    int d = 0;
    if (fabs(n[1]) > fabs(n[d])) d = 1;
    if (fabs(n[2]) > fabs(n[d])) d = 2;
    const int e1 = d == 0 ? 1 : 0;
    const int e2 = d == 2 ? 1 : 2;
    T.d = d;
    T.e1 = e1;
    T.e2 = e2;
    T.direct = 0;
    if (n[d] == 0.0) {  // degenerate plane: let every pixel gather directly
        T.direct = 1;
        return;
    }
    T.beta1 = -n[e1] / n[d];
    T.beta2 = -n[e2] / n[d];
    T.alpha = G0[d] - T.beta1 * G0[e1] - T.beta2 * G0[e2];
    T.spread = fabs(T.beta1) + fabs(T.beta2);
    // bounding box of the tile's corner pixels in (e1, e2); affine => extremes at corners
    double lo1 = 1e300, hi1 = -1e300, lo2 = 1e300, hi2 = -1e300;
    for (int k = 0; k < 4; ++k) {
        const double u = (k & 1) ? u1 : u0, v = (k & 2) ? v1 : v0;
        const double g1 = G0[e1] + u * A[e1] + v * B[e1];
        const double g2 = G0[e2] + u * A[e2] + v * B[e2];
        lo1 = fmin(lo1, g1); hi1 = fmax(hi1, g1);
        lo2 = fmin(lo2, g2); hi2 = fmax(hi2, g2);
    }
    const double big = 1e9;
    lo1 = fmax(fmin(lo1, big), -big); hi1 = fmax(fmin(hi1, big), -big);
    lo2 = fmax(fmin(lo2, big), -big); hi2 = fmax(fmin(hi2, big), -big);
    const int b1 = max(0, static_cast<int>(floor(lo1)));
    const int t1 = min(J.dims[e1] - 1, static_cast<int>(floor(hi1)) + 1);
    const int b2 = max(0, static_cast<int>(floor(lo2)));
    const int t2 = min(J.dims[e2] - 1, static_cast<int>(floor(hi2)) + 1);
    T.b1 = b1;
    T.b2 = b2;
    T.n1 = max(0, t1 - b1 + 1);
    T.n2 = max(0, t2 - b2 + 1);
    // levels floor(gd - spread) .. floor(gd + spread) + 1: at most floor(2 spread) + 3
    T.levels = static_cast<int>(floor(2.0 * T.spread + 2e-6)) + 3;
    const long long ncol = static_cast<long long>(T.n1) * T.n2;
    if (ncol > kColMax || ncol * T.levels > kSlotMax) T.direct = 1;
    // inverse of the 2x2 map (u, v) -> (g_e1, g_e2)
    const double det = A[e1] * B[e2] - A[e2] * B[e1];
    if (det == 0.0) {
        T.direct = 1;
        return;
    }
    T.m00 = B[e2] / det;
    T.m01 = -B[e1] / det;
    T.m10 = -A[e2] / det;
    T.m11 = A[e1] / det;
    T.ou = -(T.m00 * G0[e1] + T.m01 * G0[e2]);
    T.ov = -(T.m10 * G0[e1] + T.m11 * G0[e2]);
    T.hu = fabs(T.m00) + fabs(T.m01) + 1e-6;
    T.hv = fabs(T.m10) + fabs(T.m11) + 1e-6;
}

template <int K, typename VT, typename WT>
__device__ __forceinline__ float2 collapse_voxel(const ResliceJob& J, int64_t vi) {
    uint4 r[RecShape<K, VT>::kVec];
    load_record<K, VT>(J.rec + vi * RecShape<K, VT>::kBytes, r);
    const WT* wt = static_cast<const WT*>(J.wtab);
    float A = 0.0f, B = 0.0f;
#pragma unroll
    for (int s = 0; s < K; ++s) {
        const uint32_t id = slot_id<K, VT>(r, s);
        if (id == DARE_EMPTY_FRAME) break;
        const float w = weight_of(wt, static_cast<int>(id));
        A = fmaf(w, slot_value<K, VT>(r, s), A);
        B += w;
    }
    return make_float2(A, B);
}

template <int K, typename VT, typename WT>
__device__ __forceinline__ void direct_pixel(const ResliceJob& J, int u, int v, float& num, float& den) {
    const PixelCoord pc = pixel_coord(J, u, v);
    if (!pc.any) return;
#pragma unroll 1
    for (int corner = 0; corner < 8; ++corner) {
        const int dx = corner & 1, dy = (corner >> 1) & 1, dz = corner >> 2;
        const int cx = pc.c0[0] + dx, cy = pc.c0[1] + dy, cz = pc.c0[2] + dz;
        if (cx < 0 || cy < 0 || cz < 0 || cx >= J.dims[0] || cy >= J.dims[1] || cz >= J.dims[2]) continue;
        const float t = (dx ? pc.fr[0] : 1.0f - pc.fr[0]) * (dy ? pc.fr[1] : 1.0f - pc.fr[1]) *
                        (dz ? pc.fr[2] : 1.0f - pc.fr[2]);
        const int64_t vi = cx + static_cast<int64_t>(J.dims[0]) * (cy + static_cast<int64_t>(J.dims[1]) * cz);
        const float2 ab = collapse_voxel<K, VT, WT>(J, vi);
        num = fmaf(t, ab.x, num);
        den = fmaf(t, ab.y, den);
    }
}

template <int K, typename VT, typename WT>
__global__ void __launch_bounds__(kThreads) k_reslice_tiled(const ResliceJob* __restrict__ jobs, int n_jobs,
                                                            int tile_offset, const __grid_constant__ ResliceJob one) {
    extern __shared__ float2 sAB[];
    __shared__ int sCol[kColMax];  // per column: lowest level | (level count << 16)
    __shared__ TileGeom T;
    __shared__ int sJob;

    const int tile = tile_offset + static_cast<int>(blockIdx.x);
    if (threadIdx.x == 0) sJob = jobs ? find_job(jobs, n_jobs, tile) : 0;
    __syncthreads();
    const ResliceJob& J = jobs ? jobs[sJob] : one;
    const int lt = tile - J.tile_base;
    const int tx = lt % J.tiles_x, ty = lt / J.tiles_x;
    const int u0 = tx * kTileW, v0 = ty * kTileH;
    const int u1 = min(u0 + kTileW, J.width) - 1, v1 = min(v0 + kTileH, J.height) - 1;
    if (threadIdx.x == 0) tile_geometry(J, u0, v0, u1, v1, T);
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool direct = T.direct != 0;
    const int n1 = T.n1, ncol = T.n1 * T.n2, L = T.levels;
    const int e1 = T.e1, e2 = T.e2, d = T.d;

    if (!direct) {
        // (1) per-column level range, pruned against the tile parallelogram
        for (int c = threadIdx.x; c < ncol; c += kThreads) {
            const int c1 = T.b1 + c % n1, c2 = T.b2 + c / n1;
            const double uc = T.ou + T.m00 * c1 + T.m01 * c2;
            const double vc = T.ov + T.m10 * c1 + T.m11 * c2;
            const bool near = fabs(uc - fmin(fmax(uc, double(u0)), double(u1))) <= T.hu &&
                              fabs(vc - fmin(fmax(vc, double(v0)), double(v1))) <= T.hv;
            int lo = 0, cnt = 0;
            if (near) {
                const double gd = T.alpha + T.beta1 * c1 + T.beta2 * c2;
                lo = static_cast<int>(floor(gd - T.spread - 1e-6));
                int hi = static_cast<int>(floor(gd + T.spread + 1e-6)) + 1;
                lo = max(lo, 0);
                hi = min(hi, J.dims[d] - 1);
                cnt = max(0, min(hi - lo + 1, L));
            }
            sCol[c] = (lo & 0xFFFF) | (cnt << 16);
        }
        __syncthreads();
        // (2) one record read per candidate voxel -> (A_c, B_c)
        const int nslot = ncol * L;
        for (int sidx = threadIdx.x; sidx < nslot; sidx += kThreads) {
            int c, lev;
            if (d == 0) {  // levels run along x, the contiguous axis
                c = sidx / L;
                lev = sidx % L;
            } else {       // columns run along x first
                c = sidx % ncol;
                lev = sidx / ncol;
            }
            const int info = sCol[c];
            if (lev >= (info >> 16)) continue;
            int cc[3];
            cc[e1] = T.b1 + c % n1;
            cc[e2] = T.b2 + c / n1;
            cc[d] = (info & 0xFFFF) + lev;
            const int64_t vi = cc[0] + static_cast<int64_t>(J.dims[0]) * (cc[1] + static_cast<int64_t>(J.dims[1]) * cc[2]);
            sAB[c * L + lev] = collapse_voxel<K, VT, WT>(J, vi);
        }
        __syncthreads();
    }
    // (3) pixels: a warp walks the 32 pixels of a tile row
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
                const PixelCoord pc = pixel_coord(J, u, v);
                if (pc.any) {
#pragma unroll
                    for (int corner = 0; corner < 8; ++corner) {
                        int cc[3] = {pc.c0[0] + (corner & 1), pc.c0[1] + ((corner >> 1) & 1), pc.c0[2] + (corner >> 2)};
                        if (cc[0] < 0 || cc[1] < 0 || cc[2] < 0 || cc[0] >= J.dims[0] || cc[1] >= J.dims[1] ||
                            cc[2] >= J.dims[2])
                            continue;
                        const int k1 = cc[e1] - T.b1, k2 = cc[e2] - T.b2;
                        if (static_cast<unsigned>(k1) >= static_cast<unsigned>(n1) ||
                            static_cast<unsigned>(k2) >= static_cast<unsigned>(T.n2))
                            continue;
                        const int c = k1 + n1 * k2;
                        const int info = sCol[c];
                        const int lev = cc[d] - (info & 0xFFFF);
                        if (static_cast<unsigned>(lev) >= static_cast<unsigned>(info >> 16)) continue;
                        const float t = ((corner & 1) ? pc.fr[0] : 1.0f - pc.fr[0]) *
                                        ((corner & 2) ? pc.fr[1] : 1.0f - pc.fr[1]) *
                                        ((corner & 4) ? pc.fr[2] : 1.0f - pc.fr[2]);
                        const float2 ab = sAB[c * L + lev];
                        num = fmaf(t, ab.x, num);
                        den = fmaf(t, ab.y, den);
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
cudaError_t tiled_launch(const ResliceJob* jobs_dev, const ResliceJob* one, int n_jobs, int tile_offset,
                         int n_tiles, cudaStream_t st) {
    static unsigned long long configured = 0;  // one bit per device ordinal
    const int smem = kSlotMax * static_cast<int>(sizeof(float2));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(k_reslice_tiled<K, VT, WT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    ResliceJob dummy{};
    k_reslice_tiled<K, VT, WT><<<n_tiles, kThreads, smem, st>>>(one ? nullptr : jobs_dev, n_jobs, tile_offset,
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
