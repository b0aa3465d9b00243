// Tiled DARE reslice (sm_103a): one CTA per 32 x TH pixel tile (TH = 8, 16, 32 or
// 64, chosen per plane on the host so that the tile's voxel-column box fits
// shared memory).
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
// shared memory gathers per pixel instead, with the same result, and is counted.
//
// Two launch forms: a grid of one CTA per tile, and a persistent grid of one
// CTA per resident slot that takes tiles from a work queue in device memory
// (its tile count is read on the device, so a captured graph stays valid when
// new poses change the planes' tile heights).
#include <algorithm>
#include <cfloat>

#include "dare_internal.h"
#include "device_common.cuh"

namespace dare {
namespace {

using namespace dev;

constexpr int kThreads = 256;
constexpr int kColMax = kTiledColMax;
constexpr int kSlotMax = kTiledSlotMax;   // (A, B) float2 slots: 32 KB
#ifndef DARE_TILED_MIN_BLOCKS
#define DARE_TILED_MIN_BLOCKS 5  // 48 registers, a few spills: faster than 4 CTAs without spills
#endif
constexpr float kMargin = 0.02f; // voxel; > FP32 error of the plane height for |g| < 2^14

// tiles that gathered per pixel because their column box did not fit shared memory
__device__ unsigned long long g_fallback_tiles;

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

// Returned by value: sums passed by reference would live in the caller's
// stack frame, and the pixel loop would store them to local memory every row.
template <int K, typename VT, typename WT>
__device__ __noinline__ float2 direct_pixel(const ResliceJob& J, int u, int v) {
    float num = 0.0f, den = 0.0f;
    const PixelCoord pc = pixel_coord(J, u, v);
    if (!pc.any) return make_float2(num, den);
    const WT* wt = static_cast<const WT*>(J.wtab);
    for (int corner = 0; corner < 8; ++corner) {
        const int dx = corner & 1, dy = (corner >> 1) & 1, dz = corner >> 2;
        const int cx = pc.c0[0] + dx, cy = pc.c0[1] + dy, cz = pc.c0[2] + dz;
        if (cx < 0 || cy < 0 || cz < 0 || cx >= J.dims[0] || cy >= J.dims[1] || cz >= J.dims[2]) continue;
        const float t = (dx ? pc.fr[0] : 1.0f - pc.fr[0]) * (dy ? pc.fr[1] : 1.0f - pc.fr[1]) *
                        (dz ? pc.fr[2] : 1.0f - pc.fr[2]);
        const int64_t vi = cx + static_cast<int64_t>(J.dims[0]) * (cy + static_cast<int64_t>(J.dims[1]) * cz);
        const float2 ab = collapse_voxel<K, VT, WT, 1>(J.rec, vi, wt);
        num = fmaf(t, ab.x, num);
        den = fmaf(t, ab.y, den);
    }
    return make_float2(num, den);
}

// (r mod 2^20) / 2^20, exactly: the 20-bit fraction placed in the mantissa of
// a float in [1, 2), minus one (integer operations instead of a conversion)
__device__ __forceinline__ float frac20(int r) {
    static_assert(kFixBits == 20, "20-bit fixed point");
    return __int_as_float(0x3F800000 | ((r << 3) & 0x007FFFF8)) - 1.0f;
}

__device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t lmax(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ int64_t axis_fix(const ResliceJob& J, int a, int u, int v) {
    return J.g0[a] + static_cast<int64_t>(u) * J.a[a] + static_cast<int64_t>(v) * J.b[a];
}

// Per-tile set-up, computed by one thread and shared through shared memory.
struct TileSetup {
    int job;
    int u0, v0, u1, v1;      // pixel range of the tile
    int b1, b2, n1, n2;      // column box
    int direct;
    int empty;               // no pixel of the tile reaches the grid
    int R1, R2, Rd;          // 20-bit remainders of the tile origin's coordinates
    int O1, O2, Od;          // integer parts, relative to the box (clamped far outside when irrelevant)
};

// Per-tile set-up by the 32 lanes of warp 0: lanes 0-11 take the fixed-point
// coordinate of one (corner, axis) and lanes 12-14 the tile origin's on one
// axis, in parallel; lanes 0-2 reduce their axis over the four corners; lane 0
// writes the result.
template <int D>
__device__ void tile_setup(const ResliceJob& J, int u0, int v0, int u1, int v1, TileSetup& T) {
    constexpr int E1 = Axes<D>::E1, E2 = Axes<D>::E2;
    const int lane = threadIdx.x & 31;
    const int ai = lane < 12 ? lane % 3 : lane - 12;  // 0: e1, 1: e2, 2: d
    const int ax = ai == 0 ? E1 : (ai == 1 ? E2 : D);
    const int k = lane / 3;
    const int u = lane < 12 ? ((k & 1) ? u1 : u0) : u0, v = lane < 12 ? ((k & 2) ? v1 : v0) : v0;
    const int64_t G = lane < 15 ? axis_fix(J, ax < 3 ? ax : 0, u, v) : 0;
    const int64_t f = G >> kFixBits;
    const int64_t f3 = __shfl_down_sync(0xFFFFFFFFu, f, 3), f6 = __shfl_down_sync(0xFFFFFFFFu, f, 6);
    const int64_t f9 = __shfl_down_sync(0xFFFFFFFFu, f, 9);
    const int64_t lo = lmin(lmin(f, f3), lmin(f6, f9)), hi = lmax(lmax(f, f3), lmax(f6, f9));  // lanes 0-2
    const int64_t lo1 = __shfl_sync(0xFFFFFFFFu, lo, 0), hi1 = __shfl_sync(0xFFFFFFFFu, hi, 0);
    const int64_t lo2 = __shfl_sync(0xFFFFFFFFu, lo, 1), hi2 = __shfl_sync(0xFFFFFFFFu, hi, 1);
    const int64_t lod = __shfl_sync(0xFFFFFFFFu, lo, 2), hid = __shfl_sync(0xFFFFFFFFu, hi, 2);
    const int64_t G1 = __shfl_sync(0xFFFFFFFFu, G, 12), G2 = __shfl_sync(0xFFFFFFFFu, G, 13);
    const int64_t Gd = __shfl_sync(0xFFFFFFFFu, G, 14);
    if (lane != 0) return;
    // a pixel reads floors f .. f + 1 on each axis; when on some axis that
    // range misses the grid for every pixel of the tile, the tile is unassigned
    T.empty = hi1 + 1 < 0 || lo1 > J.dims[E1] - 1 || hi2 + 1 < 0 || lo2 > J.dims[E2] - 1 || hid + 1 < 0 ||
              lod > J.dims[D] - 1;
    // The box is not clipped to the grid: by convexity every pixel's column
    // (k1, k2) and its +1 neighbours lie inside it, so the pixel pass needs no
    // bounds tests; columns outside the grid hold zeros.
    const int64_t n1 = hi1 + 2 - lo1, n2 = hi2 + 2 - lo2;
    T.direct = !T.empty && (J.direct || n1 > kColMax || n2 > kColMax || n1 * n2 > kColMax || n1 * n2 * J.levels > kSlotMax ||
               lo1 < -(1 << 30) || lo2 < -(1 << 30) || hi1 > (1 << 30) || hi2 > (1 << 30));
    T.b1 = static_cast<int>(lmax(lmin(lo1, 1 << 30), -(1 << 30)));
    T.b2 = static_cast<int>(lmax(lmin(lo2, 1 << 30), -(1 << 30)));
    T.n1 = T.direct || T.empty ? 0 : static_cast<int>(n1);
    T.n2 = T.direct || T.empty ? 0 : static_cast<int>(n2);
    T.R1 = static_cast<int>(G1 & (kFixOne - 1));
    T.R2 = static_cast<int>(G2 & (kFixOne - 1));
    T.Rd = static_cast<int>(Gd & (kFixOne - 1));
    T.O1 = static_cast<int>(lmax(lmin((G1 >> kFixBits) - T.b1, 1 << 24), -(1 << 24)));
    T.O2 = static_cast<int>(lmax(lmin((G2 >> kFixBits) - T.b2, 1 << 24), -(1 << 24)));
    T.Od = static_cast<int>(lmax(lmin(Gd >> kFixBits, 1 << 24), -(1 << 24)));
}

template <int K, typename VT, typename WT, int D>
__device__ __forceinline__ void tile_body(const ResliceJob& J, const TileSetup& T, int u0, int v0, int u1, int v1,
                                          float2* sAB, int* sCol) {
    constexpr int E1 = Axes<D>::E1, E2 = Axes<D>::E2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WT* wt = static_cast<const WT*>(J.wtab);
    const int b1 = T.b1, b2 = T.b2, n1 = T.n1, n2 = T.n2, ncol = n1 * n2, L = J.levels;
    const bool direct = T.direct != 0, empty = T.empty != 0;

    if (!direct && !empty) {
        // (A) per column: its lowest level, then L slots (A_c, B_c) of levels
        // lo .. lo + L - 1; slots outside the grid, past the column's level
        // range or of columns no pixel of the tile reaches hold zeros
        const float inv_n1 = 1.0f / static_cast<float>(n1);
        const float sm = J.spread + kMargin;
        const int dd = J.dims[D], d1 = J.dims[E1], d2 = J.dims[E2];
        const float ou = J.ou, ov = J.ov, m00 = J.m00, m01 = J.m01, m10 = J.m10, m11 = J.m11, hu = J.hu, hv = J.hv;
        const float alpha = J.alpha, beta1 = J.beta1, beta2 = J.beta2;
        const float fu0 = static_cast<float>(u0), fu1 = static_cast<float>(u1);
        const float fv0 = static_cast<float>(v0), fv1 = static_cast<float>(v1);
        const uint8_t* const rec = J.rec;
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
                lo = static_cast<int>(floorf(gd - sm));
                top = min(static_cast<int>(floorf(gd + sm)) + 1, dd - 1);
            }
            sCol[c] = lo;
            const int64_t base = c1 * st1 + c2 * st2;
            for (int lev = 0; lev < L; ++lev) {
                const int g = lo + lev;
                sAB[c * L + lev] = (g >= 0 && g <= top) ? collapse_voxel<K, VT, WT>(rec, base + g * std_, wt)
                                                        : make_float2(0.0f, 0.0f);
            }
        }
        __syncthreads();
    }
    // (B) pixels: a warp walks the 32 pixels of a tile row; int32 steps from the tile origin.
    // Everything the loop reads besides the slots sits in registers: the output
    // stores go through generic pointers, which could otherwise alias the
    // shared-memory copies and force reloads.
    float* const out = J.out;
    uint32_t* const mask = J.mask;
    const int64_t width = J.width, mstride = J.mask_stride;
    const float unassigned = J.unassigned;
    const int u = u0 + lane;
    const bool active = u <= u1;
    const int rows = v1 - v0 + 1;
    if (direct || empty) {
        for (int r = warp; r < rows; r += kThreads / 32) {
            const int v = v0 + r;
            float num = 0.0f, den = 0.0f;
            if (active) {
                if (direct) {
                    const float2 nd = direct_pixel<K, VT, WT>(J, u, v);
                    num = nd.x;
                    den = nd.y;
                }
                out[v * width + u] = den > 0.0f ? num / den : unassigned;
            }
            const unsigned bits = __ballot_sync(0xFFFFFFFFu, active && den > 0.0f);
            if (lane == 0) mask[v * mstride + u0 / 32] = bits;
        }
        return;
    }
    const int A1 = static_cast<int>(J.a[E1]), B1 = static_cast<int>(J.b[E1]);
    const int A2 = static_cast<int>(J.a[E2]), B2 = static_cast<int>(J.b[E2]);
    const int Ad = static_cast<int>(J.a[D]), Bd = static_cast<int>(J.b[D]);
    const int R1 = T.R1 + lane * A1, R2 = T.R2 + lane * A2, Rd = T.Rd + lane * Ad;
    const int O1 = T.O1, O2 = T.O2, Od = T.Od;
    for (int r = warp; r < rows; r += kThreads / 32) {
        const int v = v0 + r;
        float num = 0.0f, den = 0.0f;
        if (active) {
            const int r1 = R1 + r * B1, r2 = R2 + r * B2, rd = Rd + r * Bd;
            // k1 in [0, n1 - 2], k2 in [0, n2 - 2] by construction of the box
            const int c00 = (r1 >> kFixBits) + O1 + n1 * ((r2 >> kFixBits) + O2);
            const int fd = (rd >> kFixBits) + Od;
            const float p1 = frac20(r1), p2 = frac20(r2), pd = frac20(rd);
            // TENT weights are separable: (A, B) pairs mixed along the depth
            // axis, then e1, then e2, with packed pair arithmetic (1 - p is
            // exact for a 20-bit fraction)
            const float2 wd = make_float2(pd, pd), wd0 = make_float2(1.0f - pd, 1.0f - pd);
            float2 q[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                float2 col[2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    // Levels fd, fd + 1 lie in the column's range wherever the
                    // column's weight is not zero.  The clamp keeps every read
                    // among the column's own (written, finite) slots: a pixel
                    // also reads its zero-weight neighbours, and 0 x NaN from
                    // stale shared memory would not be zero.
                    const int c = c00 + i + n1 * j;
                    const int lev = min(max(fd - sCol[c], 0), L - 2);
                    col[i] = f2_mix(sAB[c * L + lev], sAB[c * L + lev + 1], wd0, wd);
                }
                q[j] = f2_mix(col[0], col[1], make_float2(1.0f - p1, 1.0f - p1), make_float2(p1, p1));
            }
            const float2 nd = f2_mix(q[0], q[1], make_float2(1.0f - p2, 1.0f - p2), make_float2(p2, p2));
            num = nd.x;
            den = nd.y;
            // The fast division (2 ulp, far below the path's tolerance) holds
            // for den in [2^-126, 2^126]; tiny weights (thresholds opened
            // wide) can leave den below that, where the IEEE division runs.
            out[v * width + u] = den > 0.0f ? (den >= 0x1p-100f ? __fdividef(num, den) : num / den) : unassigned;
        }
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, active && den > 0.0f);
        if (lane == 0) mask[v * mstride + u0 / 32] = bits;
    }
}

// Warp 0: copy the tile's job into shared memory (one coalesced pass), then
// set the tile up (all 32 lanes); lt is the tile's index within its job.
__device__ __forceinline__ void tile_start(const ResliceJob* src, int job, int lt, ResliceJob& sJob, TileSetup& T) {
    static_assert(sizeof(ResliceJob) % 4 == 0, "job copied as 32-bit words");
    const uint32_t* s32 = reinterpret_cast<const uint32_t*>(src);
    uint32_t* d32 = reinterpret_cast<uint32_t*>(&sJob);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(ResliceJob) / 4); i += 32) d32[i] = s32[i];
    __syncwarp();
    const ResliceJob& J0 = sJob;
    const int th = J0.tile_h;
    const int ty = lt / J0.tiles_x, tx = lt - ty * J0.tiles_x;
    const int u0 = tx * kTileW, v0 = ty * th;
    const int u1 = min(u0 + kTileW, J0.width) - 1, v1 = min(v0 + th, J0.height) - 1;
    if (threadIdx.x == 0) {
        T.job = job;
        T.u0 = u0;
        T.v0 = v0;
        T.u1 = u1;
        T.v1 = v1;
    }
    const int d = J0.d;  // warp-uniform
    if (d == 0) tile_setup<0>(J0, u0, v0, u1, v1, T);
    else if (d == 1) tile_setup<1>(J0, u0, v0, u1, v1, T);
    else tile_setup<2>(J0, u0, v0, u1, v1, T);
    if (threadIdx.x == 0 && T.direct && !J0.direct) atomicAdd(&g_fallback_tiles, 1ull);
}

template <int K, typename VT, typename WT>
__device__ __forceinline__ void tile_run(const ResliceJob& J, const TileSetup& T, float2* sAB, int* sCol) {
    switch (J.d) {
    case 0: tile_body<K, VT, WT, 0>(J, T, T.u0, T.v0, T.u1, T.v1, sAB, sCol); break;
    case 1: tile_body<K, VT, WT, 1>(J, T, T.u0, T.v0, T.u1, T.v1, sAB, sCol); break;
    default: tile_body<K, VT, WT, 2>(J, T, T.u0, T.v0, T.u1, T.v1, sAB, sCol); break;
    }
}

// One CTA per tile.  With `uniform` every job has `n_tiles` tiles and the job
// is blockIdx.y; otherwise blockIdx.x runs over all tiles of the launch and
// the first warp finds the job by binary search over tile_base.
template <int K, typename VT, typename WT>
__global__ void __launch_bounds__(kThreads, DARE_TILED_MIN_BLOCKS) k_reslice_tiled(const ResliceJob* __restrict__ jobs,
                                                                                   int n_jobs, int tile_offset,
                                                                                   int uniform,
                                                                                   const __grid_constant__ ResliceJob one) {
    __shared__ float2 sAB[kSlotMax];
    __shared__ int sCol[kColMax];  // per column: its lowest level (slot 0)
    __shared__ TileSetup T;
    __shared__ ResliceJob sJob;  // the tile's job: one coalesced copy, then shared-memory reads
    if (threadIdx.x < 32) {
        int job = 0, lt = static_cast<int>(blockIdx.x);
        if (jobs && uniform) {
            job = static_cast<int>(blockIdx.y);
        } else if (jobs) {
            const int tile = tile_offset + static_cast<int>(blockIdx.x);
            job = find_job(jobs, n_jobs, tile);
            lt = tile - __ldg(&jobs[job].tile_base);
        }
        tile_start(jobs ? jobs + job : &one, job, lt, sJob, T);
    }
    __syncthreads();
    // launched with programmatic serialization after the weight-table kernel: its
    // table is complete and visible from here (no effect on an ordinary launch)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    tile_run<K, VT, WT>(sJob, T, sAB, sCol);
}

// Persistent form: CTA b first takes tile b, then tiles gridDim.x + k for the
// values k of an atomic counter (taken while the current tile runs), until
// the queue's total is reached.  The queue is written by the host with the
// job descriptors before every launch, so `next` starts at 0.
template <int K, typename VT, typename WT>
__global__ void __launch_bounds__(kThreads, DARE_TILED_MIN_BLOCKS)
    k_reslice_tiled_persistent(const ResliceJob* __restrict__ jobs, int n_jobs, TileQueue* __restrict__ queue) {
    __shared__ float2 sAB[kSlotMax];
    __shared__ int sCol[kColMax];
    __shared__ TileSetup T;
    __shared__ ResliceJob sJob;
    __shared__ int sNext;
    const int total = *reinterpret_cast<volatile int32_t*>(&queue->total);
    int tile = static_cast<int>(blockIdx.x);
    while (tile < total) {  // CTA-uniform
        if (threadIdx.x < 32) {
            int next = 0;
            if (threadIdx.x == 0) next = atomicAdd(&queue->next, 1) + static_cast<int>(gridDim.x);
            const int job = find_job(jobs, n_jobs, tile);
            tile_start(jobs + job, job, tile - __ldg(&jobs[job].tile_base), sJob, T);
            if (threadIdx.x == 0) sNext = next;
        }
        __syncthreads();
        tile_run<K, VT, WT>(sJob, T, sAB, sCol);
        tile = sNext;
        __syncthreads();  // shared memory is free for the next tile
    }
}

// Resident CTAs per SM of a kernel (queried once per kernel and device) times the SM count.
template <typename F>
int persistent_grid(F kernel) {
    static int grid[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!grid[dev]) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        grid[dev] = std::max(per_sm, 1) * std::max(sms, 1);
    }
    return grid[dev];
}

// n_tiles: tiles of the whole launch, or per job when `uniform`; queue: persistent form.
template <int K, typename VT, typename WT>
cudaError_t tiled_launch(const ResliceJob* jobs_dev, const ResliceJob* one, int n_jobs, int tile_offset,
                         int n_tiles, int uniform, TileQueue* queue, int pdl, cudaStream_t st) {
    if (queue) {
        const int grid = persistent_grid(k_reslice_tiled_persistent<K, VT, WT>);
        if (grid <= 0) return cudaErrorInvalidValue;
        k_reslice_tiled_persistent<K, VT, WT><<<grid, kThreads, 0, st>>>(jobs_dev, n_jobs, queue);
        return cudaPeekAtLastError();
    }
    ResliceJob dummy{};
    const dim3 grid(n_tiles, (one || !uniform) ? 1 : n_jobs);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_reslice_tiled<K, VT, WT>, one ? nullptr : jobs_dev, n_jobs, tile_offset, uniform,
                              one ? *one : dummy);
}

template <int K, typename VT>
cudaError_t tiled_launch_w(const ResliceJob* jobs_dev, const ResliceJob* one, int n_jobs, int tile_offset,
                           int n_tiles, int uniform, TileQueue* queue, int half_w, int pdl, cudaStream_t st) {
    return half_w ? tiled_launch<K, VT, __half>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, queue, pdl, st)
                  : tiled_launch<K, VT, float>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, queue, pdl, st);
}

template <int K>
cudaError_t tiled_launch_k(const ResliceJob* jobs_dev, const ResliceJob* one, int n_jobs, int tile_offset,
                           int n_tiles, int uniform, TileQueue* queue, int dtype, int half_w, int pdl, cudaStream_t st) {
    switch (dtype) {
    case DARE_U8:
        return tiled_launch_w<K, uint8_t>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, queue, half_w, pdl, st);
    case DARE_F16:
        return tiled_launch_w<K, __half>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, queue, half_w, pdl, st);
    case DARE_BF16:
        return tiled_launch_w<K, __nv_bfloat16>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, queue, half_w,
                                                pdl, st);
    case DARE_F32:
        return tiled_launch_w<K, float>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, queue, half_w, pdl, st);
    }
    return cudaErrorInvalidValue;
}

// The persistent kernel's grid for (K, dtype, weights), queried once per device
// (loads the kernel): call before a stream capture that launches it.
template <int K, typename VT>
cudaError_t persistent_prepare_w(int half_w) {
    const int g = half_w ? persistent_grid(k_reslice_tiled_persistent<K, VT, __half>)
                         : persistent_grid(k_reslice_tiled_persistent<K, VT, float>);
    return g > 0 ? cudaSuccess : cudaErrorInvalidValue;
}

template <int K>
cudaError_t persistent_prepare_k(int dtype, int half_w) {
    switch (dtype) {
    case DARE_U8: return persistent_prepare_w<K, uint8_t>(half_w);
    case DARE_F16: return persistent_prepare_w<K, __half>(half_w);
    case DARE_BF16: return persistent_prepare_w<K, __nv_bfloat16>(half_w);
    case DARE_F32: return persistent_prepare_w<K, float>(half_w);
    }
    return cudaErrorInvalidValue;
}

cudaError_t tiled_any(const ResliceJob* jobs_dev, const ResliceJob* one, int n_jobs, int tile_offset, int n_tiles,
                      int uniform, TileQueue* queue, int K, int dtype, int hw, int pdl, cudaStream_t st) {
    switch (K) {
    case 4: return tiled_launch_k<4>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, queue, dtype, hw, pdl, st);
    case 8: return tiled_launch_k<8>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, queue, dtype, hw, pdl, st);
    case 12: return tiled_launch_k<12>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, queue, dtype, hw, pdl, st);
    case 16: return tiled_launch_k<16>(jobs_dev, one, n_jobs, tile_offset, n_tiles, uniform, queue, dtype, hw, pdl, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_reslice_tiled(const ResliceJob* jobs_dev, const ResliceJob* one_job, int n_jobs, int tile_offset,
                                 int n_tiles, int uniform, int K, int dtype, int half_weights, int after_table,
                                 cudaStream_t st) {
    if (n_jobs <= 0 || n_tiles <= 0) return cudaSuccess;
    return tiled_any(jobs_dev, one_job, n_jobs, tile_offset, n_tiles, uniform, nullptr, K, dtype, half_weights,
                     after_table, st);
}

namespace {
template <int K, typename VT, typename WT>
void* tiled_fn() {
    return reinterpret_cast<void*>(k_reslice_tiled<K, VT, WT>);
}
template <int K>
void* tiled_fn_k(int dtype, int half_w) {
    switch (dtype) {
    case DARE_U8: return half_w ? tiled_fn<K, uint8_t, __half>() : tiled_fn<K, uint8_t, float>();
    case DARE_F16: return half_w ? tiled_fn<K, __half, __half>() : tiled_fn<K, __half, float>();
    case DARE_BF16: return half_w ? tiled_fn<K, __nv_bfloat16, __half>() : tiled_fn<K, __nv_bfloat16, float>();
    case DARE_F32: return half_w ? tiled_fn<K, float, __half>() : tiled_fn<K, float, float>();
    }
    return nullptr;
}
}  // namespace

cudaError_t reslice_tiled_node(const ResliceJob& one, int n_tiles, int K, int dtype, int half_weights, NodeArgs& args,
                               cudaKernelNodeParams* out) {
    if (n_tiles <= 0 || !out) return cudaErrorInvalidValue;
    void* fn = nullptr;
    switch (K) {
    case 4: fn = tiled_fn_k<4>(dtype, half_weights); break;
    case 8: fn = tiled_fn_k<8>(dtype, half_weights); break;
    case 12: fn = tiled_fn_k<12>(dtype, half_weights); break;
    case 16: fn = tiled_fn_k<16>(dtype, half_weights); break;
    }
    if (!fn) return cudaErrorInvalidValue;
    args.null_ptr = nullptr;
    args.ints[0] = 1;  // n_jobs
    args.ints[1] = 0;  // tile_offset
    args.ints[2] = 0;  // uniform
    args.rj = one;
    args.ptrs[0] = &args.null_ptr;  // jobs: none (one job by value)
    args.ptrs[1] = &args.ints[0];
    args.ptrs[2] = &args.ints[1];
    args.ptrs[3] = &args.ints[2];
    args.ptrs[4] = &args.rj;
    *out = cudaKernelNodeParams{};
    out->func = fn;
    out->gridDim = dim3(n_tiles);
    out->blockDim = dim3(kThreads);
    out->sharedMemBytes = 0;
    out->kernelParams = args.ptrs;
    return cudaSuccess;
}

cudaError_t launch_reslice_tiled_persistent(const ResliceJob* jobs_dev, int n_jobs, TileQueue* queue, int K,
                                            int dtype, int half_weights, cudaStream_t st) {
    if (n_jobs <= 0) return cudaSuccess;
    if (!jobs_dev || !queue) return cudaErrorInvalidValue;
    return tiled_any(jobs_dev, nullptr, n_jobs, 0, 0, 0, queue, K, dtype, half_weights, 0, st);
}

cudaError_t prepare_reslice_tiled_persistent(int K, int dtype, int half_weights) {
    switch (K) {
    case 4: return persistent_prepare_k<4>(dtype, half_weights);
    case 8: return persistent_prepare_k<8>(dtype, half_weights);
    case 12: return persistent_prepare_k<12>(dtype, half_weights);
    case 16: return persistent_prepare_k<16>(dtype, half_weights);
    }
    return cudaErrorInvalidValue;
}

cudaError_t read_fallback_tiles_tiled(unsigned long long* out, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_fallback_tiles, sizeof(*out));
    if (e != cudaSuccess || !reset) return e;
    const unsigned long long zero = 0;
    return cudaMemcpyToSymbol(g_fallback_tiles, &zero, sizeof(zero));
}

}  // namespace dare
