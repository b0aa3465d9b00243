// Reconstruction kernels (Sec. 2.1 "Volume reconstruction", Fig. 1) for
// sm_103a: pixel -> nearest voxel, one sample per (voxel, frame) holding the
// mean of that frame's pixels in the voxel, samples kept per voxel in frame
// order.
//
// Pipeline per chunk of frames:
//   count  -- each CTA takes a 32 x 64 pixel region of one frame (two 2 x 2
//             pixel blocks a thread; a 32 x 32 tile when the build lists the
//             voxels it reaches) and sums its pixels per voxel in shared
//             memory: a direct-mapped box of the region's voxels (one packed
//             32-bit add per voxel a 2 x 2 block reaches) when that box is
//             small, a hash table otherwise.  Every (voxel, region) entry
//             takes a slot from the voxel's counter; the first kBucket entries
//             of a voxel go straight into its bucket, later ones (rare) to the
//             overflow list;
//   scan   -- exclusive prefix sum of the overflow counts max(count - kBucket, 0)
//             (kernels.cu);
//   place  -- every overflow pair writes its entry into its voxel's overflow
//             range (tiles without overflow return at once);
//   (after a reset, alloc + place instead: the pair holding a voxel's first
//             entry past its bucket reserves the voxel's range from a cursor,
//             then every pair writes its entry at its slot in that range, and
//             the counters keep the full counts);
//   finalize -- one thread per voxel groups its entries (bucket, then overflow
//             range) by frame id (a frame split across tiles has several),
//             appends the new samples after the stored ones (their ids are all
//             lower), applies the capacity rule when more than K samples exist,
//             and returns the counter to zero.  After a reset every voxel is
//             written; voxels with entries past their bucket are left to a
//             second kernel (a thread each, no barrier).
// Integer sums make the result independent of scheduling order.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>

#include "dare_internal.h"

namespace dare {
namespace {

constexpr int kTile = kScatterTile;   // frame tile: 32 x 32 pixels
constexpr int kThreads = 256;         // a 2 x 2 pixel block per thread
#ifndef DARE_COUNT_MIN_BLOCKS
#define DARE_COUNT_MIN_BLOCKS 6  // 40 registers: faster than 5 CTAs at 46
#endif
#ifndef DARE_COUNT2_MIN_BLOCKS
#define DARE_COUNT2_MIN_BLOCKS 6  // 32 x 64 regions: 40 registers (a few spills), faster than 5 at 48 or 7 at 32
#endif
constexpr int kHash = 2048;           // >= 2 x pixels per tile: never full
constexpr int kEmptyKey = -1;
#ifndef DARE_BOX_CELLS
#define DARE_BOX_CELLS 4096
#endif
constexpr int kBoxCells = DARE_BOX_CELLS;  // largest direct-mapped voxel box of a tile (16 KB)
constexpr int kSmemWords = 3 * kHash + kTile * kTile;  // hash keys, counts, sums, list; or the box
static_assert(kBoxCells >= 0 && kBoxCells <= kSmemWords, "the box fits the shared buffer");
// packed per-voxel accumulator of the box: npix (<= 1024) above bit 18, sum (<= 1024 x 255 < 2^18) below
constexpr int kPackShift = 18;

// A thread's 2 x 2 pixel block.  The values are loaded first (they need only
// the frame and the pixel positions, so the loads overlap the CTA's set-up);
// the nearest voxels follow once the tile origin is known.  q-th pixel: its
// coordinates, in-grid flag and value.
struct BlockPixels {
    int c[4][3];
    bool in[4];
    unsigned val[4];
};

// In-image (and in-mask) flags and raw values of the block's pixels.  With an
// even width and an even frames address a pixel pair (u, u + 1) is one aligned
// 16-bit load.
__device__ __forceinline__ void block_values(const ScatterArgs& A, int f, int u0, int v0, BlockPixels& P) {
    const uint8_t* img = A.frames + static_cast<int64_t>(f) * A.width * A.height;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int u = u0 + 2 * tx, v = v0 + 2 * ty;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int uu = u + (q & 1), vv = v + (q >> 1);
        bool ok = uu < A.width && vv < A.height;
        if (ok && A.pix_mask)
            ok = (__ldg(A.pix_mask + static_cast<int64_t>(vv) * ((A.width + 31) >> 5) + (uu >> 5)) >> (uu & 31)) & 1u;
        P.in[q] = ok;
    }
    const bool pairs = ((reinterpret_cast<uintptr_t>(A.frames) | static_cast<uintptr_t>(A.width)) & 1u) == 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint8_t* row = img + static_cast<int64_t>(v + h) * A.width + u;
        if (pairs) {
            const unsigned pair = P.in[2 * h] || P.in[2 * h + 1] ? __ldg(reinterpret_cast<const unsigned short*>(row)) : 0u;
            P.val[2 * h] = pair & 0xFFu;
            P.val[2 * h + 1] = pair >> 8;
        } else {
            P.val[2 * h] = P.in[2 * h] ? __ldg(row) : 0u;
            P.val[2 * h + 1] = P.in[2 * h + 1] ? __ldg(row + 1) : 0u;
        }
    }
}

// Nearest voxels of the block's pixels; in[q] becomes "in the image and in the
// grid".  With small steps (|A|, |B| < 2^25, host flag) the tile origin's
// coordinates come from org (per axis: integer part, 20-bit remainder, steps
// per u and per v, set once per CTA) and each pixel adds int32 steps to them;
// otherwise int64 per pixel.
__device__ __forceinline__ void block_voxels(const ScatterArgs& A, const int64_t* aff, const int4* org, int u0, int v0,
                                             BlockPixels& P) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int u = u0 + 2 * tx, v = v0 + 2 * ty;
    if (A.small_steps) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int4 o = org[a];
            const int r00 = o.y + (2 * tx) * o.z + (2 * ty) * o.w, r10 = r00 + o.z, r01 = r00 + o.w, r11 = r10 + o.w;
            P.c[0][a] = o.x + (r00 >> kFixBits);
            P.c[1][a] = o.x + (r10 >> kFixBits);
            P.c[2][a] = o.x + (r01 >> kFixBits);
            P.c[3][a] = o.x + (r11 >> kFixBits);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            P.in[q] = P.in[q] && static_cast<unsigned>(P.c[q][0]) < static_cast<unsigned>(A.dims[0]) &&
                      static_cast<unsigned>(P.c[q][1]) < static_cast<unsigned>(A.dims[1]) &&
                      static_cast<unsigned>(P.c[q][2]) < static_cast<unsigned>(A.dims[2]);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int uu = u + (q & 1), vv = v + (q >> 1);
            bool in = P.in[q];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int64_t G = aff[a] + static_cast<int64_t>(uu) * aff[3 + a] + static_cast<int64_t>(vv) * aff[6 + a];
                const int64_t qq = (G + kFixOne / 2) >> kFixBits;
                in = in && qq >= 0 && qq < A.dims[a];
                P.c[q][a] = in ? static_cast<int>(qq) : 0;
            }
            P.in[q] = in;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (!P.in[q]) P.val[q] = 0u;
}

// Sums the block's pixels per distinct key (pixels of the block that share a
// voxel are combined before touching shared memory) and hands each distinct
// key with its pixel count and sum to `add`.
template <typename Add>
__device__ __forceinline__ void block_combine(const int (&key)[4], const unsigned (&val)[4], Add add) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        bool first = key[j] >= 0;
#pragma unroll
        for (int k = 0; k < j; ++k) first = first && key[k] != key[j];
        if (!first) continue;
        unsigned n = 1u, sm = val[j];
#pragma unroll
        for (int k = j + 1; k < 4; ++k)
            if (key[k] == key[j]) ++n, sm += val[k];
        add(key[j], n, sm);
    }
}

// A new key also appends its slot to `list` (the tile's distinct voxels).
__device__ __forceinline__ void hash_add(int* keys, unsigned* npx, unsigned* sums, int* list, int* n_list, int vi,
                                         unsigned n, unsigned s) {
    unsigned h = (static_cast<unsigned>(vi) * 2654435761u) >> 21;  // 11-bit Fibonacci hash
    for (;;) {  // at most kTile^2 distinct keys in kHash slots: terminates
        const int k0 = atomicCAS(keys + h, kEmptyKey, vi);
        if (k0 == kEmptyKey || k0 == vi) {
            atomicAdd(npx + h, n);  // two 32-bit adds: faster here than one 64-bit shared-memory add
            atomicAdd(sums + h, s);
            if (k0 == kEmptyKey) list[atomicAdd(n_list, 1)] = static_cast<int>(h);
            return;
        }
        h = (h + 1) & (kHash - 1);
    }
}

// The nearest-voxel box of a tile: by convexity its corner pixels bound every
// pixel's nearest voxel on each axis; clipped to the grid.  cells = 0 when no
// pixel of the tile can land in the grid.
struct TileBox {
    int b[3];
    int n[3];
    int cells;  // n0 n1 n2, or INT_MAX when above kBoxCells
};

// Computed by the 32 lanes of one warp: lanes 0-11 take one (corner, axis)
// each, lanes 0-2 reduce their axis over the corners, lane 0 writes B.
__device__ void tile_box(const int64_t* aff, const int4* org, bool small_steps, const int* dims, int u0, int v0, int u1,
                         int v1, TileBox& B) {
    const int lane = threadIdx.x & 31;
    const int k = lane / 3, a = lane < 12 ? lane % 3 : 0;
    const int u = (k & 1) ? u1 : u0, v = (k & 2) ? v1 : v0;
    int64_t q = 0;
    if (lane < 12) {
        if (small_steps) {  // the corner from the tile origin in int32 steps, as the pixels do
            const int4 o = org[a];
            q = o.x + ((o.y + (u - u0) * o.z + (v - v0) * o.w) >> kFixBits);
        } else {
            q = (aff[a] + static_cast<int64_t>(u) * aff[3 + a] + static_cast<int64_t>(v) * aff[6 + a] + kFixOne / 2) >>
                kFixBits;
        }
    }
    const int64_t q3 = __shfl_down_sync(0xFFFFFFFFu, q, 3), q6 = __shfl_down_sync(0xFFFFFFFFu, q, 6);
    const int64_t q9 = __shfl_down_sync(0xFFFFFFFFu, q, 9);
    const int64_t lo_a = min(min(q, q3), min(q6, q9)), hi_a = max(max(q, q3), max(q6, q9));  // lanes 0-2
    int64_t lo[3], hi[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        lo[i] = __shfl_sync(0xFFFFFFFFu, lo_a, i);
        hi[i] = __shfl_sync(0xFFFFFFFFu, hi_a, i);
    }
    if (lane != 0) return;
    int64_t cells = 1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int64_t l = lo[i] < 0 ? 0 : lo[i];
        const int64_t h = hi[i] > dims[i] - 1 ? dims[i] - 1 : hi[i];
        const int64_t n = h >= l ? h - l + 1 : 0;
        B.b[i] = static_cast<int>(l < dims[i] ? l : 0);
        B.n[i] = static_cast<int>(n);
        cells *= n;
    }
    B.cells = cells > kBoxCells ? INT_MAX : static_cast<int>(cells);
}

// Up to four (voxel, entry) results per thread and round: counter slots are
// taken with four returning atomics in flight; the first kBucket entries of a
// voxel go to its bucket (kBucket consecutive entries per voxel), later ones to
// the overflow list.  With s_new, a voxel whose first entry this is
// (slot 0) is also listed as touched by this build.
__device__ __forceinline__ void emit4(const int (&vi)[4], const unsigned long long (&e)[4], int32_t* count,
                                      unsigned long long* buckets, uint4* ovf, int* n_ovf, int* s_new, int* s_n_new) {
    int slot[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) slot[j] = vi[j] >= 0 ? atomicAdd(count + vi[j], 1) : 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (vi[j] < 0) continue;
        if (slot[j] < kBucket) {
            buckets[static_cast<int64_t>(vi[j]) * kBucket + slot[j]] = e[j];
            if (s_new && slot[j] == 0) s_new[atomicAdd(s_n_new, 1)] = vi[j];  // one per distinct voxel of the tile
        } else {
            const int k = atomicAdd(n_ovf, 1);  // at most one pair per pixel of the chunk
            ovf[k] = make_uint4(static_cast<unsigned>(vi[j]), static_cast<unsigned>(slot[j]),
                                static_cast<unsigned>(e[j]), static_cast<unsigned>(e[j] >> 32));
        }
    }
}

// One CTA per 32 x 32 frame tile (blockIdx.z = frame): per-voxel sums of the
// tile's pixels, then one (voxel, entry) per distinct voxel, entry = frame id
// << 48 | npix << 32 | sum.  Overflow pairs (a voxel's entries past its
// bucket, rare) are appended to one list, pairs[0, *n_pairs), which the host
// empties before the chunk's first count launch.  With `touched`, the
// voxels this build reaches for the first time are listed: touched[i], and
// tindex[v] = i, i < *n_touched.
template <bool kTouched>
__global__ void __launch_bounds__(kThreads, DARE_COUNT_MIN_BLOCKS)
    k_scatter_count(const __grid_constant__ ScatterArgs A,
                                                            int32_t* __restrict__ count,
                                                            unsigned long long* __restrict__ buckets,
                                                            uint4* __restrict__ pairs, int32_t* __restrict__ n_pairs,
                                                            int32_t* __restrict__ touched, int32_t* __restrict__ tindex,
                                                            int32_t* __restrict__ n_touched) {
    __shared__ __align__(16) unsigned smem[kSmemWords];
    __shared__ int64_t aff[9];
    __shared__ int4 org[3];  // small steps: the tile origin per axis (integer part, remainder, steps)
    __shared__ TileBox B;
    __shared__ int n_list, n_new, new_base;
    __shared__ int s_new[kTouched ? kTile * kTile : 1];  // voxels whose first entry this tile made
    const int f = blockIdx.z;
    const int u0 = blockIdx.x * kTile, v0 = blockIdx.y * kTile;
    if (threadIdx.x < 9) aff[threadIdx.x] = A.affines[9 * static_cast<int64_t>(f) + threadIdx.x];
    if (A.small_steps && threadIdx.x >= 32 && threadIdx.x < 35) {  // (warp 0 sets up the box later)
        const int a = threadIdx.x - 32;
        const int64_t* af = A.affines + 9 * static_cast<int64_t>(f);
        const int64_t ga = af[3 + a], gb = af[6 + a];
        const int64_t G = af[a] + static_cast<int64_t>(u0) * ga + static_cast<int64_t>(v0) * gb + kFixOne / 2;
        const int64_t F = G >> kFixBits;
        org[a] = make_int4(static_cast<int>(F < -(1 << 24) ? -(1 << 24) : (F > (1 << 24) ? (1 << 24) : F)),
                           static_cast<int>(G & (kFixOne - 1)), static_cast<int>(ga), static_cast<int>(gb));
    }
    if (threadIdx.x == 0) {
        n_list = 0;
        n_new = 0;
    }
    // the box of the direct-mapped path, cleared while the affine arrives
    BlockPixels P;
    block_values(A, f, u0, v0, P);  // in flight during the set-up
    uint4* c4 = reinterpret_cast<uint4*>(smem);
    for (int i = threadIdx.x; i < kBoxCells / 4; i += kThreads) c4[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    if (threadIdx.x < 32)
        tile_box(aff, org, A.small_steps != 0, A.dims, u0, v0, min(u0 + kTile, A.width) - 1,
                 min(v0 + kTile, A.height) - 1, B);
    block_voxels(A, aff, org, u0, v0, P);  // (the other warps meanwhile)
    __syncthreads();
    const int cells = B.cells;
    if (cells == 0) return;  // no pixel of the tile lands in the grid
    const unsigned long long fid = static_cast<unsigned long long>(A.frame_base + f) << 48;
    if (cells <= kBoxCells) {
        // direct-mapped box: one packed counter per voxel of the box
        const int b0 = B.b[0], b1 = B.b[1], b2 = B.b[2], n0 = B.n[0], n1 = B.n[1];
        int key[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) key[q] = P.in[q] ? (P.c[q][0] - b0) + n0 * ((P.c[q][1] - b1) + n1 * (P.c[q][2] - b2)) : -1;
        block_combine(key, P.val, [&](int k, unsigned n, unsigned sm) { atomicAdd(smem + k, (n << kPackShift) | sm); });
        __syncthreads();
        const int64_t d0 = A.dims[0], d01 = static_cast<int64_t>(A.dims[0]) * A.dims[1];
        // cell -> (i0, i1, i2) by FP32 reciprocals: exact for indices below 2^12
        const float inv01 = 1.0f / static_cast<float>(n0 * n1), inv0 = 1.0f / static_cast<float>(n0);
        for (int r = 0; r < cells; r += 4 * kThreads) {
            int vi[4];
            unsigned long long e[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int idx = r + j * kThreads + threadIdx.x;
                const unsigned x = idx < cells ? smem[idx] : 0u;
                vi[j] = -1;
                e[j] = 0;
                if (x) {
                    const int i2 = static_cast<int>((static_cast<float>(idx) + 0.5f) * inv01);
                    const int rem = idx - i2 * (n0 * n1);
                    const int i1 = static_cast<int>((static_cast<float>(rem) + 0.5f) * inv0), i0 = rem - i1 * n0;
                    vi[j] = static_cast<int>((b0 + i0) + d0 * (b1 + i1) + d01 * (b2 + i2));
                    e[j] = fid | (static_cast<unsigned long long>(x >> kPackShift) << 32) | (x & ((1u << kPackShift) - 1));
                }
            }
            emit4(vi, e, count, buckets, pairs, n_pairs, kTouched ? s_new : nullptr, &n_new);
        }
    } else {
        // hash table over voxel indices
        int* keys = reinterpret_cast<int*>(smem);
        unsigned* npx = smem + kHash;
        unsigned* sums = smem + 2 * kHash;
        int* list = reinterpret_cast<int*>(smem + 3 * kHash);
        uint4* keys4 = reinterpret_cast<uint4*>(keys);
        uint4* both4 = reinterpret_cast<uint4*>(npx);
        static_assert(kEmptyKey == -1, "keys cleared to all-ones words");
        for (int i = threadIdx.x; i < kHash / 4; i += kThreads) keys4[i] = make_uint4(~0u, ~0u, ~0u, ~0u);
        for (int i = threadIdx.x; i < kHash / 2; i += kThreads) both4[i] = make_uint4(0u, 0u, 0u, 0u);
        int key[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) key[q] = P.in[q] ? P.c[q][0] + A.dims[0] * (P.c[q][1] + A.dims[1] * P.c[q][2]) : -1;
        __syncthreads();  // table cleared
        block_combine(key, P.val, [&](int k, unsigned n, unsigned sm) { hash_add(keys, npx, sums, list, &n_list, k, n, sm); });
        __syncthreads();
        const int n = n_list;
        for (int r = 0; r < n; r += 4 * kThreads) {
            int vi[4];
            unsigned long long e[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = r + j * kThreads + threadIdx.x;
                vi[j] = -1;
                e[j] = 0;
                if (i < n) {
                    const int h = list[i];
                    vi[j] = keys[h];
                    e[j] = fid | (static_cast<unsigned long long>(npx[h]) << 32) | sums[h];
                }
            }
            emit4(vi, e, count, buckets, pairs, n_pairs, kTouched ? s_new : nullptr, &n_new);
        }
    }
    if constexpr (kTouched) {
        __syncthreads();
        if (threadIdx.x == 0) new_base = n_new ? atomicAdd(n_touched, n_new) : 0;
        __syncthreads();
        for (int k = threadIdx.x; k < n_new; k += kThreads) {
            const int v = s_new[k];
            touched[new_base + k] = v;
            tindex[v] = new_base + k;
        }
    }
}

// The count pass of builds that do not list the voxels they reach (full
// rebuilds, large appends): one CTA per 32 x 64 pixel region of a frame (two
// 32-row halves, a 2 x 2 block of each per thread), so the set-up
// (affine, origins, box clear, tile box) and the three barriers serve 2048
// pixels.  Each half has its own fixed-point origin, so the int32 pixel steps
// stay within the range of the 32-row form.  Boxes past kBoxCells take the
// hash table one half at a time (at most kTile^2 keys per pass).  The packed
// box accumulator holds npix <= 2048 above bit 19 and sum <= 2048 x 255 below.
// No touched list: used where the count pass need not list new voxels.
constexpr int kRows2 = 2 * kTile;
constexpr int kPackShift2 = 19;

// Corner coordinates from the origin of the half a corner lies in (small steps).
__device__ void tile_box2(const int64_t* aff, const int4* org, const int4* org2, bool small_steps, const int* dims,
                          int u0, int v0, int u1, int v1, TileBox& B) {
    const int lane = threadIdx.x & 31;
    const int k = lane / 3, a = lane < 12 ? lane % 3 : 0;
    const int u = (k & 1) ? u1 : u0, v = (k & 2) ? v1 : v0;
    int64_t q = 0;
    if (lane < 12) {
        if (small_steps) {
            const bool hi = v >= v0 + kTile;
            const int4 o = hi ? org2[a] : org[a];
            q = o.x + ((o.y + (u - u0) * o.z + (v - v0 - (hi ? kTile : 0)) * o.w) >> kFixBits);
        } else {
            q = (aff[a] + static_cast<int64_t>(u) * aff[3 + a] + static_cast<int64_t>(v) * aff[6 + a] + kFixOne / 2) >>
                kFixBits;
        }
    }
    const int64_t q3 = __shfl_down_sync(0xFFFFFFFFu, q, 3), q6 = __shfl_down_sync(0xFFFFFFFFu, q, 6);
    const int64_t q9 = __shfl_down_sync(0xFFFFFFFFu, q, 9);
    const int64_t lo_a = min(min(q, q3), min(q6, q9)), hi_a = max(max(q, q3), max(q6, q9));
    int64_t lo[3], hi[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        lo[i] = __shfl_sync(0xFFFFFFFFu, lo_a, i);
        hi[i] = __shfl_sync(0xFFFFFFFFu, hi_a, i);
    }
    if (lane != 0) return;
    int64_t cells = 1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int64_t l = lo[i] < 0 ? 0 : lo[i];
        const int64_t h = hi[i] > dims[i] - 1 ? dims[i] - 1 : hi[i];
        const int64_t n = h >= l ? h - l + 1 : 0;
        B.b[i] = static_cast<int>(l < dims[i] ? l : 0);
        B.n[i] = static_cast<int>(n);
        cells *= n;
    }
    B.cells = cells > kBoxCells ? INT_MAX : static_cast<int>(cells);
}

__global__ void __launch_bounds__(kThreads, DARE_COUNT2_MIN_BLOCKS)
    k_scatter_count2(const __grid_constant__ ScatterArgs A, int32_t* __restrict__ count,
                     unsigned long long* __restrict__ buckets, uint4* __restrict__ pairs,
                     int32_t* __restrict__ n_pairs) {
    __shared__ __align__(16) unsigned smem[kSmemWords];
    __shared__ int64_t aff[9];
    __shared__ int4 org[2][3];  // small steps: each half's origin per axis (integer part, remainder, steps)
    __shared__ TileBox B;
    __shared__ int n_list;
    const int f = blockIdx.z;
    const int u0 = blockIdx.x * kTile, v0 = blockIdx.y * kRows2;
    if (threadIdx.x < 9) aff[threadIdx.x] = A.affines[9 * static_cast<int64_t>(f) + threadIdx.x];
    if (A.small_steps && threadIdx.x >= 32 && threadIdx.x < 38) {  // (warp 0 sets up the box later)
        const int a = (threadIdx.x - 32) % 3, h = (threadIdx.x - 32) / 3;
        const int64_t* af = A.affines + 9 * static_cast<int64_t>(f);
        const int64_t ga = af[3 + a], gb = af[6 + a];
        const int64_t G = af[a] + static_cast<int64_t>(u0) * ga + static_cast<int64_t>(v0 + h * kTile) * gb + kFixOne / 2;
        const int64_t F = G >> kFixBits;
        org[h][a] = make_int4(static_cast<int>(F < -(1 << 24) ? -(1 << 24) : (F > (1 << 24) ? (1 << 24) : F)),
                              static_cast<int>(G & (kFixOne - 1)), static_cast<int>(ga), static_cast<int>(gb));
    }
    if (threadIdx.x == 0) n_list = 0;
    BlockPixels P0, P1;
    block_values(A, f, u0, v0, P0);  // both halves' pixels in flight during the set-up
    block_values(A, f, u0, v0 + kTile, P1);
    uint4* c4 = reinterpret_cast<uint4*>(smem);
    for (int i = threadIdx.x; i < kBoxCells / 4; i += kThreads) c4[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    if (threadIdx.x < 32)
        tile_box2(aff, org[0], org[1], A.small_steps != 0, A.dims, u0, v0, min(u0 + kTile, A.width) - 1,
                  min(v0 + kRows2, A.height) - 1, B);
    block_voxels(A, aff, org[0], u0, v0, P0);  // (the second half's voxels once the first half is summed)
    __syncthreads();
    const int cells = B.cells;
    if (cells == 0) return;  // no pixel of the region lands in the grid
    const unsigned long long fid = static_cast<unsigned long long>(A.frame_base + f) << 48;
    if (cells <= kBoxCells) {
        const int b0 = B.b[0], b1 = B.b[1], b2 = B.b[2], n0 = B.n[0], n1 = B.n[1];
        auto add = [&](int k, unsigned n, unsigned sm) { atomicAdd(smem + k, (n << kPackShift2) | sm); };
        int key[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) key[q] = P0.in[q] ? (P0.c[q][0] - b0) + n0 * ((P0.c[q][1] - b1) + n1 * (P0.c[q][2] - b2)) : -1;
        block_combine(key, P0.val, add);
        block_voxels(A, aff, org[1], u0, v0 + kTile, P1);
#pragma unroll
        for (int q = 0; q < 4; ++q) key[q] = P1.in[q] ? (P1.c[q][0] - b0) + n0 * ((P1.c[q][1] - b1) + n1 * (P1.c[q][2] - b2)) : -1;
        block_combine(key, P1.val, add);
        __syncthreads();
        const int64_t d0 = A.dims[0], d01 = static_cast<int64_t>(A.dims[0]) * A.dims[1];
        const float inv01 = 1.0f / static_cast<float>(n0 * n1), inv0 = 1.0f / static_cast<float>(n0);
        for (int r = 0; r < cells; r += 4 * kThreads) {
            int vi[4];
            unsigned long long e[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int idx = r + j * kThreads + threadIdx.x;
                const unsigned x = idx < cells ? smem[idx] : 0u;
                vi[j] = -1;
                e[j] = 0;
                if (x) {
                    const int i2 = static_cast<int>((static_cast<float>(idx) + 0.5f) * inv01);
                    const int rem = idx - i2 * (n0 * n1);
                    const int i1 = static_cast<int>((static_cast<float>(rem) + 0.5f) * inv0), i0 = rem - i1 * n0;
                    vi[j] = static_cast<int>((b0 + i0) + d0 * (b1 + i1) + d01 * (b2 + i2));
                    e[j] = fid | (static_cast<unsigned long long>(x >> kPackShift2) << 32) | (x & ((1u << kPackShift2) - 1));
                }
            }
            emit4(vi, e, count, buckets, pairs, n_pairs, nullptr, nullptr);
        }
    } else {
        // hash table over voxel indices, one half at a time
        int* keys = reinterpret_cast<int*>(smem);
        unsigned* npx = smem + kHash;
        unsigned* sums = smem + 2 * kHash;
        int* list = reinterpret_cast<int*>(smem + 3 * kHash);
        uint4* keys4 = reinterpret_cast<uint4*>(keys);
        uint4* both4 = reinterpret_cast<uint4*>(npx);
        static_assert(kEmptyKey == -1, "keys cleared to all-ones words");
        auto hash_half = [&](const BlockPixels& P) {
            for (int i = threadIdx.x; i < kHash / 4; i += kThreads) keys4[i] = make_uint4(~0u, ~0u, ~0u, ~0u);
            for (int i = threadIdx.x; i < kHash / 2; i += kThreads) both4[i] = make_uint4(0u, 0u, 0u, 0u);
            if (threadIdx.x == 0) n_list = 0;
            int key[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) key[q] = P.in[q] ? P.c[q][0] + A.dims[0] * (P.c[q][1] + A.dims[1] * P.c[q][2]) : -1;
            __syncthreads();  // table cleared
            block_combine(key, P.val, [&](int k, unsigned n, unsigned sm) { hash_add(keys, npx, sums, list, &n_list, k, n, sm); });
            __syncthreads();
            const int n = n_list;
            for (int r = 0; r < n; r += 4 * kThreads) {
                int vi[4];
                unsigned long long e[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int i = r + j * kThreads + threadIdx.x;
                    vi[j] = -1;
                    e[j] = 0;
                    if (i < n) {
                        const int hh = list[i];
                        vi[j] = keys[hh];
                        e[j] = fid | (static_cast<unsigned long long>(npx[hh]) << 32) | sums[hh];
                    }
                }
                emit4(vi, e, count, buckets, pairs, n_pairs, nullptr, nullptr);
            }
            __syncthreads();  // the list and table are read before the next half clears them
        };
        hash_half(P0);
        block_voxels(A, aff, org[1], u0, v0 + kTile, P1);
        hash_half(P1);
    }
}

// Overflow counts of the touched voxels, max(count - kBucket, 0), in list order;
// zeros from *n_touched up to max_t (the scan that follows covers max_t).
__global__ void __launch_bounds__(256) k_touched_overflow(const int32_t* __restrict__ count,
                                                          const int32_t* __restrict__ touched,
                                                          const int32_t* __restrict__ n_touched, int64_t max_t,
                                                          int32_t* __restrict__ ovf_cnt) {
    const int64_t n = *n_touched;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < max_t;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        ovf_cnt[i] = i < n ? max(count[touched[i]] - kBucket, 0) : 0;
}

// Overflow pairs (entries of a voxel beyond its bucket), from the list the
// count pass appended them to: a grid-stride loop, so the work is even however
// the pairs cluster.  Each pair takes a position in its voxel's overflow range
// (by voxel, or by its place in the touched list with tindex) from the voxel's
// counter, which counts back down to kBucket.
__global__ void __launch_bounds__(256) k_scatter_place(const uint4* __restrict__ pairs,
                                                       const int32_t* __restrict__ n_pairs,
                                                       int32_t* __restrict__ count, const int32_t* __restrict__ offsets,
                                                       const int32_t* __restrict__ tindex,
                                                       unsigned long long* __restrict__ entries) {
    const int64_t n = *n_pairs;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint4 p = __ldg(pairs + i);
        const int pos = offsets[tindex ? tindex[p.x] : p.x] + atomicSub(count + p.x, 1) - 1 - kBucket;
        entries[pos] = (static_cast<unsigned long long>(p.w) << 32) | p.z;
    }
}

// Full-write mode (after a reset): each voxel with entries past its bucket gets
// an overflow range of count - kBucket entries, reserved by the one pair that
// took the voxel's first slot past the bucket; a CTA scans its pairs' lengths
// and takes its share of the cursor with one atomic.  The ranges' starts go to
// offsets[v] (other voxels' offsets are not written).  This replaces the scan
// of every voxel's counter that appends need.
__global__ void __launch_bounds__(256) k_overflow_alloc(const uint4* __restrict__ pairs,
                                                        const int32_t* __restrict__ n_pairs,
                                                        const int32_t* __restrict__ count,
                                                        int32_t* __restrict__ offsets, int32_t* __restrict__ cursor) {
    __shared__ int s_warp[8];
    __shared__ int s_base;
    const int64_t n = *n_pairs;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t i0 = static_cast<int64_t>(blockIdx.x) * 256; i0 < n; i0 += static_cast<int64_t>(gridDim.x) * 256) {
        const int64_t i = i0 + threadIdx.x;
        int len = 0;
        unsigned v = 0;
        if (i < n) {
            const uint4 p = __ldg(pairs + i);
            if (p.y == kBucket) {
                v = p.x;
                len = count[v] - kBucket;
            }
        }
        int x = len;  // inclusive warp scan
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            int total = 0;
            for (int k = 0; k < 8; ++k) total += s_warp[k];
            s_base = total ? atomicAdd(cursor, total) : 0;
        }
        __syncthreads();
        int base = s_base;
        for (int k = 0; k < warp; ++k) base += s_warp[k];
        if (len) offsets[v] = base + x - len;
        __syncthreads();  // s_warp and s_base are rewritten by the next round
    }
}

// Full-write mode: every overflow pair's entry at its voxel's range start plus
// (its slot - kBucket).
__global__ void __launch_bounds__(256) k_overflow_place(const uint4* __restrict__ pairs,
                                                        const int32_t* __restrict__ n_pairs,
                                                        const int32_t* __restrict__ offsets,
                                                        unsigned long long* __restrict__ entries) {
    const int64_t n = *n_pairs;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint4 p = __ldg(pairs + i);
        entries[offsets[p.x] + static_cast<int>(p.y) - kBucket] = (static_cast<unsigned long long>(p.w) << 32) | p.z;
    }
}

// ------------------------------------------------------------------ finalize

template <typename VT>
__device__ __forceinline__ VT round_store(int sum, int cnt);
template <>
__device__ __forceinline__ float round_store<float>(int sum, int cnt) {
    return __fdiv_rn(static_cast<float>(sum), static_cast<float>(cnt));
}
template <>
__device__ __forceinline__ __half round_store<__half>(int sum, int cnt) {
    return __float2half_rn(__fdiv_rn(static_cast<float>(sum), static_cast<float>(cnt)));
}
template <>
__device__ __forceinline__ __nv_bfloat16 round_store<__nv_bfloat16>(int sum, int cnt) {
    return __float2bfloat16_rn(__fdiv_rn(static_cast<float>(sum), static_cast<float>(cnt)));
}
template <>
__device__ __forceinline__ uint8_t round_store<uint8_t>(int sum, int cnt) {
    const unsigned r = __float2uint_rn(__fdiv_rn(static_cast<float>(sum), static_cast<float>(cnt)));
    return static_cast<uint8_t>(r > 255u ? 255u : r);
}

__device__ __forceinline__ int ent_frame(unsigned long long e) { return static_cast<int>(e >> 48); }
__device__ __forceinline__ int ent_npix(unsigned long long e) { return static_cast<int>((e >> 32) & 0xFFFFu); }
__device__ __forceinline__ int ent_sum(unsigned long long e) { return static_cast<int>(e & 0xFFFFFFFFu); }

// A voxel's entries: c in its bucket, then its overflow range [s, s + n - c).
struct VoxelEntries {
    const unsigned long long* bucket;
    const unsigned long long* ovf;
    int c, s, n;
    __device__ __forceinline__ unsigned long long at(int i) const {
        return i < c ? __ldg(bucket + i) : __ldg(ovf + s + (i - c));
    }
};

// All four 16-byte pieces of a voxel's bucket, loaded together (entries past
// the voxel's count are stale and ignored).
__device__ __forceinline__ void bucket_load(const unsigned long long* bucket, ulonglong2 (&b)[kBucket / 2]) {
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(bucket);
#pragma unroll
    for (int i = 0; i < kBucket / 2; ++i) b[i] = __ldg(q + i);
}

// Sorts the c <= kBucket entries held in b ascending, by frame id (the
// entry's top 16 bits); the slots past c become all ones and sort last.
__device__ __forceinline__ void bucket_sort(const ulonglong2 (&b)[kBucket / 2], int c, unsigned long long (&e)[kBucket]) {
    static_assert(kBucket == 8, "sorting network for 8 entries");
#pragma unroll
    for (int i = 0; i < kBucket / 2; ++i) {
        e[2 * i] = 2 * i < c ? b[i].x : ~0ull;
        e[2 * i + 1] = 2 * i + 1 < c ? b[i].y : ~0ull;
    }
    // Batcher's odd-even merge sort, 19 compare-exchanges
#define DARE_CX(a, b)                                        \
    {                                                        \
        const unsigned long long lo = e[a] < e[b] ? e[a] : e[b]; \
        const unsigned long long hi = e[a] < e[b] ? e[b] : e[a]; \
        e[a] = lo;                                           \
        e[b] = hi;                                           \
    }
    DARE_CX(0, 1) DARE_CX(2, 3) DARE_CX(4, 5) DARE_CX(6, 7)
    DARE_CX(0, 2) DARE_CX(1, 3) DARE_CX(4, 6) DARE_CX(5, 7)
    DARE_CX(1, 2) DARE_CX(5, 6)
    DARE_CX(0, 4) DARE_CX(1, 5) DARE_CX(2, 6) DARE_CX(3, 7)
    DARE_CX(2, 4) DARE_CX(3, 5)
    DARE_CX(1, 2) DARE_CX(3, 4) DARE_CX(5, 6)
#undef DARE_CX
}

// The c <= kBucket entries of a voxel without overflow, sorted; only the
// 16-byte loads that hold entries are issued.
__device__ __forceinline__ void bucket_sorted(const unsigned long long* bucket, int c,
                                              unsigned long long (&e)[kBucket]) {
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(bucket);
    ulonglong2 b[kBucket / 2];
#pragma unroll
    for (int i = 0; i < kBucket / 2; ++i) b[i] = 2 * i < c ? __ldg(q + i) : make_ulonglong2(~0ull, ~0ull);
    bucket_sort(b, c, e);
}

// General merge: the m_old stored samples plus the new entries grouped by
// frame; more than K samples keep the K of largest npix (ties: lower id).
template <int K, typename VT>
__device__ __noinline__ bool merge_general(const VoxelEntries E, int m_old, uint16_t* ids, VT* vals, uint16_t* np) {
    int Lid[K], Lnp[K], Lcnt[K], Lsum[K];
    VT Lraw[K];
    bool Lnew[K];
    for (int k = 0; k < m_old; ++k) {
        Lid[k] = ids[k];
        Lnp[k] = np[k];
        Lcnt[k] = 0;
        Lsum[k] = 0;
        Lraw[k] = vals[k];
        Lnew[k] = false;
    }
    int m = m_old;
    bool over = false;
    int last = -1;
    for (;;) {
        int next = 0xFFFF, cnt = 0, sum = 0;
        for (int i = 0; i < E.n; ++i) {
            const unsigned long long x = E.at(i);
            const int f = ent_frame(x);
            if (f > last && f < next) {
                next = f;
                cnt = ent_npix(x);
                sum = ent_sum(x);
            } else if (f == next) {
                cnt += ent_npix(x);
                sum += ent_sum(x);
            }
        }
        if (next == 0xFFFF) break;
        last = next;
        const int cs = cnt < 65535 ? cnt : 65535;
        int slot = -1;
        if (m < K) {
            slot = m++;
        } else {
            over = true;
            int wi = 0;
            for (int k = 1; k < K; ++k)
                if (Lnp[k] < Lnp[wi] || (Lnp[k] == Lnp[wi] && Lid[k] > Lid[wi])) wi = k;
            if (cs > Lnp[wi] || (cs == Lnp[wi] && next < Lid[wi])) slot = wi;
        }
        if (slot >= 0) {
            Lid[slot] = next;
            Lnp[slot] = cs;
            Lcnt[slot] = cnt;
            Lsum[slot] = sum;
            Lnew[slot] = true;
        }
    }
    for (int i = 1; i < m; ++i) {  // order by frame id
        const int id = Lid[i], pn = Lnp[i], c = Lcnt[i], sm = Lsum[i];
        const VT raw = Lraw[i];
        const bool nw = Lnew[i];
        int j = i - 1;
        while (j >= 0 && Lid[j] > id) {
            Lid[j + 1] = Lid[j]; Lnp[j + 1] = Lnp[j]; Lcnt[j + 1] = Lcnt[j];
            Lsum[j + 1] = Lsum[j]; Lraw[j + 1] = Lraw[j]; Lnew[j + 1] = Lnew[j];
            --j;
        }
        Lid[j + 1] = id; Lnp[j + 1] = pn; Lcnt[j + 1] = c; Lsum[j + 1] = sm; Lraw[j + 1] = raw; Lnew[j + 1] = nw;
    }
    for (int k = 0; k < K; ++k) {
        if (k < m) {
            ids[k] = static_cast<uint16_t>(Lid[k]);
            vals[k] = Lnew[k] ? round_store<VT>(Lsum[k], Lcnt[k]) : Lraw[k];
            np[k] = static_cast<uint16_t>(Lnp[k]);
        } else {
            ids[k] = static_cast<uint16_t>(DARE_EMPTY_FRAME);
            vals[k] = VT(0);
            np[k] = 0;
        }
    }
    return over;
}

// Fast path: new samples (ascending frame id) go after the stored ones; each
// pass re-reads the voxel's entries (from L1) and takes the next frame.
// Returns false when more than K samples exist (the capacity rule needs the
// general merge).
template <int K, typename VT>
__device__ __forceinline__ bool append_in_order(const VoxelEntries& E, int m_old, uint16_t* ids, VT* vals,
                                                uint16_t* np) {
    int m = m_old, last = -1;
    for (;;) {
        int next = 0xFFFF, cnt = 0, sum = 0;
        for (int i = 0; i < E.n; ++i) {
            const unsigned long long x = E.at(i);
            const int f = ent_frame(x);
            const bool lower = f > last && f < next;
            const bool same = f == next;
            cnt = lower ? ent_npix(x) : (same ? cnt + ent_npix(x) : cnt);
            sum = lower ? ent_sum(x) : (same ? sum + ent_sum(x) : sum);
            next = lower ? f : next;
        }
        if (next == 0xFFFF) return true;
        if (m == K) return false;  // more than K samples: capacity rule
        ids[m] = static_cast<uint16_t>(next);
        vals[m] = round_store<VT>(sum, cnt);
        np[m] = static_cast<uint16_t>(cnt < 65535 ? cnt : 65535);
        ++m;
        last = next;
    }
}

// Sorted entries (frame id ascending, all-ones padding last) appended after
// the m_old stored samples, entries of one frame merged.  Returns the new
// sample count, or -1 when more than K samples exist (the general merge then
// redoes the voxel from its stored samples).
template <int K, typename VT, int N = kBucket>
__device__ __forceinline__ int append_sorted(const unsigned long long (&e)[N], int m_old, uint16_t* ids,
                                             VT* vals, uint16_t* np) {
    int m = m_old, cur = -1, cnt = 0, sum = 0;
#pragma unroll
    for (int j = 0; j <= N; ++j) {
        const bool end = j == N || e[j] == ~0ull;
        const int f = end ? -2 : ent_frame(e[j]);
        if (f != cur) {
            if (cur >= 0) {
                if (m == K) return -1;
                ids[m] = static_cast<uint16_t>(cur);
                vals[m] = round_store<VT>(sum, cnt);
                np[m] = static_cast<uint16_t>(cnt < 65535 ? cnt : 65535);
                ++m;
            }
            if (end) break;
            cur = f;
            cnt = 0;
            sum = 0;
        }
        cnt += ent_npix(e[j]);
        sum += ent_sum(e[j]);
    }
    return m;
}

// A voxel's new samples after its m_old stored ones, and the totals of its
// entries (mean-compounding comparator).  Returns true when the capacity rule
// dropped samples.
template <int K, typename VT>
__device__ __forceinline__ bool voxel_merge_sorted(const VoxelEntries& E, const unsigned long long (&ev)[kBucket],
                                                   int m_old, uint16_t* ids, VT* vals, uint16_t* np,
                                                   uint32_t& tot_sum, uint32_t& tot_cnt) {
    tot_sum = 0;
    tot_cnt = 0;
#pragma unroll
    for (int j = 0; j < kBucket; ++j)
        if (j < E.c) {
            tot_sum += static_cast<uint32_t>(ent_sum(ev[j]));
            tot_cnt += static_cast<uint32_t>(ent_npix(ev[j]));
        }
    if (append_sorted<K, VT>(ev, m_old, ids, vals, np) >= 0) return false;
    return merge_general<K, VT>(E, m_old, ids, vals, np);
}

template <int K, typename VT>
__device__ __forceinline__ bool voxel_merge(const VoxelEntries& E, int m_old, uint16_t* ids, VT* vals, uint16_t* np,
                                            uint32_t& tot_sum, uint32_t& tot_cnt) {
    tot_sum = 0;
    tot_cnt = 0;
    if (E.n == E.c) {  // every entry in the bucket: sorted in registers
        unsigned long long ev[kBucket];
        bucket_sorted(E.bucket, E.c, ev);
        return voxel_merge_sorted<K, VT>(E, ev, m_old, ids, vals, np, tot_sum, tot_cnt);
    } else {
        for (int i = 0; i < E.n; ++i) {
            const unsigned long long x = E.at(i);
            tot_sum += static_cast<uint32_t>(ent_sum(x));
            tot_cnt += static_cast<uint32_t>(ent_npix(x));
        }
        if (append_in_order<K, VT>(E, m_old, ids, vals, np)) return false;
    }
    return merge_general<K, VT>(E, m_old, ids, vals, np);
}

// kMode 0: merge into the stored records.  1 (fresh): the volume holds no
// sample at all, so the stored records are known to be empty and are not read.
// 2 (full): as 1, and the volume has not been cleared since a reset: every
// voxel is written, empty ones with the empty record, zero npix and zero
// scalar totals, which spares the reset a pass over the whole volume.
// With `touched` (modes 0 and 1) only the listed voxels are visited, item i
// being voxel touched[i] with overflow range offsets[i] .. offsets[i + 1]; else
// every voxel v with offsets[v] .. offsets[v + 1].
template <int K, typename VT, int kMode>
__global__ void __launch_bounds__(256, kMode == 2 ? 6 : 4) k_finalize(int32_t* __restrict__ count,
                                                  const unsigned long long* __restrict__ buckets,
                                                  const int32_t* __restrict__ offsets,
                                                  const unsigned long long* __restrict__ entries, int64_t n_vox,
                                                  uint8_t* __restrict__ rec, uint16_t* __restrict__ npix,
                                                  uint32_t* __restrict__ scal_sum, uint32_t* __restrict__ scal_cnt,
                                                  unsigned long long* overflow, const int32_t* __restrict__ touched,
                                                  const int32_t* __restrict__ n_touched) {
    constexpr int RB = (2 * K + K * static_cast<int>(sizeof(VT)) + 15) / 16 * 16;
    // each thread edits its voxel's record and npix row in shared memory and
    // writes them back whole (full sectors, vector stores)
    __shared__ uint4 s_rec[256 * RB / 16];
    __shared__ uint2 s_np[256 * K / 4];
    uint4* my_rec = s_rec + threadIdx.x * (RB / 16);
    uint2* my_np = s_np + threadIdx.x * (K / 4);
    constexpr bool kFresh = kMode != 0;
    const int64_t n_items = touched ? static_cast<int64_t>(*n_touched) : n_vox;
    for (int64_t it = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; it < n_items;
         it += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t v = touched ? static_cast<int64_t>(touched[it]) : it;
        // the counter and the whole bucket in one round trip; a voxel has
        // overflow entries (its offsets differ) only when its bucket is full
        const int c = count[v];
        ulonglong2 b[kBucket / 2];
        bucket_load(buckets + v * kBucket, b);
        int s = 0, e = 0;
        if (c == kBucket) {
            s = offsets[it];
            e = offsets[it + 1];
        }
        uint4* g_rec = reinterpret_cast<uint4*>(rec + v * RB);
        uint2* g_np = reinterpret_cast<uint2*>(npix + v * K);
        if (c == 0) {  // no entry (the overflow range is empty too)
            if (kMode == 2) {
#pragma unroll
                for (int i = 0; i < RB / 16; ++i) {
                    uint4 q = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const int b = 16 * i + 4 * w;
                        uint32_t x = 0u;
#pragma unroll
                        for (int h = 0; h < 2; ++h)
                            if (b + 2 * h < 2 * K) x |= 0xFFFFu << (16 * h);
                        (w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w) = x;
                    }
                    g_rec[i] = q;
                }
#pragma unroll
                for (int i = 0; i < K / 4; ++i) g_np[i] = make_uint2(0u, 0u);
                if (scal_sum) {
                    scal_sum[v] = 0u;
                    scal_cnt[v] = 0u;
                }
            }
            continue;
        }
        if (kFresh) {
            // empty record: ids 0xFFFF, values and npix 0
#pragma unroll
            for (int i = 0; i < RB / 16; ++i) {
                uint4 q = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const int b = 16 * i + 4 * w;  // byte offset of this word
                    uint32_t x = 0u;
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        if (b + 2 * h < 2 * K) x |= 0xFFFFu << (16 * h);
                    (w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w) = x;
                }
                my_rec[i] = q;
            }
#pragma unroll
            for (int i = 0; i < K / 4; ++i) my_np[i] = make_uint2(0u, 0u);
        } else {
#pragma unroll
            for (int i = 0; i < RB / 16; ++i) my_rec[i] = g_rec[i];
#pragma unroll
            for (int i = 0; i < K / 4; ++i) my_np[i] = g_np[i];
        }
        uint16_t* ids = reinterpret_cast<uint16_t*>(my_rec);
        VT* vals = reinterpret_cast<VT*>(reinterpret_cast<uint8_t*>(my_rec) + 2 * K);
        uint16_t* np = reinterpret_cast<uint16_t*>(my_np);
        int m_old = 0;
        if (!kFresh)
            while (m_old < K && ids[m_old] != DARE_EMPTY_FRAME) ++m_old;
        const VoxelEntries E{buckets + v * kBucket, entries, c, s, c + (e - s)};
        count[v] = 0;
        uint32_t tot_sum, tot_cnt;
        bool over;
        if (E.n == c) {
            unsigned long long ev[kBucket];
            bucket_sort(b, c, ev);
            over = voxel_merge_sorted<K, VT>(E, ev, m_old, ids, vals, np, tot_sum, tot_cnt);
        } else {
            over = voxel_merge<K, VT>(E, m_old, ids, vals, np, tot_sum, tot_cnt);
        }
#pragma unroll
        for (int i = 0; i < RB / 16; ++i) g_rec[i] = my_rec[i];
#pragma unroll
        for (int i = 0; i < K / 4; ++i) g_np[i] = my_np[i];
        if (scal_sum) {
            scal_sum[v] = kMode == 2 ? tot_sum : scal_sum[v] + tot_sum;
            scal_cnt[v] = kMode == 2 ? tot_cnt : scal_cnt[v] + tot_cnt;
        }
        if (over) atomicAdd(overflow, 1ull);
    }
}

// Empty record of a voxel: ids 0xFFFF, values 0.
template <int K, int RB>
__device__ __forceinline__ void empty_record(uint4* r) {
#pragma unroll
    for (int i = 0; i < RB / 16; ++i) {
        uint4 q = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int b = 16 * i + 4 * w;
            uint32_t x = 0u;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (b + 2 * h < 2 * K) x |= 0xFFFFu << (16 * h);
            (w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w) = x;
        }
        r[i] = q;
    }
}

// Shared -> global bulk copy (the asynchronous copy engine), one thread.
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
    const uint32_t saddr = static_cast<uint32_t>(__cvta_generic_to_shared(ssrc));
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 :: "l"(gdst), "r"(saddr), "r"(bytes) : "memory");
}

// Finalize writing every voxel (mode 2: the volume has not been cleared since
// a reset).  A CTA takes runs of 256 consecutive voxels; each thread builds its
// voxel's record and npix row in shared memory (the empty ones too), then the
// whole run (20 KB of f32 K=12 records) goes out in one piece: with kBulk (the
// volume in device memory) by two bulk copies from one thread, otherwise (a
// volume in mapped host memory) by all threads in consecutive 16-byte stores,
// so the host link sees whole lines.  A run shorter than 256 voxels (the
// grid's tail) is stored thread by thread.
// A voxel's counter and bucket are loaded in one round trip, empty buckets too;
// kSparse (a build of few pixels per voxel, where most buckets are empty) loads
// only the bucket's used 16-byte pairs once the counter is in: a second round
// trip, but none of the empty buckets' bytes (400 frames into 256^3: 0.43 ->
// 0.37 ms; 1600 frames: 0.439 -> 0.446 ms, so not taken there).
// 6 CTAs per SM (40 registers)
template <int K, typename VT, bool kBulk, bool kSparse>
__global__ void __launch_bounds__(256, 6) k_finalize_full(int32_t* __restrict__ count,
                                                       const unsigned long long* __restrict__ buckets,
                                                       const int32_t* __restrict__ offsets,
                                                       const unsigned long long* __restrict__ entries,
                                                       int64_t n_vox, uint8_t* __restrict__ rec,
                                                       uint16_t* __restrict__ npix, uint32_t* __restrict__ scal_sum,
                                                       uint32_t* __restrict__ scal_cnt,
                                                       unsigned long long* overflow, int32_t* __restrict__ deferred,
                                                       int32_t* __restrict__ deferred_cnt,
                                                       int32_t* __restrict__ n_deferred) {
    constexpr int RB = (2 * K + K * static_cast<int>(sizeof(VT)) + 15) / 16 * 16;
    __shared__ __align__(128) uint4 s_rec[256 * RB / 16];
    __shared__ __align__(128) uint2 s_np[256 * K / 4];
    uint4* my_rec = s_rec + threadIdx.x * (RB / 16);
    uint2* my_np = s_np + threadIdx.x * (K / 4);
    for (int64_t v0 = static_cast<int64_t>(blockIdx.x) * 256; v0 < n_vox; v0 += static_cast<int64_t>(gridDim.x) * 256) {
        const int64_t v = v0 + threadIdx.x;
        const bool whole = n_vox - v0 >= 256;  // block-uniform
        if (v < n_vox) {
            empty_record<K, RB>(my_rec);
#pragma unroll
            for (int i = 0; i < K / 4; ++i) my_np[i] = make_uint2(0u, 0u);
            // the counter (all of the voxel's entries: in this mode the place
            // pass does not count it down) and the whole bucket in one round trip
            const int n_all = count[v];
            ulonglong2 b[kBucket / 2];
            if constexpr (kSparse) {
                const ulonglong2* q = reinterpret_cast<const ulonglong2*>(buckets + v * kBucket);
#pragma unroll
                for (int i = 0; i < kBucket / 2; ++i)
                    b[i] = (2 * i < n_all && n_all <= kBucket) ? __ldg(q + i) : make_ulonglong2(0ull, 0ull);
            } else {
                bucket_load(buckets + v * kBucket, b);
            }
            uint32_t tot_sum = 0, tot_cnt = 0;
            bool over = false;
            if (n_all > kBucket) {
                // entries past the bucket (rare, clustered): left to k_finalize_deferred, a
                // thread per voxel, so that no thread holds its CTA at the barrier below; the
                // empty record written here is overwritten there.  The list takes the voxel and
                // its entry count; the counter is cleared here, with the others.
                const int i = atomicAdd(n_deferred, 1);
                deferred[i] = static_cast<int32_t>(v);
                deferred_cnt[i] = n_all;
                count[v] = 0;
            } else if (n_all > 0) {
                const VoxelEntries E{buckets + v * kBucket, entries, n_all, 0, n_all};
                count[v] = 0;
                uint16_t* ids = reinterpret_cast<uint16_t*>(my_rec);
                VT* vals = reinterpret_cast<VT*>(reinterpret_cast<uint8_t*>(my_rec) + 2 * K);
                uint16_t* np = reinterpret_cast<uint16_t*>(my_np);
                unsigned long long ev[kBucket];
                bucket_sort(b, n_all, ev);
                over = voxel_merge_sorted<K, VT>(E, ev, 0, ids, vals, np, tot_sum, tot_cnt);
            }
            if (!whole) {
                uint4* g_rec = reinterpret_cast<uint4*>(rec + v * RB);
                uint2* g_np = reinterpret_cast<uint2*>(npix + v * K);
#pragma unroll
                for (int i = 0; i < RB / 16; ++i) g_rec[i] = my_rec[i];
#pragma unroll
                for (int i = 0; i < K / 4; ++i) g_np[i] = my_np[i];
            }
            if (scal_sum) {
                scal_sum[v] = tot_sum;
                scal_cnt[v] = tot_cnt;
            }
            if (over) atomicAdd(overflow, 1ull);
        }
        if (whole) {
            __syncthreads();  // the run's records and npix rows are in shared memory
            if constexpr (kBulk) {
                if (threadIdx.x == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    // offsets are multiples of 256 records and 256 npix rows: 16-byte aligned, sizes multiples of 16
                    bulk_store(rec + v0 * RB, s_rec, 256u * RB);
                    bulk_store(npix + v0 * K, s_np, 256u * K * 2u);
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // shared memory free again
                }
            } else {
                uint4* g_rec = reinterpret_cast<uint4*>(rec + v0 * RB);
                for (int i = threadIdx.x; i < 256 * RB / 16; i += 256) g_rec[i] = s_rec[i];
                uint4* g_np = reinterpret_cast<uint4*>(npix + v0 * K);
                const uint4* s_np4 = reinterpret_cast<const uint4*>(s_np);
                for (int i = threadIdx.x; i < 256 * K * 2 / 16; i += 256) g_np[i] = s_np4[i];
            }
            // only a CTA with another run waits here: otherwise the other warps exit
            // while thread 0 waits for its copies to leave shared memory
            if (v0 + static_cast<int64_t>(gridDim.x) * 256 < n_vox) __syncthreads();
        }
    }
    // Each run already waited until its copies had read shared memory; their
    // global writes complete with the grid, so the CTA exits without waiting.
}

// Voxels the full-write finalize deferred (entries past their bucket: about 3 %
// of the working volume's covered voxels), one thread each, without barriers.
// Up to kDeferSort entries are loaded together into registers, sorted by a
// bitonic network and merged in one pass (a frame split across tiles summed);
// more entries, or more samples than K (the capacity rule), take the general
// merge.  The record and npix row are staged in shared memory and stored whole
// over the empty ones the full-write pass left; the scalar totals sum every entry.
constexpr int kDeferSort = 16;

__device__ __forceinline__ void sort16(unsigned long long (&e)[kDeferSort]) {
#pragma unroll
    for (int k = 2; k <= kDeferSort; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < kDeferSort; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long a = e[i], b = e[l];
                    const bool swap = ((i & k) == 0) ? (a > b) : (a < b);
                    e[i] = swap ? b : a;
                    e[l] = swap ? a : b;
                }
            }
}

template <int K, typename VT>
__global__ void __launch_bounds__(256) k_finalize_deferred(const int32_t* __restrict__ deferred,
                                                         const int32_t* __restrict__ deferred_cnt,
                                                         const int32_t* __restrict__ n_deferred,
                                                         const unsigned long long* __restrict__ buckets,
                                                         const int32_t* __restrict__ offsets,
                                                         const unsigned long long* __restrict__ entries,
                                                         uint8_t* __restrict__ rec, uint16_t* __restrict__ npix,
                                                         uint32_t* __restrict__ scal_sum,
                                                         uint32_t* __restrict__ scal_cnt,
                                                         unsigned long long* overflow) {
    constexpr int RB = (2 * K + K * static_cast<int>(sizeof(VT)) + 15) / 16 * 16;
    __shared__ __align__(16) uint4 s_rec[256 * RB / 16];
    __shared__ __align__(16) uint2 s_np[256 * K / 4];
    uint4* my_rec = s_rec + threadIdx.x * (RB / 16);
    uint2* my_np = s_np + threadIdx.x * (K / 4);
    uint16_t* ids = reinterpret_cast<uint16_t*>(my_rec);
    VT* vals = reinterpret_cast<VT*>(reinterpret_cast<uint8_t*>(my_rec) + 2 * K);
    uint16_t* np = reinterpret_cast<uint16_t*>(my_np);
    const int n_items = *n_deferred;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < n_items; it += gridDim.x * blockDim.x) {
        const int64_t v = deferred[it];
        const int n = deferred_cnt[it], s0 = offsets[v];  // all entries; the first kBucket in the bucket
        empty_record<K, RB>(my_rec);
#pragma unroll
        for (int i = 0; i < K / 4; ++i) my_np[i] = make_uint2(0u, 0u);
        const VoxelEntries E{buckets + v * kBucket, entries, kBucket, s0, n};
        uint32_t ts = 0, tc = 0;
        bool over = false;
        bool done = false;
        if (n <= kDeferSort) {
            unsigned long long e[kDeferSort];
#pragma unroll
            for (int j = 0; j < kDeferSort; ++j)
                e[j] = j < kBucket ? __ldg(E.bucket + j) : (j < n ? __ldg(entries + s0 + (j - kBucket)) : ~0ull);
#pragma unroll
            for (int j = 0; j < kDeferSort; ++j)
                if (j < n) {
                    ts += static_cast<uint32_t>(ent_sum(e[j]));
                    tc += static_cast<uint32_t>(ent_npix(e[j]));
                }
            sort16(e);
            done = append_sorted<K, VT, kDeferSort>(e, 0, ids, vals, np) >= 0;
            if (!done) {  // more than K samples: redone by the general merge below
                empty_record<K, RB>(my_rec);
#pragma unroll
                for (int i = 0; i < K / 4; ++i) my_np[i] = make_uint2(0u, 0u);
            }
        }
        if (!done) over = voxel_merge<K, VT>(E, 0, ids, vals, np, ts, tc);
        uint4* g_rec = reinterpret_cast<uint4*>(rec + v * RB);
        uint2* g_np = reinterpret_cast<uint2*>(npix + v * K);
#pragma unroll
        for (int i = 0; i < RB / 16; ++i) g_rec[i] = my_rec[i];
#pragma unroll
        for (int i = 0; i < K / 4; ++i) g_np[i] = my_np[i];
        if (scal_sum) {
            scal_sum[v] = ts;
            scal_cnt[v] = tc;
        }
        if (over) atomicAdd(overflow, 1ull);
    }
}

template <int K, typename VT>
cudaError_t finalize_full_v(int32_t* cnt, const unsigned long long* bk, const int32_t* off,
                            const unsigned long long* ent, int64_t n_vox, uint8_t* rec, uint16_t* npix, uint32_t* ss,
                            uint32_t* sc, unsigned long long* ovf, bool bulk, bool sparse, int32_t* dl, int32_t* dc,
                            int32_t* dn, cudaStream_t st) {
    const int64_t want = (n_vox + 255) / 256;
    const int blocks = static_cast<int>(want < (1 << 30) ? want : (1 << 30));  // one run per CTA
    if (bulk && sparse)
        k_finalize_full<K, VT, true, true><<<blocks, 256, 0, st>>>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, ovf, dl, dc, dn);
    else if (bulk)
        k_finalize_full<K, VT, true, false><<<blocks, 256, 0, st>>>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, ovf, dl, dc, dn);
    else  // a volume in mapped host memory: bound by the host link, not by these loads
        k_finalize_full<K, VT, false, false><<<blocks, 256, 0, st>>>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, ovf, dl, dc, dn);
    return cudaPeekAtLastError();
}

template <int K, typename VT>
cudaError_t finalize_deferred_v(const int32_t* dl, const int32_t* dc, const int32_t* dn, const unsigned long long* bk,
                                const int32_t* off,
                                const unsigned long long* ent, uint8_t* rec, uint16_t* npix, uint32_t* ss,
                                uint32_t* sc, unsigned long long* ovf, int64_t max_items, cudaStream_t st) {
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaErrorInvalidDevice;
    // a thread per listed voxel up to 16 CTAs of 256 per SM, then grid-stride
    const int64_t want = std::max<int64_t>(1, (max_items + 255) / 256);
    const int blocks = static_cast<int>(std::min<int64_t>(want, int64_t(sms[dev]) * 16));
    k_finalize_deferred<K, VT><<<blocks, 256, 0, st>>>(dl, dc, dn, bk, off, ent, rec, npix, ss, sc, ovf);
    return cudaPeekAtLastError();
}

template <int K>
cudaError_t finalize_deferred_k(const int32_t* dl, const int32_t* dc, const int32_t* dn, const unsigned long long* bk, const int32_t* off,
                                const unsigned long long* ent, uint8_t* rec, uint16_t* npix, uint32_t* ss,
                                uint32_t* sc, int dtype, unsigned long long* ovf, int64_t max_items, cudaStream_t st) {
    switch (dtype) {
    case DARE_U8: return finalize_deferred_v<K, uint8_t>(dl, dc, dn, bk, off, ent, rec, npix, ss, sc, ovf, max_items, st);
    case DARE_F16: return finalize_deferred_v<K, __half>(dl, dc, dn, bk, off, ent, rec, npix, ss, sc, ovf, max_items, st);
    case DARE_BF16:
        return finalize_deferred_v<K, __nv_bfloat16>(dl, dc, dn, bk, off, ent, rec, npix, ss, sc, ovf, max_items, st);
    case DARE_F32: return finalize_deferred_v<K, float>(dl, dc, dn, bk, off, ent, rec, npix, ss, sc, ovf, max_items, st);
    }
    return cudaErrorInvalidValue;
}

template <int K, int kMode>
cudaError_t finalize_kf(int32_t* cnt, const unsigned long long* bk, const int32_t* off,
                        const unsigned long long* ent, int64_t n_vox, uint8_t* rec, uint16_t* npix, uint32_t* ss,
                        uint32_t* sc, int dtype, unsigned long long* ovf, const int32_t* tl, const int32_t* tn,
                        int64_t max_t, cudaStream_t st) {
    const int threads = 256;
    const int64_t want = ((tl ? max_t : n_vox) + threads - 1) / threads;
    const int blocks = static_cast<int>(want < 148 * 64 ? want : 148 * 64);
    switch (dtype) {
    case DARE_U8:
        k_finalize<K, uint8_t, kMode><<<blocks, threads, 0, st>>>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, ovf, tl,
                                                               tn);
        break;
    case DARE_F16:
        k_finalize<K, __half, kMode><<<blocks, threads, 0, st>>>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, ovf, tl,
                                                               tn);
        break;
    case DARE_BF16:
        k_finalize<K, __nv_bfloat16, kMode><<<blocks, threads, 0, st>>>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, ovf, tl,
                                                               tn);
        break;
    case DARE_F32:
        k_finalize<K, float, kMode><<<blocks, threads, 0, st>>>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, ovf, tl,
                                                               tn);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaPeekAtLastError();
}

template <int K>
cudaError_t finalize_k(int32_t* cnt, const unsigned long long* bk, const int32_t* off, const unsigned long long* ent,
                       int64_t n_vox, uint8_t* rec, uint16_t* npix, uint32_t* ss, uint32_t* sc, int dtype, int mode,
                       int bulk, int sparse_in, unsigned long long* ovf, const int32_t* tl, const int32_t* tn,
                       int64_t max_t, int32_t* dl, int32_t* dc, int32_t* dn, cudaStream_t st) {
    if (mode == 2 && (tl || !dl || !dc || !dn)) return cudaErrorInvalidValue;  // a full write visits every voxel
    if (mode == 2) {
        const bool b = bulk != 0, sparse = sparse_in != 0;
        switch (dtype) {
        case DARE_U8: return finalize_full_v<K, uint8_t>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, ovf, b, sparse, dl, dc, dn, st);
        case DARE_F16: return finalize_full_v<K, __half>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, ovf, b, sparse, dl, dc, dn, st);
        case DARE_BF16:
            return finalize_full_v<K, __nv_bfloat16>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, ovf, b, sparse, dl, dc, dn, st);
        case DARE_F32: return finalize_full_v<K, float>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, ovf, b, sparse, dl, dc, dn, st);
        }
        return cudaErrorInvalidValue;
    }
    switch (mode) {
    case 0: return finalize_kf<K, 0>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, dtype, ovf, tl, tn, max_t, st);
    case 1: return finalize_kf<K, 1>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, dtype, ovf, tl, tn, max_t, st);
    case 2: return finalize_kf<K, 2>(cnt, bk, off, ent, n_vox, rec, npix, ss, sc, dtype, ovf, nullptr, nullptr, 0, st);
    }
    return cudaErrorInvalidValue;
}

// (tile column, tile row, frame); tiles numbered in that order
dim3 scatter_grid(const ScatterArgs& a) {
    return dim3((a.width + kTile - 1) / kTile, (a.height + kTile - 1) / kTile, a.n);
}

}  // namespace

cudaError_t launch_scatter_count(const ScatterArgs& a, int32_t* count, unsigned long long* buckets, uint4* pairs,
                                 int32_t* n_pairs, int32_t* touched, int32_t* tindex, int32_t* n_touched,
                                 cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    if (touched)
        k_scatter_count<true><<<scatter_grid(a), kThreads, 0, st>>>(a, count, buckets, pairs, n_pairs, touched, tindex,
                                                                    n_touched);
    else  // every voxel's list is visited anyway: the 32 x 64 form
        k_scatter_count2<<<dim3((a.width + kTile - 1) / kTile, (a.height + kRows2 - 1) / kRows2, a.n), kThreads, 0,
                           st>>>(a, count, buckets, pairs, n_pairs);
    return cudaPeekAtLastError();
}

cudaError_t launch_touched_overflow(const int32_t* count, const int32_t* touched, const int32_t* n_touched,
                                    int64_t max_t, int32_t* ovf_cnt, cudaStream_t st) {
    if (max_t <= 0) return cudaSuccess;
    const int64_t want = (max_t + 255) / 256;
    const int blocks = static_cast<int>(want < 148 * 16 ? want : 148 * 16);
    k_touched_overflow<<<blocks, 256, 0, st>>>(count, touched, n_touched, max_t, ovf_cnt);
    return cudaPeekAtLastError();
}

cudaError_t launch_scatter_place(const ScatterArgs& a, const uint4* pairs, const int32_t* n_pairs, int32_t* count,
                                 const int32_t* offsets, const int32_t* tindex, unsigned long long* entries,
                                 cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaErrorInvalidDevice;
    k_scatter_place<<<sms[dev] * 2, 256, 0, st>>>(pairs, n_pairs, count, offsets, tindex, entries);
    return cudaPeekAtLastError();
}

cudaError_t launch_overflow_alloc(const uint4* pairs, const int32_t* n_pairs, const int32_t* count, int32_t* offsets,
                                  int32_t* cursor, cudaStream_t st) {
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaErrorInvalidDevice;
    k_overflow_alloc<<<sms[dev] * 2, 256, 0, st>>>(pairs, n_pairs, count, offsets, cursor);
    return cudaPeekAtLastError();
}

cudaError_t launch_overflow_place(const uint4* pairs, const int32_t* n_pairs, const int32_t* offsets,
                                  unsigned long long* entries, cudaStream_t st) {
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaErrorInvalidDevice;
    k_overflow_place<<<sms[dev] * 2, 256, 0, st>>>(pairs, n_pairs, offsets, entries);
    return cudaPeekAtLastError();
}

cudaError_t launch_finalize_deferred(const int32_t* deferred, const int32_t* deferred_cnt, const int32_t* n_deferred,
                                     const unsigned long long* buckets, const int32_t* offsets,
                                     const unsigned long long* entries, uint8_t* rec, uint16_t* npix,
                                     uint32_t* scal_sum, uint32_t* scal_cnt, int K, int dtype,
                                     unsigned long long* overflow, int64_t max_items, cudaStream_t st) {
    switch (K) {
    case 4: return finalize_deferred_k<4>(deferred, deferred_cnt, n_deferred, buckets, offsets, entries, rec, npix, scal_sum, scal_cnt, dtype, overflow, max_items, st);
    case 8: return finalize_deferred_k<8>(deferred, deferred_cnt, n_deferred, buckets, offsets, entries, rec, npix, scal_sum, scal_cnt, dtype, overflow, max_items, st);
    case 12: return finalize_deferred_k<12>(deferred, deferred_cnt, n_deferred, buckets, offsets, entries, rec, npix, scal_sum, scal_cnt, dtype, overflow, max_items, st);
    case 16: return finalize_deferred_k<16>(deferred, deferred_cnt, n_deferred, buckets, offsets, entries, rec, npix, scal_sum, scal_cnt, dtype, overflow, max_items, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_finalize(int32_t* count, const unsigned long long* buckets, const int32_t* offsets,
                            const unsigned long long* entries, int64_t n_vox, uint8_t* rec, uint16_t* npix,
                            uint32_t* scal_sum, uint32_t* scal_cnt, int K, int dtype, int mode, int bulk,
                            int sparse, unsigned long long* overflow, const int32_t* touched, const int32_t* n_touched,
                            int64_t max_t, int32_t* deferred, int32_t* deferred_cnt, int32_t* n_deferred, cudaStream_t st) {
    int32_t* dl = deferred;
    int32_t* dc = deferred_cnt;
    int32_t* dn = n_deferred;
    const int32_t* tl = touched;
    const int32_t* tn = n_touched;
    switch (K) {
    case 4: return finalize_k<4>(count, buckets, offsets, entries, n_vox, rec, npix, scal_sum, scal_cnt, dtype, mode, bulk, sparse, overflow, tl, tn, max_t, dl, dc, dn, st);
    case 8: return finalize_k<8>(count, buckets, offsets, entries, n_vox, rec, npix, scal_sum, scal_cnt, dtype, mode, bulk, sparse, overflow, tl, tn, max_t, dl, dc, dn, st);
    case 12: return finalize_k<12>(count, buckets, offsets, entries, n_vox, rec, npix, scal_sum, scal_cnt, dtype, mode, bulk, sparse, overflow, tl, tn, max_t, dl, dc, dn, st);
    case 16: return finalize_k<16>(count, buckets, offsets, entries, n_vox, rec, npix, scal_sum, scal_cnt, dtype, mode, bulk, sparse, overflow, tl, tn, max_t, dl, dc, dn, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dare
