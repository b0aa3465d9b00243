// Brick paging for volumes beyond device memory (Sec. 4: growing datasets
// despite GPU memory limits) on sm_103a.
//
// The records live in page-locked host memory mapped into the device
// (DARE_SESSION_HOST_VOLUME).  A device cache holds whole 8^3-voxel bricks of
// records, slot by slot; table[brick] is the brick's slot or -1.  Before a
// plane is resliced the host pages in the bricks of its footprint that are
// not resident (k_page_in copies them from the mapped host records, reading
// the host link with coalesced 16-byte loads).  The reslice gathers per pixel
// over the distance kernel's support and reads each voxel's record from its
// brick's slot, or over the host link when the brick is not resident: the
// result never depends on what the cache holds (the same arithmetic either
// way), only the speed does.
#include <cfloat>

#include "dare_internal.h"
#include "device_common.cuh"

namespace dare {
namespace {

using namespace dev;

__device__ __forceinline__ float tent_factor(float d, float R) { return 1.0f - __fdiv_rn(fabsf(d), R); }
__device__ __forceinline__ float exp_weight(float d2, float kr) { return expf(-kr * sqrtf(d2)); }

// Table updates (brick, slot): evictions carry slot -1; bricks are distinct.
__global__ void k_table_set(const int2* __restrict__ upd, int n, int32_t* __restrict__ table) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) table[upd[i].x] = upd[i].y;
}

// One CTA per paged-in brick: its in-grid voxels' records, host -> slot.
__global__ void __launch_bounds__(256) k_page_in(const int2* __restrict__ pages, const uint4* __restrict__ host_rec,
                                                 uint4* __restrict__ cache, int3 dims, int3 nb, int vec) {
    const int2 pg = pages[blockIdx.x];
    const int brick = pg.x;
    const int bx = brick % nb.x, by = (brick / nb.x) % nb.y, bz = brick / (nb.x * nb.y);
    uint4* dst = cache + static_cast<int64_t>(pg.y) * kBrickVoxels * vec;
    for (int i = threadIdx.x; i < kBrickVoxels * vec; i += blockDim.x) {
        const int l = i / vec, c = i - l * vec;
        const int x = bx * kBrickSide + (l & (kBrickSide - 1));
        const int y = by * kBrickSide + ((l / kBrickSide) & (kBrickSide - 1));
        const int z = bz * kBrickSide + l / (kBrickSide * kBrickSide);
        if (x >= dims.x || y >= dims.y || z >= dims.z) continue;  // outside the grid: never read
        const int64_t vi = x + static_cast<int64_t>(dims.x) * (y + static_cast<int64_t>(dims.y) * z);
        dst[i] = host_rec[vi * vec + c];
    }
}

// Per-pixel gather over the support, records from the brick cache (or the
// mapped host volume for bricks that are not resident).
template <int K, typename VT, typename WT>
__device__ __noinline__ float2 gather_pixel_paged(const PagedJob& P, int u, int v) {
    float num = 0.0f, den = 0.0f;
    const ResliceJob& J = P.j;
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
                const int brick = static_cast<int>(cx >> 3) +
                                  P.nb[0] * (static_cast<int>(cy >> 3) + P.nb[1] * static_cast<int>(cz >> 3));
                const int slot = __ldg(P.table + brick);
                float2 ab;
                if (slot >= 0) {
                    const int64_t l = (cx & 7) + 8 * ((cy & 7) + 8 * (cz & 7));
                    ab = collapse_voxel<K, VT, WT>(P.cache, static_cast<int64_t>(slot) * kBrickVoxels + l, wt);
                } else {
                    const int64_t vi =
                        cx + static_cast<int64_t>(J.dims[0]) * (cy + static_cast<int64_t>(J.dims[1]) * cz);
                    ab = collapse_voxel<K, VT, WT>(J.rec, vi, wt);
                }
                num = fmaf(t, ab.x, num);
                den = fmaf(t, ab.y, den);
            }
        }
    }
    return make_float2(num, den);
}

template <int K, typename VT, typename WT>
__device__ __forceinline__ void paged_body(const PagedJob& P) {
    const ResliceJob& J = P.j;
    const int lane = threadIdx.x;
    const int u = blockIdx.x * 32 + lane;
    const int v = blockIdx.y * 8 + threadIdx.y;
    if (v >= J.height || static_cast<int>(blockIdx.x) * 32 >= J.width) return;  // warp-uniform
    const bool active = u < J.width;
    float num = 0.0f, den = 0.0f;
    if (active) {
        const float2 nd = gather_pixel_paged<K, VT, WT>(P, u, v);
        num = nd.x;
        den = nd.y;
        J.out[static_cast<int64_t>(v) * J.width + u] = den > 0.0f ? num / den : J.unassigned;
    }
    const unsigned bits = __ballot_sync(0xFFFFFFFFu, active && den > 0.0f);
    if (lane == 0) J.mask[static_cast<int64_t>(v) * J.mask_stride + blockIdx.x] = bits;
}

template <int K, typename VT, typename WT>
__global__ void __launch_bounds__(256) k_reslice_paged(const __grid_constant__ PagedJob P) {
    paged_body<K, VT, WT>(P);
}

// planes of one paged group (their bricks paged in together), one per grid z
template <int K, typename VT, typename WT>
__global__ void __launch_bounds__(256) k_reslice_paged_batch(const PagedJob* __restrict__ jobs) {
    paged_body<K, VT, WT>(jobs[blockIdx.z]);
}

template <int K, typename VT>
cudaError_t launch_p(const PagedJob* jobs_dev, const PagedJob* one, int n_jobs, int max_w, int max_h, int half_w,
                     cudaStream_t st) {
    const dim3 block(32, 8);
    const dim3 grid((max_w + 31) / 32, (max_h + 7) / 8, one ? 1 : n_jobs);
    if (one) {
        if (half_w)
            k_reslice_paged<K, VT, __half><<<grid, block, 0, st>>>(*one);
        else
            k_reslice_paged<K, VT, float><<<grid, block, 0, st>>>(*one);
    } else {
        if (half_w)
            k_reslice_paged_batch<K, VT, __half><<<grid, block, 0, st>>>(jobs_dev);
        else
            k_reslice_paged_batch<K, VT, float><<<grid, block, 0, st>>>(jobs_dev);
    }
    return cudaPeekAtLastError();
}

template <int K>
cudaError_t launch_p_k(const PagedJob* jobs_dev, const PagedJob* one, int n_jobs, int max_w, int max_h, int dtype,
                       int half_w, cudaStream_t st) {
    switch (dtype) {
    case DARE_U8: return launch_p<K, uint8_t>(jobs_dev, one, n_jobs, max_w, max_h, half_w, st);
    case DARE_F16: return launch_p<K, __half>(jobs_dev, one, n_jobs, max_w, max_h, half_w, st);
    case DARE_BF16: return launch_p<K, __nv_bfloat16>(jobs_dev, one, n_jobs, max_w, max_h, half_w, st);
    case DARE_F32: return launch_p<K, float>(jobs_dev, one, n_jobs, max_w, max_h, half_w, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_page_in(const int2* updates, int n_updates, const int2* pages, int n_pages, const uint8_t* host_rec,
                           uint8_t* cache, const int32_t dims[3], const int32_t nb[3], int rec_bytes, int32_t* table,
                           cudaStream_t st) {
    if (n_pages > 0) {
        k_page_in<<<n_pages, 256, 0, st>>>(pages, reinterpret_cast<const uint4*>(host_rec),
                                           reinterpret_cast<uint4*>(cache), make_int3(dims[0], dims[1], dims[2]),
                                           make_int3(nb[0], nb[1], nb[2]), rec_bytes / 16);
        cudaError_t e = cudaPeekAtLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_updates > 0) k_table_set<<<(n_updates + 255) / 256, 256, 0, st>>>(updates, n_updates, table);
    return cudaPeekAtLastError();
}

cudaError_t launch_reslice_paged(const PagedJob* jobs_dev, const PagedJob* one_job, int n_jobs, int max_w, int max_h,
                                 int K, int dtype, int half_weights, cudaStream_t st) {
    if (n_jobs <= 0 || max_w <= 0 || max_h <= 0) return cudaSuccess;
    if (!one_job && n_jobs > 65535) return cudaErrorInvalidValue;
    switch (K) {
    case 4: return launch_p_k<4>(jobs_dev, one_job, n_jobs, max_w, max_h, dtype, half_weights, st);
    case 8: return launch_p_k<8>(jobs_dev, one_job, n_jobs, max_w, max_h, dtype, half_weights, st);
    case 12: return launch_p_k<12>(jobs_dev, one_job, n_jobs, max_w, max_h, dtype, half_weights, st);
    case 16: return launch_p_k<16>(jobs_dev, one_job, n_jobs, max_w, max_h, dtype, half_weights, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dare
