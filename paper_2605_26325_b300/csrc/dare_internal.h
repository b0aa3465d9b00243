// Internal types shared by the host side (api.cpp) and the kernels (*.cu).
//
// Device record layout (one per voxel, 16-byte aligned, stride rec_bytes =
// round_up(2 K + K sizeof(value), 16)):
//   bytes [0, 2K)          K frame ids, uint16, ascending, 0xFFFF = empty (last)
//   bytes [2K, 2K + K vb)  K stored intensities of the storage type
// The build-only npix plane holds K uint16 per voxel in a separate array.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/dare.h"

namespace dare {

constexpr int kFixBits = DARE_FIX_BITS;
constexpr int64_t kFixOne = int64_t(1) << kFixBits;
constexpr int kMaxPixelsPerChunk = 1 << 28;  // pixels of one scatter pass (one 8-byte entry and one 16-byte pair per pixel at most)
constexpr int kScatterTile = 32;              // frame tiles of the scatter passes: 32 x 32 pixels
constexpr int kBucket = 8;                    // entries per voxel the count pass stores in place (8 bytes each)

inline int value_bytes(int dtype) { return dtype == DARE_U8 ? 1 : (dtype == DARE_F32 ? 4 : 2); }
inline int record_bytes(int K, int dtype) { return (2 * K + K * value_bytes(dtype) + 15) / 16 * 16; }

// One plane to reslice, as the kernels see it.
struct ResliceJob {
    int64_t g0[3], a[3], b[3];  // fixed-point pixel -> voxel affine (2^-20 voxel)
    const uint8_t* rec;         // records of the plane's volume
    const void* wtab;           // per-frame weight table (float or __half)
    float* out;                 // height x width
    uint32_t* mask;             // height x mask_stride
    int32_t dims[3];
    int32_t width, height;
    int32_t mask_stride;        // ceil(width / 32)
    int32_t tile_base;          // first tile of this job in a batched launch
    int32_t tiles_x;            // tiles per tile row
    float unassigned;
    // plane geometry for the tiled kernel (host FP64, stored as FP32 with margins):
    // d = axis of the largest normal component in voxel space; on the plane
    // g_d = alpha + beta1 g_e1 + beta2 g_e2; (u, v) = (ou, ov) + M (g_e1, g_e2).
    int32_t d;                  // 0, 1, 2
    int32_t levels;             // level slots per column, floor(2 spread + 0.05) + 3
    int32_t direct;             // 1: every pixel gathers directly (degenerate plane, or no tile height fits)
    int32_t n_frames;           // entries of wtab
    float alpha, beta1, beta2, spread;
    float m00, m01, m10, m11, ou, ov, hu, hv;
    // distance kernel (Sec. 2.1 "Reslicing"): radius R in voxels, TENT / BOX / EXP,
    // EXP rate; a pixel with floor(g) = f reads voxels f - ext_lo .. f + ext_hi
    // per axis at most (TENT, EXP: R - 1, R; BOX: R, R + 1)
    int32_t radius, kernel;
    int32_t ext_lo, ext_hi;
    float k_dist;
    int32_t tile_h;             // rows of the tiled kernel's tiles for this plane (8, 16, 32 or 64)
    const uint16_t* npix;       // per-pixel samples: weight each sample by its npix (general kernels); NULL: 1
};

// Inputs of the per-(plane, frame) weight table of Eq. 1 / Eq. 2.
struct TableJob {
    double n_r[3];          // plane normal (beam or elevation) in the volume frame
    double x_r[3];          // plane lateral direction in the volume frame
    const double* frames;   // n_frames x 9 row-major rotations (volume frame)
    void* wtab;             // output, n_frames entries
    int32_t n_frames;
    int32_t pad;
};

struct TableParams {
    double k_normal, k_inplane;
    double cos_normal, cos_inplane;
    int32_t use_normal, use_inplane;  // thresholds active
    int32_t normal_axis;              // 1: beam column, 2: elevation column
    int32_t half;                     // table in FP16
};

struct ScatterArgs {
    const uint8_t* frames;    // n x H x W
    const int64_t* affines;   // n x 9 (G0, A, B)
    int32_t n, width, height;
    int32_t dims[3];
    int32_t frame_base;       // global id of frame 0 of this chunk
    int32_t small_steps;      // every |A|, |B| < 2^25: tiles step pixels in int32
    int64_t tile_base;        // unused (kept for the layout)
    const uint32_t* pix_mask; // H rows of ceil(W / 32) words, bit set = pixel used; NULL: every pixel
};

// Per-frame probe geometry for curvilinear reslicing, kGeomFloats floats per
// frame (five float4): the voxel -> apex-relative image point rows
// tx, ty (p_x = tx . (i, j, k, 1), likewise p_y), the frame's image axes in
// the volume frame c0 (lateral), c1 (beam), c2 (elevation), the sample side of
// the FP32 error bound k1 (the direction error is at most k1 / |p|), and kind
// (0 linear: tx = 0, ty = (0, 0, 0, 1), k1 = 0; 1 curvilinear).
constexpr int kGeomFloats = 20;

// One plane of a curvilinear reslice (any session whose frames include a
// curvilinear probe, or a curvilinear virtual probe).  Eq. 1 / Eq. 2 are
// evaluated per (pixel, sample) in FP32; a threshold decision within the FP32
// error bound of its cosine is re-taken in FP64 from rot64 / off64.
struct CurvJob {
    ResliceJob j;             // pixel -> voxel map, records, outputs, support (wtab unused)
    const float4* geom;       // per-frame FP32 geometry, 5 float4 per frame
    const double* rot64;      // per-frame rotations in the volume frame (9 FP64, row-major)
    const double* off64;      // per-frame apex-relative offsets (ox, oy) FP64; with rot64 and h:
                              //   p_x = h sum_r R[r][0] c_r + ox, p_y = h sum_r R[r][1] c_r + oy
    double R[9];              // plane rotation in the volume frame, row-major
    double h;                 // grid spacing
    double half_w, sx, sy;    // pixel (u, v) at image point ((u - half_w) sx, v sy)
    double ax, ay;            // virtual fan apex (image mm)
    double cos_n64, cos_i64;  // thresholds
    float Rf[9];
    float oxf, oyf;           // FP32: p = (u sx + oxf, v sy + oyf) relative to the virtual apex
    float sxf, syf;
    float k1p;                // pixel side of the FP32 error bound
    float k_n, k_i;           // Eq. 2
    float cos_n, cos_i;       // thresholds, FP32 copies
    int32_t use_n, use_i;     // thresholds active
    int32_t elevation;        // 1: Eq. 1's normal is the elevation axis
    int32_t curv_out;         // 1: curvilinear virtual probe
    int32_t pad;
};

// ------------------------------------------------------------ launchers (kernels.cu, kernels_build.cu)
cudaError_t launch_weight_tables(const TableJob* jobs_dev, const TableJob* one_job, int n_jobs, int max_frames,
                                 const TableParams& p, cudaStream_t st);
cudaError_t launch_reslice_plain(const ResliceJob* jobs_dev, const ResliceJob* one_job, int n_jobs, int max_w,
                                 int max_h, int K, int dtype, int half_weights, cudaStream_t st);
// count: per-voxel entry counters (zero on entry; finalize returns them to zero); buckets: kBucket
// 8-byte entries per voxel; pairs: the overflow list of 16-byte (voxel, entry) pairs, room for one
// per pixel; *n_pairs: its length (zero before the chunk's first count launch)
// touched (optional): voxels reached for the first time are listed, touched[i] = v and tindex[v] = i
// for i < *n_touched (zero on entry)
cudaError_t launch_scatter_count(const ScatterArgs& a, int32_t* count, unsigned long long* buckets, uint4* pairs,
                                 int32_t* n_pairs, int32_t* touched, int32_t* tindex, int32_t* n_touched,
                                 cudaStream_t st);
// ovf_cnt[i] = max(count[touched[i]] - kBucket, 0) for i < *n_touched, 0 up to max_t
cudaError_t launch_touched_overflow(const int32_t* count, const int32_t* touched, const int32_t* n_touched,
                                    int64_t max_t, int32_t* ovf_cnt, cudaStream_t st);
// overflow pairs into their voxels' ranges (offsets: scan of the overflow counts by voxel, or by
// touched-list position when tindex is given); leaves min(count, kBucket) in the counters
cudaError_t launch_scatter_place(const ScatterArgs& a, const uint4* pairs, const int32_t* n_pairs, int32_t* count,
                                 const int32_t* offsets, const int32_t* tindex, unsigned long long* entries,
                                 cudaStream_t st);
// out[i] = sum_{j < i} max(in[j] - bias, 0), out[n] the total
cudaError_t launch_exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int32_t* block_sums,
                                  int64_t block_sums_len, int bias, cudaStream_t st);
int64_t scan_block_sums_needed(int64_t n);
// mode 0: merge into the stored records; 1: the volume holds no sample (created or
// reset since), stored records are not read; 2: as 1 and not cleared since a reset:
// every voxel's record, npix row and scalar totals are written (empty where no entry)
// bulk: records and npix in device memory, so mode 2 may store whole runs with bulk copies
// sparse (mode 2 with bulk): few pixels per voxel, most buckets empty: a bucket is read only as far as
// its counter says (a second round trip) instead of together with the counter
// a voxel's entries: count[v] (<= kBucket) in its bucket, then entries[offsets[v], offsets[v + 1]);
// count is returned to zero
// touched / n_touched (modes 0 and 1): only the listed voxels, offsets by list position, at most max_t
// deferred / deferred_cnt / n_deferred (mode 2; *n_deferred zero on entry, room for every voxel with
// entries past its bucket): the full-write pass lists such voxels with their entry counts, clears
// their counters and leaves their records empty for launch_finalize_deferred;
// in mode 2 the counters hold every entry (launch_overflow_alloc / _place instead of scan and place)
cudaError_t launch_finalize(int32_t* count, const unsigned long long* buckets, const int32_t* offsets,
                            const unsigned long long* entries, int64_t n_vox, uint8_t* rec, uint16_t* npix,
                            uint32_t* scal_sum, uint32_t* scal_cnt, int K, int dtype, int mode, int bulk,
                            int sparse, unsigned long long* overflow, const int32_t* touched, const int32_t* n_touched,
                            int64_t max_t, int32_t* deferred, int32_t* deferred_cnt, int32_t* n_deferred,
                            cudaStream_t st);
// full-write mode (after a reset), in place of the scan and the counting-down place pass: each
// voxel with entries past its bucket gets a range of count - kBucket overflow entries starting at
// offsets[v] (reserved from *cursor, zero on entry; other offsets are not written) ...
cudaError_t launch_overflow_alloc(const uint4* pairs, const int32_t* n_pairs, const int32_t* count, int32_t* offsets,
                                  int32_t* cursor, cudaStream_t st);
// ... and every overflow pair's entry goes to its range by its slot; the counters keep every
// voxel's entry count
cudaError_t launch_overflow_place(const uint4* pairs, const int32_t* n_pairs, const int32_t* offsets,
                                  unsigned long long* entries, cudaStream_t st);
// the voxels a full-write finalize listed (at most max_items), one thread each: record, npix row,
// scalar totals and the capacity-rule count from all deferred_cnt[i] of the voxel's entries
cudaError_t launch_finalize_deferred(const int32_t* deferred, const int32_t* deferred_cnt, const int32_t* n_deferred,
                                     const unsigned long long* buckets, const int32_t* offsets,
                                     const unsigned long long* entries, uint8_t* rec, uint16_t* npix,
                                     uint32_t* scal_sum, uint32_t* scal_cnt, int K, int dtype,
                                     unsigned long long* overflow, int64_t max_items, cudaStream_t st);
cudaError_t launch_reslice_scalar(const ResliceJob& job, const uint32_t* scal_sum, const uint32_t* scal_cnt,
                                  cudaStream_t st);
cudaError_t launch_footprint(const ResliceJob& job, uint32_t* bitmap, unsigned long long* count, cudaStream_t st);
// hole filling of the compounded volume (NaN = still empty) and the trilinear reslice of such a volume
cudaError_t launch_fill_holes(const int32_t dims[3], int radius, int min_neighbours, const uint32_t* scal_sum,
                              const uint32_t* scal_cnt, float* out, cudaStream_t st);
cudaError_t launch_reslice_values(const ResliceJob& job, const float* values, cudaStream_t st);
cudaError_t launch_fill_records(uint8_t* rec, int64_t n_vox, int rec_bytes, int K, cudaStream_t st);
// L2 read-bandwidth measurement: `reps` passes over `bytes` (multiple of 16) of buf, `blocks` CTAs of 256
cudaError_t launch_l2_read(const void* buf, int64_t bytes, int reps, void* sink, int blocks, cudaStream_t st);

// any radius and distance kernel (kernels_radius.cu): per-pixel gather, and the
// tiled kernel with col_cap columns and slot_cap (A, B) slots of dynamic shared memory
cudaError_t launch_reslice_plain_r(const ResliceJob* jobs_dev, const ResliceJob* one_job, int n_jobs, int max_w,
                                   int max_h, int K, int dtype, int half_weights, cudaStream_t st);
cudaError_t launch_reslice_tiled_r(const ResliceJob* jobs_dev, const ResliceJob* one_job, int n_jobs,
                                   int tile_offset, int n_tiles, int uniform, int col_cap, int slot_cap, int K,
                                   int dtype, int half_weights, cudaStream_t st);
// brick paging (kernels_paged.cu): 8^3-voxel bricks of records in a device cache
constexpr int kBrickSide = 8;
constexpr int kBrickVoxels = kBrickSide * kBrickSide * kBrickSide;
struct PagedJob {
    ResliceJob j;             // rec = the mapped host records (bricks that are not resident)
    const uint8_t* cache;     // slots of kBrickVoxels records, voxel x fastest within the brick
    const int32_t* table;     // per brick: its slot, or -1
    int32_t nb[3];            // bricks per axis
    int32_t pad;
};
// updates: (brick, slot or -1) table writes; pages: (brick, slot) copies host -> cache
cudaError_t launch_page_in(const int2* updates, int n_updates, const int2* pages, int n_pages, const uint8_t* host_rec,
                           uint8_t* cache, const int32_t dims[3], const int32_t nb[3], int rec_bytes, int32_t* table,
                           cudaStream_t st);
// one plane (one_job) or n_jobs planes of a paged group (jobs_dev, grid z)
cudaError_t launch_reslice_paged(const PagedJob* jobs_dev, const PagedJob* one_job, int n_jobs, int max_w, int max_h,
                                 int K, int dtype, int half_weights, cudaStream_t st);

// curvilinear probes (kernels_curv.cu): per-pixel gather with in-kernel Eq. 1 / Eq. 2
cudaError_t launch_reslice_curv(const CurvJob* jobs_dev, const CurvJob* one_job, int n_jobs, int max_w, int max_h,
                                int K, int dtype, cudaStream_t st);
constexpr int kMaxSupport = 9;           // tiled general path: support of at most 9 voxels per axis (R <= 4)
constexpr int kGeneralSmemCap = 200 << 10;  // dynamic shared memory of the general tiled kernel, at most

// tiled kernel (kernels_tiled.cu): 32 x tile_h pixel tiles (tile_h per job); a tile's voxel-column
// box must fit kTiledColMax columns and kTiledSlotMax (A, B) slots of shared memory, or it gathers
// per pixel (counted by read_fallback_tiles)
constexpr int kTileW = 32;
constexpr int kTiledColMax = 1024;
constexpr int kTiledSlotMax = 4096;
// uniform != 0: every job has n_tiles tiles (2-D grid, no job search); after_table != 0: the launch
// directly follows the weight-table kernel on `st` and overlaps its set-up with it (programmatic
// dependent launch; the kernel waits for the table before reading it)
cudaError_t launch_reslice_tiled(const ResliceJob* jobs_dev, const ResliceJob* one_job, int n_jobs,
                                 int tile_offset, int n_tiles, int uniform, int K, int dtype, int half_weights,
                                 int after_table, cudaStream_t st);
// Work queue of the persistent tiled kernel, in device memory: `total` tiles over the jobs'
// tile_base ranges; `next` counts the tiles handed out beyond the first grid-size ones (0 at launch).
struct TileQueue {
    int32_t total;
    int32_t next;
    int32_t pad[2];
};
// persistent form: one CTA per resident slot of the device, tiles taken from the queue
// Kernel-node parameters of the single-plane weight table and tiled reslice,
// for a session's two-node CUDA graph: out->kernelParams points into `args`,
// which must outlive the call that consumes out (node creation or update).
struct NodeArgs {
    const void* null_ptr = nullptr;
    int32_t ints[3] = {0, 0, 0};
    TableJob tj{};
    TableParams tp{};
    ResliceJob rj{};
    void* ptrs[5] = {};
};
cudaError_t weight_table_node(const TableJob& one, int max_frames, const TableParams& p, NodeArgs& args,
                              cudaKernelNodeParams* out);
cudaError_t reslice_tiled_node(const ResliceJob& one, int n_tiles, int K, int dtype, int half_weights, NodeArgs& args,
                               cudaKernelNodeParams* out);
cudaError_t launch_reslice_tiled_persistent(const ResliceJob* jobs_dev, int n_jobs, TileQueue* queue, int K,
                                            int dtype, int half_weights, cudaStream_t st);
// sizes (and loads) the persistent kernel for (K, dtype, weights): before a stream capture launches it
cudaError_t prepare_reslice_tiled_persistent(int K, int dtype, int half_weights);
// tiles that gathered per pixel inside the tiled kernels (kernels_tiled.cu, kernels_radius.cu) since
// the last reset, on the current device
cudaError_t read_fallback_tiles_tiled(unsigned long long* out, bool reset);
cudaError_t read_fallback_tiles_general(unsigned long long* out, bool reset);

// batch helpers and memory accounting (api.cpp), used by the server
// allow_paged: sessions with a brick cache are accepted (dare_reslice_batch runs them plane by plane)
dare_status check_batch(const dare_reslice_req* reqs, int32_t n, const dare_params* params, bool allow_paged = false);
void batch_sizes(const dare_reslice_req* reqs, int32_t n, const dare_params* params, size_t* ws_need,
                 size_t* desc_bytes);
void batch_sizes_bound(int32_t n, int32_t max_frames, size_t* ws_need, size_t* desc_bytes);
int session_max_frames(dare_session s);
dare_status queue_batch(const dare_reslice_req* reqs, int32_t n, const dare_params* params, cudaStream_t st,
                        uint8_t* ws, uint8_t* pin);
dare_status reserve_bytes(int64_t bytes);
void release_bytes(int64_t bytes);

// a clear deferred by dare_session_reset, queued and ordered before work on st (server batches)
dare_status settle_session(dare_session s, cudaStream_t st);

// allocation-free reslice support (api.cpp)
dare_status set_error(dare_status st, const char* msg);
int session_device(dare_session s);
dare_status reslice_with_table(dare_session s, const dare_plane* plane, const dare_params* params, float* out_dev,
                               uint32_t* mask_dev, void* stream, void* wtab, size_t wtab_bytes, int max_frames);
constexpr int kTileH = 64;  // largest tile height of the tiled kernel

}  // namespace dare
