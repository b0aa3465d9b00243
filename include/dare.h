/*
 * dare.h -- C ABI of libdare, a CUDA (sm_103a) implementation of DARE,
 * Directionality-Aware Reslicing of tracked freehand ultrasound
 * (Jaeggi, Black, Salcudean).
 *
 * DARE has two operations:
 *   - reconstruction (Sec. 2.1 "Volume reconstruction", Fig. 1): tracked 2D
 *     frames are placed at their poses and voxelised; every voxel keeps a
 *     list of samples, each an intensity with the orientation of the frame it
 *     came from;
 *   - reslicing (Sec. 2.1 "Reslicing", Eq. 1, Eq. 2, Fig. 2): every pixel of a
 *     virtual plane gathers the samples of its voxel neighbourhood, drops
 *     samples whose orientation disagrees with the plane's beyond angular
 *     thresholds, and averages the rest with exponential orientation weights
 *     (times a distance weight); a pixel with no valid sample is unassigned.
 *
 * ---------------------------------------------------------------- conventions
 * Units are mm.  Poses are row-major 4x4 FP64 rigid transforms.
 *
 * Image frame: pixel (u, v) of a W x H image with spacing (sx, sy) sits at
 * image point q = ((u - (W-1)/2) sx, v sy, 0).  Image x is the lateral
 * (in-plane) direction of Eq. 1, image y the beam (depth) direction, image z
 * = x cross y the elevation.
 *
 * Grid: dims (nx, ny, nz), spacing h, vol_to_world V.  Voxel (i, j, k) has
 * its centre at V * (i h, j h, k h); its linear index is i + nx (j + ny k).
 *
 * Fixed-point geometry.  For a plane with pose T, the pixel -> voxel map is
 * g(u, v) = G0 + u A + v B, all in units of 2^-20 voxel (int64), where
 * G0, A, B are the FP64 values below multiplied by 2^20 and rounded to the
 * nearest integer, ties to even.  Canonical FP64 evaluation order (no fused
 * multiply-add; sums left to right), with R_v, t_v and R_t, t_t the rotation
 * and translation of V and T:
 *     d    = t_t - t_v
 *     c0_r = R_v[0][r] R_t[0][0] + R_v[1][r] R_t[1][0] + R_v[2][r] R_t[2][0]
 *     c1_r = (same with column 1 of R_t)
 *     tm_r = R_v[0][r] d[0] + R_v[1][r] d[1] + R_v[2][r] d[2]
 *     G0_r = (tm_r - (0.5 (W-1) sx) c0_r) / h,  A_r = (c0_r sx) / h,
 *     B_r  = (c1_r sy) / h
 * Every later index, weight and coverage decision uses these integers, so
 * any two correct implementations agree on them bit for bit.
 *
 * Reconstruction (Fig. 1): a frame pixel lands in the voxel
 * floor(g / 2^20 + 1/2) per axis (nearest voxel, ties up); pixels outside the
 * grid are dropped.  One sample is kept per (voxel, frame): the frame id and
 * the mean of that frame's pixels in the voxel, stored as
 * round_dtype(RN_fp32(sum / npix)) (u8: round-half-even, clamped to
 * [0, 255]; f16, bf16: round-to-nearest-even).  The frame's orientation
 * (the paper stores it as a quaternion per sample) lives once per frame in
 * the session's frame table; a sample refers to it by frame id.  A voxel
 * holds at most max_slots samples: beyond that it keeps the samples of
 * largest npix (ties: lower frame id).
 *
 * Reslicing (Eq. 1, Eq. 2): for a sample of frame f and a plane r, with n =
 * the "acquisition normal" (beam direction R y by default; the image-plane
 * normal R z on request) and x = the lateral direction R x, both expressed
 * in the volume frame:
 *     d_normal = n_f . n_r            (signed)
 *     d_inplane = |x_f . x_r|
 *     valid iff d_normal >= cos(thr_normal) and d_inplane >= cos(thr_inplane)
 *       (a threshold of 180 degrees or more is off)
 *     w_f = exp(k_normal (d_normal - 1) + k_inplane (d_inplane - 1))
 * The decisions are taken in FP64 once per (plane, frame).
 *
 * Curvilinear probes (an extension: the paper's probe is a linear array,
 * Sec. 2.2).  The beams fan out from an apex a = (a_x, a_y) of the image plane
 * (image mm; a_y < 0 above the transducer face): the beam through image point
 * p runs along u = (p - a) / |p - a| (u = (0, 1) at p = a), and the image axes
 * there are turned about image z: beam R (u_x, u_y, 0), lateral
 * R (u_y, -u_x, 0), elevation R z.  A sample of a curvilinear frame takes the
 * turn at the centre of its voxel expressed in the frame's image coordinates
 * (in-plane part); a curvilinear virtual plane (dare_params.probe) takes it at
 * every output pixel.  Eq. 1 and Eq. 2 apply to the turned axes, so a
 * session with curvilinear frames, or a curvilinear virtual probe, evaluates
 * them per (pixel, sample): in FP32, with a threshold decision re-taken in
 * FP64 whenever the FP32 dot product lies within its error bound of the
 * cosine, so that every decision is the FP64 one.  With the TENT
 * distance kernel of radius R = 1 (the default; R is the interpolation
 * distance in voxels) a pixel at g reads the 8 voxels floor(g) + {0,1}^3
 * with trilinear weights t_c, and
 *     out = sum t_c w_f I / sum t_c w_f   over the valid samples of those
 *           voxels, accumulated in FP32;
 *     a pixel whose denominator is 0 is unassigned: its mask bit is 0 and it
 *     receives params.unassigned.
 *
 * Layouts.
 *   frames_dev: n x H x W uint8, row-major, frame-major (device memory).
 *   out_dev:    H x W float32, row-major (device memory).
 *   mask_dev:   H rows of ceil(W/32) uint32 words; bit (u mod 32) of word
 *               (v ceil(W/32) + u/32) is pixel (u, v)'s coverage bit; padding
 *               bits are 0 (device memory).
 *   records (dare_session_read_records): per voxel, K frame ids (uint16,
 *               ascending, 0xFFFF = empty, empties last), K values (storage
 *               type, 0 where empty) and K npix (uint16, saturating).
 *
 * Ownership.  The caller owns every *_dev buffer and every host array; host
 * arrays are read (or written) before the call returns.  A session owns its
 * volume, frame table and workspace, allocated through its allocator.
 *
 * Streams and errors.  Calls that take a stream are asynchronous on it (a
 * NULL stream is the legacy default stream) unless stated otherwise.
 * Arguments are checked on the host before anything is queued: a bad
 * argument returns DARE_E_INVALID (or the status named) and queues nothing.
 * A CUDA error seen while queueing returns DARE_E_CUDA.  Nothing aborts or
 * traps.  The message of the last failure on the calling thread is returned
 * by dare_last_error().  A session is externally synchronised: do not call
 * into the same session from two threads at once.  Successive calls on one
 * session may use different streams; the library orders them.
 */
#ifndef DARE_H
#define DARE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DARE_ABI_VERSION 3
#define DARE_FIX_BITS 20
#define DARE_EMPTY_FRAME 0xFFFFu
#define DARE_MAX_FRAMES 65535
#define DARE_MAX_SLOTS 16

typedef enum {
    DARE_OK = 0,
    DARE_E_INVALID = 1,     /* bad argument, nothing queued */
    DARE_E_OOM = 2,         /* the allocator returned NULL */
    DARE_E_CUDA = 3,        /* a CUDA call failed */
    DARE_E_ADMISSION = 4,   /* the device-memory budget would be exceeded */
    DARE_E_CAPACITY = 5,    /* frame ids would pass the session's max_frames */
    DARE_E_TIMEOUT = 6,     /* a bounded device wait gave up */
    DARE_E_STATE = 7,       /* the object is in the wrong state for the call */
    DARE_E_UNSUPPORTED = 8  /* valid but not implemented on this path */
} dare_status;

typedef enum { DARE_U8 = 0, DARE_F16 = 1, DARE_BF16 = 2, DARE_F32 = 3 } dare_dtype;
typedef enum { DARE_TENT = 0, DARE_BOX = 1, DARE_EXP = 2 } dare_dist_kernel;
typedef enum { DARE_NORMAL_BEAM = 0, DARE_NORMAL_ELEVATION = 1 } dare_normal_axis;
typedef enum { DARE_WEIGHTS_F32 = 0, DARE_WEIGHTS_F16 = 1 } dare_weight_dtype;
/* Kernel choice for linear probes: AUTO (tiled for single planes and batches;
 * plans time the candidates), PLAIN (one thread per pixel, every record read
 * per pixel), TILED (per-voxel reduction in shared-memory tiles whose height
 * follows dare_params.tile_rows), TILED_FIXED (the tiled kernel with exactly
 * tile_rows rows, 64 when 0, for every plane: tiles whose voxel-column box does
 * not fit shared memory gather per pixel inside the kernel and are counted by
 * dare_trace_counters_read; for measurements and tests). */
typedef enum { DARE_PATH_AUTO = 0, DARE_PATH_PLAIN = 1, DARE_PATH_TILED = 2, DARE_PATH_TILED_FIXED = 3 } dare_path;
typedef enum { DARE_PROBE_LINEAR = 0, DARE_PROBE_CURVILINEAR = 1 } dare_probe_kind;
/* What a stored sample stands for (Sec. 2.1 stores "the intensity values at
 * that voxel"): MEAN, one sample per (voxel, frame), the mean of that frame's
 * pixels in the voxel (default); PIXELS, every pixel its own sample with its
 * frame's orientation, which is the stored sample weighted by its pixel count
 * (the frame's pixels in a voxel share one orientation weight).  PIXELS runs
 * on the general kernels. */
typedef enum { DARE_SAMPLE_MEAN = 0, DARE_SAMPLE_PIXELS = 1 } dare_sample_weight;

/* Probe geometry (see "Curvilinear probes"): kind, and for a curvilinear
 * probe the apex of its beam fan as an image point (x, y) in mm. */
typedef struct {
    int32_t kind;        /* dare_probe_kind */
    int32_t reserved;
    double apex_mm[2];
} dare_probe;

typedef struct dare_session_s* dare_session;

/* Voxel grid: dims, spacing (mm) and the rigid volume pose. */
typedef struct {
    int32_t dims[3];
    int32_t reserved;
    double spacing_mm;
    double vol_to_world[16];
} dare_grid;

/*
 * Device-memory allocator used by a session for its volume and workspace.
 * alloc returns device memory of at least `bytes` (256-byte aligned) or NULL;
 * free releases it.  `stream` is the stream of the call that allocates (may
 * be NULL).  Both NULL: the library uses cudaMalloc / cudaFree.  A block that
 * is not 256-byte aligned is handed back to free at once and the call that
 * wanted it fails with DARE_E_OOM (the kernels use 16-byte vector and bulk
 * copies on it).
 */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
    void* ctx;
} dare_allocator;

#define DARE_SESSION_SCALAR 1 /* also keep the mean-compounding totals (dare_reslice_scalar) */
/* Keep the volume's records resident in L2 while this session is resliced: its
 * reslice launches run under a persisting access-policy window over the
 * records (up to the device's persisting-L2 size), so output writes stream past
 * them.  Meant for volumes under about 100 MB.  The window is set on the
 * caller's stream for the library's own launches and the stream's previous
 * window is restored before the call returns.  Not applied on the legacy
 * default (NULL) stream or inside plans.  Destroying such a session returns
 * every persisting L2 line of the device context to normal, so that the freed
 * records keep no share of L2 from later kernels; another such session's
 * records are marked again by its next reslice. */
#define DARE_SESSION_L2_PERSIST 2
/* Keep the records, npix and scalar totals in page-locked host memory mapped
 * into the device's address space instead of device memory, for volumes
 * beyond device memory (Sec. 4: growing datasets despite GPU memory limits).
 * Every kernel reads and writes them in place over the host link, through the
 * device's caches; results are those of a device-resident session, bit for
 * bit.  The host memory is not counted by the device-memory budget
 * (dare_set_memory_budget); the session's volume_bytes counts only its device
 * part. */
#define DARE_SESSION_HOST_VOLUME 4

typedef struct {
    dare_grid grid;
    int32_t dtype;       /* dare_dtype of the stored intensities */
    int32_t max_slots;   /* K, samples per voxel: 4, 8, 12 or 16 */
    int32_t max_frames;  /* frame ids available to this session, <= 65535 */
    int32_t device;      /* CUDA device ordinal */
    int32_t flags;       /* DARE_SESSION_* */
    int32_t reserved;
    dare_allocator alloc;
} dare_session_config;

/* Reslicing parameters (Sec. 2.1; defaults from dare_params_default). */
typedef struct {
    double k_normal;        /* Eq. 2, paper: 10 */
    double k_inplane;       /* Eq. 2, paper: 5 */
    double thr_normal_deg;  /* paper: 25 */
    double thr_inplane_deg; /* paper: 15 */
    double k_dist;          /* rate of the EXP distance kernel (>= 0) */
    float unassigned;       /* value of an unassigned pixel (default 0) */
    int32_t radius_vox;     /* R, interpolation distance in voxels, 1..16 (default 1) */
    int32_t dist_kernel;    /* dare_dist_kernel (default TENT): a pixel at g reads, per axis,
                               TENT: floor(g) - R + 1 .. floor(g) + R, t = prod (1 - |g - c| / R);
                               BOX:  round(g) - R .. round(g) + R,    t = 1;
                               EXP:  as TENT,                          t = exp(-k_dist |g - c| / R) */
    int32_t normal_axis;    /* dare_normal_axis (default BEAM) */
    int32_t weight_dtype;   /* dare_weight_dtype of the per-frame weight table */
    int32_t path;           /* dare_path: kernel choice (linear probes) */
    dare_probe probe;       /* virtual probe of the planes (default linear) */
    int32_t sample_weight;  /* dare_sample_weight (default MEAN) */
    int32_t tile_rows;      /* tiled kernel (TENT, R = 1): rows of its 32-pixel-wide tiles.  0 (default):
                               per plane, the largest of 64, 32, 16, 8 for which every tile's
                               voxel-column box fits the kernel's shared memory (the box grows with
                               the pixel-to-voxel pitch and the in-plane rotation); 8, 16, 32, 64: the
                               same choice, capped at that value.  A plane for which no height fits
                               goes to the per-pixel kernel (counted).  DARE_PATH_TILED_FIXED: exactly
                               this many rows. */
} dare_params;

/* A virtual image plane: output size, pixel spacing and pose. */
typedef struct {
    int32_t width, height;
    double px_mm[2];
    double image_to_world[16];
} dare_plane;

typedef struct {
    dare_session session;
    dare_plane plane;
    float* out;       /* device, height x width */
    uint32_t* mask;   /* device, height x ceil(width/32) words */
} dare_reslice_req;

typedef struct {
    int64_t volume_bytes;     /* device bytes held for the volume and tables */
    int64_t workspace_bytes;  /* device bytes held as reusable workspace */
    int64_t overflow_voxels;  /* voxels that hit max_slots (capacity rule applied) */
    int64_t version;          /* number of completed dare_build_volume calls */
    int32_t n_frames;         /* frame ids used so far */
    int32_t slots;            /* K */
    int32_t dtype;
    int32_t record_bytes;     /* device bytes per voxel record */
    int32_t dims[3];
    int32_t flags;
    double spacing_mm;
    double vol_to_world[16];
} dare_session_info;

/* Message of the last failure on this thread ("" if none). */
const char* dare_last_error(void);

int32_t dare_abi_version(void);

/* The paper's parameters (Sec. 2.1): k 10 / 5, thresholds 25 / 15 degrees,
 * R = 1, TENT, beam normal, FP32 weights, unassigned 0, automatic path. */
dare_status dare_params_default(dare_params* p);

/*
 * Bounding box "from the collected transducer positions" (Sec. 2.1): an
 * axis-aligned grid (identity rotation) of spacing spacing_mm covering every
 * corner of the n frames (image_to_world: n x 16 host FP64), grown by
 * margin_vox voxels on each side.  Host only, synchronous.
 */
dare_status dare_grid_from_frames(int32_t n, int32_t width, int32_t height, const double px_mm[2],
                                  const double* image_to_world, double spacing_mm, int32_t margin_vox,
                                  dare_grid* out);

/* The fixed-point pixel -> voxel affine [G0, A, B] of a plane in a grid
 * (see "Fixed-point geometry").  Host only. */
dare_status dare_pixel_affine(const dare_grid* grid, const dare_plane* plane, int64_t out[9]);

/*
 * Create a session holding an empty directional volume (Fig. 1's grid and
 * flat sample storage) on cfg->device.  Allocates the volume through
 * cfg->alloc and clears it (synchronously).  DARE_E_OOM if an allocation
 * fails, DARE_E_ADMISSION if the device-memory budget set by
 * dare_set_memory_budget would be exceeded.
 */
dare_status dare_session_create(const dare_session_config* cfg, dare_session* out);

/* Wait for the session's queued work, then free everything it holds. */
dare_status dare_session_destroy(dare_session s);

/* Wait for the session's queued work; report a device-side failure.  The
 * calling thread first polls the completion of the session's last call for up
 * to 200 microseconds (a preview loop waiting on one plane resumes as soon as
 * it is ready, without a blocking wait's wake-up), then blocks. */
dare_status dare_session_sync(dare_session s);

dare_status dare_session_query(dare_session s, dare_session_info* out);

/*
 * Copy the volume to host arrays (synchronous): frame_ids n_vox x K uint16,
 * values n_vox x K of the storage type, npix n_vox x K uint16; scalar_sum and
 * scalar_count n_vox uint32 each (only with DARE_SESSION_SCALAR).  Any
 * pointer may be NULL to skip that array.
 */
dare_status dare_session_read_records(dare_session s, uint16_t* frame_ids, void* values, uint16_t* npix,
                                      uint32_t* scalar_sum, uint32_t* scalar_count);

/* Frame table: n_frames x 9 FP64, row-major rotation of each frame in the
 * volume frame (columns: lateral, beam, elevation). */
dare_status dare_session_read_frames(dare_session s, double* rotations);

/*
 * Save / load a session (checkpoint, resume): a versioned header (grid,
 * dtype, K, frames), the frame table and the records, with a CRC-32.  A
 * loaded session reslices bit-identically to the saved one.  load takes the
 * device, allocator and flags from cfg and everything else from the file;
 * DARE_E_INVALID on a malformed or corrupted file.
 */
dare_status dare_session_save(dare_session s, const char* path);
dare_status dare_session_load(const dare_session_config* cfg, const char* path, dare_session* out);

/*
 * Reconstruction (Sec. 2.1, Fig. 1): append n tracked frames to the volume.
 * frames_dev: n x height x width uint8 on the session's device;
 * image_to_world: n x 16 host FP64 poses (copied before return).  The frames
 * get the next n frame ids.  The result is independent of thread scheduling
 * and equals one call over all frames ever appended.  DARE_E_CAPACITY if the
 * ids would pass max_frames (nothing queued).  The caller keeps frames_dev
 * valid until the stream reaches the end of the call.
 */
dare_status dare_build_volume(dare_session s, const uint8_t* frames_dev, int32_t n, int32_t width,
                              int32_t height, const double px_mm[2], const double* image_to_world,
                              void* stream);

/*
 * Probe of the frames appended from now on (default: linear, every pixel).
 * probe->kind DARE_PROBE_CURVILINEAR gives those frames the fan of apex
 * probe->apex_mm.  pixel_mask (host, height x width bytes, row-major; NULL
 * for none) excludes the pixels whose byte is 0 from voxelisation, e.g. the
 * dark corners outside a fan image; later builds must then use frames of
 * exactly width x height (DARE_E_INVALID otherwise).  The mask is copied
 * before return.  Waits for the session's queued work (synchronous).
 */
dare_status dare_session_set_probe(dare_session s, const dare_probe* probe, const uint8_t* pixel_mask,
                                   int32_t width, int32_t height);

/*
 * Brick cache for a DARE_SESSION_HOST_VOLUME session (Sec. 4: growing
 * datasets despite GPU memory limits): `bytes` of device memory hold whole
 * bricks of 8 x 8 x 8 voxels' records (512 x record_bytes each).  Before each
 * plane of dare_reslice / dare_reslice_batch (linear probes, per-(voxel,
 * frame) samples) the bricks its support can reach are paged in from the host
 * volume unless resident, replacing bricks in clock order that the plane does
 * not use; the plane then reads resident bricks from device memory and any
 * other from the host volume.  Results are bit-identical whatever the cache
 * holds.  A build or reset makes every cached brick stale.  bytes = 0 frees
 * the cache.  DARE_E_STATE for a device-resident session.  Synchronous.
 * dare_reslice_batch takes consecutive planes of such a session in groups
 * (up to 64 planes whose bricks fit the cache: one paging pass and one launch
 * per group); dare_reslice_batch_host, plans, the server and the
 * allocation-free call refuse them (DARE_E_UNSUPPORTED).
 */
dare_status dare_session_set_cache(dare_session s, int64_t bytes);

/* Brick cache counters: out[0] slots, out[1] resident bricks, out[2] bricks
 * paged in, out[3] bricks found resident, since dare_session_set_cache. */
dare_status dare_session_cache_stats(dare_session s, int64_t out[4]);

/*
 * Reslicing (Sec. 2.1, Eq. 1, Eq. 2, Fig. 2) of one plane into out_dev /
 * mask_dev (see Layouts).  Every distance kernel (TENT, BOX, EXP) runs on
 * both paths for radius_vox 1..16 (the tiled kernel up to a support of 9
 * voxels per axis, i.e. radius 4; planes beyond it, or whose tiles do not fit
 * shared memory, gather per pixel).  DARE_E_UNSUPPORTED above radius 16.
 * A tiled TENT R = 1 plane runs as the session's two-node CUDA graph (weight
 * table, reslice), built on the first such call and updated on later ones;
 * with tracing on, on an L2-persist session or while `stream` is being
 * captured, as two kernel launches.  The results are the same either way.
 */
dare_status dare_reslice(dare_session s, const dare_plane* plane, const dare_params* params, float* out_dev,
                         uint32_t* mask_dev, void* stream);

/*
 * Reslice n planes, possibly of different sessions and sizes, with one set of
 * parameters in as few launches as the sessions' storage types allow.  Each
 * result equals what dare_reslice gives for that request alone.
 */
dare_status dare_reslice_batch(const dare_reslice_req* reqs, int32_t n, const dare_params* params, void* stream);

/*
 * Host-buffer forms of the two calls above, for callers whose recorded
 * frames sit in host memory (Sec. 2.1: the recorded stream is processed on
 * the GPU after acquisition) and whose preview images go back to the host for
 * display (Sec. 4: reslicing runs on the physician's side).  Results are
 * those of the device-buffer calls, bit for bit.  Page-locked host buffers (cudaHostAlloc / cudaHostRegister) let the
 * copies overlap the kernels; pageable buffers work, with the copies staged
 * by the driver.  Both calls are asynchronous: the caller keeps the host
 * buffers valid and unchanged until `stream` reaches the end of the call.
 *
 * dare_build_volume_host: frames_host is n x height x width uint8 in host
 * memory.  The frames go to the device in slices of slice_frames frames (0:
 * about 32 MB a slice) through a two-slot device ring owned by the session;
 * a slice's upload runs on the session's upload stream and overlaps the
 * scatter of the previous slice.  Uploads do not wait for earlier work on
 * `stream` (they only write the ring), so they may also overlap the
 * downloads of a previous dare_reslice_batch_host.  Errors as
 * dare_build_volume; DARE_E_INVALID for slice_frames < 0.
 *
 * dare_reslice_batch_host: out and mask of every request are host pointers
 * (layouts as in dare_reslice).  The requests are resliced in groups of
 * group_planes planes (0: about 128 MB of output a group) into a device
 * staging buffer of 2 to 8 group slots (about 1 GB at most) owned by the
 * first request's session; groups are resliced ahead while earlier ones are
 * copied back on the session's download stream.  Consecutive requests whose host outputs (or masks) are
 * adjacent in memory are copied back in one transfer.  `stream` waits for the
 * last copy, so once it is synchronised every output is in host memory.
 * Errors as dare_reslice_batch; DARE_E_INVALID for group_planes < 0.
 */
dare_status dare_build_volume_host(dare_session s, const uint8_t* frames_host, int32_t n, int32_t width,
                                   int32_t height, const double px_mm[2], const double* image_to_world,
                                   int32_t slice_frames, void* stream);
dare_status dare_reslice_batch_host(const dare_reslice_req* reqs, int32_t n, const dare_params* params,
                                    int32_t group_planes, void* stream);

/*
 * Reslice plans: a fixed set of requests (sessions, output sizes and buffers)
 * prepared once and replayed many times, for a stream of batches whose poses
 * change (the batched workloads behind Sec. 3's timing and a serving loop).
 * dare_plan_create groups the requests by storage type and slot count and
 * chooses each group's kernel: with params->path == DARE_PATH_AUTO by timing,
 * on these very requests, the plain kernel and the persistent tiled kernel
 * with tiles of at most 64, 32 and 16 rows (each plane then takes the largest
 * height up to that cap whose tiles fit shared memory, recomputed for every
 * new pose; a plane that no height fits is gathered per pixel inside the
 * persistent kernel).  The persistent tiled kernel runs one CTA per resident
 * slot of the device and takes tiles from a work queue over every plane of
 * the group.  Choices are cached per shape (storage type, K, weights, output
 * pixels and planes rounded to powers of two, median pixel-to-voxel pitch in
 * eighths of a voxel, L2 mode, frame count, SM count) for the process, and in
 * the file named by dare_tune_cache_file when one is set.  The plan then
 * allocates its device workspace and pinned staging and captures the
 * descriptor upload, the weight tables and the reslice launches into one
 * CUDA graph (synchronous; writes the outputs while tuning).
 * dare_plan_set_poses replaces every request's image_to_world (n x 16 host
 * FP64, copied; waits for the previous launch's upload to finish).
 * dare_plan_launch replays the graph on `stream`; each result equals
 * dare_reslice of that request.  A session whose frame count changed since
 * the plan was created makes launch fail with DARE_E_STATE (re-create the
 * plan); rebuilding it to the same frame count is fine.  Plans cover linear
 * probes: a request whose session holds curvilinear frames, or a curvilinear
 * params->probe, gives DARE_E_UNSUPPORTED (use dare_reslice_batch).
 * The plan's workspace comes from the first request's session allocator (a
 * copy of it is kept), so dare_plan_destroy touches no session and may follow
 * the sessions' destruction; set_poses and launch need every session alive.
 */
typedef struct dare_plan_s* dare_plan;

typedef struct {
    int32_t n_requests;
    int32_t n_groups;        /* launches per replay (one per storage type / K) */
    int32_t choice[8];       /* per group: 0 = plain kernel, else the tiled kernel's largest tile height */
    float tune_ms[8][4];     /* per group: measured plain, tiled <= 64, <= 32, <= 16 rows (0 if not timed) */
    int64_t workspace_bytes;
} dare_plan_info;

/* File (JSON object of "shape key": choice) that plan tuning reads now and
 * rewrites, with every choice known to the process, now and after each new
 * choice; NULL or "" stops using a file.  A file that cannot be read is treated
 * as empty; DARE_E_INVALID if it cannot be written (then, or later from the
 * dare_plan_create that tuned).  Synchronous, host only. */
dare_status dare_tune_cache_file(const char* path);

dare_status dare_plan_create(const dare_reslice_req* reqs, int32_t n, const dare_params* params, void* stream,
                             dare_plan* out);
dare_status dare_plan_set_poses(dare_plan p, const double* image_to_world);
dare_status dare_plan_launch(dare_plan p, void* stream);
dare_status dare_plan_query(dare_plan p, dare_plan_info* out);
dare_status dare_plan_destroy(dare_plan p);

/*
 * Serving loop: many sessions' reslice requests arriving over time (the
 * expert console's haptic pose stream, Sec. 1) plus live frame ingestion
 * (incremental integration, Sec. 4).  A dispatcher thread batches the pending
 * requests whenever one of `lanes` streams is free (continuous batching:
 * requests arriving while others run join the next batch), so the batches of
 * different lanes overlap on the device; requests of different sessions and
 * output sizes go out in one dare_reslice_batch.  With coalesce_us > 0 a batch
 * that is not full waits until its oldest request is coalesce_us old before it
 * is issued, so that more requests join it (fewer launches for a bounded added
 * latency); an ingest queued behind it, or a stop, issues it at once.  A batch
 * waits only for the ingests of the sessions it reads; an ingest waits for
 * the reslices in flight, then runs dare_build_volume on the server's ingest
 * stream; requests of a session whose ingest is still running go out in a
 * batch of their own, so an ingest holds up only its own session's requests.
 * Every result equals dare_reslice of that request against the
 * volume as of its submission.  The dispatcher thread completes requests when
 * it sees their stream reach them (no host callbacks on the lanes), on the
 * clock of dare_clock_seconds.
 *
 * Sessions given to a server must be idle (dare_session_sync) and must not be
 * used outside the server until dare_server_drain returns.  frames_dev of an
 * ingest must stay valid until its completion is polled.  Submission is
 * thread-safe.  dare_server_create allocates every lane's device workspace
 * and pinned staging for max_batch requests of sessions with up to
 * max_frames frames (counted by the device-memory budget; DARE_E_ADMISSION or
 * DARE_E_OOM when that fails), so the dispatcher never allocates; a request
 * whose session allows more frames (its max_frames) is refused by submit
 * with DARE_E_INVALID.
 */
typedef struct dare_server_s* dare_server;

typedef struct {
    int32_t device;
    int32_t lanes;        /* batches in flight at once, 1..8 (default 2 when 0) */
    int32_t max_batch;    /* requests per batch, 1..4096 (default 64 when 0) */
    int32_t coalesce_us;  /* coalescing window of a batch, 0..1000000 microseconds (0: none) */
    dare_params params;
    int32_t max_frames;   /* largest max_frames of the sessions served (0: DARE_MAX_FRAMES) */
    int32_t reserved;
} dare_server_config;

typedef struct {
    uint64_t tag;
    int32_t status;     /* dare_status of the request */
    int32_t kind;       /* 0 reslice, 1 ingest */
    double submit_s;    /* dare_clock_seconds at submission */
    double done_s;      /* dare_clock_seconds when the dispatcher saw its stream finish it (it polls
                           every 20 us while work is in flight) */
    double issue_s;     /* dare_clock_seconds when the dispatcher queued it on a stream */
    int32_t batch;      /* requests in the batch it went out with (1 for an ingest) */
    int32_t lane;       /* stream lane of that batch (-1 for an ingest) */
} dare_completion;

typedef struct {
    int64_t submitted, completed, batches, ingests;
    int64_t max_batch_seen;
    int32_t lanes, reserved;
} dare_server_stats;

double dare_clock_seconds(void);
dare_status dare_server_create(const dare_server_config* cfg, dare_server* out);
dare_status dare_server_submit(dare_server sv, const dare_reslice_req* req, uint64_t tag);
dare_status dare_server_ingest(dare_server sv, dare_session s, const uint8_t* frames_dev, int32_t n, int32_t width,
                               int32_t height, const double px_mm[2], const double* image_to_world, uint64_t tag);
dare_status dare_server_poll(dare_server sv, dare_completion* out, int32_t capacity, int32_t* n_out);
dare_status dare_server_drain(dare_server sv, double timeout_s);
dare_status dare_server_stats_get(dare_server sv, dare_server_stats* out);
dare_status dare_server_destroy(dare_server sv);

/*
 * Allocation-free variant of dare_reslice.  The paper has no counterpart:
 * this entry point exists for callers that must not ask for device memory
 * while they run, e.g. a preview loop on the expert's console thread with a
 * fixed latency budget (cudaMalloc / cudaFree can block and synchronise the
 * device), or an application whose device memory is entirely owned by
 * another component once it has started.
 *
 * Same arguments, checks and result as dare_reslice (same kernels), except
 * that the plane's per-frame weight table goes to a fixed array in device
 * memory inside the library instead of the session's workspace.  That array
 * holds DARE_NOALLOC_MAX_FRAMES weights (64 KB): a session with more frames
 * is rejected with DARE_E_INVALID and nothing is queued.  Every GPU that
 * loads the library keeps the array until the process exits.  All calls
 * share it: calls that overlap on the GPU (unordered streams) race and give
 * wrong images; order them or use dare_reslice.  The first call on a device
 * looks up the array's device address on that device.  That lookup asks for
 * no memory itself, but under CUDA's lazy module loading (the default) it is
 * what loads the part of the library that holds the array, and loading takes
 * device memory; so make the first call during set-up, before the phase that
 * must not allocate and before any stream capture.  The session, its volume
 * and the outputs must already exist; after that first call, calls allocate
 * nothing.
 * Linear probes only: curvilinear frames or a curvilinear params->probe give
 * DARE_E_UNSUPPORTED.
 */
#define DARE_NOALLOC_MAX_FRAMES 16384
dare_status dare_reslice_noalloc(dare_session s, const dare_plane* plane, const dare_params* params,
                                 float* out_dev, uint32_t* mask_dev, void* stream);

/*
 * Mean-compounding comparator (the scalar reading of the PLUS baseline,
 * Sec. 2.2): each voxel holds RN_fp32(total / count) of every pixel that
 * landed in it; a pixel is the trilinear blend of its occupied corners,
 * renormalised by their weights, or unassigned.  Needs DARE_SESSION_SCALAR.
 */
dare_status dare_reslice_scalar(dare_session s, const dare_plane* plane, float unassigned, float* out_dev,
                                uint32_t* mask_dev, void* stream);

/*
 * Hole filling of the compounded volume (the PLUS baseline of Sec. 2.2 runs
 * mean compounding "with hole-filling"; one pass, this library's reading):
 * every voxel with pixels keeps RN_fp32(total / count); an empty voxel takes
 * the mean of the occupied voxels of the (2 radius_vox + 1)^3 cube around it,
 * each weighted by 1 / its Euclidean distance in voxels, when at least
 * min_neighbours of them are occupied, and stays empty otherwise.  The result
 * (FP32 per voxel, NaN = empty) is kept in the session (allocated on first
 * use, n_vox x 4 bytes) until the next build or reset makes it stale.
 * radius_vox 1..8, min_neighbours 0..(2 radius_vox + 1)^3 - 1.  Needs
 * DARE_SESSION_SCALAR (DARE_E_STATE otherwise).  Asynchronous on `stream`.
 */
dare_status dare_fill_holes(dare_session s, int32_t radius_vox, int32_t min_neighbours, void* stream);

/* The comparator's trilinear reslice (as dare_reslice_scalar) of the
 * hole-filled volume: non-empty corners only, renormalised.  DARE_E_STATE
 * without a current dare_fill_holes result. */
dare_status dare_reslice_scalar_filled(dare_session s, const dare_plane* plane, float unassigned, float* out_dev,
                                       uint32_t* mask_dev, void* stream);

/* Host copy of the hole-filled volume, n_vox FP32 (NaN = empty); synchronous. */
dare_status dare_session_read_filled(dare_session s, float* values);

/*
 * Footprint: for each of n planes, the number of distinct in-grid voxels in
 * the TENT support of radius 1 of any pixel -- the voxel records a reslice
 * must read at least once.  counts: n int64 on the host.  Synchronous.
 */
dare_status dare_footprint(dare_session s, const dare_plane* planes, int32_t n, int64_t* counts, void* stream);

/*
 * Empty the volume (all samples, frame ids and scalar totals), keeping its
 * allocation, grid and configuration; the next build starts at frame id 0.
 * Asynchronous.  The device-side clear is deferred: the next build writes
 * every voxel in its finalize pass (so a reset + rebuild costs no separate
 * pass over the volume), and any other call that reads the volume first
 * queues the clear on its own stream.  Every call sees an empty volume.
 */
dare_status dare_session_reset(dare_session s, void* stream);

/*
 * Kernel tracing.  While enabled, every kernel the library launches is
 * bracketed by two CUDA events recorded on the stream it is launched on;
 * dare_trace_read waits for them and returns, per kernel name, the number of
 * launches and their summed device time.  dare_launch_count counts every
 * kernel launched since the process started, traced or not.
 */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
} dare_kernel_time;

dare_status dare_trace_enable(int32_t on);
dare_status dare_trace_read(dare_kernel_time* out, int32_t capacity, int32_t* n_out);
int64_t dare_launch_count(void);

/*
 * Path counters of the reslice kernels, counted whether tracing is on or not:
 * tiled_planes, planes given to the tiled kernels; per_pixel_planes, planes
 * that the automatic tile choice sent to the per-pixel kernels because no
 * tile height fits them (or the plane is degenerate); fallback_tiles, tiles
 * of the tiled kernels that gathered per pixel inside the kernel because
 * their voxel-column box did not fit shared memory (0 unless
 * DARE_PATH_TILED_FIXED forces a tile height).  fallback_tiles is read from
 * the current device (synchronous: waits for that device's queued work).
 * reset != 0 sets the counters back to 0 after reading.
 */
typedef struct {
    int64_t tiled_planes;
    int64_t per_pixel_planes;
    int64_t fallback_tiles;
} dare_trace_counters;

dare_status dare_trace_counters_read(dare_trace_counters* out, int32_t reset);

/*
 * Measurement aid for the roofline of the reslice kernels, whose gathers L2
 * serves for the most part: the device's L2-to-SM read bandwidth in GB/s, from
 * 16-byte loads that bypass L1 over a buffer of `bytes` (1 MiB .. 1 GiB; keep
 * it well under the L2 size) read `reps` times by 8 CTAs of 256 threads per
 * SM after one warm-up pass.  Allocates and frees its own buffer; synchronous.
 */
dare_status dare_measure_l2_bandwidth(int32_t device, int64_t bytes, int32_t reps, double* read_gbs);

/* Device-memory budget (bytes) shared by all sessions of this process;
 * 0 = unlimited.  Sessions that would exceed it fail with DARE_E_ADMISSION. */
dare_status dare_set_memory_budget(int64_t bytes);
int64_t dare_memory_in_use(void);

#ifdef __cplusplus
}
#endif

#endif /* DARE_H */
