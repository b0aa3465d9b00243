// Host side of libdare's C ABI: argument checks, FP64 pose composition, the
// fixed-point affine, sessions (volume, frame table, workspace), ordering of
// a session's work across streams, device-memory admission, checkpoints.
//
// Compile with -ffp-contract=off: the fixed-point affine follows the
// canonical FP64 evaluation order documented in dare.h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "dare_internal.h"

using namespace dare;

namespace {

thread_local std::string g_err;
std::atomic<int64_t> g_budget{0};
std::atomic<int64_t> g_in_use{0};

dare_status fail(dare_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CUDA_TRY(expr)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess) return fail(DARE_E_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool finite_all(const double* x, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

// Rigid: finite, last row (0 0 0 1), orthonormal rotation with det +1.
bool rigid_ok(const double* T) {
    if (!finite_all(T, 16)) return false;
    if (std::fabs(T[12]) > 1e-9 || std::fabs(T[13]) > 1e-9 || std::fabs(T[14]) > 1e-9 || std::fabs(T[15] - 1.0) > 1e-9)
        return false;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double d = T[0 * 4 + i] * T[0 * 4 + j] + T[1 * 4 + i] * T[1 * 4 + j] + T[2 * 4 + i] * T[2 * 4 + j];
            if (std::fabs(d - (i == j ? 1.0 : 0.0)) > 1e-6) return false;
        }
    const double det = T[0] * (T[5] * T[10] - T[6] * T[9]) - T[1] * (T[4] * T[10] - T[6] * T[8]) +
                       T[2] * (T[4] * T[9] - T[5] * T[8]);
    return det > 0;
}

int64_t fix_round(double x) { return static_cast<int64_t>(std::nearbyint(x * static_cast<double>(kFixOne))); }

// Fixed-point pixel -> voxel affine in the canonical order of dare.h.
void compose_affine(const double* V, double h, const double* T, int32_t W, double sx, double sy, int64_t out[9]) {
    double d[3], c0[3], c1[3], tm[3];
    for (int k = 0; k < 3; ++k) d[k] = T[4 * k + 3] - V[4 * k + 3];
    for (int r = 0; r < 3; ++r) {
        c0[r] = V[0 * 4 + r] * T[0 * 4 + 0] + V[1 * 4 + r] * T[1 * 4 + 0] + V[2 * 4 + r] * T[2 * 4 + 0];
        c1[r] = V[0 * 4 + r] * T[0 * 4 + 1] + V[1 * 4 + r] * T[1 * 4 + 1] + V[2 * 4 + r] * T[2 * 4 + 1];
        tm[r] = V[0 * 4 + r] * d[0] + V[1 * 4 + r] * d[1] + V[2 * 4 + r] * d[2];
    }
    const double half_w = 0.5 * static_cast<double>(W - 1) * sx;
    for (int r = 0; r < 3; ++r) {
        out[r] = fix_round((tm[r] - half_w * c0[r]) / h);
        out[3 + r] = fix_round((c0[r] * sx) / h);
        out[6 + r] = fix_round((c1[r] * sy) / h);
    }
}

// Rotation of pose T in the volume frame, R_v^T R_t (row-major 3x3).
void relative_rotation(const double* V, const double* T, double R[9]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            R[3 * r + c] = V[0 * 4 + r] * T[0 * 4 + c] + V[1 * 4 + r] * T[1 * 4 + c] + V[2 * 4 + r] * T[2 * 4 + c];
}

// Apex-relative image coordinates of voxel centres in a frame: for voxel c,
// p_x = h sum_r R[r][0] c_r + off[0], p_y = h sum_r R[r][1] c_r + off[1], with
// R = R_v^T R_f (row-major) and tm = R_v^T (t_f - t_v): p = R^T (h c - tm) - apex.
void probe_offsets(const double* V, const double* T, const double R[9], const double apex[2], double off[2]) {
    double d[3], tm[3];
    for (int k = 0; k < 3; ++k) d[k] = T[4 * k + 3] - V[4 * k + 3];
    for (int r = 0; r < 3; ++r) tm[r] = V[0 * 4 + r] * d[0] + V[1 * 4 + r] * d[1] + V[2 * 4 + r] * d[2];
    for (int c = 0; c < 2; ++c) off[c] = -(R[c] * tm[0] + R[3 + c] * tm[1] + R[6 + c] * tm[2]) - apex[c];
}

// FP32 geometry row of a frame for the curvilinear kernel (layout in
// dare_internal.h).  k1 = 17 eps S bounds the FP32 direction error times |p|,
// S the largest operand sum of the point computation over the grid.
void geometry_row(const dare_grid& g, const double R[9], int kind, const double off[2], float* row) {
    const double h = g.spacing_mm;
    std::fill(row, row + kGeomFloats, 0.0f);
    if (kind == DARE_PROBE_CURVILINEAR) {
        double S = 0.0;
        for (int c = 0; c < 2; ++c) {
            double sum = std::fabs(off[c]);
            for (int r = 0; r < 3; ++r) {
                row[4 * c + r] = static_cast<float>(h * R[3 * r + c]);
                sum += std::fabs(h * R[3 * r + c]) * static_cast<double>(std::max(g.dims[r] - 1, 0));
            }
            row[4 * c + 3] = static_cast<float>(off[c]);
            S = std::max(S, sum);
        }
        row[17] = static_cast<float>(17.0 * std::ldexp(1.0, -24) * S * (1.0 + 1e-6));
        row[18] = 1.0f;
    } else {
        row[7] = 1.0f;  // p = (0, 1): the beam is image y
    }
    for (int r = 0; r < 3; ++r) {
        row[8 + r] = static_cast<float>(R[3 * r + 0]);
        row[11 + r] = static_cast<float>(R[3 * r + 1]);
        row[14 + r] = static_cast<float>(R[3 * r + 2]);
    }
}

// Largest coefficient magnitude that keeps g = G0 + u A + v B inside int64
// for any u, v < 2^16 (and keeps voxel coordinates far from overflow).
constexpr double kMaxFix = 9.0e15;

bool affine_ok(const double* V, double h, const double* T, int32_t W, double sx, double sy) {
    // evaluate the unrounded magnitudes before quantising
    double Rrel[9];
    relative_rotation(V, T, Rrel);
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = T[4 * k + 3] - V[4 * k + 3];
    for (int r = 0; r < 3; ++r) {
        double tm = V[0 * 4 + r] * d[0] + V[1 * 4 + r] * d[1] + V[2 * 4 + r] * d[2];
        double g0 = (tm - 0.5 * (W - 1) * sx * Rrel[3 * r]) / h * static_cast<double>(kFixOne);
        double a = Rrel[3 * r] * sx / h * static_cast<double>(kFixOne);
        double b = Rrel[3 * r + 1] * sy / h * static_cast<double>(kFixOne);
        if (!(std::fabs(g0) < kMaxFix && std::fabs(a) * 65536.0 < kMaxFix && std::fabs(b) * 65536.0 < kMaxFix))
            return false;
    }
    return true;
}

uint32_t crc32_update(uint32_t crc, const void* data, size_t n) {
    static uint32_t table[256];
    static std::once_flag once;
    std::call_once(once, [] {
        for (uint32_t i = 0; i < 256; ++i) {
            uint32_t c = i;
            for (int k = 0; k < 8; ++k) c = (c & 1) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
            table[i] = c;
        }
    });
    const uint8_t* p = static_cast<const uint8_t*>(data);
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
    return ~crc;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------- tracing

std::atomic<int64_t> g_launches{0};
std::atomic<int64_t> g_tiled_planes{0}, g_per_pixel_planes{0};
std::atomic<bool> g_trace_on{false};
std::mutex g_trace_mu;
struct TraceRec {
    const char* name;
    int device;
    cudaEvent_t a, b;
};
std::vector<TraceRec> g_trace_pending;
std::map<int, std::vector<cudaEvent_t>> g_event_pool;
std::map<std::string, std::pair<int64_t, double>> g_trace_acc;

cudaEvent_t pooled_event(int dev) {
    auto& pool = g_event_pool[dev];
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Brackets the kernel launches of one launcher call (n_kernels of them).
struct KernelScope {
    const char* name;
    cudaStream_t st;
    int dev = 0;
    cudaEvent_t a = nullptr, b = nullptr;
    KernelScope(const char* n, cudaStream_t s, int n_kernels) : name(n), st(s) {
        g_launches += n_kernels;
        if (!g_trace_on.load()) return;
        std::lock_guard<std::mutex> lk(g_trace_mu);
        cudaGetDevice(&dev);
        a = pooled_event(dev);
        b = pooled_event(dev);
        if (a && b) cudaEventRecord(a, st);
    }
    ~KernelScope() {
        if (!a || !b) return;
        std::lock_guard<std::mutex> lk(g_trace_mu);
        cudaEventRecord(b, st);
        g_trace_pending.push_back({name, dev, a, b});
    }
};

// Persisting-L2 window over a record range for the launches between
// construction and destruction (DARE_SESSION_L2_PERSIST).
struct L2Window {
    cudaStream_t st = nullptr;
    bool set = false;
    cudaStreamAttrValue prev{};
    L2Window(const void* base, size_t bytes, cudaStream_t stream) {
        if (!stream || !base || bytes == 0) return;
        static std::mutex mu;
        static int max_persist[64] = {}, max_window[64] = {};
        static bool limit_set[64] = {};
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
        {
            std::lock_guard<std::mutex> lk(mu);
            if (!max_window[dev]) {
                cudaDeviceGetAttribute(&max_persist[dev], cudaDevAttrMaxPersistingL2CacheSize, dev);
                cudaDeviceGetAttribute(&max_window[dev], cudaDevAttrMaxAccessPolicyWindowSize, dev);
                if (!max_window[dev]) max_window[dev] = -1;
            }
            if (max_window[dev] <= 0 || max_persist[dev] <= 0) return;
            if (!limit_set[dev]) {
                if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, static_cast<size_t>(max_persist[dev])) != cudaSuccess) {
                    cudaGetLastError();
                    return;
                }
                limit_set[dev] = true;
            }
        }
        if (cudaStreamGetAttribute(stream, cudaStreamAttributeAccessPolicyWindow, &prev) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        cudaStreamAttrValue v{};
        const size_t n = std::min(bytes, static_cast<size_t>(max_window[dev]));
        v.accessPolicyWindow.base_ptr = const_cast<void*>(base);
        v.accessPolicyWindow.num_bytes = n;
        v.accessPolicyWindow.hitRatio = std::min(1.0f, static_cast<float>(max_persist[dev]) / static_cast<float>(n));
        v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        if (cudaStreamSetAttribute(stream, cudaStreamAttributeAccessPolicyWindow, &v) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        st = stream;
        set = true;
    }
    ~L2Window() {
        if (set) cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &prev);
    }
};

}  // namespace

// ---------------------------------------------------------------- session

// Hands a device block back through the allocator it came from (cudaFree
// when the caller supplied none).
static void allocator_free(const dare_allocator& a, void* p, size_t bytes, cudaStream_t st) {
    if (!p) return;
    if (a.free)
        a.free(p, bytes, st, a.ctx);
    else if (!a.alloc)
        cudaFree(p);
}

struct dare_session_s {
    dare_session_config cfg{};
    int64_t n_vox = 0;
    int32_t K = 0, dtype = 0, rec_bytes = 0;
    uint8_t* rec = nullptr;
    uint16_t* npix = nullptr;
    uint32_t* ssum = nullptr;
    uint32_t* scnt = nullptr;
    int32_t* count = nullptr;              // scatter counters, all zero between calls
    double* frames_dev = nullptr;          // max_frames x 9
    float* geom_dev = nullptr;             // max_frames x kGeomFloats: probe geometry (curvilinear kernel)
    double* geom_off_dev = nullptr;        // max_frames x 2: its FP64 apex-relative offsets
    unsigned long long* overflow_dev = nullptr;
    // single-plane graph: the weight table and the tiled reslice as two kernel
    // nodes, their parameters replaced on every call (one launch on the host)
    cudaGraph_t sp_graph = nullptr;
    cudaGraphExec_t sp_exec = nullptr;
    cudaGraphNode_t sp_node[2] = {nullptr, nullptr};
    void* sp_fn[2] = {nullptr, nullptr};
    std::vector<double> frames_host;       // n_frames x 9
    std::vector<double> probe_host;        // n_frames x 3: probe kind, FP64 offsets
    int32_t n_curv = 0;                    // frames from a curvilinear probe
    dare_probe probe{};                    // probe of the frames appended from now on
    uint32_t* pix_mask = nullptr;          // its pixel mask (device bitmap), or NULL
    // brick cache (dare_session_set_cache, host volumes): slots of 8^3-voxel bricks of records
    uint8_t* cache = nullptr;
    size_t cache_bytes = 0;
    int32_t n_slots = 0;
    int32_t* brick_table = nullptr;        // per brick: slot or -1 (device)
    size_t table_bytes = 0;
    int32_t nb[3] = {0, 0, 0};
    std::vector<int32_t> slot_of_brick, brick_of_slot;
    std::vector<int64_t> slot_stamp;       // plane count at the slot's last use
    std::vector<uint8_t> brick_mark;       // scratch of plane_bricks
    int64_t stamp = 0;
    int32_t hand = 0;                      // next eviction candidate (clock)
    int64_t pages_in = 0, page_hits = 0;
    float* filled = nullptr;               // hole-filled compounded volume (NaN = empty), or NULL
    size_t filled_bytes = 0;
    int64_t filled_version = -1;           // session version it was computed at
    size_t pix_mask_bytes = 0;
    int32_t pm_w = 0, pm_h = 0;
    int32_t n_frames = 0;
    int64_t version = 0;
    bool fresh = true;                     // no sample stored since create / reset: finalize skips reading records
    bool pending_clear = false;            // reset but not yet cleared: the next build writes every voxel,
                                           // any other call clears the volume first
    int64_t volume_bytes = 0;
    void* host_vol = nullptr;              // DARE_SESSION_HOST_VOLUME: the mapped host block
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // pinned host staging: [0] and [9] frame affines / rotations of builds in
    // turn, [1..8] batch descriptors in turn, so the host can run a few calls ahead
    static constexpr int kPinSlots = 10;
    void* pinned[kPinSlots] = {};
    size_t pinned_bytes[kPinSlots] = {};
    cudaEvent_t pinned_ev[kPinSlots] = {};  // last copy out of each staging buffer
    int next_desc = 0;
    int next_build = 0;
    cudaEvent_t order_ev = nullptr;        // end of the session's last queued call
    cudaStream_t last_stream = nullptr;
    // host-buffer calls: a two-slot upload ring (build) and a two-slot download
    // staging buffer (reslice), each with its own copy stream and slot events
    uint8_t* ring = nullptr;
    size_t ring_slot = 0;
    int ring_n = 0;
    static constexpr int kStageSlots = 8;  // download staging: up to 8 slots, about 1 GB in all
    uint8_t* stage = nullptr;
    size_t stage_slot = 0;
    int stage_n = 0;
    cudaStream_t up_st = nullptr, down_st = nullptr;
    cudaEvent_t ring_free[2] = {nullptr, nullptr};   // last scatter count that read the slot
    cudaEvent_t ring_full[2] = {nullptr, nullptr};   // upload into the slot done
    cudaEvent_t stage_free[kStageSlots] = {};        // download out of the slot done
    cudaEvent_t stage_full[kStageSlots] = {};        // reslices into the slot done
    std::vector<std::pair<void*, size_t>> allocs;

    void* dev_alloc(size_t bytes, cudaStream_t st) {
        void* p = nullptr;
        if (cfg.alloc.alloc) {
            p = cfg.alloc.alloc(bytes, st, cfg.alloc.ctx);
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (p && (reinterpret_cast<uintptr_t>(p) & 255u) != 0) {
            // a caller-supplied allocator broke the 256-byte alignment the kernels rely on
            dev_free(p, bytes, st);
            p = nullptr;
        }
        return p;
    }
    void dev_free(void* p, size_t bytes, cudaStream_t st) { allocator_free(cfg.alloc, p, bytes, st); }
};

namespace {

dare_status admit(int64_t bytes) {
    const int64_t budget = g_budget.load();
    int64_t cur = g_in_use.load();
    for (;;) {
        if (budget > 0 && cur + bytes > budget)
            return fail(DARE_E_ADMISSION, "device-memory budget exceeded: %lld in use + %lld requested > %lld",
                        (long long)cur, (long long)bytes, (long long)budget);
        if (g_in_use.compare_exchange_weak(cur, cur + bytes)) return DARE_OK;
    }
}

// Every cached brick is stale once the records change (a build or a clear).
dare_status invalidate_cache(dare_session s, cudaStream_t st) {
    if (!s->cache) return DARE_OK;
    CUDA_TRY(cudaMemsetAsync(s->brick_table, 0xFF, s->table_bytes, st));
    std::fill(s->slot_of_brick.begin(), s->slot_of_brick.end(), -1);
    std::fill(s->brick_of_slot.begin(), s->brick_of_slot.end(), -1);
    std::fill(s->slot_stamp.begin(), s->slot_stamp.end(), 0);
    return DARE_OK;
}

// Empty volume on st: empty records, zero npix and scalar totals.
dare_status clear_volume(dare_session s, cudaStream_t st) {
    dare_status rc0 = invalidate_cache(s, st);
    if (rc0 != DARE_OK) return rc0;
    {
        KernelScope ks("fill_records", st, 1);
        CUDA_TRY(launch_fill_records(s->rec, s->n_vox, s->rec_bytes, s->K, st));
    }
    CUDA_TRY(cudaMemsetAsync(s->npix, 0, size_t(s->n_vox) * s->K * 2, st));
    if (s->ssum) {
        CUDA_TRY(cudaMemsetAsync(s->ssum, 0, size_t(s->n_vox) * 4, st));
        CUDA_TRY(cudaMemsetAsync(s->scnt, 0, size_t(s->n_vox) * 4, st));
    }
    return DARE_OK;
}

// Order a call after the session's previous one, whatever stream that used.
// A clear deferred by dare_session_reset is queued first, unless the caller
// takes it over (a build: its first finalize writes every voxel).
dare_status session_begin(dare_session s, cudaStream_t st, bool settle = true) {
    CUDA_TRY(cudaStreamWaitEvent(st, s->order_ev, 0));
    if (settle && s->pending_clear) {
        dare_status rc = clear_volume(s, st);
        if (rc != DARE_OK) return rc;
        s->pending_clear = false;
    }
    return DARE_OK;
}

dare_status session_end(dare_session s, cudaStream_t st) {
    CUDA_TRY(cudaEventRecord(s->order_ev, st));
    s->last_stream = st;
    return DARE_OK;
}

// A deferred clear queued now (legacy stream) for the synchronous calls and
// for callers with their own ordering; they then wait for order_ev.
dare_status settle_now(dare_session s) {
    if (!s->pending_clear) return DARE_OK;
    dare_status rc = session_begin(s, nullptr);
    if (rc != DARE_OK) return rc;
    return session_end(s, nullptr);
}

dare_status ensure_workspace(dare_session s, size_t bytes, cudaStream_t st) {
    if (s->ws_bytes >= bytes) return DARE_OK;
    size_t want = std::max(bytes, s->ws_bytes + s->ws_bytes / 2);
    want = align_up(want, size_t(1) << 20);
    if (s->ws) {
        s->dev_free(s->ws, s->ws_bytes, st);
        g_in_use -= static_cast<int64_t>(s->ws_bytes);
        s->ws = nullptr;
        s->ws_bytes = 0;
    }
    dare_status a = admit(static_cast<int64_t>(want));
    if (a != DARE_OK) {
        a = admit(static_cast<int64_t>(bytes));
        if (a != DARE_OK) return a;
        want = bytes;
    }
    s->ws = s->dev_alloc(want, st);
    if (!s->ws) {
        g_in_use -= static_cast<int64_t>(want);
        return fail(DARE_E_OOM, "workspace allocation of %zu bytes failed", want);
    }
    s->ws_bytes = want;
    return DARE_OK;
}

// Host staging in pinned memory; waits until the previous copy out of it is done.
dare_status ensure_pinned(dare_session s, int slot, size_t bytes) {
    CUDA_TRY(cudaEventSynchronize(s->pinned_ev[slot]));
    if (s->pinned_bytes[slot] >= bytes) return DARE_OK;
    if (s->pinned[slot]) cudaFreeHost(s->pinned[slot]);
    s->pinned[slot] = nullptr;
    s->pinned_bytes[slot] = 0;
    const size_t want = align_up(std::max(bytes, size_t(1) << 16), 4096);
    CUDA_TRY(cudaHostAlloc(&s->pinned[slot], want, cudaHostAllocDefault));
    s->pinned_bytes[slot] = want;
    return DARE_OK;
}

// Copy streams and slot events of the host-buffer calls, made on first use.
dare_status ensure_host_io(dare_session s) {
    if (s->up_st) return DARE_OK;
    CUDA_TRY(cudaStreamCreateWithFlags(&s->up_st, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&s->down_st, cudaStreamNonBlocking));
    std::vector<cudaEvent_t*> evs;
    for (int k = 0; k < 2; ++k) evs.insert(evs.end(), {&s->ring_free[k], &s->ring_full[k]});
    for (int k = 0; k < dare_session_s::kStageSlots; ++k) evs.insert(evs.end(), {&s->stage_free[k], &s->stage_full[k]});
    for (cudaEvent_t* e : evs) {
        CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        CUDA_TRY(cudaEventRecord(*e, s->up_st));  // completes at once: every slot starts free
    }
    return DARE_OK;
}

// A device buffer of n_want slots of at least `slot` bytes; growing it first
// waits (on the host) until no slot is in use (the events in_use).
dare_status ensure_slots(dare_session s, uint8_t*& buf, size_t& have, int& n_have, size_t slot, int n_want,
                         const std::vector<cudaEvent_t>& in_use, cudaStream_t st) {
    if (have >= slot && n_have >= n_want) return DARE_OK;
    for (cudaEvent_t e : in_use) CUDA_TRY(cudaEventSynchronize(e));
    if (buf) {
        s->dev_free(buf, size_t(n_have) * have, st);
        g_in_use -= static_cast<int64_t>(size_t(n_have) * have);
        buf = nullptr;
    }
    have = std::max(have, align_up(slot, size_t(1) << 20));
    n_have = std::max(n_have, n_want);
    const size_t bytes = size_t(n_have) * have;
    dare_status a = admit(static_cast<int64_t>(bytes));
    if (a != DARE_OK) {
        have = 0;
        n_have = 0;
        return a;
    }
    buf = static_cast<uint8_t*>(s->dev_alloc(bytes, st));
    if (!buf) {
        g_in_use -= static_cast<int64_t>(bytes);
        have = 0;
        n_have = 0;
        return fail(DARE_E_OOM, "staging allocation of %zu bytes failed", bytes);
    }
    return DARE_OK;
}

dare_status check_plane(const dare_plane* p) {
    if (!p) return fail(DARE_E_INVALID, "plane is NULL");
    if (p->width < 1 || p->height < 1 || p->width > 65535 || p->height > 65535)
        return fail(DARE_E_INVALID, "plane size %dx%d outside [1, 65535]", p->width, p->height);
    if (!(p->px_mm[0] > 0 && p->px_mm[1] > 0) || !std::isfinite(p->px_mm[0]) || !std::isfinite(p->px_mm[1]))
        return fail(DARE_E_INVALID, "pixel spacing must be positive and finite");
    if (!rigid_ok(p->image_to_world)) return fail(DARE_E_INVALID, "image_to_world is not a rigid transform");
    return DARE_OK;
}

dare_status check_params(const dare_params* p) {
    if (!p) return fail(DARE_E_INVALID, "params is NULL");
    const double xs[5] = {p->k_normal, p->k_inplane, p->thr_normal_deg, p->thr_inplane_deg, p->k_dist};
    if (!finite_all(xs, 5)) return fail(DARE_E_INVALID, "non-finite parameter");
    if (p->k_normal < 0 || p->k_inplane < 0) return fail(DARE_E_INVALID, "k_normal and k_inplane must be >= 0");
    if (p->thr_normal_deg < 0 || p->thr_inplane_deg < 0) return fail(DARE_E_INVALID, "thresholds must be >= 0");
    if (p->radius_vox < 1) return fail(DARE_E_INVALID, "radius_vox must be >= 1");
    if (p->dist_kernel < 0 || p->dist_kernel > 2) return fail(DARE_E_INVALID, "unknown distance kernel");
    if (p->normal_axis < 0 || p->normal_axis > 1) return fail(DARE_E_INVALID, "unknown normal axis");
    if (p->weight_dtype < 0 || p->weight_dtype > 1) return fail(DARE_E_INVALID, "unknown weight dtype");
    if (p->path < 0 || p->path > 3) return fail(DARE_E_INVALID, "unknown path");
    if (p->tile_rows != 0 && p->tile_rows != 8 && p->tile_rows != 16 && p->tile_rows != 32 && p->tile_rows != 64)
        return fail(DARE_E_INVALID, "tile_rows must be 0, 8, 16, 32 or 64");
    if (p->radius_vox > 16) return fail(DARE_E_UNSUPPORTED, "radius_vox above 16 is not implemented");
    if (p->dist_kernel == DARE_EXP && !(p->k_dist >= 0)) return fail(DARE_E_INVALID, "k_dist must be >= 0");
    if (p->probe.kind != DARE_PROBE_LINEAR && p->probe.kind != DARE_PROBE_CURVILINEAR)
        return fail(DARE_E_INVALID, "unknown virtual probe kind %d", p->probe.kind);
    if (!finite_all(p->probe.apex_mm, 2)) return fail(DARE_E_INVALID, "virtual probe apex is not finite");
    if (p->sample_weight != DARE_SAMPLE_MEAN && p->sample_weight != DARE_SAMPLE_PIXELS)
        return fail(DARE_E_INVALID, "unknown sample weighting %d", p->sample_weight);
    return DARE_OK;
}

TableParams table_params(const dare_params* p) {
    TableParams t{};
    t.k_normal = p->k_normal;
    t.k_inplane = p->k_inplane;
    t.use_normal = p->thr_normal_deg < 180.0;
    t.use_inplane = p->thr_inplane_deg < 180.0;
    t.cos_normal = std::cos(p->thr_normal_deg * (M_PI / 180.0));
    t.cos_inplane = std::cos(p->thr_inplane_deg * (M_PI / 180.0));
    t.normal_axis = p->normal_axis == DARE_NORMAL_ELEVATION ? 2 : 1;
    t.half = p->weight_dtype == DARE_WEIGHTS_F16;
    return t;
}

void plane_vectors(const dare_session s, const dare_plane* pl, int normal_axis, TableJob* tj) {
    double R[9];
    relative_rotation(s->cfg.grid.vol_to_world, pl->image_to_world, R);
    const int col = normal_axis == DARE_NORMAL_ELEVATION ? 2 : 1;
    for (int r = 0; r < 3; ++r) {
        tj->n_r[r] = R[3 * r + col];
        tj->x_r[r] = R[3 * r + 0];
    }
}

// The distance kernel of params (TENT at radius 1 when NULL) goes into the job.
ResliceJob make_job(const dare_session s, const dare_plane* pl, const void* wtab, float* out, uint32_t* mask,
                    float unassigned, const dare_params* params = nullptr) {
    ResliceJob j{};
    const int R = params ? params->radius_vox : 1;
    j.radius = R;
    j.kernel = params ? params->dist_kernel : DARE_TENT;
    j.k_dist = params ? static_cast<float>(params->k_dist) : 1.0f;
    j.ext_lo = j.kernel == DARE_BOX ? R : R - 1;  // a pixel with floor f reads f - ext_lo .. f + ext_hi
    j.ext_hi = j.kernel == DARE_BOX ? R + 1 : R;
    // pixels reading a voxel column lie within `reach` voxels of it on each in-plane axis
    const double reach = static_cast<double>(std::max(j.ext_hi, j.ext_lo + 1));
    int64_t aff[9];
    compose_affine(s->cfg.grid.vol_to_world, s->cfg.grid.spacing_mm, pl->image_to_world, pl->width, pl->px_mm[0],
                   pl->px_mm[1], aff);
    for (int a = 0; a < 3; ++a) {
        j.g0[a] = aff[a];
        j.a[a] = aff[3 + a];
        j.b[a] = aff[6 + a];
    }
    j.rec = s->rec;
    j.npix = (params && params->sample_weight == DARE_SAMPLE_PIXELS) ? s->npix : nullptr;
    j.wtab = wtab;
    j.out = out;
    j.mask = mask;
    for (int a = 0; a < 3; ++a) j.dims[a] = s->cfg.grid.dims[a];
    j.width = pl->width;
    j.height = pl->height;
    j.mask_stride = (pl->width + 31) / 32;
    j.tiles_x = (pl->width + kTileW - 1) / kTileW;
    j.unassigned = unassigned;
    j.n_frames = s->n_frames;
    // plane geometry for the tiled kernel, from the quantised affine
    const double sc = 1.0 / static_cast<double>(kFixOne);
    double A[3], B[3], G0[3];
    for (int a = 0; a < 3; ++a) {
        A[a] = static_cast<double>(aff[3 + a]) * sc;
        B[a] = static_cast<double>(aff[6 + a]) * sc;
        G0[a] = static_cast<double>(aff[a]) * sc;
    }
    const double n[3] = {A[1] * B[2] - A[2] * B[1], A[2] * B[0] - A[0] * B[2], A[0] * B[1] - A[1] * B[0]};
    int d = 0;
    if (std::fabs(n[1]) > std::fabs(n[d])) d = 1;
    if (std::fabs(n[2]) > std::fabs(n[d])) d = 2;
    const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
    j.d = d;
    const double det = A[e1] * B[e2] - A[e2] * B[e1];
    bool small_steps = true;  // the tiled kernel steps pixels in int32: |A|, |B| < 2^25 (2^-20 voxel units)
    for (int a = 0; a < 3; ++a)
        small_steps = small_steps && std::llabs(aff[3 + a]) < (int64_t(1) << 25) && std::llabs(aff[6 + a]) < (int64_t(1) << 25);
    if (n[d] == 0.0 || det == 0.0 || !small_steps) {
        j.direct = 1;
        return j;
    }
    const double b1 = -n[e1] / n[d], b2 = -n[e2] / n[d];
    const double spread = std::fabs(b1) + std::fabs(b2);
    j.beta1 = static_cast<float>(b1);
    j.beta2 = static_cast<float>(b2);
    j.alpha = static_cast<float>(G0[d] - b1 * G0[e1] - b2 * G0[e2]);
    j.spread = static_cast<float>(spread);
    j.levels = static_cast<int32_t>(std::floor((2.0 * spread + 0.05) * reach)) + j.ext_lo + j.ext_hi + 2;
    const double m00 = B[e2] / det, m01 = -B[e1] / det, m10 = -A[e2] / det, m11 = A[e1] / det;
    j.m00 = static_cast<float>(m00);
    j.m01 = static_cast<float>(m01);
    j.m10 = static_cast<float>(m10);
    j.m11 = static_cast<float>(m11);
    j.ou = static_cast<float>(-(m00 * G0[e1] + m01 * G0[e2]));
    j.ov = static_cast<float>(-(m10 * G0[e1] + m11 * G0[e2]));
    j.hu = static_cast<float>((std::fabs(m00) + std::fabs(m01)) * reach + 0.25);
    j.hv = static_cast<float>((std::fabs(m10) + std::fabs(m11)) * reach + 0.25);
    return j;
}

// Any distance kernel but TENT at radius 1 runs on the general kernels (kernels_radius.cu).
bool general_support(const dare_params* p) {
    return p->radius_vox != 1 || p->dist_kernel != DARE_TENT || p->sample_weight == DARE_SAMPLE_PIXELS;
}
constexpr int kTileHGeneral = 32;  // tile rows of the general tiled kernel

// Shared memory of the general tiled kernel for these jobs: a bound on any
// tile's column box and (A, B) slots.  A plane whose tiles cannot fit gathers
// per pixel (direct).
void general_caps(ResliceJob* jobs, int n, int* col_cap, int* slot_cap) {
    int64_t cols_max = 1, slots_max = 1;
    for (int i = 0; i < n; ++i) {
        ResliceJob& j = jobs[i];
        if (j.direct) continue;
        const int S = j.kernel == DARE_BOX ? 2 * j.radius + 1 : 2 * j.radius;
        const int e1 = j.d == 0 ? 1 : 0, e2 = j.d == 2 ? 1 : 2;
        const double sc = 1.0 / static_cast<double>(kFixOne);
        const double x1 = (std::llabs(j.a[e1]) * double(kTileW - 1) + std::llabs(j.b[e1]) * double(kTileHGeneral - 1)) * sc;
        const double x2 = (std::llabs(j.a[e2]) * double(kTileW - 1) + std::llabs(j.b[e2]) * double(kTileHGeneral - 1)) * sc;
        const int64_t n1 = static_cast<int64_t>(x1) + 2 + j.ext_lo + j.ext_hi;
        const int64_t n2 = static_cast<int64_t>(x2) + 2 + j.ext_lo + j.ext_hi;
        const int64_t cols = n1 * n2, slots = cols * j.levels;
        if (S > kMaxSupport || slots * 8 + cols * 4 > kGeneralSmemCap) {
            j.direct = 1;
            continue;
        }
        cols_max = std::max(cols_max, cols);
        slots_max = std::max(slots_max, slots);
    }
    *col_cap = static_cast<int>(cols_max);
    *slot_cap = static_cast<int>(slots_max);
}

int tiles_of(const dare_plane* pl, int tile_h) {
    return ((pl->width + kTileW - 1) / kTileW) * ((pl->height + tile_h - 1) / tile_h);
}

bool use_tiled(const dare_params* p) { return p->path != DARE_PATH_PLAIN; }

// Rows of the tiled kernel's tiles for a plane (TENT, R = 1).  A tile of 32 x th
// pixels has corner coordinates that differ by at most D = |a| 31 + |b| (th - 1)
// (fixed point) along each in-plane voxel axis, so its floors differ by at most
// floor(D / 2^20) + 1 and the kernel's column box (floors + 2) is at most
// floor(D / 2^20) + 3 wide: the largest th <= cap whose bound fits the kernel's
// columns and (A, B) slots makes every tile fit.  0: none fits (per-pixel kernel).
int tile_rows_fit(const ResliceJob& j, int cap) {
    if (j.direct) return 0;
    const int e1 = j.d == 0 ? 1 : 0, e2 = j.d == 2 ? 1 : 2;
    for (int th = kTileH; th >= 8; th /= 2) {
        if (th > cap) continue;
        const int64_t D1 = std::llabs(j.a[e1]) * (kTileW - 1) + std::llabs(j.b[e1]) * (th - 1);
        const int64_t D2 = std::llabs(j.a[e2]) * (kTileW - 1) + std::llabs(j.b[e2]) * (th - 1);
        const int64_t n1 = (D1 >> kFixBits) + 3, n2 = (D2 >> kFixBits) + 3;
        if (n1 <= kTiledColMax && n2 <= kTiledColMax && n1 * n2 <= kTiledColMax && n1 * n2 * j.levels <= kTiledSlotMax)
            return th;
    }
    return 0;
}

// Tile rows of a job on the tiled path of params (TENT, R = 1): the fit above
// (capped by params->tile_rows), or exactly tile_rows with DARE_PATH_TILED_FIXED.
int tile_rows_for(const ResliceJob& j, const dare_params* p) {
    if (p->path == DARE_PATH_TILED_FIXED) return p->tile_rows ? p->tile_rows : kTileH;
    return tile_rows_fit(j, p->tile_rows ? p->tile_rows : kTileH);
}

// Multiprocessors of the current device (queried once per device).
int sm_count() {
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 148;
    }
    return sms[dev];
}

// A single plane's tile height for low latency: its tiles must spread over the
// device (at least two per multiprocessor where 8 rows allow it) rather than
// take one large tile per multiprocessor, so the automatic choice is capped at
// the largest height that still gives that many tiles.
int tile_rows_single(const ResliceJob& j, const dare_plane* pl, const dare_params* p) {
    if (p->path == DARE_PATH_TILED_FIXED || p->tile_rows != 0) return tile_rows_for(j, p);
    int cap = 8;
    for (int th = kTileH; th > 8; th /= 2)
        if (tiles_of(pl, th) >= 2 * sm_count()) {
            cap = th;
            break;
        }
    return tile_rows_fit(j, cap);
}

// One plane's reslice launch on the path params choose; after_table: the
// plane's weight table was launched just before on `st`.
cudaError_t launch_one(ResliceJob& job, const dare_plane* plane, const dare_params* params, int K, int dtype,
                       int half_w, int after_table, cudaStream_t st) {
    job.tile_base = 0;
    if (general_support(params)) {
        if (use_tiled(params)) {
            int col_cap = 0, slot_cap = 0;
            general_caps(&job, 1, &col_cap, &slot_cap);
            if (!job.direct) {
                g_tiled_planes += 1;
                KernelScope ks("reslice_tiled_r", st, 1);
                return launch_reslice_tiled_r(nullptr, &job, 1, 0, tiles_of(plane, kTileHGeneral), 0, col_cap,
                                              slot_cap, K, dtype, half_w, st);
            }
            g_per_pixel_planes += 1;
        }
        KernelScope ks("reslice_plain_r", st, 1);
        return launch_reslice_plain_r(nullptr, &job, 1, plane->width, plane->height, K, dtype, half_w, st);
    }
    if (use_tiled(params)) {
        const int th = tile_rows_single(job, plane, params);
        if (th > 0) {
            job.tile_h = th;
            g_tiled_planes += 1;
            KernelScope ks("reslice_tiled", st, 1);
            // while tracing, the event recorded between the two launches keeps them apart
            return launch_reslice_tiled(nullptr, &job, 1, 0, tiles_of(plane, th), 0, K, dtype, half_w,
                                        after_table && !g_trace_on.load(), st);
        }
        g_per_pixel_planes += 1;
    }
    KernelScope ks("reslice_plain", st, 1);
    return launch_reslice_plain(nullptr, &job, 1, plane->width, plane->height, K, dtype, half_w, st);
}

// Curvilinear kernel (kernels_curv.cu) for this session and params: the
// session holds frames of a curvilinear probe, or the virtual probe is one.
bool curv_path(const dare_session s, const dare_params* p) {
    return s->n_curv > 0 || p->probe.kind == DARE_PROBE_CURVILINEAR;
}

CurvJob make_curv_job(const dare_session s, const dare_plane* pl, float* out, uint32_t* mask, const dare_params* p) {
    CurvJob c{};
    c.j = make_job(s, pl, nullptr, out, mask, p->unassigned, p);
    c.geom = reinterpret_cast<const float4*>(s->geom_dev);
    c.rot64 = s->frames_dev;
    c.off64 = s->geom_off_dev;
    relative_rotation(s->cfg.grid.vol_to_world, pl->image_to_world, c.R);
    c.h = s->cfg.grid.spacing_mm;
    c.half_w = 0.5 * static_cast<double>(pl->width - 1);
    c.sx = pl->px_mm[0];
    c.sy = pl->px_mm[1];
    c.curv_out = p->probe.kind == DARE_PROBE_CURVILINEAR;
    c.ax = c.curv_out ? p->probe.apex_mm[0] : 0.0;
    c.ay = c.curv_out ? p->probe.apex_mm[1] : 0.0;
    for (int i = 0; i < 9; ++i) c.Rf[i] = static_cast<float>(c.R[i]);
    // pixel (u, v) relative to the virtual apex: (u sx + ox, v sy + oy)
    const double ox = -c.half_w * c.sx - c.ax, oy = -c.ay;
    c.oxf = static_cast<float>(ox);
    c.oyf = static_cast<float>(oy);
    c.sxf = static_cast<float>(c.sx);
    c.syf = static_cast<float>(c.sy);
    const double S = std::max(std::fabs(static_cast<double>(pl->width - 1) * c.sx) + std::fabs(ox),
                              std::fabs(static_cast<double>(pl->height - 1) * c.sy) + std::fabs(oy));
    c.k1p = c.curv_out ? static_cast<float>(17.0 * std::ldexp(1.0, -24) * S * (1.0 + 1e-6)) : 0.0f;
    c.k_n = static_cast<float>(p->k_normal);
    c.k_i = static_cast<float>(p->k_inplane);
    c.use_n = p->thr_normal_deg < 180.0;
    c.use_i = p->thr_inplane_deg < 180.0;
    c.cos_n64 = std::cos(p->thr_normal_deg * (M_PI / 180.0));
    c.cos_i64 = std::cos(p->thr_inplane_deg * (M_PI / 180.0));
    c.cos_n = static_cast<float>(c.cos_n64);
    c.cos_i = static_cast<float>(c.cos_i64);
    c.elevation = p->normal_axis == DARE_NORMAL_ELEVATION;
    return c;
}

// Bricks whose records a plane's support can read: a conservative cover from
// 32 x 32-pixel cells (inside a cell g lies between its values at the cell's
// corners, g being affine in the pixel), each cell's voxel box widened by the
// support's extent below and above floor(g).  Coarser cells cost fewer host
// cycles per plane and add a few boundary bricks to the cover.
void plane_bricks(const dare_session s, const ResliceJob& j, std::vector<uint8_t>& mark, std::vector<int32_t>& out) {
    const int64_t n_b = int64_t(s->nb[0]) * s->nb[1] * s->nb[2];
    mark.assign(size_t(n_b), 0);
    out.clear();
    constexpr int kCell = 32;
    for (int v0 = 0; v0 < j.height; v0 += kCell)
        for (int u0 = 0; u0 < j.width; u0 += kCell) {
            const int u1 = std::min(u0 + kCell - 1, j.width - 1), v1 = std::min(v0 + kCell - 1, j.height - 1);
            int blo[3], bhi[3];
            bool empty = false;
            for (int a = 0; a < 3 && !empty; ++a) {
                const int64_t c[4] = {j.g0[a] + u0 * j.a[a] + v0 * j.b[a], j.g0[a] + u1 * j.a[a] + v0 * j.b[a],
                                      j.g0[a] + u0 * j.a[a] + v1 * j.b[a], j.g0[a] + u1 * j.a[a] + v1 * j.b[a]};
                const int64_t gmin = std::min(std::min(c[0], c[1]), std::min(c[2], c[3]));
                const int64_t gmax = std::max(std::max(c[0], c[1]), std::max(c[2], c[3]));
                const int64_t lo = std::max<int64_t>((gmin >> kFixBits) - j.ext_lo, 0);
                const int64_t hi = std::min<int64_t>((gmax >> kFixBits) + j.ext_hi, j.dims[a] - 1);
                if (lo > hi) {
                    empty = true;
                } else {
                    blo[a] = static_cast<int>(lo / kBrickSide);
                    bhi[a] = static_cast<int>(hi / kBrickSide);
                }
            }
            if (empty) continue;
            for (int bz = blo[2]; bz <= bhi[2]; ++bz)
                for (int by = blo[1]; by <= bhi[1]; ++by)
                    for (int bx = blo[0]; bx <= bhi[0]; ++bx) {
                        const int32_t id = bx + s->nb[0] * (by + s->nb[1] * bz);
                        if (!mark[size_t(id)]) {
                            mark[size_t(id)] = 1;
                            out.push_back(id);
                        }
                    }
        }
}

// Make the bricks of `need` resident: hits keep their slots, misses take the
// next slots (clock order) that this plane does not use; the copies and table
// updates are queued on st from `lists` (device workspace).  A plane needing
// more bricks than the cache has slots pages nothing and reads the missing
// bricks over the host link.
dare_status page_bricks(dare_session s, const std::vector<int32_t>& need, uint8_t* lists, cudaStream_t st) {
    s->stamp += 1;
    if (int64_t(need.size()) > s->n_slots) return DARE_OK;
    std::vector<int32_t> miss;
    for (int32_t b : need) {
        const int32_t sl = s->slot_of_brick[size_t(b)];
        if (sl >= 0) {
            s->slot_stamp[size_t(sl)] = s->stamp;
            s->page_hits += 1;
        } else {
            miss.push_back(b);
        }
    }
    if (miss.empty()) return DARE_OK;
    std::vector<int2> lst;  // table updates (evictions, then insertions), then page copies
    std::vector<int2> ins;
    lst.reserve(2 * miss.size());
    for (int32_t b : miss) {
        int32_t sl = s->hand;
        while (s->slot_stamp[size_t(sl)] == s->stamp) sl = (sl + 1) % s->n_slots;  // need <= n_slots: ends
        s->hand = (sl + 1) % s->n_slots;
        const int32_t old = s->brick_of_slot[size_t(sl)];
        if (old >= 0) {
            s->slot_of_brick[size_t(old)] = -1;
            lst.push_back(make_int2(old, -1));
        }
        s->brick_of_slot[size_t(sl)] = b;
        s->slot_of_brick[size_t(b)] = sl;
        s->slot_stamp[size_t(sl)] = s->stamp;
        ins.push_back(make_int2(b, sl));
    }
    const int n_upd = static_cast<int>(lst.size() + ins.size());
    lst.insert(lst.end(), ins.begin(), ins.end());  // insertions double as the page list
    const size_t bytes = lst.size() * sizeof(int2);
    const int pin = 1 + (s->next_desc++ & 7);
    dare_status rc = ensure_pinned(s, pin, bytes);
    if (rc != DARE_OK) return rc;
    std::memcpy(s->pinned[pin], lst.data(), bytes);
    CUDA_TRY(cudaMemcpyAsync(lists, s->pinned[pin], bytes, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaEventRecord(s->pinned_ev[pin], st));
    const auto* dl = reinterpret_cast<const int2*>(lists);
    {
        KernelScope ks("page_in", st, 2);
        CUDA_TRY(launch_page_in(dl, n_upd, dl + (n_upd - int(ins.size())), static_cast<int>(ins.size()), s->rec,
                                s->cache, s->cfg.grid.dims, s->nb, s->rec_bytes, s->brick_table, st));
    }
    s->pages_in += static_cast<int64_t>(ins.size());
    return DARE_OK;
}

// The paged reslice applies to a session with a brick cache, linear probes
// and per-(voxel, frame) samples; other reslices of such a session read the
// host volume directly.
bool paged_path(const dare_session s, const dare_params* p) {
    return s->cache && !curv_path(s, p) && p->sample_weight == DARE_SAMPLE_MEAN;
}

// n planes of one paged session in one go: the union of their bricks paged in
// once, their weight tables in one launch, one launch of the paged kernel.
// Each plane's result is that of dare_reslice.
dare_status paged_group(dare_session s, const dare_reslice_req* reqs, int n, const std::vector<int32_t>& bricks,
                        const dare_params* params, cudaStream_t st) {
    const int wb = params->weight_dtype == DARE_WEIGHTS_F16 ? 2 : 4;
    const size_t wt = align_up(size_t(std::max(s->n_frames, 1)) * wb, 256);
    const size_t o_tj = wt * size_t(n);
    const size_t o_pj = align_up(o_tj + size_t(n) * sizeof(TableJob), 256);
    const size_t o_ls = align_up(o_pj + size_t(n) * sizeof(PagedJob), 256);
    const size_t need = o_ls + (2 * bricks.size() + 2) * sizeof(int2);
    dare_status rc = session_begin(s, st);
    if (rc != DARE_OK) return rc;
    rc = ensure_workspace(s, need, st);
    if (rc != DARE_OK) return rc;
    uint8_t* ws = static_cast<uint8_t*>(s->ws);
    const int pin = 1 + (s->next_desc++ & 7);
    const size_t desc = o_ls - o_tj;
    rc = ensure_pinned(s, pin, desc);
    if (rc != DARE_OK) return rc;
    uint8_t* pinned = static_cast<uint8_t*>(s->pinned[pin]);
    auto* tjs = reinterpret_cast<TableJob*>(pinned);
    auto* pjs = reinterpret_cast<PagedJob*>(pinned + (o_pj - o_tj));
    int max_w = 0, max_h = 0;
    for (int k = 0; k < n; ++k) {
        TableJob tj{};
        plane_vectors(s, &reqs[k].plane, params->normal_axis, &tj);
        tj.frames = s->frames_dev;
        tj.wtab = ws + size_t(k) * wt;
        tj.n_frames = s->n_frames;
        tjs[k] = tj;
        PagedJob pj{};
        pj.j = make_job(s, &reqs[k].plane, ws + size_t(k) * wt, reqs[k].out, reqs[k].mask, params->unassigned, params);
        pj.cache = s->cache;
        pj.table = s->brick_table;
        for (int a = 0; a < 3; ++a) pj.nb[a] = s->nb[a];
        pjs[k] = pj;
        max_w = std::max(max_w, reqs[k].plane.width);
        max_h = std::max(max_h, reqs[k].plane.height);
    }
    CUDA_TRY(cudaMemcpyAsync(ws + o_tj, pinned, desc, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaEventRecord(s->pinned_ev[pin], st));
    if (s->n_frames > 0) {
        KernelScope ks("weight_table", st, 1);
        CUDA_TRY(launch_weight_tables(reinterpret_cast<const TableJob*>(ws + o_tj), nullptr, n, s->n_frames,
                                      table_params(params), st));
    }
    rc = page_bricks(s, bricks, ws + o_ls, st);
    if (rc != DARE_OK) return rc;
    {
        KernelScope ks("reslice_paged", st, 1);
        CUDA_TRY(launch_reslice_paged(reinterpret_cast<const PagedJob*>(ws + o_pj), nullptr, n, max_w, max_h, s->K,
                                      s->dtype, params->weight_dtype == DARE_WEIGHTS_F16, st));
    }
    return session_end(s, st);
}

}  // namespace

// ---------------------------------------------------------------- batch helpers (shared with the server)

namespace dare {

dare_status check_batch(const dare_reslice_req* reqs, int32_t n, const dare_params* params, bool allow_paged) {
    dare_status rc = check_params(params);
    if (rc != DARE_OK) return rc;
    for (int32_t i = 0; i < n; ++i) {
        const dare_reslice_req& r = reqs[i];
        if (!r.session) return fail(DARE_E_INVALID, "request %d has no session", i);
        if (r.session->cache && !allow_paged)
            return fail(DARE_E_UNSUPPORTED, "request %d: a session with a brick cache (use dare_reslice_batch)", i);
        if (r.session->cfg.device != reqs[0].session->cfg.device) return fail(DARE_E_INVALID, "requests span devices");
        rc = check_plane(&r.plane);
        if (rc != DARE_OK) return fail(rc, "request %d: %s", i, g_err.c_str());
        if (!r.out || !r.mask) return fail(DARE_E_INVALID, "request %d: output pointers are NULL", i);
        if (!affine_ok(r.session->cfg.grid.vol_to_world, r.session->cfg.grid.spacing_mm, r.plane.image_to_world,
                       r.plane.width, r.plane.px_mm[0], r.plane.px_mm[1]))
            return fail(DARE_E_INVALID, "request %d: plane too far from the grid", i);
    }
    return DARE_OK;
}

// Device workspace (weight tables + descriptors) and pinned descriptor bytes of a batch.
void batch_sizes(const dare_reslice_req* reqs, int32_t n, const dare_params* params, size_t* ws_need,
                 size_t* desc_bytes) {
    const int wb = params->weight_dtype == DARE_WEIGHTS_F16 ? 2 : 4;
    size_t o = 0;
    for (int32_t i = 0; i < n; ++i) o = align_up(o + size_t(std::max(reqs[i].session->n_frames, 1)) * wb, 256);
    const size_t o_tj = o;
    const size_t o_rj = align_up(o_tj + size_t(n) * sizeof(TableJob), 256);
    const size_t o_cj = align_up(o_rj + size_t(n) * sizeof(ResliceJob), 256);
    *ws_need = align_up(o_cj + size_t(n) * sizeof(CurvJob), 256);
    *desc_bytes = *ws_need - o_tj;
}

// A bound on batch_sizes for any batch of n requests whose sessions hold at most
// max_frames frames each.
void batch_sizes_bound(int32_t n, int32_t max_frames, size_t* ws_need, size_t* desc_bytes) {
    const size_t o_tj = size_t(n) * align_up(size_t(std::max(max_frames, 1)) * 4, 256);
    const size_t o_rj = align_up(o_tj + size_t(n) * sizeof(TableJob), 256);
    const size_t o_cj = align_up(o_rj + size_t(n) * sizeof(ResliceJob), 256);
    *ws_need = align_up(o_cj + size_t(n) * sizeof(CurvJob), 256);
    *desc_bytes = *ws_need - o_tj;
}

// Queue weight tables and reslice launches for a checked batch on `st`, using
// device workspace `ws` and pinned staging `pin` (sized by batch_sizes).  No
// ordering against the sessions' other work: the caller provides it.
dare_status queue_batch(const dare_reslice_req* reqs, int32_t n, const dare_params* params, cudaStream_t st,
                        uint8_t* ws, uint8_t* pin) {
    const int wb = params->weight_dtype == DARE_WEIGHTS_F16 ? 2 : 4;
    std::vector<size_t> t_off(n);
    size_t o = 0;
    int max_frames = 0;
    for (int32_t i = 0; i < n; ++i) {
        t_off[i] = o;
        o = align_up(o + size_t(std::max(reqs[i].session->n_frames, 1)) * wb, 256);
        max_frames = std::max(max_frames, reqs[i].session->n_frames);
    }
    const size_t o_tj = o;
    const size_t o_rj = align_up(o_tj + size_t(n) * sizeof(TableJob), 256);
    const size_t o_cj = align_up(o_rj + size_t(n) * sizeof(ResliceJob), 256);
    const size_t desc_bytes = align_up(o_cj + size_t(n) * sizeof(CurvJob), 256) - o_tj;
    auto* tjs = reinterpret_cast<TableJob*>(pin);
    auto* rjs = reinterpret_cast<ResliceJob*>(pin + (o_rj - o_tj));
    auto* cjs = reinterpret_cast<CurvJob*>(pin + (o_cj - o_tj));
    const bool general = general_support(params);
    const bool tiled = use_tiled(params);
    // every request's job and route: 0 tiled kernel, 1 per-pixel kernel (the plain
    // path, or a plane no tile fits), 2 curvilinear kernel
    std::vector<ResliceJob> jobs(n);
    std::vector<char> route(n);
    for (int32_t i = 0; i < n; ++i) {
        const dare_reslice_req& r = reqs[i];
        jobs[i] = make_job(r.session, &r.plane, ws + t_off[i], r.out, r.mask, params->unassigned, params);
        if (curv_path(r.session, params)) {
            route[i] = 2;
        } else if (!tiled) {
            route[i] = 1;
        } else if (!general) {
            jobs[i].tile_h = tile_rows_for(jobs[i], params);
            route[i] = jobs[i].tile_h > 0 ? 0 : 1;
        }
    }
    int col_cap = 0, slot_cap = 0;
    if (general && tiled) {
        std::vector<int32_t> idx;
        std::vector<ResliceJob> gj;
        for (int32_t i = 0; i < n; ++i)
            if (route[i] != 2) {
                idx.push_back(i);
                gj.push_back(jobs[i]);
            }
        general_caps(gj.data(), static_cast<int>(gj.size()), &col_cap, &slot_cap);
        for (size_t k = 0; k < idx.size(); ++k) {
            jobs[idx[k]] = gj[k];
            route[idx[k]] = gj[k].direct ? 1 : 0;
        }
    }
    // order jobs by (kernel family, K, dtype) so each launch covers one group
    std::vector<int32_t> order(n);
    for (int32_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        const auto* sa = reqs[a].session;
        const auto* sb = reqs[b].session;
        if ((route[a] == 2) != (route[b] == 2)) return route[a] < route[b];
        if (sa->K != sb->K) return sa->K < sb->K;
        if (sa->dtype != sb->dtype) return sa->dtype < sb->dtype;
        return route[a] < route[b];
    });
    max_frames = 0;
    for (int32_t i = 0; i < n; ++i)
        if (route[i] != 2) max_frames = std::max(max_frames, reqs[i].session->n_frames);
    const int th_general = kTileHGeneral;
    int total_tiles = 0;
    for (int32_t k = 0; k < n; ++k) {
        const int32_t i = order[k];
        const dare_reslice_req& r = reqs[i];
        TableJob tj{};
        plane_vectors(r.session, &r.plane, params->normal_axis, &tj);
        tj.frames = r.session->frames_dev;
        tj.wtab = ws + t_off[i];
        tj.n_frames = route[i] == 2 ? 0 : r.session->n_frames;  // the curvilinear kernel needs no table
        tjs[k] = tj;
        rjs[k] = jobs[i];
        if (route[i] == 2) cjs[k] = make_curv_job(r.session, &r.plane, r.out, r.mask, params);
        rjs[k].tile_base = total_tiles;
        if (route[i] == 0) total_tiles += tiles_of(&r.plane, general ? th_general : rjs[k].tile_h);
    }
    CUDA_TRY(cudaMemcpyAsync(ws + o_tj, pin, desc_bytes, cudaMemcpyHostToDevice, st));
    const auto* tj_dev = reinterpret_cast<const TableJob*>(ws + o_tj);
    const auto* rj_dev = reinterpret_cast<const ResliceJob*>(ws + o_rj);
    const auto* cj_dev = reinterpret_cast<const CurvJob*>(ws + o_cj);
    if (max_frames > 0) {
        KernelScope ks("weight_table", st, 1);
        CUDA_TRY(launch_weight_tables(tj_dev, nullptr, n, max_frames, table_params(params), st));
    }
    const int half_w = params->weight_dtype == DARE_WEIGHTS_F16;
    for (int32_t k0 = 0; k0 < n;) {
        const int32_t i0 = order[k0];
        const auto* sg = reqs[i0].session;
        const char rg = route[i0];
        int32_t k1 = k0;
        int max_w = 0, max_h = 0;
        while (k1 < n && route[order[k1]] == rg && reqs[order[k1]].session->K == sg->K &&
               reqs[order[k1]].session->dtype == sg->dtype) {
            max_w = std::max(max_w, reqs[order[k1]].plane.width);
            max_h = std::max(max_h, reqs[order[k1]].plane.height);
            ++k1;
        }
        if (rg == 2) {
            KernelScope ks("reslice_curv", st, 1);
            CUDA_TRY(launch_reslice_curv(cj_dev + k0, nullptr, k1 - k0, max_w, max_h, sg->K, sg->dtype, st));
        } else if (rg == 0) {
            g_tiled_planes += k1 - k0;
            const int base = rjs[k0].tile_base;
            const int end = (k1 < n && route[order[k1]] == 0) ? rjs[k1].tile_base : total_tiles;
            // same tile count for every job of the group: 2-D grid without a job search
            const int per = tiles_of(&reqs[i0].plane, general ? th_general : rjs[k0].tile_h);
            bool uniform = k1 - k0 <= 65535;
            for (int32_t k = k0; uniform && k < k1; ++k)
                uniform = tiles_of(&reqs[order[k]].plane, general ? th_general : rjs[k].tile_h) == per;
            if (general) {
                KernelScope ks("reslice_tiled_r", st, 1);
                CUDA_TRY(launch_reslice_tiled_r(rj_dev + k0, nullptr, k1 - k0, base, uniform ? per : end - base,
                                                uniform ? 1 : 0, col_cap, slot_cap, sg->K, sg->dtype, half_w, st));
            } else {
                KernelScope ks("reslice_tiled", st, 1);
                CUDA_TRY(launch_reslice_tiled(rj_dev + k0, nullptr, k1 - k0, base, uniform ? per : end - base,
                                              uniform ? 1 : 0, sg->K, sg->dtype, half_w,
                                              k0 == 0 && max_frames > 0 && !g_trace_on.load(), st));
            }
        } else {
            if (tiled) g_per_pixel_planes += k1 - k0;
            if (general) {
                KernelScope ks("reslice_plain_r", st, 1);
                CUDA_TRY(launch_reslice_plain_r(rj_dev + k0, nullptr, k1 - k0, max_w, max_h, sg->K, sg->dtype, half_w,
                                                st));
            } else {
                KernelScope ks("reslice_plain", st, 1);
                CUDA_TRY(launch_reslice_plain(rj_dev + k0, nullptr, k1 - k0, max_w, max_h, sg->K, sg->dtype, half_w,
                                              st));
            }
        }
        k0 = k1;
    }
    return DARE_OK;
}

}  // namespace dare

// ---------------------------------------------------------------- ABI

extern "C" {

const char* dare_last_error(void) { return g_err.c_str(); }

int32_t dare_abi_version(void) { return DARE_ABI_VERSION; }

dare_status dare_params_default(dare_params* p) {
    if (!p) return fail(DARE_E_INVALID, "params is NULL");
    std::memset(p, 0, sizeof(*p));
    p->k_normal = 10.0;
    p->k_inplane = 5.0;
    p->thr_normal_deg = 25.0;
    p->thr_inplane_deg = 15.0;
    p->k_dist = 1.0;
    p->unassigned = 0.0f;
    p->radius_vox = 1;
    p->dist_kernel = DARE_TENT;
    p->normal_axis = DARE_NORMAL_BEAM;
    p->weight_dtype = DARE_WEIGHTS_F32;
    p->path = DARE_PATH_AUTO;
    return DARE_OK;
}

dare_status dare_set_memory_budget(int64_t bytes) {
    if (bytes < 0) return fail(DARE_E_INVALID, "budget must be >= 0");
    g_budget = bytes;
    return DARE_OK;
}

int64_t dare_memory_in_use(void) { return g_in_use.load(); }

dare_status dare_grid_from_frames(int32_t n, int32_t width, int32_t height, const double px_mm[2],
                                  const double* image_to_world, double spacing_mm, int32_t margin_vox,
                                  dare_grid* out) {
    if (n < 1 || width < 1 || height < 1 || !px_mm || !image_to_world || !out || !(spacing_mm > 0) || margin_vox < 0)
        return fail(DARE_E_INVALID, "bad arguments to dare_grid_from_frames");
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int32_t f = 0; f < n; ++f) {
        const double* T = image_to_world + 16 * static_cast<size_t>(f);
        if (!rigid_ok(T)) return fail(DARE_E_INVALID, "pose %d is not rigid", f);
        for (int cu = 0; cu < 2; ++cu)
            for (int cv = 0; cv < 2; ++cv) {
                const double x = ((cu ? width - 1 : 0) - 0.5 * (width - 1)) * px_mm[0];
                const double y = (cv ? height - 1 : 0) * px_mm[1];
                for (int a = 0; a < 3; ++a) {
                    const double w = T[4 * a] * x + T[4 * a + 1] * y + T[4 * a + 3];
                    lo[a] = std::min(lo[a], w);
                    hi[a] = std::max(hi[a], w);
                }
            }
    }
    std::memset(out, 0, sizeof(*out));
    out->spacing_mm = spacing_mm;
    for (int a = 0; a < 3; ++a) {
        const double ext = std::ceil((hi[a] - lo[a]) / spacing_mm);
        if (!(ext < 1e6)) return fail(DARE_E_INVALID, "bounding box too large");
        out->dims[a] = static_cast<int32_t>(ext) + 1 + 2 * margin_vox;
        out->vol_to_world[4 * a + a] = 1.0;
        out->vol_to_world[4 * a + 3] = lo[a] - margin_vox * spacing_mm;
    }
    out->vol_to_world[15] = 1.0;
    return DARE_OK;
}

dare_status dare_pixel_affine(const dare_grid* grid, const dare_plane* plane, int64_t out[9]) {
    if (!grid || !out) return fail(DARE_E_INVALID, "NULL argument");
    dare_status st = check_plane(plane);
    if (st != DARE_OK) return st;
    if (!(grid->spacing_mm > 0) || !rigid_ok(grid->vol_to_world)) return fail(DARE_E_INVALID, "bad grid");
    if (!affine_ok(grid->vol_to_world, grid->spacing_mm, plane->image_to_world, plane->width, plane->px_mm[0],
                   plane->px_mm[1]))
        return fail(DARE_E_INVALID, "plane too far from the grid for fixed-point coordinates");
    compose_affine(grid->vol_to_world, grid->spacing_mm, plane->image_to_world, plane->width, plane->px_mm[0],
                   plane->px_mm[1], out);
    return DARE_OK;
}

dare_status dare_session_create(const dare_session_config* cfg, dare_session* out) {
    if (!cfg || !out) return fail(DARE_E_INVALID, "NULL argument");
    *out = nullptr;
    const dare_grid& g = cfg->grid;
    if (g.dims[0] < 1 || g.dims[1] < 1 || g.dims[2] < 1 || g.dims[0] > 4096 || g.dims[1] > 4096 || g.dims[2] > 4096)
        return fail(DARE_E_INVALID, "grid dims must be in [1, 4096]");
    if (!(g.spacing_mm > 0) || !std::isfinite(g.spacing_mm)) return fail(DARE_E_INVALID, "spacing must be > 0");
    if (!rigid_ok(g.vol_to_world)) return fail(DARE_E_INVALID, "vol_to_world is not a rigid transform");
    if (cfg->dtype < DARE_U8 || cfg->dtype > DARE_F32) return fail(DARE_E_INVALID, "unknown dtype");
    if (cfg->max_slots != 4 && cfg->max_slots != 8 && cfg->max_slots != 12 && cfg->max_slots != 16)
        return fail(DARE_E_INVALID, "max_slots must be 4, 8, 12 or 16");
    if (cfg->max_frames < 1 || cfg->max_frames > DARE_MAX_FRAMES)
        return fail(DARE_E_INVALID, "max_frames must be in [1, 65535]");
    if ((cfg->alloc.alloc == nullptr) != (cfg->alloc.free == nullptr))
        return fail(DARE_E_INVALID, "allocator needs both alloc and free");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return fail(DARE_E_INVALID, "device %d not available (%d devices)", cfg->device, ndev);
    }
    const int64_t n_vox = int64_t(g.dims[0]) * g.dims[1] * g.dims[2];
    if (n_vox >= (int64_t(1) << 31)) return fail(DARE_E_INVALID, "grid has 2^31 voxels or more");
    DeviceGuard dg(cfg->device);
    if (!dg.ok) return fail(DARE_E_CUDA, "cannot select device %d", cfg->device);

    auto* s = new dare_session_s();
    s->cfg = *cfg;
    s->n_vox = n_vox;
    s->K = cfg->max_slots;
    s->dtype = cfg->dtype;
    s->rec_bytes = record_bytes(s->K, s->dtype);
    const bool scalar = (cfg->flags & DARE_SESSION_SCALAR) != 0;
    const size_t b_rec = align_up(size_t(n_vox) * s->rec_bytes, 256);
    const size_t b_np = align_up(size_t(n_vox) * s->K * 2, 256);
    const size_t b_sc = scalar ? align_up(size_t(n_vox) * 4, 256) : 0;
    const size_t b_cnt = align_up(size_t(n_vox) * 4, 256);
    const size_t b_fr = align_up(size_t(cfg->max_frames) * 9 * 8, 256);
    const size_t b_geo = align_up(size_t(cfg->max_frames) * kGeomFloats * 4, 256);
    const size_t b_goff = align_up(size_t(cfg->max_frames) * 2 * 8, 256);
    const size_t b_ovf = 256;
    // records, npix and scalar totals: device memory, or mapped host memory (DARE_SESSION_HOST_VOLUME)
    const bool host_vol = (cfg->flags & DARE_SESSION_HOST_VOLUME) != 0;
    const size_t b_vol = b_rec + b_np + 2 * b_sc;
    const size_t total = (host_vol ? 0 : b_vol) + b_cnt + b_fr + b_geo + b_goff + b_ovf;
    uint8_t* vol = nullptr;
    if (host_vol) {
        void* h = nullptr;
        if (cudaHostAlloc(&h, b_vol, cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return fail(DARE_E_OOM, "host volume allocation of %zu bytes failed", b_vol);
        }
        void* d = nullptr;
        if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(h);
            delete s;
            return fail(DARE_E_CUDA, "host volume is not mapped into the device");
        }
        s->host_vol = h;
        vol = static_cast<uint8_t*>(d);
    }
    dare_status st = admit(static_cast<int64_t>(total));
    if (st != DARE_OK) {
        if (s->host_vol) cudaFreeHost(s->host_vol);
        delete s;
        return st;
    }
    uint8_t* base = static_cast<uint8_t*>(s->dev_alloc(total, nullptr));
    if (!base) {
        g_in_use -= static_cast<int64_t>(total);
        if (s->host_vol) cudaFreeHost(s->host_vol);
        delete s;
        return fail(DARE_E_OOM, "volume allocation of %zu bytes failed", total);
    }
    s->allocs.push_back({base, total});
    s->volume_bytes = static_cast<int64_t>(total);
    size_t off = 0;
    if (!host_vol) {
        vol = base;
        off = b_vol;
    }
    s->rec = vol;
    s->npix = reinterpret_cast<uint16_t*>(vol + b_rec);
    if (scalar) {
        s->ssum = reinterpret_cast<uint32_t*>(vol + b_rec + b_np);
        s->scnt = reinterpret_cast<uint32_t*>(vol + b_rec + b_np + b_sc);
    }
    s->count = reinterpret_cast<int32_t*>(base + off);
    off += b_cnt;
    s->frames_dev = reinterpret_cast<double*>(base + off);
    off += b_fr;
    s->geom_dev = reinterpret_cast<float*>(base + off);
    off += b_geo;
    s->geom_off_dev = reinterpret_cast<double*>(base + off);
    off += b_goff;
    s->overflow_dev = reinterpret_cast<unsigned long long*>(base + off);
    auto bail = [&](dare_status code) {
        dare_session_destroy(s);
        return code;
    };
    if (cudaEventCreateWithFlags(&s->order_ev, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(DARE_E_CUDA, "event creation failed"));
    for (int k = 0; k < dare_session_s::kPinSlots; ++k)
        if (cudaEventCreateWithFlags(&s->pinned_ev[k], cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(DARE_E_CUDA, "event creation failed"));
    // clear: empty records, zero counters (synchronous)
    g_launches += 1;
    if (launch_fill_records(s->rec, n_vox, s->rec_bytes, s->K, nullptr) != cudaSuccess ||
        cudaMemset(s->npix, 0, b_np) != cudaSuccess || cudaMemset(s->count, 0, b_cnt) != cudaSuccess ||
        cudaMemset(s->overflow_dev, 0, b_ovf) != cudaSuccess ||
        (scalar && cudaMemset(s->ssum, 0, 2 * b_sc) != cudaSuccess) || cudaDeviceSynchronize() != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        return bail(fail(DARE_E_CUDA, "clearing the volume failed: %s", cudaGetErrorString(e)));
    }
    bool rec_ok = cudaEventRecord(s->order_ev, nullptr) == cudaSuccess;
    for (int k = 0; k < dare_session_s::kPinSlots; ++k)
        rec_ok = rec_ok && cudaEventRecord(s->pinned_ev[k], nullptr) == cudaSuccess;
    if (!rec_ok) return bail(fail(DARE_E_CUDA, "event record failed"));
    *out = s;
    return DARE_OK;
}

dare_status dare_session_destroy(dare_session s) {
    if (!s) return DARE_OK;
    DeviceGuard dg(s->cfg.device);
    if (s->order_ev) cudaEventSynchronize(s->order_ev);
    for (int k = 0; k < dare_session_s::kPinSlots; ++k)
        if (s->pinned_ev[k]) cudaEventSynchronize(s->pinned_ev[k]);
    if (s->sp_exec) cudaGraphExecDestroy(s->sp_exec);
    if (s->sp_graph) cudaGraphDestroy(s->sp_graph);
    // lines marked persisting stay so after the records are freed and would keep
    // their share of L2 from every later kernel; this returns all of the context's
    // persisting lines to normal (another persisting session's lines are marked
    // again by its next call)
    if ((s->cfg.flags & DARE_SESSION_L2_PERSIST) && cudaCtxResetPersistingL2Cache() != cudaSuccess) cudaGetLastError();
    if (s->ws) {
        s->dev_free(s->ws, s->ws_bytes, s->last_stream);
        g_in_use -= static_cast<int64_t>(s->ws_bytes);
    }
    for (auto& a : s->allocs) {
        s->dev_free(a.first, a.second, s->last_stream);
        g_in_use -= static_cast<int64_t>(a.second);
    }
    for (int k = 0; k < dare_session_s::kPinSlots; ++k) {
        if (s->pinned[k]) cudaFreeHost(s->pinned[k]);
        if (s->pinned_ev[k]) cudaEventDestroy(s->pinned_ev[k]);
    }
    if (s->up_st) {
        cudaStreamSynchronize(s->up_st);
        cudaStreamSynchronize(s->down_st);
        std::vector<cudaEvent_t> evs;
        for (int k = 0; k < 2; ++k) evs.insert(evs.end(), {s->ring_free[k], s->ring_full[k]});
        for (int k = 0; k < dare_session_s::kStageSlots; ++k) evs.insert(evs.end(), {s->stage_free[k], s->stage_full[k]});
        for (cudaEvent_t e : evs) {
            cudaEventSynchronize(e);
            cudaEventDestroy(e);
        }
        cudaStreamDestroy(s->up_st);
        cudaStreamDestroy(s->down_st);
    }
    if (s->ring) {
        s->dev_free(s->ring, size_t(s->ring_n) * s->ring_slot, s->last_stream);
        g_in_use -= static_cast<int64_t>(size_t(s->ring_n) * s->ring_slot);
    }
    if (s->stage) {
        s->dev_free(s->stage, size_t(s->stage_n) * s->stage_slot, s->last_stream);
        g_in_use -= static_cast<int64_t>(size_t(s->stage_n) * s->stage_slot);
    }
    if (s->host_vol) {
        cudaDeviceSynchronize();  // no kernel may still touch the mapped volume
        cudaFreeHost(s->host_vol);
    }
    if (s->pix_mask) {
        s->dev_free(s->pix_mask, s->pix_mask_bytes, s->last_stream);
        g_in_use -= static_cast<int64_t>(s->pix_mask_bytes);
    }
    if (s->filled) {
        s->dev_free(s->filled, s->filled_bytes, s->last_stream);
        g_in_use -= static_cast<int64_t>(s->filled_bytes);
    }
    if (s->cache) {
        s->dev_free(s->cache, s->cache_bytes + s->table_bytes, s->last_stream);
        g_in_use -= static_cast<int64_t>(s->cache_bytes + s->table_bytes);
    }
    if (s->order_ev) cudaEventDestroy(s->order_ev);
    delete s;
    return DARE_OK;
}

dare_status dare_session_sync(dare_session s) {
    if (!s) return fail(DARE_E_INVALID, "session is NULL");
    DeviceGuard dg(s->cfg.device);
    // poll first (short waits resume at once), then block
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(s->order_ev);
        if (e == cudaSuccess) return DARE_OK;
        if (e != cudaErrorNotReady) {
            cudaGetLastError();
            return fail(DARE_E_CUDA, "device failure: %s", cudaGetErrorString(e));
        }
        if (std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(200)) break;
    }
    CUDA_TRY(cudaEventSynchronize(s->order_ev));
    return DARE_OK;
}

dare_status dare_session_query(dare_session s, dare_session_info* out) {
    if (!s || !out) return fail(DARE_E_INVALID, "NULL argument");
    DeviceGuard dg(s->cfg.device);
    CUDA_TRY(cudaEventSynchronize(s->order_ev));
    unsigned long long ovf = 0;
    CUDA_TRY(cudaMemcpy(&ovf, s->overflow_dev, sizeof(ovf), cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(*out));
    out->volume_bytes = s->volume_bytes;
    out->workspace_bytes = static_cast<int64_t>(s->ws_bytes);
    out->overflow_voxels = static_cast<int64_t>(ovf);
    out->version = s->version;
    out->n_frames = s->n_frames;
    out->slots = s->K;
    out->dtype = s->dtype;
    out->record_bytes = s->rec_bytes;
    for (int a = 0; a < 3; ++a) out->dims[a] = s->cfg.grid.dims[a];
    out->flags = s->cfg.flags;
    out->spacing_mm = s->cfg.grid.spacing_mm;
    std::memcpy(out->vol_to_world, s->cfg.grid.vol_to_world, sizeof(out->vol_to_world));
    return DARE_OK;
}

dare_status dare_session_read_records(dare_session s, uint16_t* frame_ids, void* values, uint16_t* npix,
                                      uint32_t* scalar_sum, uint32_t* scalar_count) {
    if (!s) return fail(DARE_E_INVALID, "session is NULL");
    if ((scalar_sum || scalar_count) && !s->ssum) return fail(DARE_E_STATE, "session keeps no scalar totals");
    DeviceGuard dg(s->cfg.device);
    dare_status rc = settle_now(s);
    if (rc != DARE_OK) return rc;
    CUDA_TRY(cudaEventSynchronize(s->order_ev));
    const int vb = value_bytes(s->dtype);
    if (frame_ids || values) {
        std::vector<uint8_t> host(size_t(s->n_vox) * s->rec_bytes);
        CUDA_TRY(cudaMemcpy(host.data(), s->rec, host.size(), cudaMemcpyDeviceToHost));
        for (int64_t v = 0; v < s->n_vox; ++v) {
            const uint8_t* r = host.data() + size_t(v) * s->rec_bytes;
            if (frame_ids) std::memcpy(frame_ids + size_t(v) * s->K, r, size_t(2) * s->K);
            if (values)
                std::memcpy(static_cast<uint8_t*>(values) + size_t(v) * s->K * vb, r + 2 * s->K, size_t(s->K) * vb);
        }
    }
    if (npix) CUDA_TRY(cudaMemcpy(npix, s->npix, size_t(s->n_vox) * s->K * 2, cudaMemcpyDeviceToHost));
    if (scalar_sum) CUDA_TRY(cudaMemcpy(scalar_sum, s->ssum, size_t(s->n_vox) * 4, cudaMemcpyDeviceToHost));
    if (scalar_count) CUDA_TRY(cudaMemcpy(scalar_count, s->scnt, size_t(s->n_vox) * 4, cudaMemcpyDeviceToHost));
    return DARE_OK;
}

dare_status dare_session_read_frames(dare_session s, double* rotations) {
    if (!s || (!rotations && s->n_frames > 0)) return fail(DARE_E_INVALID, "NULL argument");
    if (s->n_frames > 0) std::memcpy(rotations, s->frames_host.data(), s->frames_host.size() * sizeof(double));
    return DARE_OK;
}

}  // extern "C"

namespace {

// Reconstruction of n frames (Fig. 1).  host: frames are in host memory and go
// through the session's upload ring in slices of slice_frames frames, each
// slice's upload overlapping the scatter count of the previous one.
dare_status build_impl(dare_session s, const uint8_t* frames, bool host, int32_t n, int32_t width, int32_t height,
                       const double px_mm[2], const double* image_to_world, int32_t slice_frames, void* stream) {
    if (!s) return fail(DARE_E_INVALID, "session is NULL");
    if (slice_frames < 0) return fail(DARE_E_INVALID, "slice_frames must be >= 0");
    if (n < 0 || width < 1 || height < 1 || width > 65535 || height > 65535)
        return fail(DARE_E_INVALID, "bad frame count or size");
    if (n == 0) return DARE_OK;
    if (!frames || !image_to_world || !px_mm) return fail(DARE_E_INVALID, "NULL argument");
    if (!(px_mm[0] > 0 && px_mm[1] > 0) || !std::isfinite(px_mm[0]) || !std::isfinite(px_mm[1]))
        return fail(DARE_E_INVALID, "pixel spacing must be positive and finite");
    if (int64_t(s->n_frames) + n > s->cfg.max_frames)
        return fail(DARE_E_CAPACITY, "%d frames + %d new exceed max_frames %d", s->n_frames, n, s->cfg.max_frames);
    const int64_t npx = int64_t(width) * height;
    // pair slots of a frame: one per pixel of its whole 32 x 32 tiles
    const int64_t tiles_pf = int64_t((width + kScatterTile - 1) / kScatterTile) * ((height + kScatterTile - 1) / kScatterTile);
    const int64_t slots_pf = tiles_pf * kScatterTile * kScatterTile;
    if (slots_pf > kMaxPixelsPerChunk) return fail(DARE_E_INVALID, "frame too large");
    if (s->pix_mask && (width != s->pm_w || height != s->pm_h))
        return fail(DARE_E_INVALID, "frames are %dx%d but the pixel mask is %dx%d", width, height, s->pm_w, s->pm_h);
    const double* V = s->cfg.grid.vol_to_world;
    const double h = s->cfg.grid.spacing_mm;
    std::vector<int64_t> aff(size_t(n) * 9);
    std::vector<double> rot(size_t(n) * 9);
    // probe geometry of the new frames: FP32 rows, FP64 offsets, (kind, offsets) for save / load
    std::vector<float> grow(size_t(n) * kGeomFloats);
    std::vector<double> goff(size_t(n) * 2), prow(size_t(n) * 3);
    const int kind = s->probe.kind;
    for (int32_t f = 0; f < n; ++f) {
        const double* T = image_to_world + 16 * size_t(f);
        if (!rigid_ok(T)) return fail(DARE_E_INVALID, "frame pose %d is not a rigid transform", f);
        if (!affine_ok(V, h, T, width, px_mm[0], px_mm[1]))
            return fail(DARE_E_INVALID, "frame %d too far from the grid for fixed-point coordinates", f);
        compose_affine(V, h, T, width, px_mm[0], px_mm[1], &aff[9 * size_t(f)]);
        relative_rotation(V, T, &rot[9 * size_t(f)]);
        probe_offsets(V, T, &rot[9 * size_t(f)], s->probe.apex_mm, &goff[2 * size_t(f)]);
        geometry_row(s->cfg.grid, &rot[9 * size_t(f)], kind, &goff[2 * size_t(f)], &grow[size_t(f) * kGeomFloats]);
        prow[3 * size_t(f)] = kind;
        prow[3 * size_t(f) + 1] = goff[2 * size_t(f)];
        prow[3 * size_t(f) + 2] = goff[2 * size_t(f) + 1];
    }
    DeviceGuard dg(s->cfg.device);
    if (!dg.ok) return fail(DARE_E_CUDA, "cannot select device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t chunk = static_cast<int32_t>(std::min<int64_t>(65535, std::max<int64_t>(1, kMaxPixelsPerChunk / slots_pf)));
    const int32_t n_chunk = std::min(n, chunk);
    // workspace: offsets (n_vox + 1), scan block sums, overflow entries (at most one per pixel),
    // buckets (kBucket entries per voxel), the overflow (voxel, entry) pair list (one slot per pixel
    // of the frame tiles) and its length, affines
    const int64_t nbs = scan_block_sums_needed(s->n_vox);
    const size_t o_off = 0;
    const size_t o_bs = align_up(o_off + size_t(s->n_vox + 1) * 4, 256);
    const size_t o_ent = align_up(o_bs + size_t(nbs) * 4, 256);
    const size_t o_bk = align_up(o_ent + size_t(n_chunk) * npx * 8, 256);
    const size_t o_pairs = align_up(o_bk + size_t(s->n_vox) * kBucket * 8, 256);
    const size_t o_np = align_up(o_pairs + size_t(n_chunk) * slots_pf * 16, 256);
    // appends that reach few voxels (a chunk of fewer pixels than a quarter of the
    // grid's voxels) list the voxels they touch and finalize only those: touched
    // list, voxel -> list position, list overflow counts, list length
    const int64_t max_t = std::min<int64_t>(s->n_vox, int64_t(n_chunk) * npx);
    const size_t o_aff = align_up(o_np + 16, 256);
    const size_t o_tl = align_up(o_aff + size_t(n) * 9 * 8, 256);
    const size_t o_ti = align_up(o_tl + size_t(max_t) * 4, 256);
    const size_t o_tc = align_up(o_ti + size_t(s->n_vox) * 4, 256);
    const size_t o_tn = align_up(o_tc + size_t(max_t) * 4, 256);
    const size_t ws_need = align_up(o_tn + 16, 256);
    // upload slices (host frames): about 32 MB each unless given
    const int32_t slice = !host ? 0
                                : static_cast<int32_t>(std::min<int64_t>(
                                      n_chunk, slice_frames > 0 ? slice_frames
                                                                : std::max<int64_t>(1, (int64_t(32) << 20) / npx)));
    dare_status rc = session_begin(s, st, false);  // a pending clear is left to the first finalize
    if (rc != DARE_OK) return rc;
    rc = ensure_workspace(s, ws_need, st);
    if (rc != DARE_OK) return rc;
    if (host) {
        rc = ensure_host_io(s);
        if (rc != DARE_OK) return rc;
        rc = ensure_slots(s, s->ring, s->ring_slot, s->ring_n, size_t(slice) * npx, 2,
                          {s->ring_free[0], s->ring_free[1], s->ring_full[0], s->ring_full[1]}, st);
        if (rc != DARE_OK) return rc;
    }
    // two staging buffers in turn, so the host can queue a build while the
    // previous one's upload is still waiting on the stream
    const int bpin = (s->next_build++ & 1) ? 9 : 0;
    rc = ensure_pinned(s, bpin, size_t(n) * (9 * 8 * 2 + kGeomFloats * 4 + 2 * 8));
    if (rc != DARE_OK) return rc;
    uint8_t* ws = static_cast<uint8_t*>(s->ws);
    int32_t* offsets = reinterpret_cast<int32_t*>(ws + o_off);
    int32_t* bsums = reinterpret_cast<int32_t*>(ws + o_bs);
    auto* entries = reinterpret_cast<unsigned long long*>(ws + o_ent);
    auto* buckets = reinterpret_cast<unsigned long long*>(ws + o_bk);
    auto* pairs = reinterpret_cast<uint4*>(ws + o_pairs);
    auto* n_pairs = reinterpret_cast<int32_t*>(ws + o_np);
    int64_t* aff_dev = reinterpret_cast<int64_t*>(ws + o_aff);
    int32_t* t_list = reinterpret_cast<int32_t*>(ws + o_tl);
    int32_t* t_index = reinterpret_cast<int32_t*>(ws + o_ti);
    int32_t* t_ovf = reinterpret_cast<int32_t*>(ws + o_tc);
    int32_t* t_n = reinterpret_cast<int32_t*>(ws + o_tn);
    uint8_t* pin = static_cast<uint8_t*>(s->pinned[bpin]);
    const size_t p_rot = aff.size() * 8, p_geo = p_rot + rot.size() * 8, p_off = p_geo + grow.size() * 4;
    std::memcpy(pin, aff.data(), aff.size() * 8);
    std::memcpy(pin + p_rot, rot.data(), rot.size() * 8);
    std::memcpy(pin + p_geo, grow.data(), grow.size() * 4);
    std::memcpy(pin + p_off, goff.data(), goff.size() * 8);
    CUDA_TRY(cudaMemcpyAsync(aff_dev, pin, aff.size() * 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(s->frames_dev + size_t(s->n_frames) * 9, pin + p_rot, rot.size() * 8,
                             cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(s->geom_dev + size_t(s->n_frames) * kGeomFloats, pin + p_geo, grow.size() * 4,
                             cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(s->geom_off_dev + size_t(s->n_frames) * 2, pin + p_off, goff.size() * 8,
                             cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaEventRecord(s->pinned_ev[bpin], st));
    for (int32_t c0 = 0; c0 < n; c0 += n_chunk) {
        const int32_t nc = std::min(n_chunk, n - c0);
        ScatterArgs a{};
        a.frames = frames + size_t(c0) * npx;
        a.affines = aff_dev + size_t(c0) * 9;
        a.n = nc;
        a.width = width;
        a.height = height;
        for (int k = 0; k < 3; ++k) a.dims[k] = s->cfg.grid.dims[k];
        a.frame_base = s->n_frames + c0;
        a.pix_mask = s->pix_mask;
        a.small_steps = 1;
        for (int32_t f = c0; f < c0 + nc; ++f)
            for (int k = 3; k < 9; ++k)
                if (std::llabs(aff[9 * size_t(f) + k]) >= (int64_t(1) << 25)) a.small_steps = 0;
        const int mode = s->pending_clear ? 2 : (s->fresh ? 1 : 0);
        const bool listed = mode != 2 && int64_t(nc) * npx * 4 < s->n_vox;
        int32_t* tl = listed ? t_list : nullptr;
        int32_t* ti = listed ? t_index : nullptr;
        int32_t* tn = listed ? t_n : nullptr;
        if (listed || mode == 2) CUDA_TRY(cudaMemsetAsync(t_n, 0, sizeof(int32_t), st));
        // the chunk's overflow list starts empty (and, in the full-write mode, the cursor of
        // its overflow ranges, n_pairs[1])
        CUDA_TRY(cudaMemsetAsync(n_pairs, 0, 2 * sizeof(int32_t), st));
        if (!host) {
            KernelScope ks("scatter_count", st, 1);
            CUDA_TRY(launch_scatter_count(a, s->count, buckets, pairs, n_pairs, tl, ti, tn, st));
        } else {
            for (int32_t j0 = 0, k = 0; j0 < nc; j0 += slice, ++k) {
                const int b = k & 1;
                const int32_t nj = std::min(slice, nc - j0);
                uint8_t* slot = s->ring + size_t(b) * s->ring_slot;
                // upload into a free slot, then count from it on the caller's stream
                CUDA_TRY(cudaStreamWaitEvent(s->up_st, s->ring_free[b], 0));
                CUDA_TRY(cudaMemcpyAsync(slot, frames + (size_t(c0) + j0) * npx, size_t(nj) * npx,
                                         cudaMemcpyHostToDevice, s->up_st));
                CUDA_TRY(cudaEventRecord(s->ring_full[b], s->up_st));
                CUDA_TRY(cudaStreamWaitEvent(st, s->ring_full[b], 0));
                ScatterArgs sa = a;
                sa.frames = slot;
                sa.affines = a.affines + size_t(j0) * 9;
                sa.n = nj;
                sa.frame_base = a.frame_base + j0;
                {
                    KernelScope ks("scatter_count", st, 1);
                    CUDA_TRY(launch_scatter_count(sa, s->count, buckets, pairs, n_pairs, tl, ti, tn, st));
                }
                CUDA_TRY(cudaEventRecord(s->ring_free[b], st));
            }
        }
        if (mode == 2) {
            // full write: an overflow range for each voxel past its bucket only, no scan of
            // every counter; the counters keep every entry for the finalize passes
            {
                KernelScope ks("overflow_alloc", st, 1);
                CUDA_TRY(launch_overflow_alloc(pairs, n_pairs, s->count, offsets, n_pairs + 1, st));
            }
            KernelScope ks("scatter_place", st, 1);
            CUDA_TRY(launch_overflow_place(pairs, n_pairs, offsets, entries, st));
        } else {
            if (listed) {
                KernelScope ks("exclusive_scan", st, 4);
                CUDA_TRY(launch_touched_overflow(s->count, t_list, t_n, max_t, t_ovf, st));
                CUDA_TRY(launch_exclusive_scan(t_ovf, offsets, max_t, bsums, nbs, 0, st));
            } else {
                KernelScope ks("exclusive_scan", st, 3);
                CUDA_TRY(launch_exclusive_scan(s->count, offsets, s->n_vox, bsums, nbs, kBucket, st));
            }
            KernelScope ks("scatter_place", st, 1);
            CUDA_TRY(launch_scatter_place(a, pairs, n_pairs, s->count, offsets, ti, entries, st));
        }
        {
            if (c0 == 0) {
                rc = invalidate_cache(s, st);  // the records are about to change
                if (rc != DARE_OK) return rc;
            }
            s->pending_clear = false;  // a full-write finalize (mode 2) writes every voxel
            s->fresh = false;          // from here on the records may hold samples
            // a full write lists the voxels with entries past their bucket, and their entry
            // counts, in the touched list and its counts (unused in that mode) for its second kernel
            {
                KernelScope ks("finalize", st, 1);
                // fewer than 8 pixels per voxel: most buckets are empty (1600 frames of 256 x 512
                // into 256^3 give 12.5 and 83 % of the voxels covered; 400 frames give 3.1)
                const int sparse = int64_t(nc) * npx < 8 * s->n_vox ? 1 : 0;
                CUDA_TRY(launch_finalize(s->count, buckets, offsets, entries, s->n_vox, s->rec, s->npix, s->ssum,
                                         s->scnt, s->K, s->dtype, mode, s->host_vol ? 0 : 1, sparse, s->overflow_dev, tl, tn,
                                         max_t, mode == 2 ? t_list : nullptr, mode == 2 ? t_ovf : nullptr,
                                         mode == 2 ? t_n : nullptr, st));
            }
            if (mode == 2) {
                KernelScope ks("finalize_deferred", st, 1);
                CUDA_TRY(launch_finalize_deferred(t_list, t_ovf, t_n, buckets, offsets, entries, s->rec, s->npix, s->ssum,
                                                  s->scnt, s->K, s->dtype, s->overflow_dev, max_t, st));
            }
        }
    }
    rc = session_end(s, st);
    if (rc != DARE_OK) return rc;
    s->frames_host.insert(s->frames_host.end(), rot.begin(), rot.end());
    s->probe_host.insert(s->probe_host.end(), prow.begin(), prow.end());
    if (kind == DARE_PROBE_CURVILINEAR) s->n_curv += n;
    s->n_frames += n;
    s->version += 1;
    return DARE_OK;
}

}  // namespace

extern "C" {

dare_status dare_build_volume(dare_session s, const uint8_t* frames_dev, int32_t n, int32_t width, int32_t height,
                              const double px_mm[2], const double* image_to_world, void* stream) {
    return build_impl(s, frames_dev, false, n, width, height, px_mm, image_to_world, 0, stream);
}

dare_status dare_build_volume_host(dare_session s, const uint8_t* frames_host, int32_t n, int32_t width,
                                   int32_t height, const double px_mm[2], const double* image_to_world,
                                   int32_t slice_frames, void* stream) {
    return build_impl(s, frames_host, true, n, width, height, px_mm, image_to_world, slice_frames, stream);
}

dare_status dare_session_set_cache(dare_session s, int64_t bytes) {
    if (!s) return fail(DARE_E_INVALID, "session is NULL");
    if (!s->host_vol) return fail(DARE_E_STATE, "a brick cache needs DARE_SESSION_HOST_VOLUME");
    if (bytes < 0) return fail(DARE_E_INVALID, "cache bytes must be >= 0");
    DeviceGuard dg(s->cfg.device);
    if (!dg.ok) return fail(DARE_E_CUDA, "cannot select device");
    CUDA_TRY(cudaEventSynchronize(s->order_ev));  // queued reslices may still read the old cache
    if (s->cache) {
        s->dev_free(s->cache, s->cache_bytes + s->table_bytes, s->last_stream);
        g_in_use -= static_cast<int64_t>(s->cache_bytes + s->table_bytes);
        s->cache = nullptr;
        s->brick_table = nullptr;
        s->cache_bytes = s->table_bytes = 0;
        s->n_slots = 0;
    }
    if (bytes == 0) return DARE_OK;
    for (int a = 0; a < 3; ++a) s->nb[a] = (s->cfg.grid.dims[a] + kBrickSide - 1) / kBrickSide;
    const int64_t n_b = int64_t(s->nb[0]) * s->nb[1] * s->nb[2];
    const size_t slot_bytes = size_t(kBrickVoxels) * s->rec_bytes;
    const int64_t slots = std::min<int64_t>(bytes / static_cast<int64_t>(slot_bytes), n_b);
    if (slots < 1) return fail(DARE_E_INVALID, "cache of %lld bytes holds no brick of %zu bytes", (long long)bytes, slot_bytes);
    if (slots > INT32_MAX / kBrickVoxels) return fail(DARE_E_INVALID, "cache too large");
    const size_t cbytes = align_up(size_t(slots) * slot_bytes, 256), tbytes = align_up(size_t(n_b) * 4, 256);
    dare_status rc = admit(static_cast<int64_t>(cbytes + tbytes));
    if (rc != DARE_OK) return rc;
    auto* base = static_cast<uint8_t*>(s->dev_alloc(cbytes + tbytes, nullptr));
    if (!base) {
        g_in_use -= static_cast<int64_t>(cbytes + tbytes);
        return fail(DARE_E_OOM, "brick cache allocation of %zu bytes failed", cbytes + tbytes);
    }
    if (cudaMemset(base + cbytes, 0xFF, tbytes) != cudaSuccess) {
        cudaGetLastError();
        s->dev_free(base, cbytes + tbytes, nullptr);
        g_in_use -= static_cast<int64_t>(cbytes + tbytes);
        return fail(DARE_E_CUDA, "brick table clear failed");
    }
    s->cache = base;
    s->cache_bytes = cbytes;
    s->brick_table = reinterpret_cast<int32_t*>(base + cbytes);
    s->table_bytes = tbytes;
    s->n_slots = static_cast<int32_t>(slots);
    s->slot_of_brick.assign(size_t(n_b), -1);
    s->brick_of_slot.assign(size_t(slots), -1);
    s->slot_stamp.assign(size_t(slots), 0);
    s->hand = 0;
    s->pages_in = s->page_hits = 0;
    return DARE_OK;
}

dare_status dare_session_cache_stats(dare_session s, int64_t out[4]) {
    if (!s || !out) return fail(DARE_E_INVALID, "NULL argument");
    int64_t resident = 0;
    for (int32_t b : s->brick_of_slot) resident += b >= 0;
    out[0] = s->n_slots;
    out[1] = resident;
    out[2] = s->pages_in;
    out[3] = s->page_hits;
    return DARE_OK;
}

dare_status dare_session_set_probe(dare_session s, const dare_probe* probe, const uint8_t* pixel_mask,
                                   int32_t width, int32_t height) {
    if (!s || !probe) return fail(DARE_E_INVALID, "NULL argument");
    if (probe->kind != DARE_PROBE_LINEAR && probe->kind != DARE_PROBE_CURVILINEAR)
        return fail(DARE_E_INVALID, "unknown probe kind %d", probe->kind);
    if (!finite_all(probe->apex_mm, 2)) return fail(DARE_E_INVALID, "probe apex is not finite");
    if (pixel_mask && (width < 1 || height < 1 || width > 65535 || height > 65535))
        return fail(DARE_E_INVALID, "pixel mask size %dx%d outside [1, 65535]", width, height);
    DeviceGuard dg(s->cfg.device);
    if (!dg.ok) return fail(DARE_E_CUDA, "cannot select device");
    CUDA_TRY(cudaEventSynchronize(s->order_ev));  // queued builds may still read the old mask
    if (s->pix_mask) {
        s->dev_free(s->pix_mask, s->pix_mask_bytes, s->last_stream);
        g_in_use -= static_cast<int64_t>(s->pix_mask_bytes);
        s->pix_mask = nullptr;
        s->pix_mask_bytes = 0;
        s->pm_w = s->pm_h = 0;
    }
    if (pixel_mask) {
        const int words = (width + 31) / 32;
        std::vector<uint32_t> bits(size_t(words) * height, 0u);
        for (int32_t y = 0; y < height; ++y)
            for (int32_t x = 0; x < width; ++x)
                if (pixel_mask[size_t(y) * width + x]) bits[size_t(y) * words + x / 32] |= 1u << (x % 32);
        const size_t bytes = align_up(bits.size() * 4, 256);
        dare_status rc = admit(static_cast<int64_t>(bytes));
        if (rc != DARE_OK) return rc;
        auto* d = static_cast<uint32_t*>(s->dev_alloc(bytes, nullptr));
        if (!d) {
            g_in_use -= static_cast<int64_t>(bytes);
            return fail(DARE_E_OOM, "pixel mask allocation failed");
        }
        if (cudaMemcpy(d, bits.data(), bits.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaError_t e = cudaGetLastError();
            s->dev_free(d, bytes, nullptr);
            g_in_use -= static_cast<int64_t>(bytes);
            return fail(DARE_E_CUDA, "pixel mask upload failed: %s", cudaGetErrorString(e));
        }
        s->pix_mask = d;
        s->pix_mask_bytes = bytes;
        s->pm_w = width;
        s->pm_h = height;
    }
    s->probe = *probe;
    return DARE_OK;
}


// One plane's weight table and tiled reslice as the session's two-node graph:
// both nodes' parameters (grid and job) are replaced and the graph is launched
// once, which costs the host about half of two kernel launches and starts the
// reslice on the device right after the table.  The graph is rebuilt when the
// kernels change (storage type, slots or weight precision), or if an update is
// refused.
dare_status single_plane_graph(dare_session s, const TableJob& tj, const ResliceJob& job, int n_tiles,
                               const TableParams& tp, int half_w, cudaStream_t st) {
    NodeArgs a_tab, a_res;
    cudaKernelNodeParams p_tab, p_res;
    CUDA_TRY(weight_table_node(tj, tj.n_frames, tp, a_tab, &p_tab));
    CUDA_TRY(reslice_tiled_node(job, n_tiles, s->K, s->dtype, half_w, a_res, &p_res));
    bool ready = s->sp_exec && s->sp_fn[0] == p_tab.func && s->sp_fn[1] == p_res.func;
    if (ready && (cudaGraphExecKernelNodeSetParams(s->sp_exec, s->sp_node[0], &p_tab) != cudaSuccess ||
                  cudaGraphExecKernelNodeSetParams(s->sp_exec, s->sp_node[1], &p_res) != cudaSuccess)) {
        cudaGetLastError();
        ready = false;
    }
    if (!ready) {
        if (s->sp_exec) cudaGraphExecDestroy(s->sp_exec);
        if (s->sp_graph) cudaGraphDestroy(s->sp_graph);
        s->sp_exec = nullptr;
        s->sp_graph = nullptr;
        s->sp_fn[0] = s->sp_fn[1] = nullptr;
        CUDA_TRY(cudaGraphCreate(&s->sp_graph, 0));
        CUDA_TRY(cudaGraphAddKernelNode(&s->sp_node[0], s->sp_graph, nullptr, 0, &p_tab));
        CUDA_TRY(cudaGraphAddKernelNode(&s->sp_node[1], s->sp_graph, nullptr, 0, &p_res));
        // a programmatic edge: the reslice's CTAs start (and set their tiles up)
        // as soon as the table kernel has begun; they wait for its results
        // (griddepcontrol.wait) before reading the table
        cudaGraphEdgeData edge{};
        edge.from_port = cudaGraphKernelNodePortProgrammatic;
        edge.type = cudaGraphDependencyTypeProgrammatic;
        CUDA_TRY(cudaGraphAddDependencies(s->sp_graph, &s->sp_node[0], &s->sp_node[1], &edge, 1));
        CUDA_TRY(cudaGraphInstantiate(&s->sp_exec, s->sp_graph, 0));
        s->sp_fn[0] = p_tab.func;
        s->sp_fn[1] = p_res.func;
    }
    g_launches += 2;
    CUDA_TRY(cudaGraphLaunch(s->sp_exec, st));
    return DARE_OK;
}

dare_status dare_reslice(dare_session s, const dare_plane* plane, const dare_params* params, float* out_dev,
                         uint32_t* mask_dev, void* stream) {
    if (!s) return fail(DARE_E_INVALID, "session is NULL");
    dare_status rc = check_plane(plane);
    if (rc != DARE_OK) return rc;
    rc = check_params(params);
    if (rc != DARE_OK) return rc;
    if (!out_dev || !mask_dev) return fail(DARE_E_INVALID, "output pointers are NULL");
    if (!affine_ok(s->cfg.grid.vol_to_world, s->cfg.grid.spacing_mm, plane->image_to_world, plane->width,
                   plane->px_mm[0], plane->px_mm[1]))
        return fail(DARE_E_INVALID, "plane too far from the grid for fixed-point coordinates");
    DeviceGuard dg(s->cfg.device);
    if (!dg.ok) return fail(DARE_E_CUDA, "cannot select device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = session_begin(s, st);
    if (rc != DARE_OK) return rc;
    if (paged_path(s, params)) {
        const int wbp = params->weight_dtype == DARE_WEIGHTS_F16 ? 2 : 4;
        const size_t wt_bytes = align_up(size_t(std::max(s->n_frames, 1)) * wbp, 256);
        std::vector<int32_t> need;
        {
            const ResliceJob probe_job = make_job(s, plane, nullptr, out_dev, mask_dev, params->unassigned, params);
            plane_bricks(s, probe_job, s->brick_mark, need);
        }
        rc = ensure_workspace(s, wt_bytes + (2 * need.size() + 2) * sizeof(int2), st);
        if (rc != DARE_OK) return rc;
        TableJob tjp{};
        plane_vectors(s, plane, params->normal_axis, &tjp);
        tjp.frames = s->frames_dev;
        tjp.wtab = s->ws;
        tjp.n_frames = s->n_frames;
        if (s->n_frames > 0) {
            KernelScope ks("weight_table", st, 1);
            CUDA_TRY(launch_weight_tables(nullptr, &tjp, 1, s->n_frames, table_params(params), st));
        }
        rc = page_bricks(s, need, static_cast<uint8_t*>(s->ws) + wt_bytes, st);
        if (rc != DARE_OK) return rc;
        PagedJob pj{};
        pj.j = make_job(s, plane, s->ws, out_dev, mask_dev, params->unassigned, params);
        pj.cache = s->cache;
        pj.table = s->brick_table;
        for (int a = 0; a < 3; ++a) pj.nb[a] = s->nb[a];
        {
            KernelScope ks("reslice_paged", st, 1);
            CUDA_TRY(launch_reslice_paged(nullptr, &pj, 1, plane->width, plane->height, s->K, s->dtype,
                                          params->weight_dtype == DARE_WEIGHTS_F16, st));
        }
        return session_end(s, st);
    }
    if (curv_path(s, params)) {
        const CurvJob cj = make_curv_job(s, plane, out_dev, mask_dev, params);
        L2Window l2((s->cfg.flags & DARE_SESSION_L2_PERSIST) ? s->rec : nullptr, size_t(s->n_vox) * s->rec_bytes, st);
        KernelScope ks("reslice_curv", st, 1);
        CUDA_TRY(launch_reslice_curv(nullptr, &cj, 1, plane->width, plane->height, s->K, s->dtype, st));
        return session_end(s, st);
    }
    const int wb = params->weight_dtype == DARE_WEIGHTS_F16 ? 2 : 4;
    rc = ensure_workspace(s, align_up(size_t(std::max(s->n_frames, 1)) * wb, 256), st);
    if (rc != DARE_OK) return rc;
    TableJob tj{};
    plane_vectors(s, plane, params->normal_axis, &tj);
    tj.frames = s->frames_dev;
    tj.wtab = s->ws;
    tj.n_frames = s->n_frames;
    ResliceJob job = make_job(s, plane, s->ws, out_dev, mask_dev, params->unassigned, params);
    const int half_w = params->weight_dtype == DARE_WEIGHTS_F16;
    if (s->n_frames > 0 && !g_trace_on.load() && !(s->cfg.flags & DARE_SESSION_L2_PERSIST) &&
        !general_support(params) && use_tiled(params)) {
        const int th = tile_rows_single(job, plane, params);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (th > 0 && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            job.tile_h = th;
            job.tile_base = 0;
            rc = single_plane_graph(s, tj, job, tiles_of(plane, th), table_params(params), half_w, st);
            if (rc != DARE_OK) return rc;
            g_tiled_planes += 1;
            return session_end(s, st);
        }
    }
    if (s->n_frames > 0) {
        KernelScope ks("weight_table", st, 1);
        CUDA_TRY(launch_weight_tables(nullptr, &tj, 1, s->n_frames, table_params(params), st));
    }
    L2Window l2((s->cfg.flags & DARE_SESSION_L2_PERSIST) ? s->rec : nullptr, size_t(s->n_vox) * s->rec_bytes, st);
    CUDA_TRY(launch_one(job, plane, params, s->K, s->dtype, half_w, s->n_frames > 0, st));
    return session_end(s, st);
}

dare_status dare_reslice_batch(const dare_reslice_req* reqs, int32_t n, const dare_params* params, void* stream) {
    if (n < 0 || (n > 0 && !reqs)) return fail(DARE_E_INVALID, "bad request list");
    if (n == 0) return DARE_OK;
    dare_status rc = dare::check_batch(reqs, n, params, true);
    if (rc != DARE_OK) return rc;
    for (int32_t i = 0; i < n; ++i)
        if (reqs[i].session->cache) {
            // sessions with a brick cache page per group of planes: consecutive requests of one such
            // session whose bricks fit its cache together (at most 64) go as one group; any other
            // request runs alone, in order
            DeviceGuard dgp(reqs[0].session->cfg.device);
            cudaStream_t sp = static_cast<cudaStream_t>(stream);
            std::vector<uint8_t> umark;
            std::vector<int32_t> uni, need;
            for (int32_t k = 0; k < n;) {
                dare_session s = reqs[k].session;
                if (!paged_path(s, params)) {
                    rc = dare_reslice(s, &reqs[k].plane, params, reqs[k].out, reqs[k].mask, stream);
                    if (rc != DARE_OK) return rc;
                    ++k;
                    continue;
                }
                umark.assign(size_t(s->nb[0]) * s->nb[1] * s->nb[2], 0);
                uni.clear();
                int32_t j = k;
                while (j < n && j - k < 64 && reqs[j].session == s) {
                    const ResliceJob pj = make_job(s, &reqs[j].plane, nullptr, reqs[j].out, reqs[j].mask,
                                                   params->unassigned, params);
                    plane_bricks(s, pj, s->brick_mark, need);
                    size_t add = 0;
                    for (int32_t b : need) add += umark[size_t(b)] ? 0 : 1;
                    if (j > k && int64_t(uni.size() + add) > s->n_slots) break;
                    for (int32_t b : need)
                        if (!umark[size_t(b)]) {
                            umark[size_t(b)] = 1;
                            uni.push_back(b);
                        }
                    ++j;
                }
                rc = paged_group(s, reqs + k, j - k, uni, params, sp);
                if (rc != DARE_OK) return rc;
                k = j;
            }
            return DARE_OK;
        }
    dare_session s0 = reqs[0].session;
    DeviceGuard dg(s0->cfg.device);
    if (!dg.ok) return fail(DARE_E_CUDA, "cannot select device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // distinct sessions, in first-seen order
    std::vector<dare_session> sess;
    for (int32_t i = 0; i < n; ++i)
        if (std::find(sess.begin(), sess.end(), reqs[i].session) == sess.end()) sess.push_back(reqs[i].session);
    for (auto* s : sess) {
        rc = session_begin(s, st);
        if (rc != DARE_OK) return rc;
    }
    size_t ws_need = 0, desc_bytes = 0;
    dare::batch_sizes(reqs, n, params, &ws_need, &desc_bytes);
    rc = ensure_workspace(s0, ws_need, st);
    if (rc != DARE_OK) return rc;
    const int pin = 1 + (s0->next_desc++ & 7);  // descriptor slots 1..8 in turn
    rc = ensure_pinned(s0, pin, desc_bytes);
    if (rc != DARE_OK) return rc;
    {
        const bool one_l2 = sess.size() == 1 && (s0->cfg.flags & DARE_SESSION_L2_PERSIST);
        L2Window l2(one_l2 ? s0->rec : nullptr, size_t(s0->n_vox) * s0->rec_bytes, st);
        rc = dare::queue_batch(reqs, n, params, st, static_cast<uint8_t*>(s0->ws),
                               static_cast<uint8_t*>(s0->pinned[pin]));
    }
    if (rc != DARE_OK) return rc;
    CUDA_TRY(cudaEventRecord(s0->pinned_ev[pin], st));
    for (auto* s : sess) {
        rc = session_end(s, st);
        if (rc != DARE_OK) return rc;
    }
    return DARE_OK;
}

dare_status dare_reslice_batch_host(const dare_reslice_req* reqs, int32_t n, const dare_params* params,
                                    int32_t group_planes, void* stream) {
    if (n < 0 || (n > 0 && !reqs)) return fail(DARE_E_INVALID, "bad request list");
    if (group_planes < 0) return fail(DARE_E_INVALID, "group_planes must be >= 0");
    if (n == 0) return DARE_OK;
    dare_status rc = dare::check_batch(reqs, n, params);
    if (rc != DARE_OK) return rc;
    dare_session s0 = reqs[0].session;
    DeviceGuard dg(s0->cfg.device);
    if (!dg.ok) return fail(DARE_E_CUDA, "cannot select device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<size_t> ob(n), mb(n);  // staging bytes of each image and mask
    for (int32_t i = 0; i < n; ++i) {
        const dare_plane& pl = reqs[i].plane;
        ob[i] = size_t(pl.width) * pl.height * 4;
        mb[i] = size_t(pl.height) * ((pl.width + 31) / 32) * 4;
    }
    // groups of consecutive requests: group_planes planes, or about 128 MB of output
    std::vector<int32_t> gs;  // first request of each group, then n
    size_t slot_need = 0, cur = 0;
    for (int32_t i = 0, cnt = 0; i < n; ++i) {
        const bool full = group_planes > 0 ? cnt == group_planes : cur + ob[i] + mb[i] > (size_t(128) << 20);
        if (cnt == 0 || full) {
            gs.push_back(i);
            cur = 0;
            cnt = 0;
        }
        cur += ob[i] + mb[i];
        ++cnt;
        slot_need = std::max(slot_need, cur);
    }
    gs.push_back(n);
    rc = ensure_host_io(s0);
    if (rc != DARE_OK) return rc;
    const int32_t ng = static_cast<int32_t>(gs.size()) - 1;
    // slots: enough for the groups to run ahead of their downloads, within about 1 GB
    const int n_slots = static_cast<int>(std::max<int64_t>(
        2, std::min<int64_t>({int64_t(dare_session_s::kStageSlots), int64_t(ng),
                              int64_t((size_t(1) << 30) / std::max<size_t>(slot_need, 1))})));
    std::vector<cudaEvent_t> stage_ev;
    for (int k = 0; k < dare_session_s::kStageSlots; ++k) stage_ev.insert(stage_ev.end(), {s0->stage_free[k], s0->stage_full[k]});
    rc = ensure_slots(s0, s0->stage, s0->stage_slot, s0->stage_n, slot_need, n_slots, stage_ev, st);
    if (rc != DARE_OK) return rc;
    std::vector<dare_reslice_req> sub;
    for (int32_t g = 0; g < ng; ++g) {
        const int32_t a = gs[g], b = gs[g + 1];
        const int sl = g % s0->stage_n;
        uint8_t* base = s0->stage + size_t(sl) * s0->stage_slot;
        // slot layout: the group's images in request order, then its masks
        size_t out_total = 0;
        for (int32_t i = a; i < b; ++i) out_total += ob[i];
        sub.assign(reqs + a, reqs + b);
        std::vector<uint8_t*> so(b - a), sm(b - a);
        size_t oo = 0, mo = 0;
        for (int32_t i = a; i < b; ++i) {
            so[i - a] = base + oo;
            sm[i - a] = base + out_total + mo;
            sub[i - a].out = reinterpret_cast<float*>(so[i - a]);
            sub[i - a].mask = reinterpret_cast<uint32_t*>(sm[i - a]);
            oo += ob[i];
            mo += mb[i];
        }
        CUDA_TRY(cudaStreamWaitEvent(st, s0->stage_free[sl], 0));
        rc = dare_reslice_batch(sub.data(), b - a, params, st);
        if (rc != DARE_OK) return rc;
        CUDA_TRY(cudaEventRecord(s0->stage_full[sl], st));
        CUDA_TRY(cudaStreamWaitEvent(s0->down_st, s0->stage_full[sl], 0));
        // downloads; requests whose host buffers follow each other go in one copy
        for (int pass = 0; pass < 2; ++pass) {
            for (int32_t i = a; i < b;) {
                uint8_t* dst = pass == 0 ? reinterpret_cast<uint8_t*>(reqs[i].out) : reinterpret_cast<uint8_t*>(reqs[i].mask);
                const uint8_t* src = pass == 0 ? so[i - a] : sm[i - a];
                size_t bytes = pass == 0 ? ob[i] : mb[i];
                int32_t j = i + 1;
                for (; j < b; ++j) {
                    const uint8_t* next = pass == 0 ? reinterpret_cast<const uint8_t*>(reqs[j].out)
                                                    : reinterpret_cast<const uint8_t*>(reqs[j].mask);
                    if (next != dst + bytes) break;
                    bytes += pass == 0 ? ob[j] : mb[j];
                }
                CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s0->down_st));
                i = j;
            }
        }
        CUDA_TRY(cudaEventRecord(s0->stage_free[sl], s0->down_st));
    }
    // the caller's stream covers the downloads (in order on the download stream)
    CUDA_TRY(cudaStreamWaitEvent(st, s0->stage_free[(ng - 1) % s0->stage_n], 0));
    return DARE_OK;
}

dare_status dare_reslice_scalar(dare_session s, const dare_plane* plane, float unassigned, float* out_dev,
                                uint32_t* mask_dev, void* stream) {
    if (!s) return fail(DARE_E_INVALID, "session is NULL");
    dare_status rc = check_plane(plane);
    if (rc != DARE_OK) return rc;
    if (!s->ssum) return fail(DARE_E_STATE, "session was created without DARE_SESSION_SCALAR");
    if (!out_dev || !mask_dev) return fail(DARE_E_INVALID, "output pointers are NULL");
    if (!affine_ok(s->cfg.grid.vol_to_world, s->cfg.grid.spacing_mm, plane->image_to_world, plane->width,
                   plane->px_mm[0], plane->px_mm[1]))
        return fail(DARE_E_INVALID, "plane too far from the grid for fixed-point coordinates");
    DeviceGuard dg(s->cfg.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = session_begin(s, st);
    if (rc != DARE_OK) return rc;
    ResliceJob job = make_job(s, plane, nullptr, out_dev, mask_dev, unassigned);
    {
        KernelScope ks("reslice_scalar", st, 1);
        CUDA_TRY(launch_reslice_scalar(job, s->ssum, s->scnt, st));
    }
    return session_end(s, st);
}

dare_status dare_fill_holes(dare_session s, int32_t radius_vox, int32_t min_neighbours, void* stream) {
    if (!s) return fail(DARE_E_INVALID, "session is NULL");
    if (!s->ssum) return fail(DARE_E_STATE, "session was created without DARE_SESSION_SCALAR");
    if (radius_vox < 1 || radius_vox > 8) return fail(DARE_E_INVALID, "radius_vox must be in [1, 8]");
    const int cube = (2 * radius_vox + 1) * (2 * radius_vox + 1) * (2 * radius_vox + 1) - 1;
    if (min_neighbours < 0 || min_neighbours > cube)
        return fail(DARE_E_INVALID, "min_neighbours must be in [0, %d]", cube);
    DeviceGuard dg(s->cfg.device);
    if (!dg.ok) return fail(DARE_E_CUDA, "cannot select device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    dare_status rc = session_begin(s, st);
    if (rc != DARE_OK) return rc;
    if (!s->filled) {
        const size_t bytes = align_up(size_t(s->n_vox) * 4, 256);
        rc = admit(static_cast<int64_t>(bytes));
        if (rc != DARE_OK) return rc;
        s->filled = static_cast<float*>(s->dev_alloc(bytes, st));
        if (!s->filled) {
            g_in_use -= static_cast<int64_t>(bytes);
            return fail(DARE_E_OOM, "hole-filled volume allocation of %zu bytes failed", bytes);
        }
        s->filled_bytes = bytes;
    }
    {
        KernelScope ks("fill_holes", st, 1);
        CUDA_TRY(launch_fill_holes(s->cfg.grid.dims, radius_vox, min_neighbours, s->ssum, s->scnt, s->filled, st));
    }
    s->filled_version = s->version;
    return session_end(s, st);
}

dare_status dare_reslice_scalar_filled(dare_session s, const dare_plane* plane, float unassigned, float* out_dev,
                                       uint32_t* mask_dev, void* stream) {
    if (!s) return fail(DARE_E_INVALID, "session is NULL");
    dare_status rc = check_plane(plane);
    if (rc != DARE_OK) return rc;
    if (!s->filled || s->filled_version != s->version)
        return fail(DARE_E_STATE, "no hole-filled volume for the session's current frames (call dare_fill_holes)");
    if (!out_dev || !mask_dev) return fail(DARE_E_INVALID, "output pointers are NULL");
    if (!affine_ok(s->cfg.grid.vol_to_world, s->cfg.grid.spacing_mm, plane->image_to_world, plane->width,
                   plane->px_mm[0], plane->px_mm[1]))
        return fail(DARE_E_INVALID, "plane too far from the grid for fixed-point coordinates");
    DeviceGuard dg(s->cfg.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = session_begin(s, st);
    if (rc != DARE_OK) return rc;
    ResliceJob job = make_job(s, plane, nullptr, out_dev, mask_dev, unassigned);
    {
        KernelScope ks("reslice_values", st, 1);
        CUDA_TRY(launch_reslice_values(job, s->filled, st));
    }
    return session_end(s, st);
}

dare_status dare_session_read_filled(dare_session s, float* values) {
    if (!s || !values) return fail(DARE_E_INVALID, "NULL argument");
    if (!s->filled || s->filled_version != s->version)
        return fail(DARE_E_STATE, "no hole-filled volume for the session's current frames (call dare_fill_holes)");
    DeviceGuard dg(s->cfg.device);
    CUDA_TRY(cudaEventSynchronize(s->order_ev));
    CUDA_TRY(cudaMemcpy(values, s->filled, size_t(s->n_vox) * 4, cudaMemcpyDeviceToHost));
    return DARE_OK;
}

dare_status dare_footprint(dare_session s, const dare_plane* planes, int32_t n, int64_t* counts, void* stream) {
    if (!s || (n > 0 && (!planes || !counts)) || n < 0) return fail(DARE_E_INVALID, "bad arguments");
    for (int32_t i = 0; i < n; ++i) {
        dare_status rc = check_plane(planes + i);
        if (rc != DARE_OK) return rc;
        if (!affine_ok(s->cfg.grid.vol_to_world, s->cfg.grid.spacing_mm, planes[i].image_to_world, planes[i].width,
                       planes[i].px_mm[0], planes[i].px_mm[1]))
            return fail(DARE_E_INVALID, "plane %d too far from the grid", i);
    }
    if (n == 0) return DARE_OK;
    DeviceGuard dg(s->cfg.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    dare_status rc = session_begin(s, st);
    if (rc != DARE_OK) return rc;
    const size_t words = size_t((s->n_vox + 31) / 32);
    const size_t need = align_up(words * 4, 256) + 256 * size_t(n);
    rc = ensure_workspace(s, need, st);
    if (rc != DARE_OK) return rc;
    uint32_t* bitmap = static_cast<uint32_t*>(s->ws);
    auto* cnt = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(s->ws) + align_up(words * 4, 256));
    CUDA_TRY(cudaMemsetAsync(cnt, 0, 256 * size_t(n), st));
    for (int32_t i = 0; i < n; ++i) {
        CUDA_TRY(cudaMemsetAsync(bitmap, 0, words * 4, st));
        ResliceJob job = make_job(s, planes + i, nullptr, nullptr, nullptr, 0.0f);
        KernelScope ks("footprint", st, 1);
        CUDA_TRY(launch_footprint(job, bitmap, cnt + 32 * size_t(i), st));
    }
    std::vector<unsigned long long> host(32 * size_t(n));
    CUDA_TRY(cudaMemcpyAsync(host.data(), cnt, host.size() * 8, cudaMemcpyDeviceToHost, st));
    rc = session_end(s, st);
    if (rc != DARE_OK) return rc;
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int32_t i = 0; i < n; ++i) counts[i] = static_cast<int64_t>(host[32 * size_t(i)]);
    return DARE_OK;
}

dare_status dare_session_reset(dare_session s, void* stream) {
    if (!s) return fail(DARE_E_INVALID, "session is NULL");
    DeviceGuard dg(s->cfg.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the volume itself is cleared lazily: by the next build's finalize, which
    // writes every voxel, or before any other call that reads it
    dare_status rc = session_begin(s, st, false);
    if (rc != DARE_OK) return rc;
    CUDA_TRY(cudaMemsetAsync(s->overflow_dev, 0, sizeof(unsigned long long), st));
    rc = session_end(s, st);
    if (rc != DARE_OK) return rc;
    s->pending_clear = true;
    s->frames_host.clear();
    s->probe_host.clear();
    s->n_curv = 0;
    s->filled_version = -1;
    s->n_frames = 0;
    s->version = 0;
    s->fresh = true;
    return DARE_OK;
}

dare_status dare_trace_enable(int32_t on) {
    g_trace_on = on != 0;
    return DARE_OK;
}

dare_status dare_trace_read(dare_kernel_time* out, int32_t capacity, int32_t* n_out) {
    if (capacity < 0 || (capacity > 0 && !out) || !n_out) return fail(DARE_E_INVALID, "bad arguments");
    std::lock_guard<std::mutex> lk(g_trace_mu);
    dare_status rc = DARE_OK;
    for (auto& r : g_trace_pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaError_t e = cudaGetLastError();
            rc = fail(DARE_E_CUDA, "trace event: %s", cudaGetErrorString(e));
        }
        auto& acc = g_trace_acc[r.name];
        acc.first += 1;
        acc.second += ms;
        g_event_pool[r.device].push_back(r.a);
        g_event_pool[r.device].push_back(r.b);
    }
    g_trace_pending.clear();
    int32_t n = 0;
    for (auto& kv : g_trace_acc) {
        if (n < capacity) {
            std::memset(&out[n], 0, sizeof(out[n]));
            std::snprintf(out[n].name, sizeof(out[n].name), "%s", kv.first.c_str());
            out[n].launches = kv.second.first;
            out[n].total_ms = kv.second.second;
        }
        ++n;
    }
    *n_out = n;
    g_trace_acc.clear();
    return rc;
}

int64_t dare_launch_count(void) { return g_launches.load(); }

dare_status dare_measure_l2_bandwidth(int32_t device, int64_t bytes, int32_t reps, double* read_gbs) {
    if (!read_gbs || bytes < (int64_t(1) << 20) || bytes > (int64_t(1) << 30) || reps < 1 || reps > 100000)
        return fail(DARE_E_INVALID, "bytes must be 1 MiB .. 1 GiB and reps 1 .. 100000");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(DARE_E_INVALID, "device %d not available", device);
    }
    DeviceGuard dg(device);
    if (!dg.ok) return fail(DARE_E_CUDA, "cannot select device %d", device);
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int64_t n = bytes / 16 * 16;
    void* buf = nullptr;
    void* sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc(&buf, size_t(n));
    if (e == cudaSuccess) e = cudaMalloc(&sink, 16);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0x5A, size_t(n), st);
    const int blocks = sms * 8;
    if (e == cudaSuccess) e = launch_l2_read(buf, n, 2, sink, blocks, st);  // warm-up: the buffer into L2
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = launch_l2_read(buf, n, reps, sink, blocks, st);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return fail(DARE_E_CUDA, "L2 bandwidth measurement: %s", cudaGetErrorString(e));
    g_launches += 2;
    *read_gbs = double(n) * reps / (double(ms) * 1e-3) / 1e9;
    return DARE_OK;
}

dare_status dare_trace_counters_read(dare_trace_counters* out, int32_t reset) {
    if (!out) return fail(DARE_E_INVALID, "out is NULL");
    unsigned long long ft = 0, fg = 0;
    if (read_fallback_tiles_tiled(&ft, reset != 0) != cudaSuccess ||
        read_fallback_tiles_general(&fg, reset != 0) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        return fail(DARE_E_CUDA, "reading the fallback counters: %s", cudaGetErrorString(e));
    }
    out->tiled_planes = reset ? g_tiled_planes.exchange(0) : g_tiled_planes.load();
    out->per_pixel_planes = reset ? g_per_pixel_planes.exchange(0) : g_per_pixel_planes.load();
    out->fallback_tiles = static_cast<int64_t>(ft + fg);
    return DARE_OK;
}

// ---------------------------------------------------------------- checkpoint

namespace {
struct FileHeader {
    char magic[8];          // "DAREVOL1"
    int32_t abi;
    int32_t dims[3];
    double spacing_mm;
    double vol_to_world[16];
    int32_t dtype, slots, max_frames, n_frames, flags, rec_bytes;
    int64_t n_vox;
    int64_t version;
    uint32_t crc;           // CRC-32 of everything after the header
    uint32_t reserved;
};
// flags bit: a probe section (n_frames x 3 FP64: kind, apex-relative offsets)
// follows the frame table; files without it hold linear-probe frames only
constexpr int32_t kFileProbes = 1 << 8;
}  // namespace

dare_status dare_session_save(dare_session s, const char* path) {
    if (!s || !path) return fail(DARE_E_INVALID, "NULL argument");
    DeviceGuard dg(s->cfg.device);
    dare_status rc0 = settle_now(s);
    if (rc0 != DARE_OK) return rc0;
    CUDA_TRY(cudaEventSynchronize(s->order_ev));
    std::vector<uint8_t> rec(size_t(s->n_vox) * s->rec_bytes);
    std::vector<uint8_t> np(size_t(s->n_vox) * s->K * 2);
    std::vector<uint8_t> sc(s->ssum ? size_t(s->n_vox) * 8 : 0);
    CUDA_TRY(cudaMemcpy(rec.data(), s->rec, rec.size(), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(np.data(), s->npix, np.size(), cudaMemcpyDeviceToHost));
    if (s->ssum) {
        CUDA_TRY(cudaMemcpy(sc.data(), s->ssum, size_t(s->n_vox) * 4, cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(sc.data() + size_t(s->n_vox) * 4, s->scnt, size_t(s->n_vox) * 4, cudaMemcpyDeviceToHost));
    }
    FileHeader hd{};
    std::memcpy(hd.magic, "DAREVOL1", 8);
    hd.abi = DARE_ABI_VERSION;
    for (int a = 0; a < 3; ++a) hd.dims[a] = s->cfg.grid.dims[a];
    hd.spacing_mm = s->cfg.grid.spacing_mm;
    std::memcpy(hd.vol_to_world, s->cfg.grid.vol_to_world, sizeof(hd.vol_to_world));
    hd.dtype = s->dtype;
    hd.slots = s->K;
    hd.max_frames = s->cfg.max_frames;
    hd.n_frames = s->n_frames;
    hd.flags = (s->cfg.flags & DARE_SESSION_SCALAR) | (s->n_curv > 0 ? kFileProbes : 0);
    const std::vector<double> none;
    const std::vector<double>& probes = s->n_curv > 0 ? s->probe_host : none;
    hd.rec_bytes = s->rec_bytes;
    hd.n_vox = s->n_vox;
    hd.version = s->version;
    uint32_t crc = 0;
    crc = crc32_update(crc, s->frames_host.data(), s->frames_host.size() * 8);
    crc = crc32_update(crc, probes.data(), probes.size() * 8);
    crc = crc32_update(crc, rec.data(), rec.size());
    crc = crc32_update(crc, np.data(), np.size());
    crc = crc32_update(crc, sc.data(), sc.size());
    hd.crc = crc;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(DARE_E_INVALID, "cannot open %s for writing", path);
    bool ok = std::fwrite(&hd, sizeof(hd), 1, fp) == 1;
    ok = ok && (s->frames_host.empty() || std::fwrite(s->frames_host.data(), 8, s->frames_host.size(), fp) == s->frames_host.size());
    ok = ok && (probes.empty() || std::fwrite(probes.data(), 8, probes.size(), fp) == probes.size());
    ok = ok && std::fwrite(rec.data(), 1, rec.size(), fp) == rec.size();
    ok = ok && std::fwrite(np.data(), 1, np.size(), fp) == np.size();
    ok = ok && (sc.empty() || std::fwrite(sc.data(), 1, sc.size(), fp) == sc.size());
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return fail(DARE_E_INVALID, "writing %s failed", path);
    return DARE_OK;
}

dare_status dare_session_load(const dare_session_config* cfg, const char* path, dare_session* out) {
    if (!cfg || !path || !out) return fail(DARE_E_INVALID, "NULL argument");
    *out = nullptr;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(DARE_E_INVALID, "cannot open %s", path);
    FileHeader hd{};
    auto close_fail = [&](const char* why) {
        std::fclose(fp);
        return fail(DARE_E_INVALID, "%s: %s", path, why);
    };
    if (std::fread(&hd, sizeof(hd), 1, fp) != 1 || std::memcmp(hd.magic, "DAREVOL1", 8) != 0)
        return close_fail("not a DARE volume file");
    if (hd.abi != 1 && hd.abi != DARE_ABI_VERSION) return close_fail("ABI version mismatch");
    if (hd.n_frames < 0 || hd.n_frames > hd.max_frames || hd.max_frames > DARE_MAX_FRAMES ||
        hd.n_vox != int64_t(hd.dims[0]) * hd.dims[1] * hd.dims[2] || hd.n_vox <= 0 ||
        hd.rec_bytes != record_bytes(hd.slots, hd.dtype))
        return close_fail("inconsistent header");
    std::vector<double> frames(size_t(hd.n_frames) * 9);
    std::vector<double> probes((hd.flags & kFileProbes) ? size_t(hd.n_frames) * 3 : 0);
    std::vector<uint8_t> rec(size_t(hd.n_vox) * hd.rec_bytes);
    std::vector<uint8_t> np(size_t(hd.n_vox) * hd.slots * 2);
    std::vector<uint8_t> sc((hd.flags & DARE_SESSION_SCALAR) ? size_t(hd.n_vox) * 8 : 0);
    bool ok = frames.empty() || std::fread(frames.data(), 8, frames.size(), fp) == frames.size();
    ok = ok && (probes.empty() || std::fread(probes.data(), 8, probes.size(), fp) == probes.size());
    ok = ok && std::fread(rec.data(), 1, rec.size(), fp) == rec.size();
    ok = ok && std::fread(np.data(), 1, np.size(), fp) == np.size();
    ok = ok && (sc.empty() || std::fread(sc.data(), 1, sc.size(), fp) == sc.size());
    if (!ok) return close_fail("truncated file");
    std::fclose(fp);
    uint32_t crc = 0;
    crc = crc32_update(crc, frames.data(), frames.size() * 8);
    crc = crc32_update(crc, probes.data(), probes.size() * 8);
    crc = crc32_update(crc, rec.data(), rec.size());
    crc = crc32_update(crc, np.data(), np.size());
    crc = crc32_update(crc, sc.data(), sc.size());
    if (crc != hd.crc) return fail(DARE_E_INVALID, "%s: CRC mismatch (corrupted file)", path);
    if (probes.empty()) probes.assign(size_t(hd.n_frames) * 3, 0.0);  // every frame linear
    for (int32_t f = 0; f < hd.n_frames; ++f) {
        const double k = probes[3 * size_t(f)];
        if ((k != DARE_PROBE_LINEAR && k != DARE_PROBE_CURVILINEAR) || !finite_all(&probes[3 * size_t(f) + 1], 2))
            return fail(DARE_E_INVALID, "%s: bad probe record of frame %d", path, f);
    }
    dare_session_config c = *cfg;
    for (int a = 0; a < 3; ++a) c.grid.dims[a] = hd.dims[a];
    c.grid.spacing_mm = hd.spacing_mm;
    std::memcpy(c.grid.vol_to_world, hd.vol_to_world, sizeof(hd.vol_to_world));
    c.dtype = hd.dtype;
    c.max_slots = hd.slots;
    c.max_frames = hd.max_frames;
    c.flags = (cfg->flags & ~DARE_SESSION_SCALAR) | (hd.flags & DARE_SESSION_SCALAR);
    dare_session s = nullptr;
    dare_status rc = dare_session_create(&c, &s);
    if (rc != DARE_OK) return rc;
    DeviceGuard dg(s->cfg.device);
    auto bail = [&](cudaError_t e) {
        dare_session_destroy(s);
        return fail(DARE_E_CUDA, "upload failed: %s", cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaMemcpy(s->rec, rec.data(), rec.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e);
    if ((e = cudaMemcpy(s->npix, np.data(), np.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e);
    if (!frames.empty() &&
        (e = cudaMemcpy(s->frames_dev, frames.data(), frames.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e);
    if (hd.n_frames > 0) {
        // probe geometry rebuilt from the rotations and the (kind, offsets) records
        std::vector<float> grow(size_t(hd.n_frames) * kGeomFloats);
        std::vector<double> goff(size_t(hd.n_frames) * 2);
        for (int32_t f = 0; f < hd.n_frames; ++f) {
            const int kind = static_cast<int>(probes[3 * size_t(f)]);
            goff[2 * size_t(f)] = probes[3 * size_t(f) + 1];
            goff[2 * size_t(f) + 1] = probes[3 * size_t(f) + 2];
            geometry_row(s->cfg.grid, &frames[9 * size_t(f)], kind, &goff[2 * size_t(f)], &grow[size_t(f) * kGeomFloats]);
            if (kind == DARE_PROBE_CURVILINEAR) s->n_curv += 1;
        }
        if ((e = cudaMemcpy(s->geom_dev, grow.data(), grow.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e);
        if ((e = cudaMemcpy(s->geom_off_dev, goff.data(), goff.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e);
    }
    if (!sc.empty()) {
        if ((e = cudaMemcpy(s->ssum, sc.data(), size_t(hd.n_vox) * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e);
        if ((e = cudaMemcpy(s->scnt, sc.data() + size_t(hd.n_vox) * 4, size_t(hd.n_vox) * 4, cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return bail(e);
    }
    s->frames_host = std::move(frames);
    s->probe_host = std::move(probes);
    s->n_frames = hd.n_frames;
    s->version = hd.version;
    s->fresh = false;
    *out = s;
    return DARE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free reslice support

namespace dare {

dare_status set_error(dare_status st, const char* msg) { return fail(st, "%s", msg); }

dare_status settle_session(dare_session s, cudaStream_t st) {
    if (!s->pending_clear) return DARE_OK;
    dare_status rc = settle_now(s);
    if (rc != DARE_OK) return rc;
    CUDA_TRY(cudaStreamWaitEvent(st, s->order_ev, 0));
    return DARE_OK;
}

dare_status reserve_bytes(int64_t bytes) { return admit(bytes); }
void release_bytes(int64_t bytes) { g_in_use -= bytes; }

int session_device(dare_session s) { return s ? s->cfg.device : -1; }
int session_max_frames(dare_session s) { return s ? s->cfg.max_frames : 0; }

// dare_reslice with a caller-provided weight table of wtab_bytes bytes on the
// session's device; queues the same kernels and allocates nothing.
dare_status reslice_with_table(dare_session s, const dare_plane* plane, const dare_params* params, float* out_dev,
                               uint32_t* mask_dev, void* stream, void* wtab, size_t wtab_bytes, int max_frames) {
    if (!s) return fail(DARE_E_INVALID, "session is NULL");
    dare_status rc = check_plane(plane);
    if (rc != DARE_OK) return rc;
    rc = check_params(params);
    if (rc != DARE_OK) return rc;
    if (!out_dev || !mask_dev) return fail(DARE_E_INVALID, "output pointers are NULL");
    if (!affine_ok(s->cfg.grid.vol_to_world, s->cfg.grid.spacing_mm, plane->image_to_world, plane->width,
                   plane->px_mm[0], plane->px_mm[1]))
        return fail(DARE_E_INVALID, "plane too far from the grid for fixed-point coordinates");
    if (curv_path(s, params))
        return fail(DARE_E_UNSUPPORTED, "the allocation-free reslice covers linear probes only (use dare_reslice)");
    if (s->cache) return fail(DARE_E_UNSUPPORTED, "a session with a brick cache pages per call (use dare_reslice)");
    const size_t wb = params->weight_dtype == DARE_WEIGHTS_F16 ? 2 : 4;
    if (s->n_frames > max_frames || size_t(s->n_frames) * wb > wtab_bytes)
        return fail(DARE_E_INVALID, "the allocation-free reslice holds weights for at most %d frames; "
                    "this session has %d (use dare_reslice)", max_frames, s->n_frames);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = session_begin(s, st);
    if (rc != DARE_OK) return rc;
    TableJob tj{};
    plane_vectors(s, plane, params->normal_axis, &tj);
    tj.frames = s->frames_dev;
    tj.wtab = wtab;
    tj.n_frames = s->n_frames;
    if (s->n_frames > 0) {
        KernelScope ks("weight_table", st, 1);
        CUDA_TRY(launch_weight_tables(nullptr, &tj, 1, s->n_frames, table_params(params), st));
    }
    ResliceJob job = make_job(s, plane, wtab, out_dev, mask_dev, params->unassigned, params);
    const int half_w = params->weight_dtype == DARE_WEIGHTS_F16;
    L2Window l2((s->cfg.flags & DARE_SESSION_L2_PERSIST) ? s->rec : nullptr, size_t(s->n_vox) * s->rec_bytes, st);
    CUDA_TRY(launch_one(job, plane, params, s->K, s->dtype, half_w, s->n_frames > 0, st));
    return session_end(s, st);
}

}  // namespace dare

// ---------------------------------------------------------------- plans (graph-replayed batches, autotuned)

struct dare_plan_s {
    static constexpr int kCands = 4;  // plain, tiled with at most 64, 32, 16 rows
    struct Group {
        int32_t k0 = 0, k1 = 0;   // range in `order`
        int K = 0, dtype = 0;
        int choice = kTileH;      // 0 = plain, else the largest tile height of the tiled kernel
        int max_w = 0, max_h = 0;
        float tune_ms[kCands] = {0, 0, 0, 0};
        int col_cap = 0, slot_cap = 0;  // general distance kernels: shared memory of the tiled kernel
        std::string key;          // tuning-cache key
    };
    std::vector<dare_reslice_req> reqs;
    dare_params params{};
    std::vector<dare_session> sessions;
    std::vector<int32_t> frames_at_create;
    std::vector<int32_t> order;
    std::vector<size_t> t_off;
    std::vector<Group> groups;
    int device = 0;
    int max_frames = 0;
    size_t o_tj = 0, o_rj = 0, o_q = 0, desc_bytes = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    dare_allocator ws_alloc{};  // the allocator ws came from (a copy: destroy needs no live session)
    void* pinned = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t done_ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// ---- tuning cache: choices per shape, in the process and optionally in a JSON file
std::mutex g_tune_mu;
std::map<std::string, int> g_tune_cache;
std::string g_tune_file;

// The file is one flat JSON object {"key": choice, ...} written by this library.
void tune_file_load(const std::string& path) {
    FILE* f = std::fopen(path.c_str(), "rb");
    if (!f) return;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
    std::fclose(f);
    size_t i = 0;
    for (;;) {
        const size_t k0 = text.find('"', i);
        if (k0 == std::string::npos) break;
        const size_t k1 = text.find('"', k0 + 1);
        if (k1 == std::string::npos) break;
        const size_t colon = text.find(':', k1);
        if (colon == std::string::npos) break;
        char* end = nullptr;
        const long v = std::strtol(text.c_str() + colon + 1, &end, 10);
        if (end == text.c_str() + colon + 1) break;
        if (v == 0 || v == 16 || v == 32 || v == 64) g_tune_cache[text.substr(k0 + 1, k1 - k0 - 1)] = static_cast<int>(v);
        i = static_cast<size_t>(end - text.c_str());
    }
}

bool tune_file_save() {
    if (g_tune_file.empty()) return true;
    const std::string tmp = g_tune_file + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return false;
    std::fputs("{\n", f);
    size_t k = 0;
    for (auto& kv : g_tune_cache) std::fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++k < g_tune_cache.size() ? "," : "");
    std::fputs("}\n", f);
    const bool ok = std::fclose(f) == 0;
    return ok && std::rename(tmp.c_str(), g_tune_file.c_str()) == 0;
}

// Pixel-to-voxel pitch of a plane: the longer of its two in-plane pixel steps, in voxels.
double plane_pitch(const dare_reslice_req& r) {
    const double h = r.session->cfg.grid.spacing_mm;
    return std::max(r.plane.px_mm[0], r.plane.px_mm[1]) / h;
}

// Tiles of a job in a plan group: its own tile height (tiled), none (plain).
int plan_tiles(const dare_plane* pl, const ResliceJob& j, int choice) {
    return choice == 0 ? 0 : tiles_of(pl, j.tile_h);
}

// Descriptors of every request for the plan's current poses and kernel choices,
// written to its pinned staging buffer: tables, jobs, one work queue per group.
void plan_fill(dare_plan p) {
    uint8_t* pin = static_cast<uint8_t*>(p->pinned);
    auto* tjs = reinterpret_cast<TableJob*>(pin);
    auto* rjs = reinterpret_cast<ResliceJob*>(pin + (p->o_rj - p->o_tj));
    auto* qs = reinterpret_cast<TileQueue*>(pin + (p->o_q - p->o_tj));
    uint8_t* ws = static_cast<uint8_t*>(p->ws);
    const bool general = general_support(&p->params);
    for (size_t gi = 0; gi < p->groups.size(); ++gi) {
        auto& g = p->groups[gi];
        int tile_base = 0;
        for (int32_t k = g.k0; k < g.k1; ++k) {
            const dare_reslice_req& r = p->reqs[p->order[k]];
            void* wtab = ws + p->t_off[p->order[k]];
            TableJob tj{};
            plane_vectors(r.session, &r.plane, p->params.normal_axis, &tj);
            tj.frames = r.session->frames_dev;
            tj.wtab = wtab;
            tj.n_frames = r.session->n_frames;
            tjs[k] = tj;
            ResliceJob j = make_job(r.session, &r.plane, wtab, r.out, r.mask, p->params.unassigned, &p->params);
            if (general) {
                j.tile_h = kTileHGeneral;
            } else if (g.choice > 0 && p->params.path == DARE_PATH_TILED_FIXED) {
                j.tile_h = g.choice;
            } else if (g.choice > 0) {
                // the persistent tiled kernel: the plane's own tile height, or per-pixel tiles
                // (32 rows each) when none fits
                j.tile_h = tile_rows_fit(j, g.choice);
                if (j.tile_h == 0) {
                    j.direct = 1;
                    j.tile_h = 32;
                }
            }
            j.tile_base = tile_base;
            rjs[k] = j;
            tile_base += plan_tiles(&r.plane, j, g.choice);
        }
        qs[gi] = TileQueue{tile_base, 0, {0, 0}};
        if (general) general_caps(rjs + g.k0, g.k1 - g.k0, &g.col_cap, &g.slot_cap);
    }
}

cudaError_t plan_group_launch(dare_plan p, size_t gi, cudaStream_t st) {
    const dare_plan_s::Group& g = p->groups[gi];
    uint8_t* ws = static_cast<uint8_t*>(p->ws);
    const auto* rj_dev = reinterpret_cast<const ResliceJob*>(ws + p->o_rj);
    auto* q_dev = reinterpret_cast<TileQueue*>(ws + p->o_q) + gi;
    const int half_w = p->params.weight_dtype == DARE_WEIGHTS_F16;
    const bool general = general_support(&p->params);
    if (g.choice == 0)
        return general ? launch_reslice_plain_r(rj_dev + g.k0, nullptr, g.k1 - g.k0, g.max_w, g.max_h, g.K, g.dtype,
                                                half_w, st)
                       : launch_reslice_plain(rj_dev + g.k0, nullptr, g.k1 - g.k0, g.max_w, g.max_h, g.K, g.dtype,
                                              half_w, st);
    if (general) {
        // fixed 32-row tiles: the tile count does not depend on the poses
        const int per = tiles_of(&p->reqs[p->order[g.k0]].plane, kTileHGeneral);
        bool uniform = g.k1 - g.k0 <= 65535;
        int total = 0;
        for (int32_t k = g.k0; k < g.k1; ++k) {
            const int t = tiles_of(&p->reqs[p->order[k]].plane, kTileHGeneral);
            uniform = uniform && t == per;
            total += t;
        }
        return launch_reslice_tiled_r(rj_dev + g.k0, nullptr, g.k1 - g.k0, 0, uniform ? per : total, uniform ? 1 : 0,
                                      g.col_cap, g.slot_cap, g.K, g.dtype, half_w, st);
    }
    return launch_reslice_tiled_persistent(rj_dev + g.k0, g.k1 - g.k0, q_dev, g.K, g.dtype, half_w, st);
}

cudaError_t plan_tables_launch(dare_plan p, cudaStream_t st) {
    const auto* tj_dev = reinterpret_cast<const TableJob*>(static_cast<uint8_t*>(p->ws) + p->o_tj);
    return launch_weight_tables(tj_dev, nullptr, static_cast<int>(p->reqs.size()), p->max_frames,
                                table_params(&p->params), st);
}

// Tuning key of a group: storage type, K, weight type, output pixels (rounded to
// a power of two) and planes, median pixel-to-voxel pitch (eighths of a voxel),
// L2 mode, frame count (rounded to a power of two) and the device's SM count.
std::string tune_key(dare_plan p, const dare_plan_s::Group& g) {
    long long px = 0;
    std::vector<double> pitch;
    bool l2 = true;
    for (int32_t k = g.k0; k < g.k1; ++k) {
        const dare_reslice_req& r = p->reqs[p->order[k]];
        px += int64_t(r.plane.width) * r.plane.height;
        pitch.push_back(plane_pitch(r));
        l2 = l2 && (r.session->cfg.flags & DARE_SESSION_L2_PERSIST);
    }
    std::nth_element(pitch.begin(), pitch.begin() + pitch.size() / 2, pitch.end());
    auto pow2 = [](long long x) {
        int e = 0;
        while ((1LL << e) < x) ++e;
        return e;
    };
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    char buf[200];
    std::snprintf(buf, sizeof(buf), "sm%d t%d K%d w%d px2^%d n2^%d pitch%d l2%d f2^%d", sms, g.dtype, g.K,
                  p->params.weight_dtype, pow2(px), pow2(g.k1 - g.k0),
                  static_cast<int>(std::lround(pitch[pitch.size() / 2] * 8.0)), l2 ? 1 : 0, pow2(p->max_frames));
    return buf;
}

// Time one group's candidate kernels on the plan's own requests; keep the fastest.
dare_status plan_tune(dare_plan p, size_t gi, cudaStream_t st) {
    auto& g = p->groups[gi];
    g.key = tune_key(p, g);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(g.key);
        if (it != g_tune_cache.end()) {
            g.choice = it->second;
            return DARE_OK;
        }
    }
    const int cands[dare_plan_s::kCands] = {0, 64, 32, 16};
    cudaEvent_t a = nullptr, b = nullptr;
    CUDA_TRY(cudaEventCreate(&a));
    CUDA_TRY(cudaEventCreate(&b));
    float best = 1e30f;
    int best_c = kTileH;
    for (int ci = 0; ci < dare_plan_s::kCands; ++ci) {
        g.choice = cands[ci];
        plan_fill(p);
        float ms = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {  // the first is a warm-up
            CUDA_TRY(cudaMemcpyAsync(static_cast<uint8_t*>(p->ws) + p->o_tj, p->pinned, p->desc_bytes,
                                     cudaMemcpyHostToDevice, st));
            CUDA_TRY(plan_tables_launch(p, st));
            CUDA_TRY(cudaEventRecord(a, st));
            CUDA_TRY(plan_group_launch(p, gi, st));
            CUDA_TRY(cudaEventRecord(b, st));
            CUDA_TRY(cudaEventSynchronize(b));
            float t = 0;
            CUDA_TRY(cudaEventElapsedTime(&t, a, b));
            if (rep > 0) ms = std::min(ms, t);
        }
        g.tune_ms[ci] = ms;
        if (ms < best) {
            best = ms;
            best_c = cands[ci];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    g.choice = best_c;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[g.key] = best_c;
    if (!tune_file_save()) return fail(DARE_E_INVALID, "cannot write the tuning file %s", g_tune_file.c_str());
    return DARE_OK;
}

}  // namespace

extern "C" {

dare_status dare_tune_cache_file(const char* path) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_file = path ? path : "";
    if (g_tune_file.empty()) return DARE_OK;
    tune_file_load(g_tune_file);
    if (!tune_file_save()) return fail(DARE_E_INVALID, "cannot write the tuning file %s", g_tune_file.c_str());
    return DARE_OK;
}

dare_status dare_plan_destroy(dare_plan p) {
    if (!p) return DARE_OK;
    DeviceGuard dg(p->device);
    if (p->done_ev) cudaEventSynchronize(p->done_ev);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->done_ev) cudaEventDestroy(p->done_ev);
    if (p->pinned) cudaFreeHost(p->pinned);
    if (p->ws) {
        allocator_free(p->ws_alloc, p->ws, p->ws_bytes, nullptr);
        g_in_use -= static_cast<int64_t>(p->ws_bytes);
    }
    delete p;
    return DARE_OK;
}

dare_status dare_plan_create(const dare_reslice_req* reqs, int32_t n, const dare_params* params, void* stream,
                             dare_plan* out) {
    if (!out) return fail(DARE_E_INVALID, "out is NULL");
    *out = nullptr;
    if (n <= 0 || !reqs) return fail(DARE_E_INVALID, "a plan needs at least one request");
    dare_status rc = check_params(params);
    if (rc != DARE_OK) return rc;
    for (int32_t i = 0; i < n; ++i) {
        const dare_reslice_req& r = reqs[i];
        if (!r.session) return fail(DARE_E_INVALID, "request %d has no session", i);
        if (curv_path(r.session, params))
            return fail(DARE_E_UNSUPPORTED, "request %d: plans cover linear probes only (use dare_reslice_batch)", i);
        if (r.session->cache)
            return fail(DARE_E_UNSUPPORTED, "request %d: a session with a brick cache (use dare_reslice_batch)", i);
        if (r.session->cfg.device != reqs[0].session->cfg.device) return fail(DARE_E_INVALID, "requests span devices");
        rc = check_plane(&r.plane);
        if (rc != DARE_OK) return fail(rc, "request %d: %s", i, g_err.c_str());
        if (!r.out || !r.mask) return fail(DARE_E_INVALID, "request %d: output pointers are NULL", i);
        if (!affine_ok(r.session->cfg.grid.vol_to_world, r.session->cfg.grid.spacing_mm, r.plane.image_to_world,
                       r.plane.width, r.plane.px_mm[0], r.plane.px_mm[1]))
            return fail(DARE_E_INVALID, "request %d: plane too far from the grid", i);
    }
    auto* p = new dare_plan_s();
    p->reqs.assign(reqs, reqs + n);
    p->params = *params;
    p->device = reqs[0].session->cfg.device;
    DeviceGuard dg(p->device);
    auto bail = [&](dare_status code) {
        dare_plan_destroy(p);
        return code;
    };
    for (int32_t i = 0; i < n; ++i)
        if (std::find(p->sessions.begin(), p->sessions.end(), reqs[i].session) == p->sessions.end()) {
            p->sessions.push_back(reqs[i].session);
            p->frames_at_create.push_back(reqs[i].session->n_frames);
        }
    p->order.resize(n);
    for (int32_t i = 0; i < n; ++i) p->order[i] = i;
    std::stable_sort(p->order.begin(), p->order.end(), [&](int32_t a, int32_t b) {
        const auto* sa = reqs[a].session;
        const auto* sb = reqs[b].session;
        return sa->K != sb->K ? sa->K < sb->K : sa->dtype < sb->dtype;
    });
    for (int32_t k0 = 0; k0 < n;) {
        dare_plan_s::Group g;
        const auto* sg = reqs[p->order[k0]].session;
        g.k0 = k0;
        g.K = sg->K;
        g.dtype = sg->dtype;
        int32_t k1 = k0;
        while (k1 < n && reqs[p->order[k1]].session->K == g.K && reqs[p->order[k1]].session->dtype == g.dtype) {
            g.max_w = std::max(g.max_w, reqs[p->order[k1]].plane.width);
            g.max_h = std::max(g.max_h, reqs[p->order[k1]].plane.height);
            ++k1;
        }
        g.k1 = k1;
        g.choice = params->path == DARE_PATH_PLAIN ? 0
                   : general_support(params)       ? kTileHGeneral
                   : params->tile_rows             ? params->tile_rows
                                                   : kTileH;
        p->groups.push_back(g);
        k0 = k1;
    }
    if (p->groups.size() > 8) return bail(fail(DARE_E_INVALID, "a plan holds at most 8 storage-type/slot groups"));
    const int wb = params->weight_dtype == DARE_WEIGHTS_F16 ? 2 : 4;
    p->t_off.resize(n);
    size_t o = 0;
    for (int32_t i = 0; i < n; ++i) {
        p->t_off[i] = o;
        o = align_up(o + size_t(std::max(reqs[i].session->n_frames, 1)) * wb, 256);
        p->max_frames = std::max(p->max_frames, reqs[i].session->n_frames);
    }
    p->o_tj = o;
    p->o_rj = align_up(p->o_tj + size_t(n) * sizeof(TableJob), 256);
    p->o_q = align_up(p->o_rj + size_t(n) * sizeof(ResliceJob), 256);
    const size_t need = align_up(p->o_q + p->groups.size() * sizeof(TileQueue), 256);
    p->desc_bytes = need - p->o_tj;
    rc = admit(static_cast<int64_t>(need));
    if (rc != DARE_OK) return bail(rc);
    p->ws_alloc = p->sessions[0]->cfg.alloc;
    p->ws = p->sessions[0]->dev_alloc(need, static_cast<cudaStream_t>(stream));
    if (!p->ws) {
        g_in_use -= static_cast<int64_t>(need);
        return bail(fail(DARE_E_OOM, "plan workspace allocation of %zu bytes failed", need));
    }
    p->ws_bytes = need;
    if (cudaHostAlloc(&p->pinned, p->desc_bytes, cudaHostAllocDefault) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(DARE_E_CUDA, "plan set-up failed"));
    }
    // tuning and capture run on the plan's own stream, after the sessions' queued work
    for (auto* s : p->sessions) {
        rc = settle_now(s);
        if (rc != DARE_OK) return bail(rc);
        if (cudaStreamWaitEvent(p->cap, s->order_ev, 0) != cudaSuccess) return bail(fail(DARE_E_CUDA, "wait failed"));
    }
    if (params->path == DARE_PATH_AUTO && !general_support(params))  // general kernels: tiled, no tuning
        for (size_t gi = 0; gi < p->groups.size(); ++gi) {
            rc = plan_tune(p, gi, p->cap);
            if (rc != DARE_OK) return bail(rc);
        }
    plan_fill(p);
    if (cudaStreamSynchronize(p->cap) != cudaSuccess) return bail(fail(DARE_E_CUDA, "plan tuning failed"));
    for (auto& g : p->groups)
        if (g.choice > 0 && !general_support(params) &&
            prepare_reslice_tiled_persistent(g.K, g.dtype, params->weight_dtype == DARE_WEIGHTS_F16) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(DARE_E_CUDA, "persistent kernel set-up failed"));
        }
    cudaError_t e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaMemcpyAsync(static_cast<uint8_t*>(p->ws) + p->o_tj, p->pinned, p->desc_bytes,
                                         cudaMemcpyHostToDevice, p->cap);
        if (e1 == cudaSuccess && p->max_frames > 0) e1 = plan_tables_launch(p, p->cap);
        for (size_t gi = 0; gi < p->groups.size(); ++gi)
            if (e1 == cudaSuccess) e1 = plan_group_launch(p, gi, p->cap);
        e = cudaStreamEndCapture(p->cap, &p->graph);
        if (e == cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(DARE_E_CUDA, "graph capture failed: %s", cudaGetErrorString(e)));
    }
    if (cudaEventRecord(p->done_ev, p->cap) != cudaSuccess) return bail(fail(DARE_E_CUDA, "event record failed"));
    *out = p;
    return DARE_OK;
}

dare_status dare_plan_set_poses(dare_plan p, const double* image_to_world) {
    if (!p || !image_to_world) return fail(DARE_E_INVALID, "NULL argument");
    const int32_t n = static_cast<int32_t>(p->reqs.size());
    for (int32_t i = 0; i < n; ++i) {
        const double* T = image_to_world + 16 * size_t(i);
        const dare_reslice_req& r = p->reqs[i];
        if (!rigid_ok(T)) return fail(DARE_E_INVALID, "pose %d is not a rigid transform", i);
        if (!affine_ok(r.session->cfg.grid.vol_to_world, r.session->cfg.grid.spacing_mm, T, r.plane.width,
                       r.plane.px_mm[0], r.plane.px_mm[1]))
            return fail(DARE_E_INVALID, "pose %d too far from the grid", i);
    }
    DeviceGuard dg(p->device);
    CUDA_TRY(cudaEventSynchronize(p->done_ev));
    for (int32_t i = 0; i < n; ++i) std::memcpy(p->reqs[i].plane.image_to_world, image_to_world + 16 * size_t(i), 128);
    plan_fill(p);
    return DARE_OK;
}

dare_status dare_plan_launch(dare_plan p, void* stream) {
    if (!p) return fail(DARE_E_INVALID, "plan is NULL");
    for (size_t i = 0; i < p->sessions.size(); ++i)
        if (p->sessions[i]->n_frames != p->frames_at_create[i])
            return fail(DARE_E_STATE, "a session's frame count changed since the plan was made; re-create the plan");
    DeviceGuard dg(p->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (auto* s : p->sessions) {
        dare_status rc = session_begin(s, st);
        if (rc != DARE_OK) return rc;
    }
    {
        KernelScope ks("plan_graph", st, (p->max_frames > 0 ? 1 : 0) + static_cast<int>(p->groups.size()));
        CUDA_TRY(cudaGraphLaunch(p->exec, st));
    }
    CUDA_TRY(cudaEventRecord(p->done_ev, st));
    for (auto* s : p->sessions) {
        dare_status rc = session_end(s, st);
        if (rc != DARE_OK) return rc;
    }
    return DARE_OK;
}

dare_status dare_plan_query(dare_plan p, dare_plan_info* out) {
    if (!p || !out) return fail(DARE_E_INVALID, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->n_requests = static_cast<int32_t>(p->reqs.size());
    out->n_groups = static_cast<int32_t>(p->groups.size());
    for (size_t g = 0; g < p->groups.size() && g < 8; ++g) {
        out->choice[g] = p->groups[g].choice;
        for (int c = 0; c < dare_plan_s::kCands; ++c) out->tune_ms[g][c] = p->groups[g].tune_ms[c];
    }
    out->workspace_bytes = static_cast<int64_t>(p->ws_bytes);
    return DARE_OK;
}

}  // extern "C"
