// Allocation-free single-plane reslice (dare_reslice_noalloc).
//
// dare_reslice keeps each plane's per-frame weight table (Eq. 1 / Eq. 2) in
// the session's workspace, which it may (re)allocate.  This entry point keeps
// that table in a fixed array in device global memory instead, so a call
// never asks for memory.  The array lives in the library image: every GPU
// that loads the library holds its DARE_NOALLOC_MAX_FRAMES * 4 bytes until
// the process exits.  All calls share it, so calls that overlap on the GPU
// (different streams, no ordering between them) race on it.  Each call
// rewrites the entries it reads before reading them, so nothing needs to be
// cleared between calls.
#include <mutex>

#include "dare_internal.h"

namespace {

// Weight table of one plane: FP32 (or FP16, half the bytes) per frame.
static __device__ __align__(256) float g_noalloc_weights[DARE_NOALLOC_MAX_FRAMES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_weights_addr[kMaxDevices] = {};

// Device address of the array on the current device `dev`, looked up once.
// In host code the array's name is only a host-side stand-in; kernels must
// be given this address.
dare_status weights_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return dare::set_error(DARE_E_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_weights_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_weights);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return dare::set_error(DARE_E_CUDA, "cudaGetSymbolAddress of the allocation-free weight table failed");
        }
        g_weights_addr[dev] = p;
    }
    *out = g_weights_addr[dev];
    return DARE_OK;
}

}  // namespace

extern "C" dare_status dare_reslice_noalloc(dare_session s, const dare_plane* plane, const dare_params* params,
                                            float* out_dev, uint32_t* mask_dev, void* stream) {
    if (!s) return dare::set_error(DARE_E_INVALID, "session is NULL");
    const int dev = dare::session_device(s);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        cudaGetLastError();
        prev = -1;
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return dare::set_error(DARE_E_CUDA, "cannot select the session's device");
    }
    void* weights = nullptr;
    dare_status rc = weights_address(dev, &weights);
    if (rc == DARE_OK)
        rc = dare::reslice_with_table(s, plane, params, out_dev, mask_dev, stream, weights,
                                      sizeof(float) * DARE_NOALLOC_MAX_FRAMES, DARE_NOALLOC_MAX_FRAMES);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    return rc;
}
