// Device helpers shared by the reslice kernels: record decoding and the
// fixed-point pixel coordinate.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dare_internal.h"

namespace dare {
namespace dev {

__device__ __forceinline__ float to_f(uint8_t v) { return static_cast<float>(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(float v) { return v; }

__device__ __forceinline__ float weight_of(const float* w, int id) { return __ldg(w + id); }
__device__ __forceinline__ float weight_of(const __half* w, int id) { return __half2float(__ldg(w + id)); }

// Packed FP32 pairs (sm_100 and later): two independent IEEE round-to-nearest
// operations per instruction, bit-identical to the scalar ones.
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
    return (static_cast<unsigned long long>(__float_as_uint(a.y)) << 32) | __float_as_uint(a.x);
}
__device__ __forceinline__ float2 f2_of(unsigned long long b) {
    return make_float2(__uint_as_float(static_cast<uint32_t>(b)), __uint_as_float(static_cast<uint32_t>(b >> 32)));
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_of(d);
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return f2_of(d);
}
// (1 - t) a + t b on both halves, for a, b >= 0 (t and 1 - t each hold the same
// weight twice).  Unlike a + t (b - a), a sum of non-negative products: no
// cancellation when a and b differ by orders of magnitude.
__device__ __forceinline__ float2 f2_mix(float2 a, float2 b, float2 omt, float2 t) {
    return f2_fma(omt, a, f2_mul(t, b));
}

template <int K, typename VT>
struct RecShape {
    static constexpr int kBytes = (2 * K + K * int(sizeof(VT)) + 15) / 16 * 16;
    static constexpr int kVec = kBytes / 16;
    static constexpr int kWords = kBytes / 4;
};

__device__ __forceinline__ uint32_t word_of(const uint4* r, int w) {
    const uint4 q = r[w >> 2];
    const int k = w & 3;
    return k == 0 ? q.x : (k == 1 ? q.y : (k == 2 ? q.z : q.w));
}

// frame id of slot s (s is a compile-time constant after unrolling)
template <int K, typename VT>
__device__ __forceinline__ uint32_t slot_id(const uint4* r, int s) {
    return (word_of(r, s >> 1) >> (16 * (s & 1))) & 0xFFFFu;
}

template <int K, typename VT>
__device__ __forceinline__ float slot_value(const uint4* r, int s) {
    if constexpr (sizeof(VT) == 1) {
        const int b = 2 * K + s;
        return static_cast<float>((word_of(r, b >> 2) >> (8 * (b & 3))) & 0xFFu);
    } else if constexpr (sizeof(VT) == 2) {
        const uint32_t w = word_of(r, K / 2 + (s >> 1));
        const unsigned short bits = static_cast<unsigned short>((w >> (16 * (s & 1))) & 0xFFFFu);
        VT v;
        memcpy(&v, &bits, 2);
        return to_f(v);
    } else {
        return __uint_as_float(word_of(r, K / 2 + s));
    }
}

template <int K, typename VT>
__device__ __forceinline__ void load_record(const uint8_t* p, uint4 (&r)[RecShape<K, VT>::kVec]) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int i = 0; i < RecShape<K, VT>::kVec; ++i) r[i] = __ldg(q + i);
}

// Slots per group of weight lookups in collapse_voxel: half the record, at least 4
// (out-of-line callers, where registers are scarcer, pass 1).
template <int K>
struct SlotGroup {
    static constexpr int G = K / 2 > 4 ? K / 2 : (K < 4 ? K : 4);
};

// (A_c, B_c) of one voxel from its whole record, read in one round trip (ids
// first, values after; empty ids sort last).  The weight-table lookups go in
// groups of G slots whose loads issue together (each predicated on its slot
// being used), so a record waits on about K / G table round trips instead of
// one per sample; the sums keep slot order, so the result does not depend on G.
template <int K, typename VT, typename WT, int G = SlotGroup<K>::G>
__device__ __forceinline__ float2 collapse_voxel(const uint8_t* rec, int64_t vi, const WT* wt) {
    using S = RecShape<K, VT>;
    const uint4* q = reinterpret_cast<const uint4*>(rec + vi * S::kBytes);
    uint4 r[S::kVec];
#pragma unroll
    for (int i = 0; i < S::kVec; ++i) r[i] = __ldg(q + i);
    float A = 0.0f, B = 0.0f;
#pragma unroll
    for (int g = 0; g < K; g += G) {
        uint32_t id[G];
        float w[G];
#pragma unroll
        for (int j = 0; j < G; ++j) id[j] = g + j < K ? slot_id<K, VT>(r, g + j) : DARE_EMPTY_FRAME;
        if (id[0] == DARE_EMPTY_FRAME) break;  // empty slots come last
#pragma unroll
        for (int j = 0; j < G; ++j) w[j] = id[j] != DARE_EMPTY_FRAME ? weight_of(wt, static_cast<int>(id[j])) : 0.0f;
#pragma unroll
        for (int j = 0; j < G; ++j)
            if (id[j] != DARE_EMPTY_FRAME) {
                A = fmaf(w[j], slot_value<K, VT>(r, g + j), A);
                B += w[j];
            }
        if (id[G - 1] == DARE_EMPTY_FRAME) break;
    }
    return make_float2(A, B);
}

// Fixed-point pixel coordinate: integer voxel part and 20-bit fraction.
struct PixelCoord {
    int c0[3];
    float fr[3];
    bool any;  // false when no corner of the TENT(R=1) support can be in the grid
};

__device__ __forceinline__ PixelCoord pixel_coord(const ResliceJob& J, int u, int v) {
    PixelCoord pc;
    pc.any = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int64_t G = J.g0[a] + static_cast<int64_t>(u) * J.a[a] + static_cast<int64_t>(v) * J.b[a];
        const int64_t c = G >> kFixBits;  // arithmetic shift: floor
        pc.fr[a] = static_cast<float>(static_cast<int32_t>(G & (kFixOne - 1))) * (1.0f / static_cast<float>(kFixOne));
        if (c < -1 || c > J.dims[a] - 1) {
            pc.any = false;
            pc.c0[a] = 0;
        } else {
            pc.c0[a] = static_cast<int>(c);
        }
    }
    return pc;
}

}  // namespace dev
}  // namespace dare
