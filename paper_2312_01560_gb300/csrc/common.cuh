// common.cuh -- shared device helpers of the RaftGP CUDA library (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "raftgp.h"

namespace raftgp {

// ------------------------------------------------------------------------------------
// Device error word: kernels that find malformed input OR a flag in instead of trapping.
// ------------------------------------------------------------------------------------
enum DeviceError : uint32_t {
    DERR_COL_RANGE = 1u,     // a column index outside [0, n)
    DERR_ROW_PTR = 2u,       // row_ptr decreasing, or row_ptr[0] != 0, or row_ptr[n] != nnz
    DERR_SELF_LOOP = 4u,     // an entry (i, i)
    DERR_LABEL_RANGE = 8u,   // a label outside [0, K)
    DERR_TIMEOUT = 16u,      // a bounded wait gave up
    DERR_NORM = 32u,         // an embedding row with norm well above 1
    DERR_BOUNDS = 64u,       // an internal index outside its array (checked, the access skipped)
};

__device__ __forceinline__ void flag_error(uint32_t* err, uint32_t bit) { atomicOr(err, bit); }

// ------------------------------------------------------------------------------------
// CSR view with either int32 or int64 row offsets.
// ------------------------------------------------------------------------------------
template <typename OffT>
struct Csr {
    int64_t n;
    int64_t nnz;
    const OffT* row_ptr;
    const int32_t* col;
    __device__ __forceinline__ int64_t begin(int64_t i) const { return (int64_t)__ldg(row_ptr + i); }
    __device__ __forceinline__ int64_t end(int64_t i) const { return (int64_t)__ldg(row_ptr + i + 1); }
};

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// ------------------------------------------------------------------------------------
struct U32x4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint64_t seed) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return U32x4{c0, c1, c2, c3};
}

// Stream tags (counter word 3) of the random streams.
constexpr uint32_t STREAM_THETA = 0x54686574u;  // "Thet"
constexpr uint32_t STREAM_W = 0x57676e6eu;      // "Wgnn"
constexpr uint32_t STREAM_KMPP = 0x4b6d7070u;   // "Kmpp"

// Box-Muller on 24-bit uniforms u = ((x >> 8) + 0.5) * 2^-24 (exact in FP32).
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& g0, float& g1) {
    const float u1 = ((float)(a >> 8) + 0.5f) * (1.0f / 16777216.0f);
    const float u2 = ((float)(b >> 8) + 0.5f) * (1.0f / 16777216.0f);
    const float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    g0 = r * c;
    g1 = r * s;
}

// ------------------------------------------------------------------------------------
// Feature storage types: FP32 or BF16, 16-byte vectors.
// ------------------------------------------------------------------------------------
template <typename T>
struct Vec;
template <>
struct Vec<float> {
    static constexpr int E = 4;  // elements per 16 bytes
    __device__ __forceinline__ static void load(const float* p, float* out) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    }
    __device__ __forceinline__ static void store(float* p, const float* in) {
        *reinterpret_cast<float4*>(p) = make_float4(in[0], in[1], in[2], in[3]);
    }
    __device__ __forceinline__ static float to_float(float v) { return v; }
    __device__ __forceinline__ static float from_float(float v) { return v; }
    // 16 raw bytes, kept packed until they are added (4 registers per gather in flight)
    __device__ __forceinline__ static uint4 load_raw(const float* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }
    __device__ __forceinline__ static void unpack(const uint4& v, float* out) {
        out[0] = __uint_as_float(v.x); out[1] = __uint_as_float(v.y);
        out[2] = __uint_as_float(v.z); out[3] = __uint_as_float(v.w);
    }
};
template <>
struct Vec<__nv_bfloat16> {
    static constexpr int E = 8;
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, float* out) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            out[2 * i] = __uint_as_float(w[i] << 16);
            out[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
    __device__ __forceinline__ static void store(__nv_bfloat16* p, const float* in) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(in[2 * i], in[2 * i + 1]);
            w[i] = *reinterpret_cast<const uint32_t*>(&h);
        }
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __device__ __forceinline__ static float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ __forceinline__ static __nv_bfloat16 from_float(float v) { return __float2bfloat16_rn(v); }
    __device__ __forceinline__ static uint4 load_raw(const __nv_bfloat16* p) {
        return __ldg(reinterpret_cast<const uint4*>(p));
    }
    __device__ __forceinline__ static void unpack(const uint4& v, float* out) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            out[2 * i] = __uint_as_float(w[i] << 16);
            out[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
};

__device__ __forceinline__ float load_elem(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float load_elem(const __nv_bfloat16* p, int64_t i) {
    return __bfloat162float(p[i]);
}

// ------------------------------------------------------------------------------------
// Warp helpers
// ------------------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

constexpr double FIXED_SCALE = 1099511627776.0;  // 2^40: centroid sums and D^2 quantisation
constexpr float FIXED_SCALE_F = 1099511627776.0f;

}  // namespace raftgp
