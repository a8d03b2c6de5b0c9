// Shared device/host helpers of the bcpp library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/bcpp.h"

namespace bcpp {

constexpr int32_t DINF = INT32_MAX;      // unreachable distance
constexpr unsigned FULL = 0xffffffffu;

// flags word indices (device-side status, one uint32 each)
enum : int {
    FLAG_SIGMA_OVF = 0,     // a path count exceeded 2^64
    FLAG_CAPACITY = 1,      // a per-batch list outgrew its buffer
    FLAG_INVALID = 2,       // input validation failed
    FLAG_INVALID_WHY = 3,   // first reason code of an invalid input
    FLAG_DEPTH = 4,         // a one-byte distance or 32-bit path count would overflow (rerun with wide rows)
    FLAG_COUNT = 8
};

// reason codes written into FLAG_INVALID_WHY
enum : uint32_t {
    WHY_NONE = 0, WHY_RANGE = 1, WHY_SELF_LOOP = 2, WHY_DUPLICATE = 3, WHY_UNSORTED = 4,
    WHY_WEIGHT_ZERO = 5, WHY_ASYMMETRIC = 6, WHY_TARGET = 7, WHY_PART = 8, WHY_ROWPTR = 9,
    WHY_WEIGHT_RANGE = 10
};

__device__ __forceinline__ void flag_invalid(uint32_t* flags, uint32_t why) {
    atomicOr(&flags[FLAG_INVALID], 1u);
    atomicCAS(&flags[FLAG_INVALID_WHY], 0u, why);
}

__device__ __forceinline__ int warp_incl_scan(int x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

__device__ __forceinline__ uint64_t shfl_u64(uint64_t x, int src) {
    uint32_t lo = __shfl_sync(FULL, (uint32_t)x, src);
    uint32_t hi = __shfl_sync(FULL, (uint32_t)(x >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}

// Neumaier (improved Kahan) compensated add into (sum, comp)
__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
    double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
}

// a + acc on uint64 with overflow detection
__device__ __forceinline__ uint64_t add_ck(uint64_t acc, uint64_t a, bool& ovf) {
    const uint64_t t = acc + a;
    if (t < acc) ovf = true;
    return t;
}

// a*b + acc on uint64 with overflow detection; factors below 2^32 (the common case) take one
// 32 x 32 -> 64-bit multiply, which cannot overflow
__device__ __forceinline__ uint64_t madd_ck(uint64_t acc, uint64_t a, uint64_t b, bool& ovf) {
    uint64_t p;
    if (((a | b) >> 32) == 0) {
        p = (uint64_t)(uint32_t)a * (uint32_t)b;
    } else {
        p = a * b;
        if (__umul64hi(a, b) != 0) ovf = true;
    }
    uint64_t t = acc + p;
    if (t < acc) ovf = true;
    return t;
}

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace bcpp
