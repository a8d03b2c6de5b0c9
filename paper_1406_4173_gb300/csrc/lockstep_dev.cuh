// Device helpers shared by the lockstep kernels (general and unit-weight).
#pragma once
#include "lockstep.cuh"

namespace bcpp {

// Mark head v in the bucket of distance nd (fire-and-forget: a stale mark only costs a
// visit that finds no lane at that distance).
__device__ __forceinline__ void mark_bucket(const LsParams& P, uint32_t* bm, uint8_t* bflag, int64_t bm_words,
                                            int v, int32_t nd, int* s_maxpush) {
    const int bk = nd % P.nb;
    atomicOr(&bm[(int64_t)bk * bm_words + (v >> 5)], 1u << (v & 31));
    bflag[bk] = 1;
    atomicMax(s_maxpush, nd);
}

// Fetch the next entry index of the current step for this warp (dynamic scheduling).
__device__ __forceinline__ int fetch_entry(int* s_next, int lane) {
    int e = 0;
    if (lane == 0) e = atomicAdd(s_next, 1);
    return __shfl_sync(FULL, e, 0);
}

__device__ __forceinline__ LsEnt load_entry(const LsEnt* order, int e, int end) {
    if (e < end) return order[e];
    LsEnt z;
    z.u = -1; z.deg = 0; z.a0 = 0;
    return z;
}

}  // namespace bcpp
