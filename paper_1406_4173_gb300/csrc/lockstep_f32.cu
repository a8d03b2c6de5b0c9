// Lockstep kernel instances with FP32 dependencies.
#include "lockstep_kernel.cuh"

namespace bcpp {

void ls_launch_f32(int spl, int cl, bool fused, bool weighted, bool mult, bool narrow, const LsArena& A,
                   const LsParams& P, const LsSlots& W, const LsItem* items, int nitems, int slots, cudaStream_t st) {
    ls_launch_dt<float>(spl, cl, fused, weighted, mult, narrow, A, P, W, items, nitems, slots, st);
}

}  // namespace bcpp
