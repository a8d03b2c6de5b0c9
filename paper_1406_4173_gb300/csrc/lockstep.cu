// Lockstep multi-source Brandes kernel (see lockstep.cuh for the layout and the modes).
//
// Forward (Sec. 3, Eq. 2; Sec. 4, Eq. 11; Dijkstra_SK Eq. 10): a node u settled at distance
// D on some lanes pulls its path count from the in-neighbours v with d(v) + w(v,u) = D
// (sigma(s,u) = sum sigma(s,v) * m(v,u)), then relaxes its out-arcs: an improved tentative
// distance D + w marks the head in bucket (D + w) mod nb.  Weights are >= 1, so every parent
// is settled in an earlier step and its count is final when it is read.
// Backward (Eq. 7 / Eq. 12): steps are replayed in reverse; u on lane s gets
// delta(s|u) = sigma(s,u) * sum over successors v (d(v) = d(u) + w) of m(u,v) * c(s,v) with
// c(s,v) = (I_{v in S} + delta(s|v)) / sigma(s,v), stores c(s,u), and its dependency is
// added (u != s) into the slot's partial betweenness.
//
// Each lane carries SPL sources (1 or 2); a node's row holds the batch's 32 * SPL sources
// contiguously, so a lane reads its SPL values with one vector load.  Unit-weight Brandes passes
// store distances in one byte per source (255 = unreached) while they stay below 254: rows four
// times smaller, so more of the slot state stays in L2.  The kernel itself is in
// lockstep_kernel.cuh, instantiated per dependency precision in lockstep_f64.cu / lockstep_f32.cu.
//
// Latency structure: a warp works on one settled entry at a time, and every dependent memory
// round trip costs it a full HBM latency, so the kernel keeps the chain per entry short: the
// entry already carries the node's arc range (filled by a parallel pass over the step's list),
// the next entry is fetched while the current one is processed, a group of arcs issues all its
// distance-row loads and then all its sigma (or c) loads together, bucket marks and
// partial-sum updates are fire-and-forget atomics.
#include <algorithm>

#include "lockstep.cuh"

namespace bcpp {

// instances per dependency precision (lockstep_f64.cu, lockstep_f32.cu)
void ls_launch_f64(int spl, int cl, bool fused, bool weighted, bool mult, bool narrow, const LsArena& A,
                   const LsParams& P, const LsSlots& W, const LsItem* items, int nitems, int slots, cudaStream_t st);
void ls_launch_f32(int spl, int cl, bool fused, bool weighted, bool mult, bool narrow, const LsArena& A,
                   const LsParams& P, const LsSlots& W, const LsItem* items, int nitems, int slots, cudaStream_t st);

namespace {

__global__ void fill_i32_kernel(int32_t* p, int32_t v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// 16-byte stores (p 16-byte aligned, n4 groups of four values)
__global__ void fill_i32x4_kernel(int4* p, int32_t v, int64_t n4) {
    const int4 q = make_int4(v, v, v, v);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = q;
}

}  // namespace

void ls_launch(bool fp32_delta, bool fused, const LsArena& A, const LsParams& P, const LsSlots& W,
               const LsItem* items, int nitems, int slots, cudaStream_t st, int spl, int cl, bool narrow) {
    if (nitems <= 0 || slots <= 0) return;
    // multiplicities > 1 only occur on skeleton arcs, whose weights then exceed 1 as well,
    // so a multiplicity array always comes with a weight array
    const bool mult = A.mu != nullptr;
    const bool weighted = A.w != nullptr;
    if (mult && !weighted) return;
    // the backward pass reads the multiplicities in the dependency type
    if (mult && !A.mud && (P.mode == LS_BRANDES || P.mode == LS_SKEL)) return;
    if (spl == 2 && P.mode != LS_BRANDES) return;   // 64-source rows: Brandes passes only
    if (cl != 1 && cl != 2 && cl != 4) return;
    narrow = narrow && !weighted && P.mode == LS_BRANDES;
    if (fp32_delta) ls_launch_f32(spl, cl, fused, weighted, mult, narrow, A, P, W, items, nitems, slots, st);
    else ls_launch_f64(spl, cl, fused, weighted, mult, narrow, A, P, W, items, nitems, slots, st);
}

// Every distance row of the first `slots` slots back to "unreached": a streaming fill of the
// whole region (slots x cap_n rows of 128 bytes) costs a fraction of a scatter over the settled
// entries, whose dependent loads of the order list leave the GPU latency-bound.
void ls_reset_launch(const LsSlots& W, int slots, cudaStream_t st) {
    if (slots > 0) fill_i32(W.d, DINF, (int64_t)slots * W.cap_n * LS_LANES, st);
}

template <typename T>
__global__ void convert_mult_kernel(const uint64_t* __restrict__ mu, int64_t m, T* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (T)mu[i];
}

void convert_mult(const uint64_t* mu, int64_t m, bool fp32, void* out, cudaStream_t st) {
    if (m <= 0) return;
    const int64_t blocks = std::min<int64_t>((m + 255) / 256, 152 * 16);
    if (fp32) convert_mult_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(mu, m, (float*)out);
    else convert_mult_kernel<double><<<(unsigned)blocks, 256, 0, st>>>(mu, m, (double*)out);
}

void fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0 && (n & 3) == 0) {
        const int64_t n4 = n / 4;
        const int64_t blocks = std::min<int64_t>((n4 + 255) / 256, 152 * 16);
        fill_i32x4_kernel<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<int4*>(p), v, n4);
        return;
    }
    int64_t blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    fill_i32_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, v, n);
}

}  // namespace bcpp
