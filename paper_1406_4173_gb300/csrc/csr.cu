// CSR build and validation for the input graph G(V, E, W) (Sec. 3): undirected graphs with
// non-negative weights, restricted here to integer weights >= 1.  Building expands every
// undirected edge into two arcs, sorts the arcs by (tail, head) with the library's radix
// sort, and rejects self-loops, repeated edges and zero weights.
#include "csr.cuh"

namespace bcpp {

namespace {

__global__ void csr_expand_kernel(int32_t n, int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                                  const uint32_t* __restrict__ ew, int directed, uint64_t* __restrict__ keys,
                                  uint32_t* __restrict__ vals, uint32_t* flags) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = eu[i], v = ev[i];
        const uint32_t w = ew ? ew[i] : 1u;
        if (u < 0 || u >= n || v < 0 || v >= n) { flag_invalid(flags, WHY_RANGE); continue; }
        if (u == v) flag_invalid(flags, WHY_SELF_LOOP);
        if (w == 0) flag_invalid(flags, WHY_WEIGHT_ZERO);
        keys[directed ? i : 2 * i] = (uint64_t)u * (uint64_t)n + (uint64_t)v;
        vals[directed ? i : 2 * i] = w;
        if (!directed) {
            keys[2 * i + 1] = (uint64_t)v * (uint64_t)n + (uint64_t)u;
            vals[2 * i + 1] = w;
        }
    }
}

__global__ void csr_split_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t na,
                                 int32_t n, int32_t* __restrict__ col, uint32_t* __restrict__ w_out, uint32_t* flags) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        col[i] = (int32_t)(k % (uint64_t)n);
        if (w_out) w_out[i] = vals[i];
        if (i > 0 && keys[i - 1] == k) flag_invalid(flags, WHY_DUPLICATE);
    }
}

// row_ptr[u] = first arc with tail >= u (binary search in the sorted keys)
__global__ void csr_rowptr_kernel(const uint64_t* __restrict__ keys, int64_t na, int32_t n, int64_t* __restrict__ rp) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= n; u += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t target = (uint64_t)u * (uint64_t)n;
        int64_t lo = 0, hi = na;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (keys[mid] < target) lo = mid + 1; else hi = mid;
        }
        rp[u] = lo;
    }
}

// One warp per row: sorted strictly increasing heads in range, no self-loop, weights >= 1,
// and for undirected graphs the reverse arc with the same weight.
// With node_off (graph arenas) heads are graph-local ids of the row's graph.
__global__ void csr_check_kernel(int32_t n, int64_t na, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const uint32_t* __restrict__ w, int directed, uint32_t* flags,
                                 unsigned long long* wmax, const int64_t* __restrict__ node_off, int32_t ngraphs) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (warp == 0 && lane == 0) {
        if (rp[0] != 0 || rp[n] != na) flag_invalid(flags, WHY_ROWPTR);
    }
    uint32_t local_max = 0;
    for (int64_t u = warp; u < n; u += nwarps) {
        const int64_t a0 = rp[u], a1 = rp[u + 1];
        if (a0 > a1 || a0 < 0 || a1 > na) {
            if (lane == 0) flag_invalid(flags, WHY_ROWPTR);
            continue;
        }
        int64_t gb = 0, ge = n;   // node range of the row's graph
        if (node_off) {
            int32_t lo = 0, hi = ngraphs;   // last g with node_off[g] <= u
            while (hi - lo > 1) {
                int32_t mid = (lo + hi) >> 1;
                if (node_off[mid] <= u) lo = mid; else hi = mid;
            }
            gb = node_off[lo];
            ge = node_off[lo + 1];
        }
        for (int64_t p = a0 + lane; p < a1; p += 32) {
            const int64_t vl = col[p];
            if (vl < 0 || vl >= ge - gb) { flag_invalid(flags, WHY_RANGE); continue; }
            const int64_t v = gb + vl;
            if (v == u) flag_invalid(flags, WHY_SELF_LOOP);
            if (p > a0 && col[p - 1] >= vl) flag_invalid(flags, WHY_UNSORTED);
            const uint32_t wv = w ? w[p] : 1u;
            if (wv == 0) flag_invalid(flags, WHY_WEIGHT_ZERO);
            if (wv > local_max) local_max = wv;
            if (!directed) {
                int64_t lo = rp[v], hi = rp[v + 1];
                if (lo < 0 || hi > na || lo > hi) { flag_invalid(flags, WHY_ROWPTR); continue; }
                const int32_t ul = (int32_t)(u - gb);
                while (lo < hi) {
                    int64_t mid = (lo + hi) >> 1;
                    if (col[mid] < ul) lo = mid + 1; else hi = mid;
                }
                if (lo >= rp[v + 1] || col[lo] != ul || (w && w[lo] != wv)) flag_invalid(flags, WHY_ASYMMETRIC);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local_max = max(local_max, __shfl_xor_sync(FULL, local_max, o));
    if (lane == 0 && local_max) atomicMax(wmax, (unsigned long long)local_max);
}

// Targets: in range and distinct; sets in_s[v] = 1 for v in S.
__global__ void targets_kernel(const int32_t* __restrict__ S, int32_t nS, int32_t n, uint8_t* in_s,
                               uint32_t* cnt, uint32_t* flags) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nS; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = S[i];
        if (s < 0 || s >= n) { flag_invalid(flags, WHY_TARGET); continue; }
        if (atomicAdd(&cnt[s], 1u) != 0) flag_invalid(flags, WHY_TARGET);
        in_s[s] = 1;
    }
}

// CSR transpose: count in-degrees (pass 0) or scatter (pass 1, cursor = row starts).
__global__ void transpose_kernel(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const uint32_t* __restrict__ w, int64_t* counts_or_cursor, int32_t* tcol,
                                 uint32_t* tw, int pass) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        for (int64_t p = rp[u] + lane; p < rp[u + 1]; p += 32) {
            const int32_t v = col[p];
            if (pass == 0) {
                atomicAdd((unsigned long long*)&counts_or_cursor[v], 1ull);
            } else {
                const int64_t q = (int64_t)atomicAdd((unsigned long long*)&counts_or_cursor[v], 1ull);
                tcol[q] = (int32_t)u;
                if (tw) tw[q] = w[p];
            }
        }
    }
}

// Disjoint union of graphs: heads must stay inside the row's graph; lcol = head - graph start.
__global__ void localize_kernel(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                const int64_t* __restrict__ node_off, int32_t ngraphs, int32_t* __restrict__ lcol,
                                uint32_t* flags) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        int32_t lo = 0, hi = ngraphs;
        while (hi - lo > 1) {
            int32_t mid = (lo + hi) >> 1;
            if (node_off[mid] <= u) lo = mid; else hi = mid;
        }
        const int64_t gb = node_off[lo], ge = node_off[lo + 1];
        for (int64_t p = rp[u] + lane; p < rp[u + 1]; p += 32) {
            const int32_t v = col[p];
            if (v < gb || v >= ge) flag_invalid(flags, WHY_RANGE);
            lcol[p] = (int32_t)(v - gb);
        }
    }
}

inline unsigned grid_for(int64_t work, int threads, int max_blocks = 8192) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (unsigned)b;
}

}  // namespace

void csr_expand(int32_t n, int64_t m, const int32_t* eu, const int32_t* ev, const uint32_t* ew, int directed,
                uint64_t* keys, uint32_t* vals, uint32_t* flags, cudaStream_t st) {
    if (m > 0) csr_expand_kernel<<<grid_for(m, 256), 256, 0, st>>>(n, m, eu, ev, ew, directed, keys, vals, flags);
}

void csr_finish(const uint64_t* keys, const uint32_t* vals, int64_t na, int32_t n, int64_t* rp, int32_t* col,
                uint32_t* w_out, uint32_t* flags, cudaStream_t st) {
    if (na > 0) csr_split_kernel<<<grid_for(na, 256), 256, 0, st>>>(keys, vals, na, n, col, w_out, flags);
    csr_rowptr_kernel<<<grid_for((int64_t)n + 1, 256), 256, 0, st>>>(keys, na, n, rp);
}

void csr_check(int32_t n, int64_t na, const int64_t* rp, const int32_t* col, const uint32_t* w, int directed,
               uint32_t* flags, unsigned long long* wmax, cudaStream_t st, const int64_t* node_off, int32_t ngraphs) {
    csr_check_kernel<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(n, na, rp, col, w, directed, flags, wmax,
                                                                      node_off, ngraphs);
}

void csr_localize(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* node_off, int32_t ngraphs,
                  int32_t* lcol, uint32_t* flags, cudaStream_t st) {
    if (n > 0 && ngraphs > 0)
        localize_kernel<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(n, rp, col, node_off, ngraphs, lcol, flags);
}

void targets_check(const int32_t* S, int32_t nS, int32_t n, uint8_t* in_s, uint32_t* cnt, uint32_t* flags,
                   cudaStream_t st) {
    if (nS > 0) targets_kernel<<<grid_for(nS, 256), 256, 0, st>>>(S, nS, n, in_s, cnt, flags);
}

void csr_transpose_count(int32_t n, const int64_t* rp, const int32_t* col, int64_t* counts, cudaStream_t st) {
    transpose_kernel<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(n, rp, col, nullptr, counts, nullptr, nullptr, 0);
}

void csr_transpose_fill(int32_t n, const int64_t* rp, const int32_t* col, const uint32_t* w, int64_t* cursor,
                        int32_t* tcol, uint32_t* tw, cudaStream_t st) {
    transpose_kernel<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(n, rp, col, w, cursor, tcol, tw, 1);
}

}  // namespace bcpp
