// Build_SK steps (Sec. 3 "The skeleton graph", Sec. 4 Alg. 1-2), the Centrality step
// (Sec. 4, Eq. 13) and the combination of partial betweenness.
#include <cuda_fp16.h>

#include "skeleton.cuh"

namespace bcpp {

namespace {

inline unsigned grid_for(int64_t work, int threads, int max_blocks = 16384) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (unsigned)b;
}

#define GRID_STRIDE(i, n) for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
                               i += (int64_t)gridDim.x * blockDim.x)
#define WARP_STRIDE(j, n)                                                        \
    const int lane = threadIdx.x & 31;                                           \
    const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; \
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;               \
    for (int64_t j = warp_id; j < (n); j += nwarps)

__global__ void partp_copy_kernel(int32_t n, const int32_t* part, int32_t k, int32_t* partp, uint32_t* flags) {
    GRID_STRIDE(v, n) {
        const int32_t p = part[v];
        if (p < 0 || p >= k) flag_invalid(flags, WHY_PART);
        partp[v] = p;
    }
}

__global__ void partp_targets_kernel(const int32_t* S, int32_t nS, int32_t k, int32_t* partp) {
    GRID_STRIDE(j, nS) partp[S[j]] = k + (int32_t)j;
}

__global__ void frontier_kernel(int32_t n, const int64_t* rp, const int32_t* col, const int32_t* partp, uint8_t* fr) {
    WARP_STRIDE(u, n) {
        const int32_t pu = partp[u];
        bool any = false;
        for (int64_t p = rp[u] + lane; p < rp[u + 1]; p += 32) {
            const int32_t v = col[p];
            if (partp[v] != pu) { fr[v] = 1; any = true; }
        }
        if (__any_sync(FULL, any) && lane == 0) fr[u] = 1;
    }
}

__global__ void group_keys_kernel(int32_t n, const int32_t* partp, const uint8_t* fr, uint64_t* keys, uint32_t* vals) {
    GRID_STRIDE(v, n) {
        keys[v] = 2ull * (uint64_t)partp[v] + (fr[v] ? 0ull : 1ull);
        vals[v] = (uint32_t)v;
    }
}

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* a, int64_t n, uint64_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void segments_kernel(const uint64_t* keys, int32_t n, int32_t kp, int32_t* pstart, int32_t* nf) {
    GRID_STRIDE(i, (int64_t)kp + 1) {
        const int64_t a = lower_bound_u64(keys, n, 2ull * (uint64_t)i);
        pstart[i] = (int32_t)a;
        if (i < kp) nf[i] = (int32_t)(lower_bound_u64(keys, n, 2ull * (uint64_t)i + 1ull) - a);
    }
}

__global__ void local_ids_kernel(int32_t n, const uint32_t* pnodes, const int32_t* partp, const int32_t* pstart,
                                 const int32_t* nf, const int32_t* skbase, int32_t* loc, int32_t* skid,
                                 int32_t* sknode) {
    GRID_STRIDE(j, n) {
        const int32_t v = (int32_t)pnodes[j];
        const int32_t i = partp[v];
        const int32_t li = (int32_t)j - pstart[i];
        loc[v] = li;
        if (li < nf[i]) {
            const int32_t x = skbase[i] + li;
            skid[v] = x;
            sknode[x] = v;
        } else {
            skid[v] = -1;
        }
    }
}

__global__ void local_count_kernel(int32_t n, const uint32_t* pnodes, const int64_t* rp, const int32_t* col,
                                   const int32_t* partp, int64_t* cnt) {
    WARP_STRIDE(j, n) {
        const int32_t v = (int32_t)pnodes[j];
        const int32_t pv = partp[v];
        int c = 0;
        for (int64_t p = rp[v] + lane; p < rp[v + 1]; p += 32) c += (partp[col[p]] == pv);
        c = warp_sum(c);
        if (lane == 0) cnt[j] = c;
    }
}

__global__ void local_fill_kernel(int32_t n, const uint32_t* pnodes, const int64_t* rp, const int32_t* col,
                                  const uint32_t* w, const int32_t* partp, const int32_t* loc, const int64_t* lrp,
                                  int32_t* lcol, int32_t* lw) {
    WARP_STRIDE(j, n) {
        const int32_t v = (int32_t)pnodes[j];
        const int32_t pv = partp[v];
        int64_t out = lrp[j];
        for (int64_t p0 = rp[v]; p0 < rp[v + 1]; p0 += 32) {
            const int64_t p = p0 + lane;
            bool keep = false;
            int32_t u = 0;
            if (p < rp[v + 1]) { u = col[p]; keep = partp[u] == pv; }
            const unsigned m = __ballot_sync(FULL, keep);
            if (keep) {
                const int64_t q = out + __popc(m & ((1u << lane) - 1u));
                lcol[q] = loc[u];
                if (lw) lw[q] = w ? (int32_t)w[p] : 1;
            }
            out += __popc(m);
        }
    }
}

// skeleton arcs of skeleton node x: R arcs (G row, other part) then clique arcs (exit table row)
__global__ void sk_arcs_count_kernel(int32_t N, const int32_t* sknode, const int64_t* rp, const int32_t* col,
                                     const int32_t* partp, const int32_t* loc, SkTables T, int64_t* cnt) {
    WARP_STRIDE(x, N) {
        const int32_t v = sknode[x];
        const int32_t i = partp[v];
        int c = 0;
        for (int64_t p = rp[v] + lane; p < rp[v + 1]; p += 32) c += (partp[col[p]] != i);
        const int32_t nfi = T.nf[i];
        if (nfi >= 2) {
            const int32_t fi = loc[v];
            const int64_t row = T.toff[i] + (int64_t)fi * nfi;
            for (int32_t q = lane; q < nfi; q += 32)
                c += (q != fi && T.tdr[row + q] != DINF && T.tsr[row + q] != 0ull);
        }
        c = warp_sum(c);
        if (lane == 0) cnt[x] = c;
    }
}

__global__ void sk_arcs_fill_kernel(int32_t N, const int32_t* sknode, const int64_t* rp, const int32_t* col,
                                    const uint32_t* w, const int32_t* partp, const int32_t* loc, const int32_t* skid,
                                    SkTables T, const int64_t* skrp, int32_t* skcol, int32_t* skw, uint64_t* skmu,
                                    unsigned long long* maxes) {
    uint32_t wmax = 0;
    unsigned long long mmax = 0;
    WARP_STRIDE(x, N) {
        const int32_t v = sknode[x];
        const int32_t i = partp[v];
        int64_t out = skrp[x];
        for (int64_t p0 = rp[v]; p0 < rp[v + 1]; p0 += 32) {
            const int64_t p = p0 + lane;
            bool keep = false;
            int32_t u = 0;
            if (p < rp[v + 1]) { u = col[p]; keep = partp[u] != i; }
            const unsigned m = __ballot_sync(FULL, keep);
            if (keep) {
                const int64_t q = out + __popc(m & ((1u << lane) - 1u));
                const uint32_t wv = w ? w[p] : 1u;
                skcol[q] = skid[u];
                skw[q] = (int32_t)wv;
                skmu[q] = 1ull;
                wmax = max(wmax, wv);
                mmax = max(mmax, 1ull);
            }
            out += __popc(m);
        }
        const int32_t nfi = T.nf[i];
        if (nfi >= 2) {
            const int32_t fi = loc[v];
            const int64_t row = T.toff[i] + (int64_t)fi * nfi;
            const int32_t xb = x - fi;   // skeleton id of the part's first frontier
            for (int32_t q0 = 0; q0 < nfi; q0 += 32) {
                const int32_t q = q0 + lane;
                bool keep = false;
                int32_t dq = 0;
                uint64_t sq = 0;
                if (q < nfi && q != fi) {
                    dq = T.tdr[row + q];
                    sq = T.tsr[row + q];
                    keep = dq != DINF && sq != 0ull;
                }
                const unsigned m = __ballot_sync(FULL, keep);
                if (keep) {
                    const int64_t o = out + __popc(m & ((1u << lane) - 1u));
                    skcol[o] = xb + q;
                    skw[o] = dq;
                    skmu[o] = sq;
                    wmax = max(wmax, (uint32_t)dq);
                    mmax = max(mmax, (unsigned long long)sq);
                }
                out += __popc(m);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wmax = max(wmax, __shfl_xor_sync(FULL, wmax, o));
        mmax = max(mmax, __shfl_xor_sync(FULL, mmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&maxes[0], (unsigned long long)wmax);
        atomicMax(&maxes[1], mmax);
    }
}

__global__ void sk_transpose_kernel(int32_t N, const int64_t* rp, const int32_t* col, const int32_t* w,
                                    const uint64_t* mu, int64_t* cursor, int32_t* tcol, int32_t* tw, uint64_t* tmu,
                                    int pass) {
    WARP_STRIDE(u, N) {
        for (int64_t p = rp[u] + lane; p < rp[u + 1]; p += 32) {
            const int32_t v = col[p];
            if (pass == 0) {
                atomicAdd((unsigned long long*)&cursor[v], 1ull);
            } else {
                const int64_t q = (int64_t)atomicAdd((unsigned long long*)&cursor[v], 1ull);
                tcol[q] = (int32_t)u;
                tw[q] = w[p];
                tmu[q] = mu[p];
            }
        }
    }
}

__global__ void gather_flags_kernel(int32_t N, const int32_t* sknode, const uint8_t* in_s, uint8_t* out) {
    GRID_STRIDE(x, N) out[x] = in_s[sknode[x]];
}

// targets as skeleton ids, position for position (-1 for a target that is no skeleton node: an
// isolated node, whose lane then stays idle), so that shards of positions are shards of S
__global__ void target_ids_kernel(const int32_t* S, int32_t nS, const int32_t* skid, int32_t* out) {
    GRID_STRIDE(j, nS) out[j] = skid[S[j]];
}

// Tiled Centrality: one block (16 warps) per unit of up to 64 non-frontier nodes and one slot,
// each warp CTV nodes, lanes are the slot's sources.  The part's frontier state rows (d, with
// sigma or c) are staged in shared memory FT frontiers at a time with coalesced loads, and each
// warp holds its nodes' table entries of the tile in registers (lane = frontier) and broadcasts
// them by shuffle, so the inner loop over (frontier, node) reads no global memory.
//
// Forward, in two sweeps over the entry frontiers: first the distance of each node, a pure
// min-plus d(s,v) = min_f d(s,f) + d_i(f,v); then its path count, summed over the frontiers
// that attain that minimum, sigma(s,v) = sum_f sigma(s,f) sigma_i(f,v), so that every count
// product is a final one (no partial sums to reset when a smaller distance turns up).
// Backward: the dependency through the exit frontiers that stay on a shortest path (Eq. 13
// with the tight-frontier tests).  Distances are handled as uint32: real distances are below
// DINF = 2^31 - 1, so a sum of two values never wraps, and a sum with an unreachable term is at
// least DINF, above every real distance.
//
// 16-bit path: when every finite table distance (h16, from the host) and every finite frontier
// distance of the block's slot and part (checked while the first sweep stages them) is at most
// CT_H16_MAX = 1023, the distance arithmetic runs on pairs of nodes packed in binary16 halves
// (one shuffle, one packed add and one packed min or compare for two nodes).  Integers up to
// 2048 are exact in binary16, so every sum of two such values is exact and the min-plus and the
// tight tests decide as in integers; a backward sum above 2048 can round but stays above every
// frontier distance, so it cannot test equal.  Unreachable is +inf in the sums and NaN where a
// value must equal nothing.  A block that finds a larger frontier distance redoes the first
// sweep in 32 bits and stays there.
constexpr int CTV = 4;          // nodes per warp
constexpr int CT_NP = CTV / 2;  // node pairs per warp (16-bit path)
constexpr int CT_WARPS = 16;    // warps per block: 64 nodes = one unit
constexpr int FT = 32;          // frontiers per tile
constexpr uint32_t CT_NONE = 0xffffffffu;   // "unreachable" after the min-plus sweep (no sum equals it)

// four or two packed half2 values, read from shared memory with one vector load
union H2x4 {
    uint4 u;
    __half2 h[4];
};
union H2x2 {
    uint2 u;
    __half2 h[2];
};

__device__ __forceinline__ __half ct_h(uint32_t x) {
    return x >= (uint32_t)DINF ? __ushort_as_half((unsigned short)0x7c00) : __uint2half_rn(x);
}
__device__ __forceinline__ __half ct_h_or_nan(uint32_t x) {
    return x >= (uint32_t)DINF ? __ushort_as_half((unsigned short)0x7e00) : __uint2half_rn(x);
}

template <typename DT>
__global__ void __launch_bounds__(CT_WARPS * 32)
centrality_tiled_kernel(const CentralityUnit* __restrict__ units, SkTables T, const uint32_t* __restrict__ pnodes,
                        const int32_t* __restrict__ skbase, const int32_t* __restrict__ d_all,
                        const uint64_t* __restrict__ sg_all, const DT* __restrict__ dl_all, int64_t cap_n,
                        double* bc_sum, double* bc_cmp, int64_t cap_bc, uint32_t* flags, int slot_major, int h16) {
    __shared__ uint32_t s_d[FT][32];
    __shared__ __half2 s_h[FT][32];       // 16-bit path: the frontier distance in both halves
    __shared__ uint64_t s_x[FT][32];      // sigma rows (forward) or c rows (backward, as DT bits)
    // 16-bit path: each warp's table tile, read with one broadcast load per frontier instead of a
    // shuffle per node pair: distances s_t[warp][f][q] (node pair q), counts s_c[warp][j][f]
    // (uint64 path counts forward, converted to DT backward)
    __shared__ __align__(16) __half2 s_t[CT_WARPS][FT][CT_NP];
    __shared__ __align__(16) uint64_t s_c[CT_WARPS][CTV][FT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const CentralityUnit U = units[slot_major ? blockIdx.y : blockIdx.x];
    const int slot = slot_major ? blockIdx.x : blockIdx.y;
    const int32_t i = U.part;
    const int32_t nfi = T.nf[i];
    const int64_t t0 = T.toff[i];
    const int32_t ps = T.pstart[i];
    const int64_t fbase = ((int64_t)slot * cap_n + skbase[i]) * 32;   // row of frontier 0 of part i
    const int32_t vb = U.v0 + warp * CTV;
    int nv = U.v1 - vb;
    nv = nv < 0 ? 0 : (nv > CTV ? CTV : nv);
    // entry-table distance of node j of this warp for frontier f0 + lane (DINF past the end)
    auto td_at = [&](const int32_t* tab, int j, int32_t f0, int nt) -> uint32_t {
        return (j < nv && lane < nt) ? (uint32_t)tab[t0 + (int64_t)(vb + j) * nfi + f0 + lane] : (uint32_t)DINF;
    };
    // ---- forward sweep 1: d(s,v) = min over entry frontiers of d(s,f) + d_i(f,v)
    uint32_t dv[CTV];
#pragma unroll
    for (int j = 0; j < CTV; j++) dv[j] = CT_NONE;
    bool use16 = h16 != 0;
    if (use16) {
        __half2 dv2[CT_NP], dv2b[CT_NP];
#pragma unroll
        for (int q = 0; q < CT_NP; q++) dv2[q] = dv2b[q] = __half2half2(ct_h(DINF));
        bool big = false;
        for (int32_t f0 = 0; f0 < nfi; f0 += FT) {
            const int nt = min(FT, nfi - f0);
            __syncthreads();
            for (int x = threadIdx.x; x < nt * 32; x += CT_WARPS * 32) {
                const uint32_t v = (uint32_t)d_all[fbase + (int64_t)(f0 + (x >> 5)) * 32 + (x & 31)];
                big |= v != (uint32_t)DINF && v > CT_H16_MAX;
                s_h[x >> 5][x & 31] = __half2half2(ct_h(v));
            }
#pragma unroll
            for (int q = 0; q < CT_NP; q++)
                s_t[warp][lane][q] = __halves2half2(ct_h(td_at(T.td, 2 * q, f0, nt)), ct_h(td_at(T.td, 2 * q + 1, f0, nt)));
            __syncthreads();
            // two frontiers per iteration into two running minima (independent chains)
            int f = 0;
            for (; f + 1 < nt; f += 2) {
                const __half2 dha = s_h[f][lane], dhb = s_h[f + 1][lane];
                H2x4 tt;
                tt.u = *reinterpret_cast<const uint4*>(&s_t[warp][f][0]);
#pragma unroll
                for (int q = 0; q < CT_NP; q++) {
                    dv2[q] = __hmin2(dv2[q], __hadd2(dha, tt.h[q]));
                    dv2b[q] = __hmin2(dv2b[q], __hadd2(dhb, tt.h[CT_NP + q]));
                }
            }
            if (f < nt) {
                const __half2 dh = s_h[f][lane];
#pragma unroll
                for (int q = 0; q < CT_NP; q++) dv2[q] = __hmin2(dv2[q], __hadd2(dh, s_t[warp][f][q]));
            }
        }
#pragma unroll
        for (int q = 0; q < CT_NP; q++) dv2[q] = __hmin2(dv2[q], dv2b[q]);
        use16 = !__syncthreads_or(big);
        if (use16) {
#pragma unroll
            for (int q = 0; q < CT_NP; q++) {
                const __half lo = __low2half(dv2[q]), hi = __high2half(dv2[q]);
                dv[2 * q] = __hisinf(lo) ? CT_NONE : __half2uint_rn(lo);
                dv[2 * q + 1] = __hisinf(hi) ? CT_NONE : __half2uint_rn(hi);
            }
        }
    }
    if (!use16) {
        for (int32_t f0 = 0; f0 < nfi; f0 += FT) {
            const int nt = min(FT, nfi - f0);
            __syncthreads();
            for (int x = threadIdx.x; x < nt * 32; x += CT_WARPS * 32)
                s_d[x >> 5][x & 31] = (uint32_t)d_all[fbase + (int64_t)(f0 + (x >> 5)) * 32 + (x & 31)];
            uint32_t tdv[CTV];
#pragma unroll
            for (int j = 0; j < CTV; j++) tdv[j] = td_at(T.td, j, f0, nt);
            __syncthreads();
            for (int f = 0; f < nt; f++) {
                const uint32_t dsf = s_d[f][lane];
#pragma unroll
                for (int j = 0; j < CTV; j++) {
                    const uint32_t tdj = __shfl_sync(FULL, tdv[j], f);
                    dv[j] = min(dv[j], dsf + tdj);
                }
            }
        }
    }
    bool any_reach = false;
#pragma unroll
    for (int j = 0; j < CTV; j++) {
        if (dv[j] >= (uint32_t)DINF) dv[j] = CT_NONE;
        any_reach |= dv[j] != CT_NONE;
    }
    // ---- forward sweep 2: sigma(s,v) = sum over the entry frontiers that attain d(s,v)
    uint64_t sv[CTV];
#pragma unroll
    for (int j = 0; j < CTV; j++) sv[j] = 0;
    bool ovf = false;
    if (__syncthreads_or(any_reach)) {
        __half2 dvh[CT_NP];   // 16-bit path: the node distances, NaN when unreachable
#pragma unroll
        for (int q = 0; q < CT_NP; q++) dvh[q] = __halves2half2(ct_h_or_nan(dv[2 * q]), ct_h_or_nan(dv[2 * q + 1]));
        for (int32_t f0 = 0; f0 < nfi; f0 += FT) {
            const int nt = min(FT, nfi - f0);
            __syncthreads();
            for (int x = threadIdx.x; x < nt * 32; x += CT_WARPS * 32) {
                const int64_t o = fbase + (int64_t)(f0 + (x >> 5)) * 32 + (x & 31);
                const uint32_t v = (uint32_t)d_all[o];
                if (use16) s_h[x >> 5][x & 31] = __half2half2(ct_h(v));
                else s_d[x >> 5][x & 31] = v;
                s_x[x >> 5][x & 31] = sg_all[o];
            }
            uint32_t tdv[CTV];
            uint64_t tsv[CTV];
#pragma unroll
            for (int j = 0; j < CTV; j++) {
                tdv[j] = td_at(T.td, j, f0, nt);
                tsv[j] = tdv[j] != (uint32_t)DINF ? T.ts[t0 + (int64_t)(vb + j) * nfi + f0 + lane] : 0ull;
            }
            if (use16) {
#pragma unroll
                for (int q = 0; q < CT_NP; q++) s_t[warp][lane][q] = __halves2half2(ct_h(tdv[2 * q]), ct_h(tdv[2 * q + 1]));
#pragma unroll
                for (int j = 0; j < CTV; j++) s_c[warp][j][lane] = tsv[j];
            }
            __syncthreads();
            if (use16) {
                for (int f = 0; f < nt; f++) {
                    const __half2 dh = s_h[f][lane];
                    H2x2 tt;
                    tt.u = *reinterpret_cast<const uint2*>(&s_t[warp][f][0]);
                    unsigned m[CT_NP], any = 0u;
#pragma unroll
                    for (int q = 0; q < CT_NP; q++) {
                        m[q] = __heq2_mask(__hadd2(dh, tt.h[q]), dvh[q]);
                        any |= m[q];
                    }
                    if (__any_sync(FULL, any != 0u)) {
                        // lanes take their own tight nodes (no shuffles below: the counts are in
                        // shared memory)
                        const uint64_t xs = s_x[f][lane];
#pragma unroll
                        for (int j = 0; j < CTV; j++)
                            if ((m[j >> 1] >> (16 * (j & 1))) & 0xffffu) sv[j] = madd_ck(sv[j], xs, s_c[warp][j][f], ovf);
                    }
                }
            } else {
                for (int f = 0; f < nt; f++) {
                    const uint32_t dsf = s_d[f][lane];
#pragma unroll
                    for (int j = 0; j < CTV; j++) {
                        const uint32_t tdj = __shfl_sync(FULL, tdv[j], f);
                        const bool tight = dsf + tdj == dv[j];
                        if (__any_sync(FULL, tight)) {
                            const uint64_t tsj = shfl_u64(tsv[j], f);
                            if (tight) sv[j] = madd_ck(sv[j], s_x[f][lane], tsj, ovf);
                        }
                    }
                }
            }
        }
    }
    // ---- backward: acc = sum over exit frontiers f on a shortest path of sigma_i(v,f) c(s,f)
    DT acc[CTV];
    bool live[CTV], any_live = false;
#pragma unroll
    for (int j = 0; j < CTV; j++) {
        acc[j] = (DT)0;
        live[j] = sv[j] != 0;
        any_live |= live[j];
    }
    if (__syncthreads_or(any_live)) {
        __half2 lvh[CT_NP];   // 16-bit path: distances of live nodes, NaN otherwise
#pragma unroll
        for (int q = 0; q < CT_NP; q++)
            lvh[q] = __halves2half2(ct_h_or_nan(live[2 * q] ? dv[2 * q] : CT_NONE),
                                    ct_h_or_nan(live[2 * q + 1] ? dv[2 * q + 1] : CT_NONE));
        for (int32_t f0 = 0; f0 < nfi; f0 += FT) {
            const int nt = min(FT, nfi - f0);
            __syncthreads();
            for (int x = threadIdx.x; x < nt * 32; x += CT_WARPS * 32) {
                const int64_t o = fbase + (int64_t)(f0 + (x >> 5)) * 32 + (x & 31);
                const uint32_t v = (uint32_t)d_all[o];
                // an unreachable frontier must equal no sum: NaN on the 16-bit path
                if (use16) s_h[x >> 5][x & 31] = __half2half2(ct_h_or_nan(v));
                else s_d[x >> 5][x & 31] = v;
                DT cv = dl_all[o];
                uint64_t bits = 0;
                memcpy(&bits, &cv, sizeof(DT));
                s_x[x >> 5][x & 31] = bits;
            }
            uint32_t tdv[CTV];
            uint64_t tsv[CTV];
#pragma unroll
            for (int j = 0; j < CTV; j++) {
                tdv[j] = td_at(T.tdr, j, f0, nt);
                tsv[j] = tdv[j] != (uint32_t)DINF ? T.tsr[t0 + (int64_t)(vb + j) * nfi + f0 + lane] : 0ull;
            }
            if (use16) {
#pragma unroll
                for (int q = 0; q < CT_NP; q++) s_t[warp][lane][q] = __halves2half2(ct_h(tdv[2 * q]), ct_h(tdv[2 * q + 1]));
                DT* cd = reinterpret_cast<DT*>(&s_c[warp][0][0]);   // [j][f] as DT
#pragma unroll
                for (int j = 0; j < CTV; j++) cd[j * FT + lane] = (DT)tsv[j];
            }
            __syncthreads();
            if (use16) {
                const DT* cd = reinterpret_cast<const DT*>(&s_c[warp][0][0]);
                for (int f = 0; f < nt; f++) {
                    const __half2 dh = s_h[f][lane];
                    H2x2 tt;
                    tt.u = *reinterpret_cast<const uint2*>(&s_t[warp][f][0]);
                    unsigned m[CT_NP], any = 0u;
#pragma unroll
                    for (int q = 0; q < CT_NP; q++) {
                        m[q] = __heq2_mask(__hadd2(lvh[q], tt.h[q]), dh);
                        any |= m[q];
                    }
                    if (__any_sync(FULL, any != 0u)) {
                        DT cf;
                        const uint64_t bits = s_x[f][lane];
                        memcpy(&cf, &bits, sizeof(DT));
#pragma unroll
                        for (int j = 0; j < CTV; j++)
                            if ((m[j >> 1] >> (16 * (j & 1))) & 0xffffu) acc[j] += cd[j * FT + f] * cf;
                    }
                }
            } else {
                for (int f = 0; f < nt; f++) {
                    const uint32_t dsf = s_d[f][lane];
                    const bool fin = dsf != (uint32_t)DINF;
#pragma unroll
                    for (int j = 0; j < CTV; j++) {
                        // a live node has a finite distance, and a sum with an unreachable exit
                        // table entry exceeds every finite frontier distance.  (The shuffle is
                        // taken by every lane before the test: a full-mask shuffle that some lanes
                        // skip never completes.)
                        const uint32_t tdj = __shfl_sync(FULL, tdv[j], f);
                        const bool on = live[j] && fin && dv[j] + tdj == dsf;
                        if (__any_sync(FULL, on)) {
                            const uint64_t tsj = shfl_u64(tsv[j], f);
                            if (on) {
                                DT cf;
                                const uint64_t bits = s_x[f][lane];
                                memcpy(&cf, &bits, sizeof(DT));
                                acc[j] += (DT)tsj * cf;
                            }
                        }
                    }
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < CTV; j++) {
        const double delta = (double)((DT)sv[j] * acc[j]);
        const double tot = warp_sum(delta);
        if (lane == 0 && j < nv && tot != 0.0) {
            const int64_t ix = (int64_t)slot * cap_bc + pnodes[ps + vb + j];
            double s0 = bc_sum[ix], c0 = bc_cmp[ix];
            neumaier_add(s0, c0, tot);
            bc_sum[ix] = s0;
            bc_cmp[ix] = c0;
        }
    }
    if (__any_sync(FULL, ovf) && lane == 0) atomicOr(&flags[FLAG_SIGMA_OVF], 1u);
}

__global__ void combine_kernel(const double* bc_sum, const double* bc_cmp, int nslots, int64_t cap_bc, int64_t n,
                               double scale, double* out) {
    GRID_STRIDE(v, n) {
        double s = 0.0, c = 0.0;
        for (int k = 0; k < nslots; k++) {
            neumaier_add(s, c, bc_sum[(int64_t)k * cap_bc + v]);
            neumaier_add(s, c, bc_cmp[(int64_t)k * cap_bc + v]);
        }
        out[v] = (s + c) * scale;
    }
}

}  // namespace

void sk_partition(int32_t n, const int32_t* part, int32_t k, const int32_t* S, int32_t nS, int32_t* partp,
                  uint32_t* flags, cudaStream_t st) {
    if (n > 0) partp_copy_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, part, k, partp, flags);
    if (nS > 0) partp_targets_kernel<<<grid_for(nS, 256), 256, 0, st>>>(S, nS, k, partp);
}
void sk_frontiers(int32_t n, const int64_t* rp, const int32_t* col, const int32_t* partp, uint8_t* fr, cudaStream_t st) {
    if (n > 0) frontier_kernel<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(n, rp, col, partp, fr);
}
void sk_group_keys(int32_t n, const int32_t* partp, const uint8_t* fr, uint64_t* keys, uint32_t* vals, cudaStream_t st) {
    if (n > 0) group_keys_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, partp, fr, keys, vals);
}
void sk_segments(const uint64_t* keys, int32_t n, int32_t kp, int32_t* pstart, int32_t* nf, cudaStream_t st) {
    segments_kernel<<<grid_for((int64_t)kp + 1, 256), 256, 0, st>>>(keys, n, kp, pstart, nf);
}
void sk_local_ids(int32_t n, const uint32_t* pnodes, const int32_t* partp, const int32_t* pstart, const int32_t* nf,
                  const int32_t* skbase, int32_t* loc, int32_t* skid, int32_t* sknode, cudaStream_t st) {
    if (n > 0) local_ids_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, pnodes, partp, pstart, nf, skbase, loc, skid, sknode);
}
void sk_local_count(int32_t n, const uint32_t* pnodes, const int64_t* rp, const int32_t* col, const int32_t* partp,
                    int64_t* cnt, cudaStream_t st) {
    if (n > 0) local_count_kernel<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(n, pnodes, rp, col, partp, cnt);
}
void sk_local_fill(int32_t n, const uint32_t* pnodes, const int64_t* rp, const int32_t* col, const uint32_t* w,
                   const int32_t* partp, const int32_t* loc, const int64_t* lrp, int32_t* lcol, int32_t* lw,
                   cudaStream_t st) {
    if (n > 0)
        local_fill_kernel<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(n, pnodes, rp, col, w, partp, loc, lrp, lcol, lw);
}
void sk_arcs_count(int32_t N, const int32_t* sknode, const int64_t* rp, const int32_t* col, const int32_t* partp,
                   const int32_t* loc, SkTables T, int64_t* cnt, cudaStream_t st) {
    if (N > 0) sk_arcs_count_kernel<<<grid_for((int64_t)N * 32, 256), 256, 0, st>>>(N, sknode, rp, col, partp, loc, T, cnt);
}
void sk_arcs_fill(int32_t N, const int32_t* sknode, const int64_t* rp, const int32_t* col, const uint32_t* w,
                  const int32_t* partp, const int32_t* loc, const int32_t* skid, SkTables T, const int64_t* skrp,
                  int32_t* skcol, int32_t* skw, uint64_t* skmu, unsigned long long* maxes, cudaStream_t st) {
    if (N > 0)
        sk_arcs_fill_kernel<<<grid_for((int64_t)N * 32, 256), 256, 0, st>>>(N, sknode, rp, col, w, partp, loc, skid, T,
                                                                           skrp, skcol, skw, skmu, maxes);
}
void sk_transpose(int32_t N, const int64_t* rp, const int32_t* col, const int32_t* w, const uint64_t* mu,
                  int64_t* cursor, int32_t* tcol, int32_t* tw, uint64_t* tmu, int pass, cudaStream_t st) {
    if (N > 0)
        sk_transpose_kernel<<<grid_for((int64_t)N * 32, 256), 256, 0, st>>>(N, rp, col, w, mu, cursor, tcol, tw, tmu, pass);
}
void sk_gather_flags(int32_t N, const int32_t* sknode, const uint8_t* in_s, uint8_t* out, cudaStream_t st) {
    if (N > 0) gather_flags_kernel<<<grid_for(N, 256), 256, 0, st>>>(N, sknode, in_s, out);
}
void sk_target_ids(const int32_t* S, int32_t nS, const int32_t* skid, int32_t* out, cudaStream_t st) {
    if (nS > 0) target_ids_kernel<<<grid_for(nS, 256), 256, 0, st>>>(S, nS, skid, out);
}

void centrality_launch(bool fp32_delta, bool h16, const CentralityUnit* units, int nunits, int nslots, SkTables T,
                       const uint32_t* pnodes, const int32_t* skbase, const int32_t* d, const uint64_t* sg,
                       const void* dl, int64_t cap_n, double* bc_sum, double* bc_cmp, int64_t cap_bc,
                       uint32_t* flags, cudaStream_t st) {
    if (nunits <= 0 || nslots <= 0) return;
    const int slot_major = nunits <= 65535 ? 1 : 0;   // grid.y is limited to 65,535
    const dim3 grid = slot_major ? dim3(nslots, nunits) : dim3(nunits, nslots);
    if (fp32_delta)
        centrality_tiled_kernel<float><<<grid, CT_WARPS * 32, 0, st>>>(units, T, pnodes, skbase, d, sg,
                                                                      (const float*)dl, cap_n, bc_sum, bc_cmp,
                                                                      cap_bc, flags, slot_major, h16 ? 1 : 0);
    else
        centrality_tiled_kernel<double><<<grid, CT_WARPS * 32, 0, st>>>(units, T, pnodes, skbase, d, sg,
                                                                       (const double*)dl, cap_n, bc_sum, bc_cmp,
                                                                       cap_bc, flags, slot_major, h16 ? 1 : 0);
}

void combine_launch(const double* bc_sum, const double* bc_cmp, int nslots, int64_t cap_bc, int64_t n, double scale,
                    double* bc_out, cudaStream_t st) {
    if (n > 0) combine_kernel<<<grid_for(n, 256), 256, 0, st>>>(bc_sum, bc_cmp, nslots, cap_bc, n, scale, bc_out);
}

}  // namespace bcpp
