// The lockstep kernel template and its launchers (see lockstep.cu for the description), included
// by one translation unit per dependency precision so that the instances compile in parallel.
#pragma once
#include <cooperative_groups.h>
#include <type_traits>

#include "lockstep.cuh"

namespace bcpp {

namespace cg = cooperative_groups;

namespace {


// Mark head v in a bucket's bitmap (fire-and-forget: a stale mark only costs a visit that
// finds no lane at that distance).
__device__ __forceinline__ void mark_head(uint32_t* bmk, int v) { atomicOr(&bmk[v >> 5], 1u << (v & 31)); }

// 1/x for a path count x >= 1.  FP64: a single-precision seed (relative error at most 2^-23
// after the two roundings) refined by one Newton-Raphson step r' = r + r (1 - x r), which
// squares the error (about 2^-46, below 1.5e-14 relative) for two FMAs instead of a full
// double-precision division.  FP32: the ordinary division.
__device__ __forceinline__ double recip_count(double x) {
    const double r = (double)__frcp_rn((float)x);
    return fma(r, fma(-x, r, 1.0), r);
}
__device__ __forceinline__ float recip_count(float x) { return 1.0f / x; }

// Row storage: distances int32 (DINF = unreached) and path counts uint64, or, for unit-weight
// Brandes passes whose distances stay below 254 and path counts below 2^32, one byte per
// distance (255 = unreached) and 32 bits per count: rows four and two times smaller.
template <bool NARROW>
struct DistT {
    using T = int32_t;
    using S = uint64_t;
    static constexpr int32_t INF = DINF;
};
template <>
struct DistT<true> {
    using T = uint8_t;
    using S = uint32_t;
    static constexpr uint8_t INF = 255;
};
constexpr int32_t NARROW_MAX_D = 254;   // a step at this distance would relax to an unstorable 255

// this lane's SPL distances of one node row, as int32: DINF for unreached in int32 rows; one-byte
// rows keep their 255, which every comparison of a unit-weight pass (distances D - 1, D, D + 1
// with D <= 253) treats like an unreached node
template <int SPL>
__device__ __forceinline__ void ld_dist(const int32_t* p, int32_t (&x)[SPL]) {
    if constexpr (SPL == 1) {
        x[0] = *p;
    } else {
        const int2 t = *reinterpret_cast<const int2*>(p);
        x[0] = t.x; x[1] = t.y;
    }
}
template <int SPL>
__device__ __forceinline__ void ld_dist(const uint8_t* p, int32_t (&x)[SPL]) {
    if constexpr (SPL == 1) {
        x[0] = *p;
    } else {
        const uchar2 t = *reinterpret_cast<const uchar2*>(p);
        x[0] = t.x;
        x[1] = t.y;
    }
}

// vector access to this lane's SPL consecutive values of one node row
template <int SPL>
__device__ __forceinline__ void ld_row(const int32_t* p, int32_t (&x)[SPL]) {
    if constexpr (SPL == 1) {
        x[0] = *p;
    } else {
        const int2 t = *reinterpret_cast<const int2*>(p);
        x[0] = t.x; x[1] = t.y;
    }
}
template <int SPL>
__device__ __forceinline__ void ld_row(const uint64_t* p, uint64_t (&x)[SPL]) {
    if constexpr (SPL == 1) {
        x[0] = *p;
    } else {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(p);
        x[0] = t.x; x[1] = t.y;
    }
}
template <int SPL>
__device__ __forceinline__ void ld_row(const uint32_t* p, uint64_t (&x)[SPL]) {
    if constexpr (SPL == 1) {
        x[0] = *p;
    } else {
        const uint2 t = *reinterpret_cast<const uint2*>(p);
        x[0] = t.x; x[1] = t.y;
    }
}
template <int SPL>
__device__ __forceinline__ void ld_row(const double* p, double (&x)[SPL]) {
    if constexpr (SPL == 1) {
        x[0] = *p;
    } else {
        const double2 t = *reinterpret_cast<const double2*>(p);
        x[0] = t.x; x[1] = t.y;
    }
}
template <int SPL>
__device__ __forceinline__ void ld_row(const float* p, float (&x)[SPL]) {
    if constexpr (SPL == 1) {
        x[0] = *p;
    } else {
        const float2 t = *reinterpret_cast<const float2*>(p);
        x[0] = t.x; x[1] = t.y;
    }
}

// One group of U arcs starting at chunk position j: heads (and weights and multiplicities)
// are broadcast by shuffle from the chunk's registers, then the distance rows of the whole
// group are loaded before the group is handed to f (with its size as a compile-time tag), so
// f can issue its own dependent loads for the whole group at once.  Positions past the row's
// end get distance DINF, which is never a parent's or a successor's distance.
// broadcast of a multiplicity: exact uint64 (path counts) or converted once per chunk to the
// dependency type (the backward pass's products)
__device__ __forceinline__ uint64_t shfl_mult(uint64_t x, int src) { return shfl_u64(x, src); }
__device__ __forceinline__ double shfl_mult(double x, int src) { return __shfl_sync(FULL, x, src); }
__device__ __forceinline__ float shfl_mult(float x, int src) { return __shfl_sync(FULL, x, src); }

template <int U, int SPL, bool WEIGHTED, bool MULT, typename MT, typename DD, class F>
__device__ __forceinline__ void arc_group(int32_t mv, int32_t mw, MT mm, int j, int cnt, const DD* dl0, F&& f) {
    constexpr int SH = SPL == 1 ? 5 : 6;
    int32_t vv[U], ww[U], dv[U][SPL];
    MT mk[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
        vv[k] = __shfl_sync(FULL, mv, (j + k) & 31);
        ww[k] = WEIGHTED ? __shfl_sync(FULL, mw, (j + k) & 31) : 1;
        mk[k] = MULT ? shfl_mult(mm, (j + k) & 31) : (MT)1;
    }
#pragma unroll
    for (int k = 0; k < U; k++) {
        if (j + k < cnt) {
            ld_dist<SPL>(dl0 + ((uint32_t)vv[k] << SH), dv[k]);
        } else {
#pragma unroll
            for (int s = 0; s < SPL; s++) dv[k][s] = DINF;
        }
    }
    f(std::integral_constant<int, U>{}, vv, ww, mk, dv, cnt - j);
}

// Visit the arcs [a0, a0 + deg) of one row: 32 heads per coalesced load, then groups of
// UNROLL arcs, or of UNROLL / 2 when at most that many are left (low-degree rows waste less).
// MT: the type the multiplicities are handed to f in (uint64_t, or the dependency type); MP: the
// type they are stored in (uint64_t, or already the dependency type).
template <int UNROLL, int SPL, bool WEIGHTED, bool MULT, typename MT = uint64_t, typename MP = uint64_t,
          typename DD, class F>
__device__ __forceinline__ void for_arc_groups(const int32_t* __restrict__ col, const int32_t* __restrict__ w,
                                               const MP* __restrict__ mu, int64_t a0, int32_t deg,
                                               const DD* dl0, int lane, F&& f) {
    for (int32_t c0 = 0; c0 < deg; c0 += 32) {
        const int cnt = min(32, deg - c0);
        int32_t mv = 0, mw = 1;
        MT mm = (MT)1;
        if (lane < cnt) {
            mv = __ldg(col + a0 + c0 + lane);
            if (WEIGHTED) mw = __ldg(w + a0 + c0 + lane);
            if (MULT) mm = (MT)__ldg(mu + a0 + c0 + lane);
        }
        for (int j = 0; j < cnt;) {
            if (cnt - j > UNROLL / 2) {
                arc_group<UNROLL, SPL, WEIGHTED, MULT, MT>(mv, mw, mm, j, cnt, dl0, f);
                j += UNROLL;
            } else {
                arc_group<UNROLL / 2, SPL, WEIGHTED, MULT, MT>(mv, mw, mm, j, cnt, dl0, f);
                j += UNROLL / 2;
            }
        }
    }
}

// Whether some value of one node's distance row (ROW int32 values, 16-byte aligned) equals D.
template <int ROW>
__device__ __forceinline__ bool row_has(const int32_t* row, int32_t D) {
    const int4* r4 = reinterpret_cast<const int4*>(row);
    int4 t[ROW / 4];
#pragma unroll
    for (int i = 0; i < ROW / 4; i++) t[i] = r4[i];
    bool hit = false;
#pragma unroll
    for (int i = 0; i < ROW / 4; i++) hit |= t[i].x == D || t[i].y == D || t[i].z == D || t[i].w == D;
    return hit;
}
template <int ROW>
__device__ __forceinline__ bool row_has(const uint8_t*, int32_t) { return true; }

// Sparse-lane visits (32-source rows).  A node is listed once per distinct distance among its
// batch's 32 sources, so many entries have only a few lanes at the step's distance: with integer
// weights about 16 listings per node with 2 active lanes on average on the directed Chung-Lu
// workloads, with unit weights about 3 listings per node with 11 active lanes on the undirected
// ones.  A lane per source then leaves most of the warp idle on every arc.  For such an entry the
// warp spreads (arc, active source) pairs over its lanes instead: with A' lanes per arc (A' the
// power of two at or above the active count a), lane L takes source index i = L mod A' and arc
// slot j = L / A' of each chunk of 32 / A' arcs; sums per source are combined by a butterfly
// over the lanes of equal i.
#ifndef BCPP_LS_SPARSE_MAX
#define BCPP_LS_SPARSE_MAX 16
#endif
#ifndef BCPP_LS_SPARSE_UNIT
#define BCPP_LS_SPARSE_UNIT 32
#endif
// most active lanes an entry takes the sparse visit with: integer weights, unit weights
constexpr int LS_SPARSE_MAX = BCPP_LS_SPARSE_MAX;
constexpr int LS_SPARSE_UNIT = BCPP_LS_SPARSE_UNIT;

struct SparseLanes {
    int lg;       // log2 A'
    int i, j;     // this lane's source index and arc slot
    bool valid;   // i < a
    int s;        // row position (source lane) of source index i
};

// scratch: LS_SPARSE_MAX ints of this warp's shared memory
__device__ __forceinline__ SparseLanes sparse_lanes(unsigned am, int lane, int* scratch) {
    const int a = __popc(am);
    SparseLanes L;
    L.lg = a <= 1 ? 0 : 32 - __clz(a - 1);
    L.i = lane & ((1 << L.lg) - 1);
    L.j = lane >> L.lg;
    L.valid = L.i < a;
    if ((am >> lane) & 1u) scratch[__popc(am & ((1u << lane) - 1u))] = lane;
    __syncwarp();
    L.s = scratch[L.valid ? L.i : 0];
    __syncwarp();   // the warp's next entry rewrites the scratch
    return L;
}

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t x, int m) {
    const uint32_t lo = __shfl_xor_sync(FULL, (uint32_t)x, m);
    const uint32_t hi = __shfl_xor_sync(FULL, (uint32_t)(x >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}

// Scalar control state of one batch; with a cluster it lives in the leader CTA's shared memory
// and the other CTAs reach it through distributed shared memory.
struct LsCtl {
    int item, pos, next, D, done, maxpush, nsteps, err, end;
    unsigned long long t0, t1;   // batch start and end of its forward pass (global timer, ns)
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Fetch the next entry index of the current step for this warp (dynamic scheduling).
__device__ __forceinline__ int fetch_entry(int* next, int lane) {
    int e = 0;
    if (lane == 0) e = atomicAdd(next, 1);
    return __shfl_sync(FULL, e, 0);
}

__device__ __forceinline__ LsEnt load_entry(const LsEnt* order, int e, int end) {
    if (e < end) return order[e];
    LsEnt z;
    z.u = -1; z.deg = 0; z.a0 = 0;
    return z;
}

template <typename DT, int SPL, int CL, bool FUSED, bool WEIGHTED, bool MULT, bool NARROW>
__global__ void __launch_bounds__(LS_THREADS, LS_MIN_CTAS)
ls_kernel(const LsArena A, const LsParams P, const LsSlots W, const LsItem* __restrict__ items, int nitems) {
    // CL CTAs (a thread-block cluster when CL > 1) share one batch and one slot
    __shared__ LsCtl s_ctl;
    __shared__ int s_scr[LS_THREADS / 32][32];   // sparse-lane visits: active lanes by rank
    LsCtl* ctl = &s_ctl;
    int crank = 0;
    if constexpr (CL > 1) {
        cg::cluster_group cluster = cg::this_cluster();
        crank = (int)cluster.block_rank();
        ctl = cluster.map_shared_rank(&s_ctl, 0);
    }
    auto sync = [&]() {
        if constexpr (CL == 1) __syncthreads();
        else cg::this_cluster().sync();
    };
    constexpr int GT = CL * LS_THREADS;            // threads sharing the batch
    const int gtid = crank * LS_THREADS + (int)threadIdx.x;
    const int gwarp = gtid >> 5;
    const bool leader = gtid == 0;
    const int lane = threadIdx.x & 31;
    const int slot = blockIdx.x / CL;
    constexpr int ROW = 32 * SPL;                 // sources per node row
    constexpr int SH = SPL == 1 ? 5 : 6;          // log2(ROW)
    // arcs handled per group (bounded by the 64 registers of two resident 512-thread CTAs).
    // Unit weights: groups of 4 in FP64 and with one CTA per batch, 8 in clustered FP32-delta
    // instances (same-box A/B on the unit-weight workloads; integer weights keep 8).
#ifndef BCPP_LS_UNROLL
#define BCPP_LS_UNROLL 8
#endif
    constexpr int UNIT_UNROLL = (std::is_same<DT, double>::value || CL == 1) ? 4 : BCPP_LS_UNROLL;
    constexpr int UNROLL = SPL == 1 ? ((WEIGHTED && FUSED) ? (MULT ? 4 : 6)
                                                           : (MULT ? 6 : (WEIGHTED ? BCPP_LS_UNROLL : UNIT_UNROLL)))
                                    : ((WEIGHTED && FUSED) ? (MULT ? 2 : 3) : (MULT ? 3 : 4));
    // Leaf entries (no successor on any active lane) are finished by the forward pass and skip
    // the backward arc scan.  Measured with the sparse-lane visits: `chunglu_1m` plain (4-CTA
    // clusters) 726 -> 679 ms, `chunglu_100k` 22.4 -> 19.5 ms, `planted_200k` 45.7 -> 39.8 ms.
    constexpr bool LEAVES = true;
    // entries with at most SMAX lanes at the step's distance take the sparse-lane visit
    constexpr int SMAX = SPL != 1 ? 0 : WEIGHTED ? LS_SPARSE_MAX : LS_SPARSE_UNIT;

    using DD = typename DistT<NARROW>::T;
    constexpr DD DD_INF = DistT<NARROW>::INF;
    using SG = typename DistT<NARROW>::S;
    LsEnt* order = W.order + (int64_t)slot * W.cap_order;
    int32_t* step_d = W.step_d + (int64_t)slot * W.cap_steps;
    int32_t* step_beg = W.step_beg + (int64_t)slot * W.cap_steps;
    uint32_t* bm = W.bm + (int64_t)slot * P.nb * W.bm_words;
    uint8_t* bflag = W.bflag + (int64_t)slot * P.nb;
    // dependencies of the current batch (at most 32 * SPL terms per node) are added into bat with
    // atomics; at the end of the batch they move into the slot's compensated sums
    double* bat = W.bc_bat ? W.bc_bat + (int64_t)slot * W.cap_bc : nullptr;
    // multiplicities in the dependency type for the backward pass (set whenever MULT)
    const DT* mud = reinterpret_cast<const DT*>(A.mud);

    bool first = true;
    for (;;) {
        if (leader) {
            if (P.items_static) ctl->item = first ? slot : nitems;
            else ctl->item = atomicAdd(P.item_counter, 1);
        }
        first = false;
        sync();
        const int it = ctl->item;
        if (it >= nitems) break;
        const LsItem I = items[it];
        // the batch's rows: the slot's, or the item's own row state (kept for the Centrality step)
        const int64_t rb = P.rows_by_item ? (int64_t)it : (int64_t)slot;
        DD* d = reinterpret_cast<DD*>(W.d) + rb * W.cap_n * ROW;
        SG* sg = reinterpret_cast<SG*>(W.sg) + rb * W.cap_n * ROW;
        DT* dlt = reinterpret_cast<DT*>(W.dl) + rb * W.cap_n * ROW;
        DD* dl0 = d + lane * SPL;                 // this lane's slice: node v at dl0[v << SH]
        SG* sl0 = sg + lane * SPL;
        DT* cl0 = dlt + lane * SPL;
        const int64_t base = A.node_off[I.g];
        const int32_t n = (int32_t)(A.node_off[I.g + 1] - base);
        const int64_t* rp = A.rp + base;
        const int64_t* irp = A.irp + base;
        const int32_t nf = P.nfront ? P.nfront[I.g] : 0;
        int32_t my_src[SPL];
#pragma unroll
        for (int s = 0; s < SPL; s++) {
            const int b = lane * SPL + s;
            my_src[s] = b < I.nsrc ? P.srcs[I.src_off + b] : -1;
        }

        // sources: d = 0, sigma = 1, bucket 0
        if (gtid < 32) {
#pragma unroll
            for (int s = 0; s < SPL; s++) {
                if (my_src[s] >= 0) {
                    dl0[((uint32_t)my_src[s] << SH) + s] = 0;
                    sl0[((uint32_t)my_src[s] << SH) + s] = 1;
                    atomicOr(&bm[my_src[s] >> 5], 1u << (my_src[s] & 31));
                }
            }
        }
        if (leader) {
            bflag[0] = 1;
            ctl->pos = 0; ctl->D = 0; ctl->maxpush = 0; ctl->nsteps = 0; ctl->err = 0;
            if (P.phase_ns) ctl->t0 = global_ns();
        }
        sync();

        // ------------------------------------------------------------------ forward
        for (;;) {
            if (leader) {
                // Integer weights: the next non-empty bucket.  Every pending tentative distance
                // lies in [D, D + max w] (a step at D' < D relaxes to at most D' + max w), so
                // the nb = max w + 1 buckets from D hold all of them and the batch is done when
                // none of them is flagged.  Unit weights: the levels are consecutive, and the
                // step after the last level finds its bucket empty and leaves maxpush below D.
                int D = ctl->D;
                if constexpr (WEIGHTED) {
                    int i = 0;
                    while (i < P.nb && bflag[(D + i) % P.nb] == 0) i++;
                    D += i;
                    ctl->done = i == P.nb || ctl->err;
                } else {
                    ctl->done = (D > ctl->maxpush) || ctl->err;
                }
                ctl->D = D;
                if (!ctl->done) {
                    if constexpr (WEIGHTED) bflag[D % P.nb] = 0;
                    if (ctl->nsteps >= W.cap_steps) {
                        ctl->err = 1; ctl->done = 1;
                    } else {
                        step_d[ctl->nsteps] = D;
                        step_beg[ctl->nsteps] = ctl->pos;
                        ctl->next = ctl->pos;
                    }
                }
            }
            sync();
            if (ctl->done) break;
            const int32_t D = ctl->D;
            const int beg = ctl->next;
            // heads relaxed to D + w go to bucket (D + w) mod nb; w < nb, so one subtraction
            // replaces the modulo
            const int dmod = D % P.nb;
            // collect bucket D into the order list
            {
                uint32_t* bmD = bm + (int64_t)dmod * W.bm_words;
                const int nwords = (n + 31) >> 5;
                const int nwr = (nwords + 31) & ~31;
                for (int wi = gtid; wi < nwr; wi += GT) {
                    uint32_t x = wi < nwords ? bmD[wi] : 0u;
                    if (x) bmD[wi] = 0u;
                    if constexpr (WEIGHTED) {
                        // A mark goes stale when the lane it was made for improves to a smaller
                        // distance (the node is then settled from that smaller bucket).  Keep only
                        // nodes with some lane at D, so that a batch lists each node at most once
                        // per distinct distance (at most 32 * SPL entries per node).
                        uint32_t keep = 0u;
                        for (uint32_t y = x; y; y &= y - 1) {
                            const int b = __ffs(y) - 1;
                            if (row_has<ROW>(d + ((int64_t)(wi * 32 + b) << SH), D)) keep |= 1u << b;
                        }
                        x = keep;
                    }
                    const int c = __popc(x);
                    const int incl = warp_incl_scan(c, lane);
                    const int tot = __shfl_sync(FULL, incl, 31);
                    int bpos = 0;
                    if (lane == 31 && tot) bpos = atomicAdd(&ctl->pos, tot);
                    bpos = __shfl_sync(FULL, bpos, 31);
                    if (tot && bpos + tot > W.cap_order) {
                        if (lane == 0) atomicExch(&ctl->err, 1);
                        continue;
                    }
                    int p = bpos + incl - c;
                    while (x) {
                        const int b = __ffs(x) - 1;
                        x &= x - 1;
                        order[p++].u = wi * 32 + b;
                    }
                }
            }
            sync();
            if (leader) {
                ctl->end = min(ctl->pos, (int)W.cap_order);
                if (NARROW && D >= NARROW_MAX_D && ctl->end > beg) {
                    // nodes deeper than one-byte distances reach: the call reruns with int32 rows
                    atomicOr(&P.flags[FLAG_DEPTH], 1u);
                    ctl->err = 1;
                }
            }
            sync();
            if (ctl->err) break;
            const int end = ctl->end;
            // attach every entry's out-arc range (independent loads, all threads)
            for (int e = beg + gtid; e < end; e += GT) {
                const int32_t u = order[e].u;
                const int64_t a0 = __ldg(rp + u);
                order[e].a0 = a0;
                order[e].deg = (int32_t)(__ldg(rp + u + 1) - a0);
            }
            sync();
            // settle the nodes of step D
            int e = fetch_entry(&ctl->next, lane);
            LsEnt cur = load_entry(order, e, end);
            while (e < end) {
                const int e2 = fetch_entry(&ctl->next, lane);
                const LsEnt nxt = load_entry(order, e2, end);
                const int u = cur.u;
                int32_t du[SPL];
                ld_dist<SPL>(dl0 + ((uint32_t)u << SH), du);
                bool act[SPL], pull[SPL], any = false;
#pragma unroll
                for (int s = 0; s < SPL; s++) {
                    act[s] = du[s] == D;
                    pull[s] = act[s] && D > 0;
                    any |= act[s];
                }
                const unsigned am = __ballot_sync(FULL, any);
                bool sparse = false;
                if constexpr (SPL == 1 && SMAX > 0) {
                    if (am != 0u && __popc(am) <= SMAX) {
                        // few lanes at D: (arc, active source) pairs over the lanes
                        sparse = true;
                        const SparseLanes L = sparse_lanes(am, lane, s_scr[threadIdx.x >> 5]);
                        const int K = 32 >> L.lg;   // arcs per chunk
                        DD* drow = d + L.s;
                        SG* srow = sg + L.s;
                        const bool pl = D > 0;
                        bool ovf = false, cand = false;
                        uint64_t acc = 0;
                        // v is a parent of u on source i: d(v) + w(v,u) = D (and, for the tables,
                        // v is not a frontier other than the source)
                        auto sp_pull = [&](int32_t v, int32_t dv, int32_t w, uint64_t m) {
                            const bool tight = WEIGHTED ? dv < D && dv + w == D : dv == D - 1;
                            if (tight && (v >= nf || dv == 0)) {
                                const uint64_t t = srow[(uint32_t)v << 5];
                                if constexpr (NARROW)
                                    acc += t;   // parents' counts < 2^32, fewer than 2^31 parents
                                else
                                    acc = MULT ? madd_ck(acc, t, m, ovf) : add_ck(acc, t, ovf);
                            }
                        };
                        // relax u -> v on source i; warp-collective (every lane calls it)
                        auto sp_relax = [&](int32_t v, int32_t dv, int32_t w, bool ok) {
                            const int64_t nd64 = (int64_t)D + w;
                            const int32_t nd = !WEIGHTED ? D + 1 : nd64 < DINF ? (int32_t)nd64 : DINF;
                            const bool imp = ok && nd < dv;
                            if constexpr (LEAVES) cand |= ok && nd <= dv;
                            const unsigned im = __ballot_sync(FULL, imp);
                            if (imp) {
                                if constexpr (WEIGHTED) atomicMin(reinterpret_cast<int32_t*>(drow) + ((uint32_t)v << 5), nd);
                                else drow[(uint32_t)v << 5] = (DD)nd;
                                // the arc's first improving lane marks the head
                                if (((im >> (L.j << L.lg)) & ((1u << L.i) - 1u)) == 0u) {
                                    int bk = dmod + w;
                                    if (bk >= P.nb) bk -= P.nb;
                                    mark_head(bm + (int64_t)bk * W.bm_words, v);
                                    if constexpr (WEIGHTED) bflag[bk] = 1;
                                }
                            }
                        };
                        // two arcs per lane and iteration (and, for directed graphs, an in-arc
                        // and an out-arc), so that their dependent load chains overlap
                        if (FUSED) {
                            for (int c0 = 0; c0 < cur.deg; c0 += 2 * K) {
                                const int k1 = c0 + L.j, k2 = k1 + K;
                                const bool ok1 = L.valid && k1 < cur.deg, ok2 = L.valid && k2 < cur.deg;
                                int32_t v1 = 0, w1 = 1, d1 = DINF, v2 = 0, w2 = 1, d2 = DINF;
                                uint64_t m1 = 1, m2 = 1;
                                if (ok1) {
                                    v1 = __ldg(A.col + cur.a0 + k1);
                                    if (WEIGHTED) w1 = __ldg(A.w + cur.a0 + k1);
                                    if (MULT) m1 = __ldg(A.mu + cur.a0 + k1);
                                }
                                if (ok2) {
                                    v2 = __ldg(A.col + cur.a0 + k2);
                                    if (WEIGHTED) w2 = __ldg(A.w + cur.a0 + k2);
                                    if (MULT) m2 = __ldg(A.mu + cur.a0 + k2);
                                }
                                if (ok1) d1 = drow[(uint32_t)v1 << 5];
                                if (ok2) d2 = drow[(uint32_t)v2 << 5];
                                if (pl) {
                                    if (ok1) sp_pull(v1, d1, w1, m1);
                                    if (ok2) sp_pull(v2, d2, w2, m2);
                                }
                                sp_relax(v1, d1, w1, ok1);
                                sp_relax(v2, d2, w2, ok2);
                            }
                        } else {
                            int64_t i0 = 0;
                            int32_t ideg = 0;
                            if (pl) {
                                i0 = __ldg(irp + u);
                                ideg = (int32_t)(__ldg(irp + u + 1) - i0);
                            }
                            const int32_t span = max(ideg, (int32_t)cur.deg);
                            for (int c0 = 0; c0 < span; c0 += K) {
                                const int k = c0 + L.j;
                                const bool okp = L.valid && k < ideg, ok = L.valid && k < cur.deg;
                                int32_t pv = 0, pw = 1, pd = DINF, v = 0, w = 1, dv = DINF;
                                uint64_t pm = 1;
                                if (okp) {
                                    pv = __ldg(A.icol + i0 + k);
                                    if (WEIGHTED) pw = __ldg(A.iw + i0 + k);
                                    if (MULT) pm = __ldg(A.imu + i0 + k);
                                }
                                if (ok) {
                                    v = __ldg(A.col + cur.a0 + k);
                                    if (WEIGHTED) w = __ldg(A.w + cur.a0 + k);
                                }
                                if (okp) pd = drow[(uint32_t)pv << 5];
                                if (ok) dv = drow[(uint32_t)v << 5];
                                if (okp) sp_pull(pv, pd, pw, pm);
                                sp_relax(v, dv, w, ok);
                            }
                        }
                        if (pl) {
#pragma unroll
                            for (int o = 1; o < 32; o <<= 1)
                                if (o >= (1 << L.lg)) acc = add_ck(acc, shfl_xor_u64(acc, o), ovf);
                        }
                        const bool head = L.valid && L.j == 0;
                        if constexpr (LEAVES) {
                            if ((P.mode == LS_BRANDES || P.mode == LS_SKEL) && !__any_sync(FULL, cand)) {
                                const bool tgt = P.in_s ? P.in_s[base + u] != 0 : true;
                                if (head)
                                    dlt[((uint32_t)u << 5) + L.s] = tgt ? recip_count((DT)(pl ? acc : 1ull)) : (DT)0;
                                if (lane == 0) order[e].deg = cur.deg | INT32_MIN;
                            }
                        }
                        if (pl && head) srow[(uint32_t)u << 5] = (SG)acc;
                        if (__any_sync(FULL, ovf) && lane == 0) atomicOr(&P.flags[FLAG_SIGMA_OVF], 1u);
                        if constexpr (NARROW) {
                            // a count past 32 bits: abort the batch, the call reruns with 64-bit rows
                            if (__any_sync(FULL, pl && head && (acc >> 32) != 0) && lane == 0) {
                                atomicOr(&P.flags[FLAG_DEPTH], 1u);
                                atomicExch(&ctl->err, 1);
                            }
                        }
                    }
                }
                if (am != 0u && !sparse) {
                    bool ovf = false;
                    bool cand = false;   // some arc relaxed to <= its head's distance: a possible successor
                    uint64_t acc[SPL];
#pragma unroll
                    for (int s = 0; s < SPL; s++) acc[s] = 0;
                    // sigma(s,u) = sum over parents v (d(v) + w(v,u) = D) of sigma(s,v) * m(v,u)
                    auto pull_group = [&](auto tag, const int32_t* vv, const int32_t* ww, const uint64_t* mk,
                                          const int32_t (*dv)[SPL]) {
                        constexpr int U = decltype(tag)::value;
                        uint64_t sp[U][SPL];
#pragma unroll
                        for (int k = 0; k < U; k++) {
                            bool par[SPL], anyp = false;
#pragma unroll
                            for (int s = 0; s < SPL; s++) {
                                const bool tight = WEIGHTED ? dv[k][s] < D && dv[k][s] + ww[k] == D : dv[k][s] == D - 1;
                                par[s] = pull[s] && tight &&
                                         (vv[k] >= nf || dv[k][s] == 0);
                                anyp |= par[s];
                            }
                            uint64_t t[SPL];
                            if (anyp) ld_row<SPL>(sl0 + ((uint32_t)vv[k] << SH), t);
#pragma unroll
                            for (int s = 0; s < SPL; s++) sp[k][s] = par[s] ? t[s] : 0ull;
                        }
#pragma unroll
                        for (int k = 0; k < U; k++)
#pragma unroll
                            for (int s = 0; s < SPL; s++)
                                if constexpr (NARROW)
                                    acc[s] += sp[k][s];   // parents' counts < 2^32, fewer than 2^31 parents
                                else if (MULT)
                                    acc[s] = madd_ck(acc[s], sp[k][s], mk[k], ovf);
                                else
                                    acc[s] = add_ck(acc[s], sp[k][s], ovf);
                    };
                    // relax the out-arcs: lower tentative distances, mark improved heads
                    auto relax_group = [&](auto tag, const int32_t* vv, const int32_t* ww, const int32_t (*dv)[SPL],
                                           int left) {
                        constexpr int U = decltype(tag)::value;
#pragma unroll
                        for (int k = 0; k < U; k++) {
                            if (k >= left) break;
                            const int64_t nd64 = (int64_t)D + ww[k];
                            const int32_t nd = !WEIGHTED ? D + 1 : nd64 < DINF ? (int32_t)nd64 : DINF;
                            bool imp[SPL], anyi = false;
#pragma unroll
                            for (int s = 0; s < SPL; s++) {
                                imp[s] = act[s] && nd < dv[k][s];
                                if constexpr (LEAVES) cand |= act[s] && nd <= dv[k][s];
                                anyi |= imp[s];
                            }
                            const unsigned im = __ballot_sync(FULL, anyi);
                            if (im) {
                                DD* pd = dl0 + ((uint32_t)vv[k] << SH);
#pragma unroll
                                for (int s = 0; s < SPL; s++) {
                                    if (imp[s]) {
                                        if constexpr (WEIGHTED) atomicMin(reinterpret_cast<int32_t*>(pd) + s, nd);
                                        else pd[s] = (DD)nd;
                                    }
                                }
                                if (lane == __ffs(im) - 1) {
                                    int bk = dmod + ww[k];
                                    if (bk >= P.nb) bk -= P.nb;
                                    mark_head(bm + (int64_t)bk * W.bm_words, vv[k]);
                                    if constexpr (WEIGHTED) bflag[bk] = 1;
                                }
                            }
                        }
                    };
                    if (FUSED) {
                        for_arc_groups<UNROLL, SPL, WEIGHTED, MULT>(A.col, A.w, A.mu, cur.a0, cur.deg, dl0, lane,
                            [&](auto tag, const int32_t* vv, const int32_t* ww, const uint64_t* mk,
                                const int32_t (*dv)[SPL], int left) {
                                pull_group(tag, vv, ww, mk, dv);
                                relax_group(tag, vv, ww, dv, left);
                            });
                    } else {
                        if (D > 0) {
                            const int64_t i0 = __ldg(irp + u);
                            const int32_t ideg = (int32_t)(__ldg(irp + u + 1) - i0);
                            for_arc_groups<UNROLL, SPL, WEIGHTED, MULT>(A.icol, A.iw, A.imu, i0, ideg, dl0, lane,
                                [&](auto tag, const int32_t* vv, const int32_t* ww, const uint64_t* mk,
                                    const int32_t (*dv)[SPL], int) { pull_group(tag, vv, ww, mk, dv); });
                        }
                        for_arc_groups<UNROLL, SPL, WEIGHTED, false>(A.col, A.w, (const uint64_t*)nullptr, cur.a0, cur.deg, dl0, lane,
                            [&](auto tag, const int32_t* vv, const int32_t* ww, const uint64_t*,
                                const int32_t (*dv)[SPL], int left) { relax_group(tag, vv, ww, dv, left); });
                    }
                    // Every shortest-path successor of u was relaxed to at most its distance here,
                    // so an entry without such an arc on any active lane is a leaf of all its
                    // lanes' DAGs: the backward pass skips its arcs (sign bit of its degree).
                    if constexpr (LEAVES) {
                        if ((P.mode == LS_BRANDES || P.mode == LS_SKEL) && !__any_sync(FULL, cand)) {
                            // a leaf is finished here: delta(s|u) = 0 and c(s,u) = I_{u in S} / sigma(s,u);
                            // the backward pass skips the entry
                            const bool tgt = P.in_s ? P.in_s[base + u] != 0 : true;
#pragma unroll
                            for (int s = 0; s < SPL; s++)
                                if (act[s])
                                    cl0[((uint32_t)u << SH) + s] = tgt ? recip_count((DT)(pull[s] ? acc[s] : 1ull)) : (DT)0;
                            if (lane == 0) order[e].deg = cur.deg | INT32_MIN;
                        }
                    }
                    bool wide = false;
#pragma unroll
                    for (int s = 0; s < SPL; s++) {
                        if (pull[s]) sl0[((uint32_t)u << SH) + s] = (SG)acc[s];
                        if constexpr (NARROW) wide |= pull[s] && (acc[s] >> 32) != 0;
                    }
                    if (__any_sync(FULL, ovf) && lane == 0) atomicOr(&P.flags[FLAG_SIGMA_OVF], 1u);
                    if constexpr (NARROW) {
                        // a count past 32 bits: abort the batch, the call reruns with 64-bit rows
                        if (__any_sync(FULL, wide) && lane == 0) {
                            atomicOr(&P.flags[FLAG_DEPTH], 1u);
                            atomicExch(&ctl->err, 1);
                        }
                    }
                }
                e = e2;
                cur = nxt;
            }
            sync();
            if (leader) {
                ctl->D = D + 1;
                if (end > beg) ctl->nsteps++;        // steps without entries are not recorded
                if (!WEIGHTED && end > beg) ctl->maxpush = D + 1;   // try the next level
            }
        }
        sync();
        const int nsteps = ctl->nsteps;
        const int olen = min(ctl->pos, (int)W.cap_order);
        if (leader && P.phase_ns) ctl->t1 = global_ns();
        if (ctl->err) {
            // a list outgrew its bound: report it and leave the slot clean for the next batch
            if (leader) atomicOr(&P.flags[FLAG_CAPACITY], 1u);
            for (int64_t i = gtid; i < (int64_t)n * ROW; i += GT) d[i] = DD_INF;
            for (int64_t i = gtid; i < (int64_t)P.nb * W.bm_words; i += GT) bm[i] = 0u;
            for (int i = gtid; i < P.nb; i += GT) bflag[i] = 0;
            if (P.mode == LS_SKEL && leader) {
                W.hdr[slot * 4 + 0] = 0; W.hdr[slot * 4 + 1] = 0; W.hdr[slot * 4 + 2] = it;
            }
            sync();
            continue;
        }

        if (P.mode == LS_BRANDES || P.mode == LS_SKEL) {
            // -------------------------------------------------------------- backward
            for (int st = nsteps - 1; st >= 0; st--) {
                if (leader) ctl->next = step_beg[st];
                sync();
                const int32_t D = step_d[st];
                const int end = (st + 1 < nsteps) ? step_beg[st + 1] : olen;
                int e = fetch_entry(&ctl->next, lane);
                LsEnt cur = load_entry(order, e, end);
                while (e < end) {
                    const int e2 = fetch_entry(&ctl->next, lane);
                    const LsEnt nxt = load_entry(order, e2, end);
                    if (LEAVES && cur.deg < 0) {   // a leaf, finished by the forward pass
                        e = e2;
                        cur = nxt;
                        continue;
                    }
                    const int u = cur.u;
                    int32_t du[SPL];
                    ld_dist<SPL>(dl0 + ((uint32_t)u << SH), du);
                    bool act[SPL], any = false;
#pragma unroll
                    for (int s = 0; s < SPL; s++) {
                        act[s] = du[s] == D;
                        any |= act[s];
                    }
                    const unsigned am = __ballot_sync(FULL, any);
                    bool sparse = false;
                    if constexpr (SPL == 1 && SMAX > 0) {
                        if (am != 0u && __popc(am) <= SMAX) {
                            // few lanes at D: (arc, active source) pairs over the lanes
                            sparse = true;
                            const SparseLanes L = sparse_lanes(am, lane, s_scr[threadIdx.x >> 5]);
                            const int K = 32 >> L.lg;
                            const DD* drow = d + L.s;
                            DT* crow = dlt + L.s;
                            DT acc = (DT)0;
                            // successors v of u on source i: d(v) = D + w(u,v)
                            auto succ = [&](int32_t dv, int32_t w) {
                                return WEIGHTED ? dv != DINF && (int64_t)dv == (int64_t)D + w : dv == D + 1;
                            };
                            // two arcs per lane and iteration (overlapping load chains)
                            for (int k1 = L.j; L.valid && k1 < cur.deg; k1 += 2 * K) {
                                const int k2 = k1 + K;
                                const bool two = k2 < cur.deg;
                                const int32_t v1 = __ldg(A.col + cur.a0 + k1);
                                const int32_t w1 = WEIGHTED ? __ldg(A.w + cur.a0 + k1) : 1;
                                int32_t v2 = 0, w2 = 1;
                                if (two) {
                                    v2 = __ldg(A.col + cur.a0 + k2);
                                    if (WEIGHTED) w2 = __ldg(A.w + cur.a0 + k2);
                                }
                                const int32_t d1 = drow[(uint32_t)v1 << 5];
                                const int32_t d2 = two ? (int32_t)drow[(uint32_t)v2 << 5] : DINF;
                                if (succ(d1, w1)) {
                                    const DT cv = crow[(uint32_t)v1 << 5];
                                    acc += MULT ? __ldg(mud + cur.a0 + k1) * cv : cv;
                                }
                                if (two && succ(d2, w2)) {
                                    const DT cv = crow[(uint32_t)v2 << 5];
                                    acc += MULT ? __ldg(mud + cur.a0 + k2) * cv : cv;
                                }
                            }
#pragma unroll
                            for (int o = 1; o < 32; o <<= 1)
                                if (o >= (1 << L.lg)) acc += __shfl_xor_sync(FULL, acc, o);
                            if (L.valid && L.j == 0) {
                                const DT sd = (DT)sg[((uint32_t)u << 5) + L.s];
                                const DT delta = sd * acc;
                                const bool is_t = P.in_s ? P.in_s[base + u] != 0 : true;
                                const int64_t ix = P.bc_map ? (int64_t)P.bc_map[base + u] : base + u;
                                crow[(uint32_t)u << 5] = is_t ? acc + recip_count(sd) : acc;
                                // D = 0 only at the source itself (weights >= 1)
                                if (D > 0 && bat && delta != (DT)0) atomicAdd(&bat[ix], (double)delta);
                            }
                        }
                    }
                    if (am != 0u && !sparse) {
                        // acc(s) = sum over successors v of m(u,v) c(s,v).  On GB300 a warp-wide
                        // FP64 add costs 16 SM cycles, so the sum skips every arc that is tight on
                        // no lane of the warp (about half of them), with a warp-uniform branch.
                        DT acc[SPL];
#pragma unroll
                        for (int s = 0; s < SPL; s++) acc[s] = (DT)0;
                        for_arc_groups<UNROLL, SPL, WEIGHTED, MULT, DT>(A.col, A.w, mud, cur.a0, cur.deg, dl0, lane,
                            [&](auto tag, const int32_t* vv, const int32_t* ww, const DT* mk,
                                const int32_t (*dv)[SPL], int) {
                                constexpr int U = decltype(tag)::value;
                                DT cv[U][SPL];
                                unsigned used = 0;
#pragma unroll
                                for (int k = 0; k < U; k++) {
                                    bool sc[SPL], anys = false;
#pragma unroll
                                    for (int s = 0; s < SPL; s++) {
                                        sc[s] = act[s] &&
                                                (WEIGHTED ? dv[k][s] != DINF && (int64_t)dv[k][s] == (int64_t)D + ww[k]
                                                          : dv[k][s] == D + 1);
                                        anys |= sc[s];
                                    }
                                    DT t[SPL];
                                    if (anys) ld_row<SPL>(cl0 + ((uint32_t)vv[k] << SH), t);
#pragma unroll
                                    for (int s = 0; s < SPL; s++) cv[k][s] = sc[s] ? t[s] : (DT)0;
                                    if constexpr (std::is_same<DT, double>::value)
                                        if (__any_sync(FULL, anys)) used |= 1u << k;
                                }
                                // FP32 adds are cheap: no vote, non-tight arcs add zero
#pragma unroll
                                for (int k = 0; k < U; k++)
                                    if (!std::is_same<DT, double>::value || (used & (1u << k)))
#pragma unroll
                                        for (int s = 0; s < SPL; s++)
                                            acc[s] += MULT ? mk[k] * cv[k][s] : cv[k][s];
                            });
                        uint64_t su[SPL];
                        ld_row<SPL>(sl0 + ((uint32_t)u << SH), su);
                        // c(s,u) = (I_{u in S} + delta(s|u)) / sigma(s,u) = acc + I_{u in S} / sigma(s,u)
                        // with delta(s|u) = sigma(s,u) acc: non-targets need no division
                        const bool is_t = P.in_s ? P.in_s[base + u] != 0 : true;
                        const int64_t ix = P.bc_map ? (int64_t)P.bc_map[base + u] : base + u;
                        // The slot owns its partial sums (no other CTA adds here) and an add needs
                        // no reply: each lane adds its own dependency (in FP64), so no FP64 warp
                        // reduction is needed.
#pragma unroll
                        for (int s = 0; s < SPL; s++) {
                            if (act[s]) {
                                const DT sd = (DT)su[s];
                                const DT delta = sd * acc[s];
                                cl0[((uint32_t)u << SH) + s] = is_t ? acc[s] + recip_count(sd) : acc[s];
                                if (u != my_src[s] && bat && delta != (DT)0) atomicAdd(&bat[ix], (double)delta);
                            }
                        }

                    }
                    e = e2;
                    cur = nxt;
                }
                sync();
            }
        } else if constexpr (SPL == 1 && !NARROW) {
            if (P.mode == LS_TABLE) {
                // ---------------------------------------------------------- tables d_i[v][f], sigma_i[v][f]
                const int64_t t0 = P.toff[I.g];
                for (int v = gwarp; v < n; v += GT / 32) {
                    if (lane < I.nsrc) {
                        const int32_t dv = dl0[(uint32_t)v << SH];
                        const int64_t o = t0 + (int64_t)v * nf + I.aux + lane;
                        P.td[o] = dv;
                        P.ts[o] = dv == DINF ? 0ull : sl0[(uint32_t)v << SH];
                    }
                }
                sync();
            } else if (P.mode == LS_SSSP) {
                for (int v = gwarp; v < n; v += GT / 32) {
                    if (lane < I.nsrc) {
                        const int32_t dv = dl0[(uint32_t)v << SH];
                        const int64_t o = (int64_t)(I.src_off + lane) * P.dbg_n + v;
                        P.dbg_d[o] = dv;
                        P.dbg_s[o] = dv == DINF ? 0ull : sl0[(uint32_t)v << SH];
                    }
                }
                sync();
            }
        }

        if (leader && P.phase_ns) {
            const unsigned long long t2 = global_ns();
            atomicAdd(&P.phase_ns[0], ctl->t1 - ctl->t0);
            atomicAdd(&P.phase_ns[1], t2 - ctl->t1);
        }
        if (bat && (P.mode == LS_BRANDES || P.mode == LS_SKEL)) {
            // Neumaier step of every touched node's batch sum into the slot's (sum, compensation):
            // the exchange hands each node's sum to exactly one of its entries (a node has one
            // entry per step it was settled at) and leaves zero for the next batch
            double* bcs = W.bc_sum + (int64_t)slot * W.cap_bc;
            double* bcc = W.bc_cmp + (int64_t)slot * W.cap_bc;
            constexpr int FK = 2;   // entries per thread and round, requested together
            for (int e0 = gtid * FK; e0 < olen; e0 += GT * FK) {
                int64_t ix[FK];
                unsigned long long x[FK];
#pragma unroll
                for (int k = 0; k < FK; k++) {
                    ix[k] = -1;
                    if (e0 + k < olen) {
                        const int32_t u = order[e0 + k].u;
                        ix[k] = P.bc_map ? (int64_t)P.bc_map[base + u] : base + u;
                    }
                }
#pragma unroll
                for (int k = 0; k < FK; k++)
                    x[k] = ix[k] >= 0 ? atomicExch(reinterpret_cast<unsigned long long*>(bat + ix[k]), 0ull) : 0ull;
#pragma unroll
                for (int k = 0; k < FK; k++) {
                    if (x[k]) {
                        double s0 = bcs[ix[k]], c0 = bcc[ix[k]];
                        neumaier_add(s0, c0, __longlong_as_double((long long)x[k]));
                        bcs[ix[k]] = s0;
                        bcc[ix[k]] = c0;
                    }
                }
            }
        }
        if (P.mode == LS_SKEL) {
            if (leader) {
                W.hdr[slot * 4 + 0] = olen;
                W.hdr[slot * 4 + 1] = nsteps;
                W.hdr[slot * 4 + 2] = it;
            }
        } else {
            // restore "unreached" on every touched row
            for (int e = gwarp; e < olen; e += GT / 32) {
                DD* pd = dl0 + ((uint32_t)order[e].u << SH);
#pragma unroll
                for (int s = 0; s < SPL; s++) pd[s] = DD_INF;
            }
        }
        sync();
    }
    // with a cluster, the leader's shared memory must outlive the other CTAs' last reads
    sync();
}

template <typename DT, int SPL, int CL, bool F, bool WT, bool M, bool NW>
void ls_go(const LsArena& A, const LsParams& P, const LsSlots& W, const LsItem* items, int nitems, int slots,
           cudaStream_t st) {
    if constexpr (CL == 1) {
        ls_kernel<DT, SPL, 1, F, WT, M, NW><<<slots, LS_THREADS, 0, st>>>(A, P, W, items, nitems);
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(slots * CL));
        cfg.blockDim = dim3(LS_THREADS);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, ls_kernel<DT, SPL, CL, F, WT, M, NW>, A, P, W, items, nitems);
    }
}

template <typename DT, int SPL, int CL>
void ls_launch_t(bool fused, bool weighted, bool mult, bool narrow, const LsArena& A, const LsParams& P,
                 const LsSlots& W, const LsItem* items, int nitems, int slots, cudaStream_t st) {
    if (fused) {
        if (!weighted && narrow) ls_go<DT, SPL, CL, true, false, false, true>(A, P, W, items, nitems, slots, st);
        else if (!weighted) ls_go<DT, SPL, CL, true, false, false, false>(A, P, W, items, nitems, slots, st);
        else if (!mult) ls_go<DT, SPL, CL, true, true, false, false>(A, P, W, items, nitems, slots, st);
        else ls_go<DT, SPL, CL, true, true, true, false>(A, P, W, items, nitems, slots, st);
    } else {
        if (!weighted && narrow) ls_go<DT, SPL, CL, false, false, false, true>(A, P, W, items, nitems, slots, st);
        else if (!weighted) ls_go<DT, SPL, CL, false, false, false, false>(A, P, W, items, nitems, slots, st);
        else if (!mult) ls_go<DT, SPL, CL, false, true, false, false>(A, P, W, items, nitems, slots, st);
        else ls_go<DT, SPL, CL, false, true, true, false>(A, P, W, items, nitems, slots, st);
    }
}

template <typename DT>
void ls_launch_dt(int spl, int cl, bool fused, bool weighted, bool mult, bool narrow, const LsArena& A,
                  const LsParams& P, const LsSlots& W, const LsItem* items, int nitems, int slots, cudaStream_t st) {
    if (spl == 2) ls_launch_t<DT, 2, 1>(fused, weighted, mult, narrow, A, P, W, items, nitems, slots, st);
    else if (cl == 4) ls_launch_t<DT, 1, 4>(fused, weighted, mult, narrow, A, P, W, items, nitems, slots, st);
    else if (cl == 2) ls_launch_t<DT, 1, 2>(fused, weighted, mult, narrow, A, P, W, items, nitems, slots, st);
    else ls_launch_t<DT, 1, 1>(fused, weighted, mult, narrow, A, P, W, items, nitems, slots, st);
}

}  // namespace

}  // namespace bcpp
