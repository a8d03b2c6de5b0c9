// Unit-weight lockstep Brandes with lane bitmasks (forward) and 8-bit levels (backward).
//
// Same batches, slots, settle order and backward recursion as the general lockstep kernel
// (Sec. 3, Eq. 2 and Eq. 7), specialised for unit weights, where the forward pass is a
// breadth-first search in which every lane's frontier advances one level per step.  Per node
// the kernel keeps four 32-bit lane masks (bit b = source lane b):
//   M[v][D mod 3]  lanes that reach v at level D (three rotating levels: previous, current, next)
//   M[v][3]        lanes that have reached v at a level <= the current step
// so the forward pass reads one 4-byte mask of a neighbour instead of its 32 distances:
//   parents of u on lane b at step D:   b in M[u][D] and b in M[v][D-1]   -> sigma pull
//   children of u on lane b:            b in M[u][D] and b not in M[v][3]  -> M[v][D+1] |= b
// Path counts are pulled from the parents (exact uint64, overflow checked); the level of
// every (node, lane) is also written as one byte, read back by the backward pass (32 lanes in
// one 32-byte sector).  A batch deeper than 253 levels stops and reports FLAG_LEVELS; the
// library then reruns the call with the general kernel.
//
// Slot layout inside the general kernel's distance region (128 bytes per node):
//   bytes [0, 16 n)      M[n][4]
//   bytes [16 n, 48 n)   level bytes [n][32] (0xFF = unreached)
#include "lockstep.cuh"
#include "lockstep_dev.cuh"

namespace bcpp {

namespace {

constexpr int BFS_UNROLL = 8;
constexpr uint8_t LV_NONE = 0xFF;
constexpr int LV_MAX = 253;              // D + 1 stays below LV_NONE

__global__ void bfs_init_kernel(int32_t* d, int64_t cap_n, int slots) {
    const int64_t per = cap_n * LS_LANES;                 // int32 words per slot
    const int64_t tot = per * slots;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = i % per;                        // word inside the slot
        d[i] = w < 4 * cap_n ? 0 : (w < 12 * cap_n ? -1 : 0);
    }
}

template <typename DT, bool FUSED>
__global__ void __launch_bounds__(LS_THREADS, 2)
bfs_kernel(const LsArena A, const LsParams P, const LsSlots W, const LsItem* __restrict__ items, int nitems) {
    __shared__ int s_item, s_pos, s_next, s_D, s_done, s_maxpush, s_nsteps, s_err, s_end;
    const int lane = threadIdx.x & 31;
    const int slot = blockIdx.x;
    const uint32_t lane_bit = 1u << lane;

    char* region = reinterpret_cast<char*>(W.d + (int64_t)slot * W.cap_n * LS_LANES);
    uint32_t* M = reinterpret_cast<uint32_t*>(region);                  // [n][4]
    uint8_t* lv = reinterpret_cast<uint8_t*>(region + 16 * W.cap_n);    // [n][32]
    uint8_t* lv0 = lv + lane;
    uint64_t* sl0 = W.sg + (int64_t)slot * W.cap_n * LS_LANES + lane;
    DT* cl0 = reinterpret_cast<DT*>(W.dl) + (int64_t)slot * W.cap_n * LS_LANES + lane;
    LsEnt* order = W.order + (int64_t)slot * W.cap_order;
    int32_t* step_d = W.step_d + (int64_t)slot * W.cap_steps;
    int32_t* step_beg = W.step_beg + (int64_t)slot * W.cap_steps;
    uint32_t* bm = W.bm + (int64_t)slot * P.nb * W.bm_words;
    uint8_t* bflag = W.bflag + (int64_t)slot * P.nb;
    double* bcs = W.bc_sum ? W.bc_sum + (int64_t)slot * W.cap_bc : nullptr;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.item_counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const LsItem I = items[it];
        const int64_t base = A.node_off[I.g];
        const int32_t n = (int32_t)(A.node_off[I.g + 1] - base);
        const int64_t* rp = A.rp + base;
        const int64_t* irp = A.irp + base;
        const int32_t my_src = lane < I.nsrc ? P.srcs[I.src_off + lane] : -1;

        if (threadIdx.x < 32 && my_src >= 0) {
            atomicOr(&M[4 * my_src + 0], lane_bit);
            sl0[(uint32_t)my_src << 5] = 1;
            atomicOr(&bm[my_src >> 5], 1u << (my_src & 31));
        }
        if (threadIdx.x == 0) {
            bflag[0] = 1;
            s_pos = 0; s_D = 0; s_maxpush = 0; s_nsteps = 0; s_err = 0;
        }
        __syncthreads();

        // ------------------------------------------------------------------ forward
        for (;;) {
            if (threadIdx.x == 0) {
                int D = s_D;
                while (D <= s_maxpush && bflag[D & 1] == 0) D++;
                s_D = D;
                s_done = (D > s_maxpush) || s_err;
                if (!s_done) {
                    bflag[D & 1] = 0;
                    if (s_nsteps >= W.cap_steps) {
                        s_err = 1; s_done = 1;
                    } else if (D > LV_MAX) {
                        s_err = 2; s_done = 1;
                    } else {
                        step_d[s_nsteps] = D;
                        step_beg[s_nsteps] = s_pos;
                        s_next = s_pos;
                    }
                }
            }
            __syncthreads();
            if (s_done) break;
            const int32_t D = s_D;
            const int cur = D % 3, prv = (D + 2) % 3, nxt = (D + 1) % 3;
            const int beg = s_next;
            {
                uint32_t* bmD = bm + (int64_t)(D & 1) * W.bm_words;
                const int nwords = (n + 31) >> 5;
                const int nwr = (nwords + 31) & ~31;
                for (int wi = threadIdx.x; wi < nwr; wi += LS_THREADS) {
                    uint32_t x = wi < nwords ? bmD[wi] : 0u;
                    if (x) bmD[wi] = 0u;
                    const int c = __popc(x);
                    const int incl = warp_incl_scan(c, lane);
                    const int tot = __shfl_sync(FULL, incl, 31);
                    int bpos = 0;
                    if (lane == 31 && tot) bpos = atomicAdd(&s_pos, tot);
                    bpos = __shfl_sync(FULL, bpos, 31);
                    if (tot && bpos + tot > W.cap_order) {
                        if (lane == 0) atomicExch(&s_err, 1);
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
            __syncthreads();
            if (threadIdx.x == 0) s_end = min(s_pos, (int)W.cap_order);
            __syncthreads();
            if (s_err) break;
            const int end = s_end;
            // arc ranges; the step's lanes join the reached set; the masks two levels back are
            // cleared so that they can collect the next level
            for (int e = beg + threadIdx.x; e < end; e += LS_THREADS) {
                const int32_t u = order[e].u;
                const int64_t a0 = __ldg(rp + u);
                order[e].a0 = a0;
                order[e].deg = (int32_t)(__ldg(rp + u + 1) - a0);
                M[4 * u + 3] |= M[4 * u + cur];
            }
            if (s_nsteps >= 2) {
                const int b2 = step_beg[s_nsteps - 2], e2 = step_beg[s_nsteps - 1];
                for (int e = b2 + threadIdx.x; e < e2; e += LS_THREADS) M[4 * order[e].u + nxt] = 0u;
            }
            __syncthreads();
            int e = fetch_entry(&s_next, lane);
            LsEnt ce = load_entry(order, e, end);
            while (e < end) {
                const int e2 = fetch_entry(&s_next, lane);
                const LsEnt ne = load_entry(order, e2, end);
                const int u = ce.u;
                const uint32_t m = M[4 * u + cur];
                if (m) {
                    const bool act = (m & lane_bit) != 0;
                    if (act) lv0[(uint32_t)u << 5] = (uint8_t)D;
                    bool ovf = false;
                    uint64_t acc = 0;
                    // pull sigma from the parents (level D-1), push the children (level D+1)
                    auto visit = [&](int64_t a0, int32_t deg, bool do_pull, bool do_push) {
                        for (int32_t c0 = 0; c0 < deg; c0 += 32) {
                            const int cnt = min(32, deg - c0);
                            const int32_t mv = lane < cnt ? __ldg((FUSED || do_push ? A.col : A.icol) + a0 + c0 + lane) : 0;
                            for (int j = 0; j < cnt; j += BFS_UNROLL) {
                                int32_t vv[BFS_UNROLL];
                                uint32_t pm[BFS_UNROLL], sm[BFS_UNROLL];
#pragma unroll
                                for (int k = 0; k < BFS_UNROLL; k++) vv[k] = __shfl_sync(FULL, mv, (j + k) & 31);
#pragma unroll
                                for (int k = 0; k < BFS_UNROLL; k++) {
                                    const bool ok = j + k < cnt;
                                    pm[k] = (ok && do_pull) ? M[4 * vv[k] + prv] : 0u;
                                    sm[k] = (ok && do_push) ? M[4 * vv[k] + 3] : ~0u;
                                }
                                if (do_pull && D > 0) {
                                    uint64_t sp[BFS_UNROLL];
#pragma unroll
                                    for (int k = 0; k < BFS_UNROLL; k++)
                                        sp[k] = (act && (pm[k] & lane_bit)) ? sl0[(uint32_t)vv[k] << 5] : 0ull;
#pragma unroll
                                    for (int k = 0; k < BFS_UNROLL; k++)
                                        if (sp[k]) acc = madd_ck(acc, sp[k], 1ull, ovf);
                                }
                                if (do_push) {
#pragma unroll
                                    for (int k = 0; k < BFS_UNROLL; k++) {
                                        const uint32_t q = m & ~sm[k];
                                        if (q && lane == k) {
                                            atomicOr(&M[4 * vv[k] + nxt], q);
                                            mark_bucket(P, bm, bflag, W.bm_words, vv[k], D + 1, &s_maxpush);
                                        }
                                    }
                                }
                            }
                        }
                    };
                    if (FUSED) {
                        visit(ce.a0, ce.deg, true, true);
                    } else {
                        if (D > 0) {
                            const int64_t i0 = __ldg(irp + u);
                            visit(i0, (int32_t)(__ldg(irp + u + 1) - i0), true, false);
                        }
                        visit(ce.a0, ce.deg, false, true);
                    }
                    if (act && D > 0) sl0[(uint32_t)u << 5] = acc;
                    if (__any_sync(FULL, ovf) && lane == 0) atomicOr(&P.flags[FLAG_SIGMA_OVF], 1u);
                }
                e = e2;
                ce = ne;
            }
            __syncthreads();
            if (threadIdx.x == 0) { s_nsteps++; s_D = D + 1; }
        }
        __syncthreads();
        const int nsteps = s_nsteps;
        const int olen = min(s_pos, (int)W.cap_order);
        if (s_err) {
            if (threadIdx.x == 0) atomicOr(&P.flags[s_err == 2 ? FLAG_LEVELS : FLAG_CAPACITY], 1u);
            for (int64_t i = threadIdx.x; i < 4 * (int64_t)n; i += LS_THREADS) M[i] = 0u;
            for (int64_t i = threadIdx.x; i < 32 * (int64_t)n; i += LS_THREADS) lv[i] = LV_NONE;
            for (int64_t i = threadIdx.x; i < 2 * W.bm_words; i += LS_THREADS) bm[i] = 0u;
            if (threadIdx.x < 2) bflag[threadIdx.x] = 0;
            __syncthreads();
            continue;
        }

        // ------------------------------------------------------------------ backward
        for (int st = nsteps - 1; st >= 0; st--) {
            if (threadIdx.x == 0) s_next = step_beg[st];
            __syncthreads();
            const int32_t D = step_d[st];
            const int end = (st + 1 < nsteps) ? step_beg[st + 1] : olen;
            int e = fetch_entry(&s_next, lane);
            LsEnt ce = load_entry(order, e, end);
            while (e < end) {
                const int e2 = fetch_entry(&s_next, lane);
                const LsEnt ne = load_entry(order, e2, end);
                const int u = ce.u;
                const bool act = lv0[(uint32_t)u << 5] == (uint8_t)D;
                if (__ballot_sync(FULL, act)) {
                    DT acc = (DT)0;
                    for (int32_t c0 = 0; c0 < ce.deg; c0 += 32) {
                        const int cnt = min(32, ce.deg - c0);
                        const int32_t mv = lane < cnt ? __ldg(A.col + ce.a0 + c0 + lane) : 0;
                        for (int j = 0; j < cnt; j += BFS_UNROLL) {
                            int32_t vv[BFS_UNROLL];
                            uint8_t lvv[BFS_UNROLL];
#pragma unroll
                            for (int k = 0; k < BFS_UNROLL; k++) vv[k] = __shfl_sync(FULL, mv, (j + k) & 31);
#pragma unroll
                            for (int k = 0; k < BFS_UNROLL; k++)
                                lvv[k] = j + k < cnt ? lv0[(uint32_t)vv[k] << 5] : LV_NONE;
                            DT cv[BFS_UNROLL];
#pragma unroll
                            for (int k = 0; k < BFS_UNROLL; k++)
                                cv[k] = (act && lvv[k] == (uint8_t)(D + 1)) ? cl0[(uint32_t)vv[k] << 5] : (DT)0;
#pragma unroll
                            for (int k = 0; k < BFS_UNROLL; k++) acc += cv[k];
                        }
                    }
                    double contrib = 0.0;
                    if (act) {
                        const DT sd = (DT)sl0[(uint32_t)u << 5];
                        const DT delta = sd * acc;
                        const DT is_t = P.in_s ? (DT)P.in_s[base + u] : (DT)1;
                        cl0[(uint32_t)u << 5] = (is_t + delta) / sd;
                        if (u != my_src) contrib = (double)delta;
                    }
                    const double tot = warp_sum(contrib);
                    if (lane == 0 && bcs && tot != 0.0) {
                        const int64_t ix = P.bc_map ? (int64_t)P.bc_map[base + u] : base + u;
                        atomicAdd(&bcs[ix], tot);
                    }
                }
                e = e2;
                ce = ne;
            }
            __syncthreads();
        }
        // restore the empty state on every touched node
        {
            const int warp = threadIdx.x >> 5;
            for (int e = warp; e < olen; e += LS_THREADS / 32) {
                const int32_t u = order[e].u;
                lv0[(uint32_t)u << 5] = LV_NONE;
                if (lane < 4) M[4 * u + lane] = 0u;
            }
        }
        __syncthreads();
    }
}

}  // namespace

void bfs_init_slots(const LsSlots& W, int slots, cudaStream_t st) {
    const int64_t tot = W.cap_n * LS_LANES * slots;
    if (tot <= 0) return;
    int64_t blocks = (tot + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    bfs_init_kernel<<<(unsigned)blocks, 256, 0, st>>>(W.d, W.cap_n, slots);
}

void bfs_launch(bool fp32_delta, bool fused, const LsArena& A, const LsParams& P, const LsSlots& W,
                const LsItem* items, int nitems, int slots, cudaStream_t st) {
    if (nitems <= 0 || slots <= 0 || P.mode != LS_BRANDES || P.nb != 2 || A.w || A.mu) return;
    if (fp32_delta) {
        if (fused) bfs_kernel<float, true><<<slots, LS_THREADS, 0, st>>>(A, P, W, items, nitems);
        else bfs_kernel<float, false><<<slots, LS_THREADS, 0, st>>>(A, P, W, items, nitems);
    } else {
        if (fused) bfs_kernel<double, true><<<slots, LS_THREADS, 0, st>>>(A, P, W, items, nitems);
        else bfs_kernel<double, false><<<slots, LS_THREADS, 0, st>>>(A, P, W, items, nitems);
    }
}

}  // namespace bcpp
