// Node partition by label propagation, for Brandes++ callers without a partition of their own.
//
// The paper takes its partitions from external tools (Sec. 6: Modularity, Graclus, Metis) and
// Brandes++ is exact for every partition (Sec. 4), so any partition is valid input; this one is
// the label propagation of Raghavan, Albert and Kumara (2007) made deterministic:
//   - labels start as the node ids;
//   - half-step t updates the nodes v with v mod 2 == t mod 2 from the labels of half-step t-1
//     (double buffered): v takes the label carried by most of its neighbours (in- and out-arcs
//     of a directed graph both count), keeps its own label when that one is among the most
//     frequent, and otherwise takes the smallest of the most frequent labels; a node without
//     neighbours keeps its label;
//   - it stops after a round of two half-steps without a change, or after max_rounds rounds;
//   - the labels in use are numbered 0..k-1 in increasing order.
#include "partition.cuh"
#include "prims.cuh"

namespace bcpp {

namespace {

// One half-step.  A warp per node: neighbour labels 32 at a time; the count of a lane's label
// over all neighbours is __match_any_sync within a chunk, and a broadcast compare across the
// other chunks for nodes with more than 32 neighbours.
__global__ void lp_step_kernel(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const int64_t* __restrict__ irp, const int32_t* __restrict__ icol,
                               const int32_t* __restrict__ lin, int32_t* __restrict__ lout, int parity,
                               unsigned int* changes) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        const int32_t cur = lin[v];
        if ((v & 1) != parity) {
            if (lane == 0) lout[v] = cur;
            continue;
        }
        const int64_t a0 = rp[v], d0 = rp[v + 1] - a0;
        const int64_t b0 = irp ? irp[v] : 0, d1 = irp ? irp[v + 1] - b0 : 0;
        const int64_t deg = d0 + d1;
        if (deg == 0) {
            if (lane == 0) lout[v] = cur;
            continue;
        }
        // neighbour i (0 <= i < deg): out-arc i, then in-arc i - d0
        auto nlab = [&](int64_t i) -> int32_t {
            const int32_t u = i < d0 ? col[a0 + i] : icol[b0 + (i - d0)];
            return lin[u];
        };
        int32_t best_cnt = 0, best_lab = INT32_MAX, cur_cnt = 0;
        for (int64_t c0 = 0; c0 < deg; c0 += 32) {
            const bool valid = c0 + lane < deg;
            const int32_t lab = valid ? nlab(c0 + lane) : -1;
            cur_cnt += __popc(__ballot_sync(FULL, valid && lab == cur));
            int32_t cnt;
            if (deg <= 32) {
                cnt = __popc(__match_any_sync(FULL, lab));
            } else {
                cnt = 0;
                for (int64_t c1 = 0; c1 < deg; c1 += 32) {
                    const int32_t lab1 = c1 + lane < deg ? nlab(c1 + lane) : -2;
                    for (int j = 0; j < 32; j++) cnt += __shfl_sync(FULL, lab1, j) == lab;
                }
            }
            if (!valid) cnt = 0;
            // chunk winner: largest count, then smallest label
            int32_t c = cnt, l = valid ? lab : INT32_MAX;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int32_t c2 = __shfl_xor_sync(FULL, c, o), l2 = __shfl_xor_sync(FULL, l, o);
                if (c2 > c || (c2 == c && l2 < l)) { c = c2; l = l2; }
            }
            if (c > best_cnt || (c == best_cnt && l < best_lab)) { best_cnt = c; best_lab = l; }
        }
        const int32_t nl = cur_cnt == best_cnt ? cur : best_lab;
        if (lane == 0) {
            lout[v] = nl;
            if (nl != cur) atomicAdd(changes, 1u);
        }
    }
}

__global__ void lp_init_kernel(int32_t n, int32_t* lab, int32_t* used) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        lab[v] = (int32_t)v;
        used[v] = 0;
    }
}
__global__ void lp_mark_kernel(int32_t n, const int32_t* lab, int32_t* used) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        used[lab[v]] = 1;
}
__global__ void lp_number_kernel(int32_t n, const int32_t* lab, const int64_t* rank, int32_t* part) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        part[v] = (int32_t)rank[lab[v]];
}

inline unsigned blocks_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 16384);
}

}  // namespace

void lp_init(int32_t n, int32_t* lab, int32_t* used, cudaStream_t st) {
    if (n > 0) lp_init_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, lab, used);
}
void lp_step(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* irp, const int32_t* icol,
             const int32_t* lin, int32_t* lout, int parity, unsigned int* changes, cudaStream_t st) {
    if (n > 0) lp_step_kernel<<<blocks_for((int64_t)n * 32, 256), 256, 0, st>>>(n, rp, col, irp, icol, lin, lout,
                                                                                parity, changes);
}
void lp_mark(int32_t n, const int32_t* lab, int32_t* used, cudaStream_t st) {
    if (n > 0) lp_mark_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, lab, used);
}
void lp_number(int32_t n, const int32_t* lab, const int64_t* rank, int32_t* part, cudaStream_t st) {
    if (n > 0) lp_number_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, lab, rank, part);
}

}  // namespace bcpp
