// Exclusive scan (three passes: tile sums, scan of tile sums, tile scans) and a stable LSD
// radix sort (8-bit digits; per-tile histograms, one scan, warp-match ranking for the
// stable scatter).  Both run on the caller's stream with caller-provided scratch.
#include "prims.cuh"

namespace bcpp {

namespace {
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename TI>
__global__ void scan_tile_sums(const TI* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
    __shared__ int64_t red[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t acc = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t idx = base + i;
        if (idx < n) acc += (int64_t)in[idx];
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; w++) t += red[w];
        sums[blockIdx.x] = t;
    }
}

// single block: exclusive scan of sums[0..nb) in place, total to sums[nb]
__global__ void scan_sums(int64_t* sums, int64_t nb) {
    __shared__ int64_t wtot[SCAN_THREADS / 32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c0 = 0; c0 < nb; c0 += SCAN_THREADS) {
        int64_t idx = c0 + threadIdx.x;
        int64_t x = idx < nb ? sums[idx] : 0;
        int64_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wtot[warp] = incl;
        __syncthreads();
        int64_t wpre = 0, tot = 0;
        for (int w = 0; w < SCAN_THREADS / 32; w++) {
            if (w < warp) wpre += wtot[w];
            tot += wtot[w];
        }
        if (idx < nb) sums[idx] = carry + wpre + incl - x;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

template <typename TI>
__global__ void scan_tiles(const TI* in, int64_t* out, int64_t n, const int64_t* __restrict__ sums,
                           int64_t* total_dev, int64_t nb) {
    __shared__ int64_t wtot[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t local = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + i;
        v[i] = idx < n ? (int64_t)in[idx] : 0;
        local += v[i];
    }
    int64_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    int64_t wpre = 0;
    for (int w = 0; w < warp; w++) wpre += wtot[w];
    int64_t run = sums[blockIdx.x] + wpre + incl - local;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && total_dev) *total_dev = sums[nb];
}
}  // namespace

int64_t scan_tmp_elems(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 2; }

template <typename TI>
void exclusive_scan(const TI* in, int64_t* out, int64_t n, int64_t* total_dev, int64_t* tmp, cudaStream_t st,
                    int64_t& launches) {
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 0) {
        if (total_dev) cudaMemsetAsync(total_dev, 0, sizeof(int64_t), st);
        return;
    }
    scan_tile_sums<TI><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, tmp);
    scan_sums<<<1, SCAN_THREADS, 0, st>>>(tmp, nb);
    scan_tiles<TI><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, tmp, total_dev, nb);
    launches += 3;
}

template void exclusive_scan<int32_t>(const int32_t*, int64_t*, int64_t, int64_t*, int64_t*, cudaStream_t, int64_t&);
template void exclusive_scan<int64_t>(const int64_t*, int64_t*, int64_t, int64_t*, int64_t*, cudaStream_t, int64_t&);
template void exclusive_scan<uint32_t>(const uint32_t*, int64_t*, int64_t, int64_t*, int64_t*, cudaStream_t, int64_t&);

// ----------------------------------------------------------------------------- radix sort
namespace {
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_CHUNKS = 16;
constexpr int RS_TILE = RS_THREADS * RS_CHUNKS;

__global__ void rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int64_t* __restrict__ hist,
                        int64_t nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        int64_t idx = base + i;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void rs_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                           uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
                           const int64_t* __restrict__ offs, int64_t nblocks) {
    __shared__ int64_t base[256];
    __shared__ uint32_t wcnt[RS_WARPS][257];
    __shared__ uint32_t chunk_tot[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    const int64_t tile = (int64_t)blockIdx.x * RS_TILE;
    for (int c = 0; c < RS_CHUNKS; c++) {
        for (int i = threadIdx.x; i < RS_WARPS * 257; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        int64_t idx = tile + (int64_t)c * RS_THREADS + threadIdx.x;
        bool valid = idx < n;
        uint64_t key = valid ? kin[idx] : 0;
        uint32_t val = valid ? vin[idx] : 0;
        int digit = valid ? (int)((key >> shift) & 255) : 256;
        unsigned peers = __match_any_sync(FULL, digit);
        int rank = __popc(peers & ((1u << lane) - 1u));
        if (rank == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {
            int t = threadIdx.x;   // one thread per digit
            uint32_t run = 0;
            for (int w = 0; w < RS_WARPS; w++) {
                uint32_t x = wcnt[w][t];
                wcnt[w][t] = run;
                run += x;
            }
            chunk_tot[t] = run;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = base[digit] + wcnt[warp][digit] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        base[threadIdx.x] += chunk_tot[threadIdx.x];
        __syncthreads();
    }
}
}  // namespace

int64_t radix_hist_elems(int64_t n) { return 256 * ((n + RS_TILE - 1) / RS_TILE) + 1; }

void radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* kbuf, uint32_t* vbuf, int64_t n, int bits,
                      int64_t* hist, int64_t* scan_tmp, cudaStream_t st, int64_t& launches) {
    if (n <= 1 || bits <= 0) return;
    int64_t nblocks = (n + RS_TILE - 1) / RS_TILE;
    int passes = (bits + 7) / 8;
    uint64_t* ka = keys; uint32_t* va = vals;
    uint64_t* kb = kbuf; uint32_t* vb = vbuf;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        rs_hist<<<(unsigned)nblocks, RS_THREADS, 0, st>>>(ka, n, shift, hist, nblocks);
        exclusive_scan<int64_t>(hist, hist, 256 * nblocks, nullptr, scan_tmp, st, launches);
        rs_scatter<<<(unsigned)nblocks, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, shift, hist, nblocks);
        launches += 2;
        uint64_t* tk = ka; ka = kb; kb = tk;
        uint32_t* tv = va; va = vb; vb = tv;
    }
    if (ka != keys) {
        cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    }
}

}  // namespace bcpp
