// C-ABI entry points of libbcpp (declared in include/bcpp.h) and the host orchestration of
// plain Brandes, Brandes++ (Alg. 1: Build_SK -> Brandes_SK -> Centrality), batched graphs and
// the inspection calls.  The context keeps a caching pool of device blocks so that repeated
// calls of the same size do not allocate.
#include <algorithm>
#include <cstring>
#include <memory>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "csr.cuh"
#include "lockstep.cuh"
#include "partition.cuh"
#include "prims.cuh"
#include "skeleton.cuh"

using namespace bcpp;

struct PoolBlock {
    void* p;
    size_t bytes;
    bool used;
};

struct bcpp_ctx {
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    std::vector<PoolBlock> pool;
    uint32_t* flags = nullptr;       // device [FLAG_COUNT], followed by the two phase timers
    uint32_t* hflags = nullptr;      // pinned host copy (same layout)
    unsigned long long* phase = nullptr;    // device [2]: forward / backward batch time (ns)
    int64_t launches = 0;
    int order_factor = 8;            // settled-entry capacity per node of a batch (retry: worst case)
    cudaEvent_t ev[8] = {};

    void* acquire(size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        int best = -1;
        for (size_t i = 0; i < pool.size(); i++) {
            const PoolBlock& b = pool[i];
            if (!b.used && b.bytes >= bytes && b.bytes <= 2 * bytes + (64u << 20) &&
                (best < 0 || b.bytes < pool[best].bytes))
                best = (int)i;
        }
        if (best >= 0) {
            pool[best].used = true;
            return pool[best].p;
        }
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            trim();
            if (cudaMalloc(&p, bytes) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
        }
        pool.push_back({p, bytes, true});
        return p;
    }
    void release(void* p) {
        if (!p) return;
        for (auto& b : pool)
            if (b.p == p) { b.used = false; return; }
    }
    void trim() {
        cudaStreamSynchronize(stream);
        std::vector<PoolBlock> keep;
        for (auto& b : pool) {
            if (b.used) keep.push_back(b);
            else cudaFree(b.p);
        }
        pool.swap(keep);
    }
    int64_t held() const {
        int64_t t = 0;
        for (auto& b : pool) t += (int64_t)b.bytes;
        return t;
    }
};

namespace {

// RAII device buffer from the context pool
template <typename T>
struct DBuf {
    bcpp_ctx* c = nullptr;
    T* p = nullptr;
    int64_t n = 0;
    DBuf() = default;
    DBuf(bcpp_ctx* ctx, int64_t count) { alloc(ctx, count); }
    bool alloc(bcpp_ctx* ctx, int64_t count) {
        free();
        c = ctx;
        n = count;
        p = (T*)ctx->acquire((size_t)std::max<int64_t>(count, 1) * sizeof(T));
        return p != nullptr;
    }
    void free() {
        if (c && p) c->release(p);
        p = nullptr;
    }
    ~DBuf() { free(); }
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    explicit operator bool() const { return p != nullptr; }
};

struct Status {
    int code = BCPP_OK;
};

#define CK_CUDA(x)                                   \
    do {                                             \
        cudaError_t e__ = (x);                       \
        if (e__ != cudaSuccess) {                    \
            cudaGetLastError();                      \
            return BCPP_ECUDA;                       \
        }                                            \
    } while (0)
#define CK_ALLOC(buf)                                \
    do {                                             \
        if (!(buf)) return BCPP_ENOMEM;              \
    } while (0)
#define CK_RC(x)                                     \
    do {                                             \
        int r__ = (x);                               \
        if (r__ != BCPP_OK) return r__;              \
    } while (0)

// status flags and the two 64-bit phase timers behind them: one allocation, one copy
constexpr size_t FLAG_BYTES = FLAG_COUNT * sizeof(uint32_t) + 2 * sizeof(unsigned long long);

int sync_flags(bcpp_ctx* c) {
    CK_CUDA(cudaMemcpyAsync(c->hflags, c->flags, FLAG_BYTES, cudaMemcpyDeviceToHost, c->stream));
    CK_CUDA(cudaStreamSynchronize(c->stream));
    CK_CUDA(cudaGetLastError());
    return BCPP_OK;
}

int reset_flags(bcpp_ctx* c) {
    CK_CUDA(cudaMemsetAsync(c->flags, 0, FLAG_BYTES, c->stream));
    return BCPP_OK;
}

template <typename T>
int to_host(bcpp_ctx* c, T* dst, const T* src, int64_t count) {
    if (count <= 0) return BCPP_OK;
    CK_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
    CK_CUDA(cudaStreamSynchronize(c->stream));
    return BCPP_OK;
}

template <typename T>
int to_dev(bcpp_ctx* c, T* dst, const T* src, int64_t count) {
    if (count <= 0) return BCPP_OK;
    CK_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    CK_CUDA(cudaStreamSynchronize(c->stream));
    return BCPP_OK;
}

__global__ void iota_kernel(int32_t* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}
void iota(int32_t* p, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    iota_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, st>>>(p, n);
}

// highest-degree node (smallest id on ties): max of (degree << 32 | ~id)
__global__ void hub_kernel(const int64_t* rp, int32_t n, unsigned long long* best) {
    unsigned long long b = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = ((unsigned long long)(rp[v + 1] - rp[v]) << 32) | (0xffffffffu - (uint32_t)v);
        b = key > b ? key : b;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(FULL, b, o);
        b = x > b ? x : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(best, b);
}

// keys[i] = key[S[i]] (a per-node sort key), vals[i] = S[i]
__global__ void level_keys_kernel(const int32_t* S, int64_t ns, const int32_t* level, uint64_t* keys, uint32_t* vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
        keys[i] = (uint64_t)(uint32_t)level[S[i]];
        vals[i] = (uint32_t)S[i];
    }
}
__global__ void part_keys_kernel(const uint32_t* vals, int64_t ns, const int32_t* part, uint64_t* keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (uint64_t)part[vals[i]];
}

__global__ void or_flags_kernel(const uint8_t* a, const uint8_t* b, int32_t n, int32_t* f) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        f[i] = (a[i] | b[i]) ? 1 : 0;
}
__global__ void compact_kernel(const int32_t* f, const int64_t* pos, int32_t n, int32_t* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (f[i]) out[pos[i]] = (int32_t)i;
}
__global__ void part_flag_kernel(const int32_t* part, int32_t n, int32_t j, uint8_t* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = part[i] == j ? 1 : 0;
}
// (sum, comp) += x, Neumaier, element-wise
// Brandes++All grouping: key = part (checked against [0, k)), value = node, and the part sizes
__global__ void group_by_part_kernel(const int32_t* part, int32_t n, int32_t k, uint64_t* keys, uint32_t* vals,
                                     int64_t* cnt, uint32_t* flags) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = part[v];
        if (p < 0 || p >= k) {
            flag_invalid(flags, WHY_PART);
            keys[v] = 0;
        } else {
            keys[v] = (uint64_t)p;
            atomicAdd(reinterpret_cast<unsigned long long*>(cnt + p), 1ull);
        }
        vals[v] = (uint32_t)v;
    }
}

// largest finite value of a distance table (DINF = unreachable) into *out
__global__ void table_max_kernel(const int32_t* t, int64_t n, unsigned* out) {
    unsigned m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = t[i];
        if (v != DINF && (unsigned)v > m) m = (unsigned)v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(FULL, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

__global__ void accumulate_kernel(const double* x, int32_t n, double* sum, double* comp) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = sum[i], c = comp[i];
        neumaier_add(s, c, x[i]);
        sum[i] = s;
        comp[i] = c;
    }
}
__global__ void finish_kernel(const double* sum, const double* comp, int32_t n, double scale, double* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (sum[i] + comp[i]) * scale;
}

__global__ void i64_from_i32_kernel(const int32_t* in, int64_t* out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

// sources [s0, s1) of shard r of R: [ns*r/R, ns*(r+1)/R) (bcpp_shard_bounds)
void shard_range(int64_t ns, int64_t r, int64_t R, int64_t& s0, int64_t& s1) {
    s0 = 0;
    s1 = ns;
    if (R > 1) {
        s0 = ns * r / R;
        s1 = ns * (r + 1) / R;
    }
}

// sources [s0, s1) of this call's shard (an out-of-range shard index is clamped)
void shard_sources(const bcpp_opts& o, int64_t ns, int64_t& s0, int64_t& s1) {
    const int64_t r = std::max(0, std::min(o.shard_index, o.shard_count - 1));
    shard_range(ns, r, o.shard_count, s0, s1);
}

// batches of `lanes` consecutive sources of [s0, s1) of graph g
std::vector<LsItem> make_items(int32_t g, int64_t s0, int64_t s1, int lanes) {
    std::vector<LsItem> v;
    for (int64_t b = s0; b < s1; b += lanes)
        v.push_back(LsItem{g, (int32_t)b, (int32_t)std::min<int64_t>(lanes, s1 - b), 0});
    return v;
}

// sources per lane: opts.batch = 64 selects two per lane (rows of 64); the default is one
// (measured on GB300: rows of 64 were slower in FP64 and within 3% in FP32)
int choose_spl(const bcpp_ctx*, int64_t, const bcpp_opts& o) {
    return o.batch == 64 ? 2 : 1;
}

int bits_for(uint64_t maxval) {
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) b++;
    return b;
}

bcpp_opts opts_or_default(const bcpp_opts* o) {
    bcpp_opts d;
    bcpp_default_opts(&d);
    return o ? *o : d;
}

int check_graph_struct(const bcpp_graph* g) {
    if (!g || g->n < 0 || g->num_arcs < 0) return BCPP_EINVAL;
    if (!g->row_ptr) return BCPP_EINVAL;
    if (g->num_arcs > 0 && !g->col) return BCPP_EINVAL;
    return BCPP_OK;
}

// Validate a CSR; on success *wmax_out = max weight (1 for unit weights).
int validate_csr(bcpp_ctx* c, const bcpp_graph* g, uint64_t* wmax_out, const int64_t* node_off = nullptr,
                 int32_t ngraphs = 0) {
    DBuf<unsigned long long> wmax(c, 1);
    CK_ALLOC(wmax);
    CK_CUDA(cudaMemsetAsync(wmax.p, 0, sizeof(unsigned long long), c->stream));
    csr_check(g->n, g->num_arcs, g->row_ptr, g->col, g->w, g->directed, c->flags, wmax.p, c->stream, node_off,
              ngraphs);
    c->launches++;
    unsigned long long hw = 0;
    CK_RC(to_host(c, &hw, (const unsigned long long*)wmax.p, 1));
    CK_RC(sync_flags(c));
    if (c->hflags[FLAG_INVALID]) return BCPP_EINVAL;
    if (hw == 0) hw = 1;
    if (g->n > 1 && (uint64_t)hw * (uint64_t)(g->n - 1) >= (1ull << 31)) return BCPP_EINVAL;
    if (hw > (1ull << 20)) return BCPP_EINVAL;   // bucket array bound (max weight <= 2^20)
    *wmax_out = hw;
    return BCPP_OK;
}

// Per-slot lockstep workspace.
struct SlotWs {
    DBuf<int32_t> d;
    DBuf<uint64_t> sg;
    DBuf<char> dl;
    DBuf<LsEnt> order;
    DBuf<int32_t> step_d, step_beg, hdr;
    DBuf<uint32_t> bm;
    DBuf<uint8_t> bflag;
    DBuf<double> bcs, bcc, bcb;
    DBuf<int> counter;
    LsSlots W{};
    int slots = 0, nb = 0;
    int row_states = 0;         // distance / count / dependency row sets (one per slot, or per item)
    int sum_slots = 0;          // partial-sum sets (one per slot, or per item)
    int64_t rows = 0;
    bool narrow = false;        // one-byte distance rows (0xff = unreached)
};

// One-byte distance rows for unit-weight Brandes passes, except on the worst-case retry (which
// also serves batches deeper than those rows reach).
bool use_narrow(const bcpp_ctx* c, bool weighted) { return !weighted && c->order_factor < 64; }

int64_t order_capacity(int64_t cap_n, int order_factor, int spl) {
    return (int64_t)std::min(order_factor, 32 * spl) * cap_n + 1024;
}

// Settled entries per node of a batch to provide for.  With unit weights a node is settled
// at few distinct distances per batch of 32 sources (2 to 3 on the graphs of this project),
// so the list holds 8 per node and a batch that outgrows it makes the call retry with the
// worst case (one per node and source).  With integer weights the distances spread (about
// 15 per node for weights in [1,16]), so weighted runs take the worst case at once.
int entry_factor(const bcpp_ctx* c, bool weighted, int spl) {
    return weighted ? 32 * spl : c->order_factor;
}

// Non-empty steps a batch can record.  Every recorded step holds at least one settled entry
// (a bucket is flagged only when a head is marked in it, and with weights below nb the window
// of tentative distances maps each bucket to a single distance), so the order capacity bounds
// them; so does the number of distinct distances, 0 .. (nb - 1)(n - 1).
int32_t step_capacity(int64_t cap_n, int nb, int64_t cap_order) {
    const int64_t dist_bound = (int64_t)(nb - 1) * std::max<int64_t>(cap_n - 1, 0) + 2;
    return (int32_t)std::min<int64_t>(cap_order, dist_bound);
}

int64_t slot_bytes(int64_t cap_n, int nb, bool fp32, int order_factor = 8, int spl = 1) {
    const int64_t cap_order = order_capacity(cap_n, order_factor, spl);
    const int64_t bm_words = (cap_n + 31) / 32;
    return cap_n * 32 * spl * (4 + 8 + (fp32 ? 4 : 8)) + cap_order * (int64_t)sizeof(LsEnt) +
           2 * (int64_t)step_capacity(cap_n, nb, cap_order) * 4 + (int64_t)nb * bm_words * 4 + nb;
}

// CTAs per batch: with fewer batches than resident CTAs (two per SM), 2 or 4 CTAs of a
// thread-block cluster share each batch so that every SM has work.
// (Measured on GB300: with 63 or 128 batches, 4-CTA clusters beat 2-CTA ones.)
int choose_cluster(const bcpp_ctx* c, int nitems, const bcpp_opts& o) {
    if (o.cluster == 1 || o.cluster == 2 || o.cluster == 4) return o.cluster;
    const int cps = o.ctas_per_sm > 0 ? o.ctas_per_sm : LS_MIN_CTAS;
    const int64_t resident = (int64_t)cps * c->num_sms;
    if (2 * (int64_t)nitems <= resident) return 4;
    if ((int64_t)nitems < resident) return 2;
    return 1;
}

// Batches in flight at most: resident CTAs / CTAs per batch.
int64_t slot_capacity(const bcpp_ctx* c, const bcpp_opts& o, int cl) {
    const int cps = o.ctas_per_sm > 0 ? o.ctas_per_sm : LS_MIN_CTAS;
    return std::max<int64_t>(1, (int64_t)cps * c->num_sms / cl);
}

// Source-batch width when 32-source batches would leave slots idle: a call with fewer batches
// than slots (one round) spreads its sources over all of them, since a batch costs about in
// proportion to its active lanes (entries with few active lanes are visited by (arc, source)
// pairs) and otherwise the idle slots' SMs wait.  Measured on one box: 200 sources on 76 slots
// (`planted_200k` plain) 107 -> 46 ms, 512 sources 34 -> 22 ms, 2,000 sources 198 -> 179 ms.
// Not for two or more rounds: 4,096 sources as 152 batches of 27 instead of 128 of 32 on 76
// slots was slower (724 -> 933 ms; narrower batches of well-ordered sources save little per
// batch, and both rounds then run full).
#ifndef BCPP_BALANCE_MAX_ROUNDS
#define BCPP_BALANCE_MAX_ROUNDS 1
#endif
int balanced_width(int64_t ns, int64_t slots_cap, int lanes) {
    if (ns <= 0 || slots_cap <= 0) return lanes;
    const int64_t rounds = (ns + (int64_t)lanes * slots_cap - 1) / ((int64_t)lanes * slots_cap);
    if (rounds > BCPP_BALANCE_MAX_ROUNDS) return lanes;
    const int64_t b = (ns + rounds * slots_cap - 1) / (rounds * slots_cap);
    return (int)std::max<int64_t>(1, std::min<int64_t>(lanes, b));
}

// Choose how many slots (batches in flight, cl CTAs each) to run, within the memory budget.
int choose_slots(bcpp_ctx* c, int nitems, int ctas_per_sm, int64_t per_slot, int64_t per_slot_bc, int cl = 1) {
    int cps = ctas_per_sm > 0 ? ctas_per_sm : LS_MIN_CTAS;
    int slots = std::min<int64_t>(nitems, std::max<int64_t>(1, (int64_t)cps * c->num_sms / cl));
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    int64_t reusable = 0;
    for (auto& b : c->pool)
        if (!b.used) reusable += (int64_t)b.bytes;
    int64_t budget = (int64_t)((double)(fr + reusable) * 0.80);
    int64_t each = per_slot + per_slot_bc;
    if (each > 0) slots = (int)std::min<int64_t>(slots, std::max<int64_t>(1, budget / each));
    return std::max(1, slots);
}

// Initial slot state: distances unreached, bucket bitmaps and headers empty, partial sums 0,
// batch counter 0.  Device work only (no host synchronization), so it can be captured.
int init_slots(bcpp_ctx* c, SlotWs& S) {
    const LsSlots& W = S.W;
    if (W.cap_bc > 0) {
        CK_CUDA(cudaMemsetAsync(S.bcs.p, 0, (size_t)S.sum_slots * W.cap_bc * sizeof(double), c->stream));
        CK_CUDA(cudaMemsetAsync(S.bcc.p, 0, (size_t)S.sum_slots * W.cap_bc * sizeof(double), c->stream));
        CK_CUDA(cudaMemsetAsync(S.bcb.p, 0, (size_t)S.sum_slots * W.cap_bc * sizeof(double), c->stream));
    }
    fill_i32(S.d.p, S.narrow ? -1 : DINF, (int64_t)S.row_states * S.rows * 32, c->stream);
    c->launches++;
    CK_CUDA(cudaMemsetAsync(S.bm.p, 0, (size_t)S.slots * S.nb * W.bm_words * sizeof(uint32_t), c->stream));
    CK_CUDA(cudaMemsetAsync(S.bflag.p, 0, (size_t)S.slots * S.nb, c->stream));
    CK_CUDA(cudaMemsetAsync(S.hdr.p, 0, (size_t)S.slots * 4 * sizeof(int32_t), c->stream));
    CK_CUDA(cudaMemsetAsync(S.counter.p, 0, sizeof(int), c->stream));
    return BCPP_OK;
}

// row_states / sum_slots: row sets and partial-sum sets when they differ from the slot count
// (Brandes_SK with one row set per batch); 0 = one per slot.
int alloc_slots(bcpp_ctx* c, SlotWs& S, int slots, int64_t cap_n, int nb, bool fp32, int64_t cap_bc, int spl,
                int factor, bool init = true, int row_states = 0, int sum_slots = 0) {
    if (cap_n >= (1 << 25)) return BCPP_EINVAL;   // 32-bit row offsets inside a slot
    const int64_t cap_order = order_capacity(cap_n, factor, spl);
    const int64_t rows = cap_n * spl;              // rows of 32 values
    const int32_t cap_steps = step_capacity(cap_n, nb, cap_order);
    const int64_t bm_words = (cap_n + 31) / 32;
    if (row_states <= 0) row_states = slots;
    if (sum_slots <= 0) sum_slots = slots;
    CK_ALLOC(S.d.alloc(c, (int64_t)row_states * rows * 32));
    CK_ALLOC(S.sg.alloc(c, (int64_t)row_states * rows * 32));
    CK_ALLOC(S.dl.alloc(c, (int64_t)row_states * rows * 32 * (fp32 ? 4 : 8)));
    CK_ALLOC(S.order.alloc(c, (int64_t)slots * cap_order));
    CK_ALLOC(S.step_d.alloc(c, (int64_t)slots * cap_steps));
    CK_ALLOC(S.step_beg.alloc(c, (int64_t)slots * cap_steps));
    CK_ALLOC(S.hdr.alloc(c, (int64_t)slots * 4));
    CK_ALLOC(S.bm.alloc(c, (int64_t)slots * nb * bm_words));
    CK_ALLOC(S.bflag.alloc(c, (int64_t)slots * nb));
    CK_ALLOC(S.counter.alloc(c, 1));
    if (cap_bc > 0) {
        CK_ALLOC(S.bcs.alloc(c, (int64_t)sum_slots * cap_bc));
        CK_ALLOC(S.bcc.alloc(c, (int64_t)sum_slots * cap_bc));
        CK_ALLOC(S.bcb.alloc(c, (int64_t)sum_slots * cap_bc));
    }
    S.slots = slots;
    S.row_states = row_states;
    S.sum_slots = sum_slots;
    S.nb = nb;
    S.rows = rows;
    LsSlots& W = S.W;
    W.d = S.d.p; W.sg = S.sg.p; W.dl = S.dl.p; W.cap_n = cap_n;
    W.order = S.order.p; W.cap_order = cap_order;
    W.step_d = S.step_d.p; W.step_beg = S.step_beg.p; W.cap_steps = cap_steps;
    W.bm = S.bm.p; W.bm_words = bm_words; W.bflag = S.bflag.p;
    W.bc_sum = cap_bc > 0 ? S.bcs.p : nullptr;
    W.bc_cmp = cap_bc > 0 ? S.bcc.p : nullptr;
    W.bc_bat = cap_bc > 0 ? S.bcb.p : nullptr;
    W.cap_bc = cap_bc;
    W.hdr = S.hdr.p;
    return init ? init_slots(c, S) : BCPP_OK;
}

// Accumulated device time of [start, stop) intervals on the context's stream.  A lazy timer
// does not wait at stop: it keeps each interval's events and adds them up in resolve(), so the
// host can go on queueing work.
struct Timer {
    bcpp_ctx* c;
    cudaEvent_t a, b;
    float acc = 0.f;
    bool lazy = false;
    cudaEvent_t la = nullptr;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> iv;
    explicit Timer(bcpp_ctx* ctx, bool lazy_ = false) : c(ctx), lazy(lazy_) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        resolve();
        if (la) cudaEventDestroy(la);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
    void start() {
        if (lazy) {
            if (!la) cudaEventCreate(&la);
            cudaEventRecord(la, c->stream);
            return;
        }
        cudaEventRecord(a, c->stream);
    }
    void stop() {
        if (lazy) {
            cudaEvent_t e = nullptr;
            if (!la || cudaEventCreate(&e) != cudaSuccess) return;
            cudaEventRecord(e, c->stream);
            iv.push_back({la, e});
            la = nullptr;
            return;
        }
        cudaEventRecord(b, c->stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        acc += ms;
    }
    float resolve() {
        for (auto& x : iv) {
            float ms = 0.f;
            if (cudaEventSynchronize(x.second) == cudaSuccess && cudaEventElapsedTime(&ms, x.first, x.second) == cudaSuccess)
                acc += ms;
            cudaEventDestroy(x.first);
            cudaEventDestroy(x.second);
        }
        iv.clear();
        cudaGetLastError();
        return acc;
    }
};

int finish_status(bcpp_ctx* c, bcpp_stats* st) {
    CK_RC(sync_flags(c));
    if (st) {
        st->sigma_overflow = c->hflags[FLAG_SIGMA_OVF] ? 1u : 0u;
        const unsigned long long* hp = reinterpret_cast<const unsigned long long*>(c->hflags + FLAG_COUNT);
        st->ms_batch_forward = (float)(hp[0] * 1e-6);
        st->ms_batch_backward = (float)(hp[1] * 1e-6);
    }
    if (c->hflags[FLAG_INVALID]) return BCPP_EINVAL;
    if (c->hflags[FLAG_CAPACITY]) return BCPP_ECAPACITY;
    if (c->hflags[FLAG_SIGMA_OVF]) return BCPP_EOVERFLOW_SIGMA;
    return BCPP_OK;
}

// in-CSR (transpose) of a graph with uint32 weights
struct InCsr {
    DBuf<int64_t> rp;
    DBuf<int32_t> col;
    DBuf<uint32_t> w;
    DBuf<int64_t> cnt, tmp;
};
int in_csr_alloc(bcpp_ctx* c, const bcpp_graph* g, InCsr& T) {
    const int32_t n = g->n;
    CK_ALLOC(T.rp.alloc(c, (int64_t)n + 1));
    CK_ALLOC(T.col.alloc(c, g->num_arcs));
    if (g->w) CK_ALLOC(T.w.alloc(c, g->num_arcs));
    CK_ALLOC(T.cnt.alloc(c, (int64_t)n + 1));
    CK_ALLOC(T.tmp.alloc(c, scan_tmp_elems((int64_t)n + 1)));
    return BCPP_OK;
}
int in_csr_emit(bcpp_ctx* c, const bcpp_graph* g, InCsr& T) {
    const int32_t n = g->n;
    CK_CUDA(cudaMemsetAsync(T.cnt.p, 0, ((size_t)n + 1) * sizeof(int64_t), c->stream));
    csr_transpose_count(n, g->row_ptr, g->col, T.cnt.p, c->stream);
    exclusive_scan<int64_t>(T.cnt.p, T.rp.p, (int64_t)n + 1, nullptr, T.tmp.p, c->stream, c->launches);
    CK_CUDA(cudaMemcpyAsync(T.cnt.p, T.rp.p, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, c->stream));
    csr_transpose_fill(n, g->row_ptr, g->col, g->w, T.cnt.p, T.col.p, g->w ? T.w.p : nullptr, c->stream);
    c->launches += 2;
    CK_CUDA(cudaGetLastError());
    return BCPP_OK;
}
int build_in_csr(bcpp_ctx* c, const bcpp_graph* g, InCsr& T) {
    CK_RC(in_csr_alloc(c, g, T));
    return in_csr_emit(c, g, T);
}

// Order the targets so that every batch holds sources close to each other: by position in the
// breadth-first discovery order from the highest-degree node (level by level; within a level
// by the position of the earliest-placed parent, then by node id), then, when a partition is
// given, stably by part.  Sources discovered from the same parent are at distance <= 2 from
// each other, so the nodes of the graph see few distinct distances per batch and a batch
// settles fewer (node, step) entries.  Only the batching order changes, not the result.
//
// The positions depend on the graph only: order_prepare computes them (a single-source run
// of the lockstep kernel for the levels, then one small sort per level; the level sizes are
// read by the host), and order_emit sorts S by them (device work only, capturable).
struct OrderWs {
    int64_t ns = 0;
    int32_t n = 0, k = 0;
    const int32_t* S = nullptr;
    const int32_t* part = nullptr;
    DBuf<int32_t> pos;        // [n] discovery position of every node
    DBuf<uint64_t> keys, kb;
    DBuf<uint32_t> vals, vb;
    DBuf<int64_t> hist, tmp;
    DBuf<int32_t> out;        // the ordered targets
};

constexpr int ORDER_MAX_LEVELS = 4096;   // deeper graphs keep plain level order past this level

__global__ void hub_src_kernel(const unsigned long long* best, int32_t* src) {
    src[0] = (int32_t)(0xffffffffu - (uint32_t)(best[0] & 0xffffffffull));
}
// Breadth-first levels from one source over unit-weight arcs, as the lockstep kernel's LS_SSSP
// mode would give them (DINF = unreached), but with the whole GPU on each level: warp w looks
// at nodes [32w, 32w + 32) and scans the arcs of those at level L with all its lanes;
// unreached heads get L + 1 (concurrent writers all write L + 1).  more[L] = some head was
// reached; a level whose predecessor reached nothing returns at once.
__global__ void bfs_seed_kernel(int32_t* level, const int32_t* src, int32_t* more, int32_t nmore) {
    level[src[0]] = 0;
    for (int i = 0; i < nmore; i++) more[i] = 0;
}
__global__ void bfs_level_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t n,
                                 int32_t* level, int32_t L, int32_t* more) {
    if (L > 0 && more[L - 1] == 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    bool found = false;
    for (int64_t b0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; b0 < n; b0 += nw * 32) {
        const int64_t v = b0 + lane;
        unsigned m = __ballot_sync(FULL, v < n && level[v] == L);
        while (m) {
            const int64_t u = b0 + (__ffs(m) - 1);
            m &= m - 1;
            const int64_t a1 = rp[u + 1];
            for (int64_t a = rp[u] + lane; a < a1; a += 32) {
                const int32_t w = col[a];
                if (level[w] == DINF) {
                    level[w] = L + 1;
                    found = true;
                }
            }
        }
    }
    if (__any_sync(FULL, found) && lane == 0) more[L] = 1;
}
// level histogram (levels >= cap counted at cap) and the deepest level
__global__ void level_hist_kernel(const int32_t* level, int32_t n, int32_t cap, int32_t* cnt, int32_t* maxl) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t L = level[v];
        if (L == DINF) continue;
        atomicAdd(&cnt[min(L, cap)], 1);
        atomicMax(maxl, L);
    }
}
// keys = level (unreached last), vals = node
__global__ void node_level_keys_kernel(const int32_t* level, int32_t n, uint64_t unreached, uint64_t* keys,
                                       uint32_t* vals) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        keys[v] = level[v] == DINF ? unreached : (uint64_t)level[v];
        vals[v] = (uint32_t)v;
    }
}
__global__ void scatter_pos_kernel(const uint32_t* vals, int64_t count, int64_t base, int32_t* pos) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        pos[vals[i]] = (int32_t)(base + i);
}
// for the nodes of one level (in id order): key = smallest position among their parents (the
// in-neighbours one level up), val = node
__global__ void parent_keys_kernel(const uint32_t* nodes, int64_t count, const int64_t* irp, const int32_t* icol,
                                   const int32_t* level, const int32_t* pos, int32_t L, uint64_t* keys,
                                   uint32_t* vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = nodes[i];
        int32_t m = INT32_MAX;
        for (int64_t p = irp[v]; p < irp[v + 1]; p++) {
            const int32_t u = icol[p];
            if (level[u] == L - 1) m = min(m, pos[u]);
        }
        keys[i] = (uint64_t)(uint32_t)m;
        vals[i] = v;
    }
}

int order_prepare(bcpp_ctx* c, const bcpp_graph* g, const int64_t* irp, const int32_t* icol, const uint32_t* iw,
                  uint64_t wmax, const int32_t* S, int64_t ns, const int32_t* part, int32_t k, OrderWs& w) {
    const int32_t n = g->n;
    w.ns = ns; w.n = n; w.k = k; w.S = S; w.part = part;
    // levels from the hub (the node of largest degree)
    DBuf<unsigned long long> best(c, 1);
    DBuf<int32_t> level(c, n), src(c, 1), cnt(c, ORDER_MAX_LEVELS + 1), maxl(c, 1);
    DBuf<uint64_t> lsig(c, n);
    DBuf<LsItem> item(c, 1);
    DBuf<int64_t> node_off(c, 2);
    CK_ALLOC(best); CK_ALLOC(level); CK_ALLOC(src); CK_ALLOC(cnt); CK_ALLOC(maxl); CK_ALLOC(lsig); CK_ALLOC(item);
    CK_ALLOC(node_off);
    const LsItem hi{0, 0, 1, 0};
    const int64_t hoff[2] = {0, n};
    CK_RC(to_dev(c, item.p, &hi, 1));
    CK_RC(to_dev(c, node_off.p, hoff, 2));
    const unsigned nblk = (unsigned)std::min<int64_t>((n + 255) / 256, 8192);
    CK_CUDA(cudaMemsetAsync(best.p, 0, sizeof(unsigned long long), c->stream));
    hub_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, c->stream>>>(g->row_ptr, n, best.p);
    hub_src_kernel<<<1, 1, 0, c->stream>>>(best.p, src.p);
    c->launches += 2;
    // Unit weights: level-synchronous breadth-first search over the whole GPU, 8 levels per
    // host check; a graph deeper than BFS_LEVELS levels falls back to the lockstep kernel.
    constexpr int32_t BFS_LEVELS = 256;
    bool have_levels = false;
    if (!g->w) {
        DBuf<int32_t> more(c, BFS_LEVELS);
        CK_ALLOC(more);
        fill_i32(level.p, DINF, n, c->stream);
        bfs_seed_kernel<<<1, 1, 0, c->stream>>>(level.p, src.p, more.p, BFS_LEVELS);
        c->launches += 2;
        const unsigned bblk = (unsigned)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)c->num_sms * 8);
        for (int32_t L0 = 0; L0 < BFS_LEVELS && !have_levels; L0 += 8) {
            for (int32_t L = L0; L < L0 + 8; L++) {
                bfs_level_kernel<<<bblk, 256, 0, c->stream>>>(g->row_ptr, g->col, n, level.p, L, more.p);
                c->launches++;
            }
            int32_t last = 1;
            CK_RC(to_host(c, &last, more.p + L0 + 7, 1));
            have_levels = last == 0;
        }
    }
    if (!have_levels) {
        // levels (or weighted distances) from the lockstep kernel: one source, one 4-CTA cluster
        const int nb = g->w ? (int)wmax + 1 : 2;
        SlotWs ws;
        CK_RC(alloc_slots(c, ws, 1, n, nb, false, 0, 1, entry_factor(c, g->w != nullptr, 1)));
        LsArena A{};
        A.rp = g->row_ptr; A.col = g->col; A.w = (const int32_t*)g->w;
        A.irp = irp; A.icol = icol; A.iw = (const int32_t*)iw;
        A.node_off = node_off.p;
        LsParams P{};
        P.mode = LS_SSSP;
        P.nb = nb;
        P.srcs = src.p;
        P.dbg_d = level.p;
        P.dbg_s = lsig.p;
        P.dbg_n = n;
        P.item_counter = ws.counter.p;
        P.flags = c->flags;
        ls_launch(false, !g->directed, A, P, ws.W, item.p, 1, 1, c->stream, 1, 4);
        c->launches++;
    }
    // level sizes
    CK_CUDA(cudaMemsetAsync(cnt.p, 0, (ORDER_MAX_LEVELS + 1) * sizeof(int32_t), c->stream));
    CK_CUDA(cudaMemsetAsync(maxl.p, 0, sizeof(int32_t), c->stream));
    level_hist_kernel<<<nblk, 256, 0, c->stream>>>(level.p, n, ORDER_MAX_LEVELS, cnt.p, maxl.p);
    c->launches++;
    int32_t hmax = 0;
    CK_RC(to_host(c, &hmax, maxl.p, 1));
    const int32_t lmax = std::min(hmax, ORDER_MAX_LEVELS);
    std::vector<int32_t> hcnt((size_t)lmax + 1);
    CK_RC(to_host(c, hcnt.data(), cnt.p, (int64_t)lmax + 1));
    // all nodes by level (stable: by id within a level), positions = level order
    DBuf<uint64_t> nk(c, n), nkb(c, n);
    DBuf<uint32_t> nv(c, n), nvb(c, n);
    DBuf<int64_t> nhist(c, radix_hist_elems(n)), ntmp(c, scan_tmp_elems(radix_hist_elems(n)));
    CK_ALLOC(nk); CK_ALLOC(nkb); CK_ALLOC(nv); CK_ALLOC(nvb); CK_ALLOC(nhist); CK_ALLOC(ntmp);
    CK_ALLOC(w.pos.alloc(c, n));
    node_level_keys_kernel<<<nblk, 256, 0, c->stream>>>(level.p, n, (uint64_t)hmax + 1, nk.p, nv.p);
    radix_sort_pairs(nk.p, nv.p, nkb.p, nvb.p, n, bits_for((uint64_t)hmax + 1), nhist.p, ntmp.p, c->stream,
                     c->launches);
    scatter_pos_kernel<<<nblk, 256, 0, c->stream>>>(nv.p, n, 0, w.pos.p);
    c->launches += 2;
    // levels 1..lmax in discovery order: by the earliest-placed parent (stable: then by id)
    const int kbits = bits_for((uint64_t)std::max(n, 1));
    int64_t beg = hcnt.empty() ? 0 : hcnt[0];
    for (int32_t L = 1; L <= lmax && L < ORDER_MAX_LEVELS; L++) {
        const int64_t cntL = hcnt[L];
        if (cntL > 1) {
            const unsigned b = (unsigned)std::min<int64_t>((cntL + 255) / 256, 8192);
            parent_keys_kernel<<<b, 256, 0, c->stream>>>(nv.p + beg, cntL, irp, icol, level.p, w.pos.p, L, nk.p,
                                                         nvb.p);
            radix_sort_pairs(nk.p, nvb.p, nkb.p, nv.p + beg, cntL, kbits, nhist.p, ntmp.p, c->stream, c->launches);
            scatter_pos_kernel<<<b, 256, 0, c->stream>>>(nvb.p, cntL, beg, w.pos.p);
            c->launches += 2;
        }
        beg += cntL;
    }
    CK_CUDA(cudaGetLastError());
    // buffers of the per-call sort of S
    CK_ALLOC(w.keys.alloc(c, ns)); CK_ALLOC(w.kb.alloc(c, ns));
    CK_ALLOC(w.vals.alloc(c, ns)); CK_ALLOC(w.vb.alloc(c, ns));
    CK_ALLOC(w.hist.alloc(c, radix_hist_elems(ns)));
    CK_ALLOC(w.tmp.alloc(c, scan_tmp_elems(radix_hist_elems(ns))));
    CK_ALLOC(w.out.alloc(c, ns));
    CK_CUDA(cudaStreamSynchronize(c->stream));   // the local buffers above go back to the pool
    return BCPP_OK;
}

int order_emit(bcpp_ctx* c, OrderWs& w, bool) {
    const int64_t ns = w.ns;
    const unsigned blocks = (unsigned)std::min<int64_t>((ns + 255) / 256, 8192);
    level_keys_kernel<<<blocks, 256, 0, c->stream>>>(w.S, ns, w.pos.p, w.keys.p, w.vals.p);
    radix_sort_pairs(w.keys.p, w.vals.p, w.kb.p, w.vb.p, ns, bits_for((uint64_t)std::max(w.n, 1)), w.hist.p, w.tmp.p,
                     c->stream, c->launches);
    c->launches++;
    if (w.part) {
        part_keys_kernel<<<blocks, 256, 0, c->stream>>>(w.vals.p, ns, w.part, w.keys.p);
        radix_sort_pairs(w.keys.p, w.vals.p, w.kb.p, w.vb.p, ns, bits_for((uint64_t)w.k), w.hist.p, w.tmp.p,
                         c->stream, c->launches);
        c->launches++;
    }
    CK_CUDA(cudaMemcpyAsync(w.out.p, w.vals.p, ns * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
    CK_CUDA(cudaGetLastError());
    return BCPP_OK;
}

int order_targets(bcpp_ctx* c, const bcpp_graph* g, const int64_t* irp, const int32_t* icol, const uint32_t* iw,
                  uint64_t wmax, const int32_t* S, int64_t ns, const int32_t* part, int32_t k, OrderWs& w) {
    CK_RC(order_prepare(c, g, irp, icol, iw, wmax, S, ns, part, k, w));
    return order_emit(c, w, g->directed != 0);
}

// --------------------------------------------------------------------------- plain Brandes
// A plain-Brandes evaluation in two parts: plain_prepare takes every host decision (input
// checks, sizes, batches, workspace) and plain_emit queues the device work only, so that the
// same sequence runs directly or is captured once into a CUDA graph and replayed.
struct PlainRun {
    bcpp_graph g{};
    const int32_t* S = nullptr;
    int32_t nS = 0;
    bcpp_opts o{};
    double* bc_out = nullptr;
    uint64_t wmax = 1;
    int64_t ns = 0;
    bool trivial = false;          // |S| < 2 or n == 0: all zeros
    DBuf<uint8_t> in_s;
    DBuf<uint32_t> cnt;
    DBuf<unsigned long long> wmaxd;
    DBuf<int32_t> all;
    InCsr T;
    OrderWs ord;
    bool ordered = false;
    DBuf<LsItem> items;
    DBuf<int64_t> node_off;
    SlotWs ws;
    int nitems = 0, slots = 0, spl = 1, cl = 1, nb = 2;
    LsArena A{};
    LsParams P{};
};

__global__ void wmax_bound_kernel(const unsigned long long* wmax, unsigned long long bound, uint32_t* flags) {
    if (wmax[0] > bound) {
        atomicOr(&flags[FLAG_INVALID], 1u);
        atomicCAS(&flags[FLAG_INVALID_WHY], 0u, WHY_WEIGHT_RANGE);
    }
}

// The input checks as device work only: flags reset, CSR check with the prepared weight bound,
// targets check (rebuilds the target indicator).  Used before every replay of a captured plan.
int plain_emit_checks(bcpp_ctx* c, PlainRun& r) {
    const bcpp_graph* g = &r.g;
    const int32_t n = g->n;
    CK_RC(reset_flags(c));
    CK_CUDA(cudaMemsetAsync(r.wmaxd.p, 0, sizeof(unsigned long long), c->stream));
    csr_check(n, g->num_arcs, g->row_ptr, g->col, g->w, g->directed, c->flags, r.wmaxd.p, c->stream, nullptr, 0);
    wmax_bound_kernel<<<1, 1, 0, c->stream>>>(r.wmaxd.p, (unsigned long long)(g->w ? r.wmax : 1), c->flags);
    c->launches += 2;
    if (r.nS > 0) {
        CK_CUDA(cudaMemsetAsync(r.in_s.p, 0, (size_t)std::max(n, 1), c->stream));
        CK_CUDA(cudaMemsetAsync(r.cnt.p, 0, (size_t)std::max(n, 1) * 4, c->stream));
        targets_check(r.S, r.nS, n, r.in_s.p, r.cnt.p, c->flags, c->stream);
        c->launches++;
    }
    CK_CUDA(cudaGetLastError());
    return BCPP_OK;
}

int plain_prepare(bcpp_ctx* c, const bcpp_graph* g, const int32_t* S, int32_t nS, const bcpp_opts& o,
                  double* bc_out, PlainRun& r) {
    CK_RC(check_graph_struct(g));
    if (nS < 0 || (nS > 0 && !S) || (g->n > 0 && !bc_out)) return BCPP_EINVAL;
    const int32_t n = g->n;
    const bool fp32 = o.precision == BCPP_FP32_DELTA;
    r.g = *g; r.S = S; r.nS = nS; r.o = o; r.bc_out = bc_out;
    CK_RC(reset_flags(c));
    CK_RC(validate_csr(c, g, &r.wmax));
    CK_ALLOC(r.wmaxd.alloc(c, 1));
    if (nS > 0) {
        CK_ALLOC(r.in_s.alloc(c, n));
        CK_ALLOC(r.cnt.alloc(c, n));
        CK_CUDA(cudaMemsetAsync(r.in_s.p, 0, (size_t)std::max(n, 1), c->stream));
        CK_CUDA(cudaMemsetAsync(r.cnt.p, 0, (size_t)std::max(n, 1) * 4, c->stream));
        targets_check(S, nS, n, r.in_s.p, r.cnt.p, c->flags, c->stream);
        c->launches++;
        CK_RC(sync_flags(c));
        if (c->hflags[FLAG_INVALID]) return BCPP_EINVAL;
    }
    r.ns = nS > 0 ? nS : n;
    if (r.ns < 2 || n == 0) {
        r.trivial = true;
        return BCPP_OK;
    }
    const int32_t* srcs = S;
    if (nS == 0) {
        CK_ALLOC(r.all.alloc(c, n));
        srcs = r.all.p;
    }
    if (g->directed) {
        // the source order below reads the in-arcs now; emit rebuilds them for every replay
        CK_RC(in_csr_alloc(c, g, r.T));
        CK_RC(in_csr_emit(c, g, r.T));
    }
    if (o.order_sources && r.ns > 2 * LS_LANES && !g->w) {   // measured to help on unit weights only
        CK_RC(order_prepare(c, g, g->directed ? r.T.rp.p : g->row_ptr, g->directed ? r.T.col.p : g->col,
                            g->directed ? (g->w ? r.T.w.p : nullptr) : g->w, r.wmax, srcs, r.ns, nullptr, 0, r.ord));
        r.ordered = true;
        srcs = r.ord.out.p;
    }
    // items: batches of 32 targets (ordered when requested)
    int64_t s0, s1;
    shard_sources(o, r.ns, s0, s1);
    r.spl = choose_spl(c, s1 - s0, o);
    std::vector<LsItem> hitems = make_items(0, s0, s1, 32 * r.spl);
    r.cl = r.spl == 1 ? choose_cluster(c, (int)hitems.size(), o) : 1;
    if (r.spl == 1) {
        const int b = balanced_width(s1 - s0, slot_capacity(c, o, r.cl), 32);
        if (b < 32) hitems = make_items(0, s0, s1, b);
    }
    r.nitems = (int)hitems.size();
    if (r.nitems <= 0) return BCPP_OK;
    CK_ALLOC(r.items.alloc(c, r.nitems));
    CK_ALLOC(r.node_off.alloc(c, 2));
    CK_RC(to_dev(c, r.items.p, hitems.data(), r.nitems));
    const int64_t hoff[2] = {0, n};
    CK_RC(to_dev(c, r.node_off.p, hoff, 2));
    r.nb = g->w ? (int)r.wmax + 1 : 2;
    const int ef = entry_factor(c, g->w != nullptr, r.spl);
    r.slots = choose_slots(c, r.nitems, o.ctas_per_sm, slot_bytes(n, r.nb, fp32, ef, r.spl), (int64_t)n * 24, r.cl);
    CK_RC(alloc_slots(c, r.ws, r.slots, n, r.nb, fp32, n, r.spl, ef, false));
    r.ws.narrow = use_narrow(c, g->w != nullptr);
    LsArena& A = r.A;
    A.rp = g->row_ptr; A.col = g->col; A.w = (const int32_t*)g->w; A.mu = nullptr;
    if (g->directed) {
        A.irp = r.T.rp.p; A.icol = r.T.col.p; A.iw = g->w ? (const int32_t*)r.T.w.p : nullptr;
    } else {
        A.irp = g->row_ptr; A.icol = g->col; A.iw = (const int32_t*)g->w;
    }
    A.imu = nullptr;
    A.node_off = r.node_off.p;
    LsParams& P = r.P;
    P.mode = LS_BRANDES;
    P.nb = r.nb;
    P.srcs = srcs;
    P.in_s = nS > 0 ? r.in_s.p : nullptr;
    P.items_static = 0;
    P.item_counter = r.ws.counter.p;
    P.flags = c->flags;
    P.phase_ns = c->phase;
    return BCPP_OK;
}

// Device work of one evaluation (no host synchronization).  tb (may be null) times the
// lockstep launch.
int plain_emit(bcpp_ctx* c, PlainRun& r, Timer* tb) {
    const bcpp_graph* g = &r.g;
    const int32_t n = g->n;
    if (r.trivial || r.nitems <= 0) {
        if (n > 0) CK_CUDA(cudaMemsetAsync(r.bc_out, 0, (size_t)n * sizeof(double), c->stream));
        return BCPP_OK;
    }
    if (r.nS == 0) {
        iota(r.all.p, n, c->stream);
        c->launches++;
    }
    if (g->directed) CK_RC(in_csr_emit(c, g, r.T));
    if (r.ordered) CK_RC(order_emit(c, r.ord, g->directed != 0));
    CK_RC(init_slots(c, r.ws));
    if (tb) tb->start();
    ls_launch(r.o.precision == BCPP_FP32_DELTA, !g->directed, r.A, r.P, r.ws.W, r.items.p, r.nitems, r.slots,
              c->stream, r.spl, r.cl, r.ws.narrow);
    c->launches++;
    if (tb) tb->stop();
    CK_CUDA(cudaGetLastError());
    const bool halve = !g->directed && r.o.halve_undirected != 0;
    combine_launch(r.ws.W.bc_sum, r.ws.W.bc_cmp, r.slots, n, n, halve ? 0.5 : 1.0, r.bc_out, c->stream);
    c->launches++;
    CK_CUDA(cudaGetLastError());
    return BCPP_OK;
}

int brandes_dev(bcpp_ctx* c, const bcpp_graph* g, const int32_t* S, int32_t nS, const bcpp_opts& o, double* bc_out,
                bcpp_stats* st) {
    Timer tt(c), tb(c);
    tt.start();
    PlainRun r;
    CK_RC(plain_prepare(c, g, S, nS, o, bc_out, r));
    CK_RC(plain_emit(c, r, &tb));
    int rc = finish_status(c, st);
    tt.stop();
    if (st) {
        st->ms_brandes_sk = tb.acc;
        st->ms_total = tt.acc;
    }
    return rc;
}

// --------------------------------------------------------------------------- Build_SK
struct Skeleton {
    int32_t n = 0, kp = 0, N = 0;
    int64_t arcs = 0, edges = 0, table_entries = 0;
    int32_t lcs = 0, k_nonempty = 0;
    uint64_t wmax_sk = 1, mmax_sk = 1;
    uint32_t tdmax = 0;   // largest finite distance in the entry and exit tables
    DBuf<int32_t> partp, pstart, nf, loc, skid, sknode, skbase;
    DBuf<uint8_t> fr;
    DBuf<uint32_t> pnodes;
    DBuf<int64_t> toff, pstart64;
    DBuf<int32_t> td, tdr;
    DBuf<uint64_t> ts, tsr;
    DBuf<int64_t> skrp;
    DBuf<int32_t> skcol, skw;
    DBuf<uint64_t> skmu;
    std::vector<int32_t> h_pstart, h_nf, h_skbase;
    std::vector<int64_t> h_toff;
    const Skeleton* shared = nullptr;   // tables owned by another skeleton (same parts, same order)
    SkTables tables() const {
        const Skeleton& o = shared ? *shared : *this;
        SkTables T;
        T.pstart = pstart.p; T.nf = nf.p; T.toff = toff.p;
        T.td = o.td.p; T.ts = o.ts.p;
        T.tdr = o.tdr.p ? o.tdr.p : o.td.p;
        T.tsr = o.tsr.p ? o.tsr.p : o.ts.p;
        return T;
    }
};

// part-local CSR over the grouped node order (graph i = part i of P')
int build_local_csr(bcpp_ctx* c, const Skeleton& K, const int64_t* rp, const int32_t* col, const uint32_t* w,
                    DBuf<int64_t>& lrp, DBuf<int32_t>& lcol, DBuf<int32_t>& lw) {
    const int32_t n = K.n;
    DBuf<int64_t> cnt(c, (int64_t)n + 1), tmp(c, scan_tmp_elems((int64_t)n + 1));
    CK_ALLOC(cnt); CK_ALLOC(tmp);
    CK_ALLOC(lrp.alloc(c, (int64_t)n + 1));
    CK_CUDA(cudaMemsetAsync(cnt.p, 0, ((size_t)n + 1) * sizeof(int64_t), c->stream));
    sk_local_count(n, K.pnodes.p, rp, col, K.partp.p, cnt.p, c->stream);
    exclusive_scan<int64_t>(cnt.p, lrp.p, (int64_t)n + 1, nullptr, tmp.p, c->stream, c->launches);
    int64_t total = 0;
    CK_RC(to_host(c, &total, lrp.p + n, 1));
    CK_ALLOC(lcol.alloc(c, total));
    if (w) CK_ALLOC(lw.alloc(c, total));
    sk_local_fill(n, K.pnodes.p, rp, col, w, K.partp.p, K.loc.p, lrp.p, lcol.p, w ? lw.p : nullptr, c->stream);
    c->launches += 2;
    CK_CUDA(cudaGetLastError());
    return BCPP_OK;
}

// reuse (may be null): a skeleton of the same graph built for `part` without singletons.  Every
// part that keeps its nodes under P' keeps its frontiers, its local order and so its Dijkstra_SK
// tables, so they are read from `reuse` instead of being recomputed (Alg. 3 builds the
// skeleton once and only expands P_i and P_j per pair).
int build_sk(bcpp_ctx* c, const bcpp_graph* g, const int32_t* S, int32_t nS_eff, const int32_t* part, int32_t k,
             uint64_t wmax, const InCsr* Tin, const bcpp_opts& o, Skeleton& K, const Skeleton* reuse = nullptr) {
    const int32_t n = g->n;
    const bool fp32 = o.precision == BCPP_FP32_DELTA;
    (void)fp32;
    K.n = n;
    K.kp = k + nS_eff;
    const int32_t kp = K.kp;
    CK_ALLOC(K.partp.alloc(c, n));
    CK_ALLOC(K.fr.alloc(c, n));
    CK_ALLOC(K.pnodes.alloc(c, n));
    CK_ALLOC(K.pstart.alloc(c, (int64_t)kp + 1));
    CK_ALLOC(K.nf.alloc(c, kp));
    CK_ALLOC(K.loc.alloc(c, n));
    CK_ALLOC(K.skid.alloc(c, n));
    // P' and frontiers
    sk_partition(n, part, k, S, nS_eff, K.partp.p, c->flags, c->stream);
    CK_CUDA(cudaMemsetAsync(K.fr.p, 0, (size_t)std::max(n, 1), c->stream));
    sk_frontiers(n, g->row_ptr, g->col, K.partp.p, K.fr.p, c->stream);
    c->launches += 3;
    // group nodes by (part, frontiers first), stable in node id
    {
        DBuf<uint64_t> keys(c, n), kb(c, n);
        DBuf<uint32_t> vb(c, n);
        DBuf<int64_t> hist(c, radix_hist_elems(n)), tmp(c, scan_tmp_elems(radix_hist_elems(n)));
        CK_ALLOC(keys); CK_ALLOC(kb); CK_ALLOC(vb); CK_ALLOC(hist); CK_ALLOC(tmp);
        sk_group_keys(n, K.partp.p, K.fr.p, keys.p, K.pnodes.p, c->stream);
        radix_sort_pairs(keys.p, K.pnodes.p, kb.p, vb.p, n, bits_for(2ull * (uint64_t)kp), hist.p, tmp.p, c->stream,
                         c->launches);
        sk_segments(keys.p, n, kp, K.pstart.p, K.nf.p, c->stream);
        c->launches += 2;
        CK_CUDA(cudaGetLastError());
    }
    K.h_pstart.resize((size_t)kp + 1);
    K.h_nf.resize(kp);
    CK_RC(to_host(c, K.h_pstart.data(), K.pstart.p, (int64_t)kp + 1));
    CK_RC(to_host(c, K.h_nf.data(), K.nf.p, kp));
    CK_RC(sync_flags(c));
    if (c->hflags[FLAG_INVALID]) return BCPP_EINVAL;
    // tables of the parts that keep their nodes can come from `reuse` if nothing else differs
    if (reuse && reuse->kp == k && reuse->n == n) {
        for (int32_t i = 0; i < k && reuse; i++) {
            const int32_t sz = K.h_pstart[i + 1] - K.h_pstart[i];
            const int32_t sz0 = reuse->h_pstart[i + 1] - reuse->h_pstart[i];
            if (sz > 0 && (sz != sz0 || K.h_nf[i] != reuse->h_nf[i])) reuse = nullptr;
        }
    } else {
        reuse = nullptr;
    }
    // host: skeleton ids, table offsets, statistics
    K.h_skbase.resize(kp);
    K.h_toff.resize((size_t)kp + 1);
    int64_t N = 0, tofs = 0, entries = 0;
    int32_t maxpart_tab = 0;
    K.lcs = 0;
    K.k_nonempty = 0;
    for (int32_t i = 0; i < kp; i++) {
        const int32_t sz = K.h_pstart[i + 1] - K.h_pstart[i];
        K.h_skbase[i] = (int32_t)N;
        N += K.h_nf[i];
        K.h_toff[i] = reuse ? (i < k ? reuse->h_toff[i] : 0) : tofs;
        if (sz >= 2 && K.h_nf[i] >= 1) {
            if (!reuse) tofs += (int64_t)sz * K.h_nf[i];
            entries += (int64_t)sz * K.h_nf[i];
            maxpart_tab = std::max(maxpart_tab, sz);
        }
        K.lcs = std::max(K.lcs, sz);
        K.k_nonempty += sz > 0;
    }
    K.h_toff[kp] = tofs;
    K.N = (int32_t)N;
    K.table_entries = entries;
    K.shared = reuse;
    CK_ALLOC(K.skbase.alloc(c, kp));
    CK_ALLOC(K.toff.alloc(c, (int64_t)kp + 1));
    CK_ALLOC(K.sknode.alloc(c, std::max<int64_t>(N, 1)));
    CK_RC(to_dev(c, K.skbase.p, K.h_skbase.data(), kp));
    CK_RC(to_dev(c, K.toff.p, K.h_toff.data(), (int64_t)kp + 1));
    sk_local_ids(n, K.pnodes.p, K.partp.p, K.pstart.p, K.nf.p, K.skbase.p, K.loc.p, K.skid.p, K.sknode.p, c->stream);
    c->launches++;
    if (!reuse) {
        CK_ALLOC(K.td.alloc(c, std::max<int64_t>(tofs, 1)));
        CK_ALLOC(K.ts.alloc(c, std::max<int64_t>(tofs, 1)));
        if (g->directed) {
            CK_ALLOC(K.tdr.alloc(c, std::max<int64_t>(tofs, 1)));
            CK_ALLOC(K.tsr.alloc(c, std::max<int64_t>(tofs, 1)));
        }
    }
    CK_ALLOC(K.pstart64.alloc(c, (int64_t)kp + 1));
    i64_from_i32_kernel<<<(unsigned)std::min<int64_t>(((int64_t)kp + 256) / 256, 8192), 256, 0, c->stream>>>(
        K.pstart.p, K.pstart64.p, (int64_t)kp + 1);
    c->launches++;
    // Dijkstra_SK (Eq. 10) in every part with a table, from every frontier
    if (tofs > 0) {
        DBuf<int64_t> lrp, lirp;
        DBuf<int32_t> lcol, lw, licol, liw;
        CK_RC(build_local_csr(c, K, g->row_ptr, g->col, g->w, lrp, lcol, lw));
        if (g->directed) CK_RC(build_local_csr(c, K, Tin->rp.p, Tin->col.p, Tin->w.p, lirp, licol, liw));
        std::vector<LsItem> hitems;
        std::vector<int32_t> order_parts;
        int32_t maxnf = 0;
        for (int32_t i = 0; i < kp; i++) {
            const int32_t sz = K.h_pstart[i + 1] - K.h_pstart[i];
            if (sz >= 2 && K.h_nf[i] >= 1) order_parts.push_back(i);
        }
        std::stable_sort(order_parts.begin(), order_parts.end(), [&](int32_t a, int32_t b) {
            return (K.h_pstart[a + 1] - K.h_pstart[a]) > (K.h_pstart[b + 1] - K.h_pstart[b]);
        });
        for (int32_t i : order_parts) {
            maxnf = std::max(maxnf, K.h_nf[i]);
            for (int32_t f0 = 0; f0 < K.h_nf[i]; f0 += LS_LANES)
                hitems.push_back(LsItem{i, f0, std::min(LS_LANES, K.h_nf[i] - f0), f0});
        }
        const int nitems = (int)hitems.size();
        DBuf<LsItem> items(c, nitems);
        DBuf<int32_t> srcs(c, maxnf);
        CK_ALLOC(items); CK_ALLOC(srcs);
        CK_RC(to_dev(c, items.p, hitems.data(), nitems));
        iota(srcs.p, maxnf, c->stream);
        c->launches++;
        const int nb = g->w ? (int)wmax + 1 : 2;
        // parts are small: provide the worst case (one entry per node and frontier source)
        const int ef = entry_factor(c, true, 1);
        const int slots = choose_slots(c, nitems, o.ctas_per_sm, slot_bytes(maxpart_tab, nb, false, ef), 0);
        for (int dir = 0; dir < (g->directed ? 2 : 1); dir++) {
            SlotWs ws;
            CK_RC(alloc_slots(c, ws, slots, maxpart_tab, nb, false, 0, 1, ef));
            LsArena A{};
            if (dir == 0) {
                A.rp = lrp.p; A.col = lcol.p; A.w = g->w ? lw.p : nullptr;
                A.irp = g->directed ? lirp.p : lrp.p;
                A.icol = g->directed ? licol.p : lcol.p;
                A.iw = g->w ? (g->directed ? liw.p : lw.p) : nullptr;
            } else {
                A.rp = lirp.p; A.col = licol.p; A.w = g->w ? liw.p : nullptr;
                A.irp = lrp.p; A.icol = lcol.p; A.iw = g->w ? lw.p : nullptr;
            }
            A.node_off = K.pstart64.p;
            LsParams P{};
            P.mode = LS_TABLE;
            P.nb = nb;
            P.srcs = srcs.p;
            P.nfront = K.nf.p;
            P.toff = K.toff.p;
            P.td = dir == 0 ? K.td.p : K.tdr.p;
            P.ts = dir == 0 ? K.ts.p : K.tsr.p;
            P.item_counter = ws.counter.p;
            P.flags = c->flags;
            ls_launch(false, !g->directed, A, P, ws.W, items.p, nitems, slots, c->stream);
            c->launches++;
            CK_CUDA(cudaGetLastError());
            // A batch whose settle list outgrew its bound leaves its table rows unwritten: stop
            // here, before the skeleton is assembled from them (the caller retries with the
            // worst-case bound).
            CK_RC(sync_flags(c));
            if (c->hflags[FLAG_CAPACITY]) return BCPP_ECAPACITY;
        }
    }
    // the largest finite table distance (the Centrality step takes a 16-bit path when it is small)
    if (reuse) {
        K.tdmax = reuse->tdmax;
    } else if (K.table_entries > 0) {
        DBuf<unsigned> tm(c, 1);
        CK_ALLOC(tm);
        CK_CUDA(cudaMemsetAsync(tm.p, 0, sizeof(unsigned), c->stream));
        const unsigned blocks = (unsigned)std::min<int64_t>((K.table_entries + 255) / 256, 152 * 8);
        table_max_kernel<<<blocks, 256, 0, c->stream>>>(K.td.p, K.table_entries, tm.p);
        c->launches++;
        if (K.tdr.p) {
            table_max_kernel<<<blocks, 256, 0, c->stream>>>(K.tdr.p, K.table_entries, tm.p);
            c->launches++;
        }
        unsigned h = 0;
        CK_RC(to_host(c, &h, tm.p, 1));
        K.tdmax = h;
    }
    // skeleton arcs: R with <w,1>, X_i with <d_i, sigma_i>
    {
        const SkTables T = K.tables();
        DBuf<int64_t> cnt(c, N + 1), tmp(c, scan_tmp_elems(N + 1));
        DBuf<unsigned long long> maxes(c, 2);
        CK_ALLOC(cnt); CK_ALLOC(tmp); CK_ALLOC(maxes);
        CK_ALLOC(K.skrp.alloc(c, N + 1));
        CK_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)(N + 1) * sizeof(int64_t), c->stream));
        CK_CUDA(cudaMemsetAsync(maxes.p, 0, 2 * sizeof(unsigned long long), c->stream));
        sk_arcs_count((int32_t)N, K.sknode.p, g->row_ptr, g->col, K.partp.p, K.loc.p, T, cnt.p, c->stream);
        exclusive_scan<int64_t>(cnt.p, K.skrp.p, N + 1, nullptr, tmp.p, c->stream, c->launches);
        CK_RC(to_host(c, &K.arcs, K.skrp.p + N, 1));
        CK_ALLOC(K.skcol.alloc(c, K.arcs));
        CK_ALLOC(K.skw.alloc(c, K.arcs));
        CK_ALLOC(K.skmu.alloc(c, K.arcs));
        sk_arcs_fill((int32_t)N, K.sknode.p, g->row_ptr, g->col, g->w, K.partp.p, K.loc.p, K.skid.p, T, K.skrp.p,
                     K.skcol.p, K.skw.p, K.skmu.p, maxes.p, c->stream);
        c->launches += 2;
        unsigned long long hm[2] = {0, 0};
        CK_RC(to_host(c, hm, maxes.p, 2));
        K.wmax_sk = std::max<unsigned long long>(hm[0], 1);
        K.mmax_sk = std::max<unsigned long long>(hm[1], 1);
        K.edges = g->directed ? K.arcs : K.arcs / 2;
    }
    CK_CUDA(cudaGetLastError());
    return BCPP_OK;
}

// --------------------------------------------------------------------------- Brandes++
// A Brandes++ evaluation in two parts, like plain Brandes: pp_prepare runs Build_SK and takes
// the host decisions of Brandes_SK and Centrality (targets as skeleton ids, batches, work units,
// workspace); pp_emit queues the per-source device work (Brandes_SK, Centrality, combine) only,
// so that it can be captured into a CUDA graph and replayed on the same skeleton.
struct PpRun {
    bcpp_graph g{};
    bcpp_opts o{};
    double scale = 1.0;
    double* bc_out = nullptr;
    const uint8_t* dflag = nullptr;
    Skeleton K;
    DBuf<int32_t> tsk;
    OrderWs ord;
    int32_t nt = 0;
    SlotWs ws;
    bool unit = true, mult = false;
    bool rows_by_item = false;   // Brandes_SK in one dynamic pass with a row set per batch
    int nb = 2, spl = 1, nitems = 0, cl = 1, slots = 1;
    std::vector<CentralityUnit> hunits;
    DBuf<uint8_t> sk_in_s;
    DBuf<int64_t> irp, icnt, itmp;
    DBuf<int32_t> icol, iw;
    DBuf<uint64_t> imu;
    DBuf<double> mud;   // skeleton multiplicities as the dependency type (float in the first half in FP32-delta)
    DBuf<int64_t> node_off;
    DBuf<CentralityUnit> units;
    DBuf<LsItem> items;
    LsArena A{};
};

int pp_prepare(bcpp_ctx* c, const bcpp_graph* g, uint64_t wmax, const InCsr* Tin, const int32_t* Ssing,
               int32_t nsing, const int32_t* Ssrc, int32_t nsrc, const uint8_t* dflag, const int32_t* part, int32_t k,
               const bcpp_opts& o, double scale, double* bc_out, PpRun& r, Timer* tb,
               const Skeleton* reuse = nullptr) {
    const int32_t n = g->n;
    const bool fp32 = o.precision == BCPP_FP32_DELTA;
    const int64_t ns = nsrc;
    r.g = *g; r.o = o; r.scale = scale; r.bc_out = bc_out; r.dflag = dflag;
    // Step 1: Build_SK on P' (every node of Ssing a singleton part)
    if (tb) tb->start();
    Skeleton& K = r.K;
    CK_RC(build_sk(c, g, Ssing, nsing, part, k, wmax, Tin, o, K, reuse));
    if (tb) tb->stop();
    const int32_t N = K.N;
    // targets in batch order (grouped by their original part when requested), as skeleton ids
    CK_ALLOC(r.tsk.alloc(c, ns));
    {
        const int32_t* Suse = Ssrc;
        if (o.order_sources && ns > 2 * LS_LANES) {
            CK_RC(order_targets(c, g, g->directed ? Tin->rp.p : g->row_ptr, g->directed ? Tin->col.p : g->col,
                                g->directed ? (g->w ? Tin->w.p : nullptr) : g->w, wmax, Ssrc, ns, part, k, r.ord));
            Suse = r.ord.out.p;
        }
        sk_target_ids(Suse, (int32_t)ns, K.skid.p, r.tsk.p, c->stream);
        c->launches++;
    }
    r.nt = (int32_t)ns;
    r.unit = K.wmax_sk == 1;
    r.mult = K.mmax_sk > 1;
    r.nb = (int)K.wmax_sk + 1;
    int64_t s0, s1;
    shard_sources(o, r.nt, s0, s1);
    // Centrality work units: chunks of 64 non-frontier nodes of parts with frontiers
    for (int32_t i = 0; i < K.kp; i++) {
        const int32_t sz = K.h_pstart[i + 1] - K.h_pstart[i];
        if (K.h_nf[i] < 1 || sz <= K.h_nf[i]) continue;
        for (int32_t v0 = K.h_nf[i]; v0 < sz; v0 += 64) r.hunits.push_back({i, v0, std::min(sz, v0 + 64), 0});
    }
    // without non-frontier nodes Brandes_SK runs alone and may use 64-source batches
    r.spl = r.hunits.empty() ? choose_spl(c, s1 - s0, o) : 1;
    std::vector<LsItem> hitems = make_items(0, s0, s1, 32 * r.spl);
    r.cl = (!hitems.empty() && r.spl == 1) ? choose_cluster(c, (int)hitems.size(), o) : 1;
    if (r.spl == 1 && r.hunits.empty()) {
        // without a Centrality step (whose cost grows with the batch count, not their width)
        const int b = balanced_width(s1 - s0, slot_capacity(c, o, r.cl), 32);
        if (b < 32) hitems = make_items(0, s0, s1, b);
    }
    r.nitems = (int)hitems.size();
    const int ef = entry_factor(c, !r.unit, r.spl);
    r.slots = r.nitems > 0 ? choose_slots(c, r.nitems, o.ctas_per_sm,
                                          slot_bytes(std::max(N, 1), r.nb, fp32, ef, r.spl), (int64_t)n * 24, r.cl)
                           : 1;
    if (!r.hunits.empty() && r.nitems > r.slots) {
        // More batches than slots.  When memory allows, every batch gets its own set of distance,
        // count and dependency rows (what the Centrality step reads) and its own partial sums, so
        // Brandes_SK schedules all batches dynamically over the slots in one launch and one
        // Centrality launch covers them all; otherwise the batches run in static chunks of
        // `slots`, each followed by Centrality, with equal chunks (128 batches on 76 slots run as
        // 64 + 64 instead of 76 + 52).
        const int64_t Nc = std::max(N, 1);
        const int64_t row_bytes = Nc * 32 * (4 + 8 + (fp32 ? 4 : 8));
        const int64_t work_bytes = slot_bytes(Nc, r.nb, fp32, ef, 1) - row_bytes;
        const int64_t need = (int64_t)r.nitems * (row_bytes + (int64_t)n * 24) + (int64_t)r.slots * work_bytes;
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        int64_t reusable = 0;
        for (auto& b : c->pool)
            if (!b.used) reusable += (int64_t)b.bytes;
        if (!o.pp_chunks && need <= (int64_t)((double)(fr + reusable) * 0.80)) {
            r.rows_by_item = true;
        } else {
            const int chunks = div_up(r.nitems, r.slots);
            r.slots = div_up(r.nitems, chunks);
        }
    }
    // partial sums live in the lockstep slots (or per batch); combine at the end
    CK_RC(alloc_slots(c, r.ws, r.slots, std::max(N, 1), r.nb, fp32, n, r.spl, ef, false,
                      r.rows_by_item ? r.nitems : 0, r.rows_by_item ? r.nitems : 0));
    r.ws.narrow = r.hunits.empty() && use_narrow(c, !r.unit);   // Centrality reads int32 rows
    if (r.nitems > 0) {
        CK_ALLOC(r.sk_in_s.alloc(c, N));
        if (g->directed) {   // skeleton in-arcs
            CK_ALLOC(r.icnt.alloc(c, (int64_t)N + 1));
            CK_ALLOC(r.itmp.alloc(c, scan_tmp_elems((int64_t)N + 1)));
            CK_ALLOC(r.irp.alloc(c, (int64_t)N + 1));
            CK_ALLOC(r.icol.alloc(c, K.arcs));
            CK_ALLOC(r.iw.alloc(c, K.arcs));
            CK_ALLOC(r.imu.alloc(c, K.arcs));
        }
        CK_ALLOC(r.node_off.alloc(c, 2));
        const int64_t hoff[2] = {0, N};
        CK_RC(to_dev(c, r.node_off.p, hoff, 2));
        LsArena& A = r.A;
        A.rp = K.skrp.p; A.col = K.skcol.p;
        A.w = r.unit ? nullptr : K.skw.p;
        A.mu = r.mult ? K.skmu.p : nullptr;
        if (r.mult) {
            CK_ALLOC(r.mud.alloc(c, K.arcs));
            convert_mult(K.skmu.p, K.arcs, r.o.precision == BCPP_FP32_DELTA, r.mud.p, c->stream);
            c->launches++;
            A.mud = r.mud.p;
        }
        if (g->directed) {
            A.irp = r.irp.p; A.icol = r.icol.p; A.iw = r.unit ? nullptr : r.iw.p; A.imu = r.mult ? r.imu.p : nullptr;
        } else {
            A.irp = A.rp; A.icol = A.col; A.iw = A.w; A.imu = A.mu;
        }
        A.node_off = r.node_off.p;
        CK_ALLOC(r.units.alloc(c, (int64_t)r.hunits.size()));
        CK_RC(to_dev(c, r.units.p, r.hunits.data(), (int64_t)r.hunits.size()));
        CK_ALLOC(r.items.alloc(c, r.nitems));
        CK_RC(to_dev(c, r.items.p, hitems.data(), r.nitems));
    }
    return BCPP_OK;
}

// Per-source device work of Brandes++ (no host synchronization); tbr / tce (may be null) time
// the Brandes_SK and Centrality launches.
int pp_emit(bcpp_ctx* c, PpRun& r, Timer* tbr, Timer* tce) {
    const bcpp_graph* g = &r.g;
    const int32_t n = g->n;
    const bool fp32 = r.o.precision == BCPP_FP32_DELTA;
    Skeleton& K = r.K;
    const int32_t N = K.N;
    CK_RC(init_slots(c, r.ws));
    if (r.nitems > 0) {
        sk_gather_flags(N, K.sknode.p, r.dflag, r.sk_in_s.p, c->stream);
        c->launches++;
        if (g->directed) {
            CK_CUDA(cudaMemsetAsync(r.icnt.p, 0, ((size_t)N + 1) * sizeof(int64_t), c->stream));
            sk_transpose(N, K.skrp.p, K.skcol.p, K.skw.p, K.skmu.p, r.icnt.p, nullptr, nullptr, nullptr, 0, c->stream);
            exclusive_scan<int64_t>(r.icnt.p, r.irp.p, (int64_t)N + 1, nullptr, r.itmp.p, c->stream, c->launches);
            CK_CUDA(cudaMemcpyAsync(r.icnt.p, r.irp.p, ((size_t)N + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                                    c->stream));
            sk_transpose(N, K.skrp.p, K.skcol.p, K.skw.p, K.skmu.p, r.icnt.p, r.icol.p, r.iw.p, r.imu.p, 1, c->stream);
            c->launches += 2;
        }
        const SkTables T = K.tables();
        if (r.hunits.empty()) {
            // no non-frontier nodes: Brandes_SK alone, batches scheduled dynamically
            LsParams P{};
            P.mode = LS_BRANDES;
            P.nb = r.nb;
            P.srcs = r.tsk.p;
            P.in_s = r.sk_in_s.p;
            P.bc_map = K.sknode.p;
            P.item_counter = r.ws.counter.p;
            P.flags = c->flags;
            P.phase_ns = c->phase;
            if (tbr) tbr->start();
            ls_launch(fp32, !g->directed, r.A, P, r.ws.W, r.items.p, r.nitems, r.slots, c->stream, r.spl, r.cl,
                      r.ws.narrow);
            c->launches++;
            if (tbr) tbr->stop();
            CK_CUDA(cudaGetLastError());
        }
        if (!r.hunits.empty() && r.rows_by_item) {
            // all batches in one dynamic Brandes_SK launch, each into its own rows, then one
            // Centrality launch over all batches (row set and partial sums of batch i: index i)
            LsParams P{};
            P.mode = LS_SKEL;
            P.nb = r.nb;
            P.srcs = r.tsk.p;
            P.in_s = r.sk_in_s.p;
            P.bc_map = K.sknode.p;
            P.item_counter = r.ws.counter.p;
            P.rows_by_item = 1;
            P.flags = c->flags;
            P.phase_ns = c->phase;
            if (tbr) tbr->start();
            ls_launch(fp32, !g->directed, r.A, P, r.ws.W, r.items.p, r.nitems, r.slots, c->stream, 1, r.cl);
            c->launches++;
            if (tbr) tbr->stop();
            CK_CUDA(cudaGetLastError());
            if (tce) tce->start();
            centrality_launch(fp32, K.tdmax <= CT_H16_MAX, r.units.p, (int)r.hunits.size(), r.nitems, T, K.pnodes.p,
                              K.skbase.p, r.ws.W.d,
                              r.ws.W.sg, r.ws.W.dl, r.ws.W.cap_n, r.ws.W.bc_sum, r.ws.W.bc_cmp, r.ws.W.cap_bc,
                              c->flags, c->stream);
            c->launches++;
            if (tce) tce->stop();
            CK_CUDA(cudaGetLastError());
        }
        for (int c0 = 0; c0 < r.nitems && !r.hunits.empty() && !r.rows_by_item; c0 += r.slots) {
            const int cn = std::min(r.slots, r.nitems - c0);
            LsParams P{};
            P.mode = LS_SKEL;
            P.nb = r.nb;
            P.srcs = r.tsk.p;
            P.in_s = r.sk_in_s.p;
            P.bc_map = K.sknode.p;
            P.items_static = 1;
            P.flags = c->flags;
            P.phase_ns = c->phase;
            if (tbr) tbr->start();
            ls_launch(fp32, !g->directed, r.A, P, r.ws.W, r.items.p + c0, cn, cn, c->stream, 1, r.cl);
            c->launches++;
            if (tbr) tbr->stop();
            CK_CUDA(cudaGetLastError());
            if (tce) tce->start();
            centrality_launch(fp32, K.tdmax <= CT_H16_MAX, r.units.p, (int)r.hunits.size(), cn, T, K.pnodes.p,
                              K.skbase.p, r.ws.W.d,
                              r.ws.W.sg, r.ws.W.dl, r.ws.W.cap_n, r.ws.W.bc_sum, r.ws.W.bc_cmp, r.ws.W.cap_bc,
                              c->flags, c->stream);
            c->launches++;
            if (tce) tce->stop();
            CK_CUDA(cudaGetLastError());
            ls_reset_launch(r.ws.W, cn, c->stream);
            c->launches++;
        }
    }
    combine_launch(r.ws.W.bc_sum, r.ws.W.bc_cmp, r.ws.sum_slots, n, n, r.scale, r.bc_out, c->stream);
    c->launches++;
    CK_CUDA(cudaGetLastError());
    return BCPP_OK;
}

void pp_fill_stats(const PpRun& r, bcpp_stats* st) {
    if (!st) return;
    st->skel_nodes = r.K.N;
    st->skel_edges = r.K.edges;
    st->k = r.K.k_nonempty;
    st->lcs = r.K.lcs;
    st->table_entries = r.K.table_entries;
}

// Brandes++ core (Alg. 1 steps, and Alg. 3's Brandes_SK(G_sk, S_sc, S_dest) + Centrality):
// every node of Ssing becomes a singleton part, the sources are Ssrc (a subset of Ssing), and
// dflag marks the destinations (the indicator of Eq. 7 / Eq. 12 / Eq. 13).  bc_out receives the
// partial betweenness of these (source, destination) pairs times `scale`.
int brandes_pp_core(bcpp_ctx* c, const bcpp_graph* g, uint64_t wmax, const InCsr* Tin, const int32_t* Ssing,
                    int32_t nsing, const int32_t* Ssrc, int32_t nsrc, const uint8_t* dflag, const int32_t* part,
                    int32_t k, const bcpp_opts& o, double scale, double* bc_out, bcpp_stats* st, Timer& tb, Timer& tbr,
                    Timer& tce, const Skeleton* reuse = nullptr) {
    PpRun r;
    CK_RC(pp_prepare(c, g, wmax, Tin, Ssing, nsing, Ssrc, nsrc, dflag, part, k, o, scale, bc_out, r, &tb, reuse));
    CK_RC(pp_emit(c, r, &tbr, &tce));
    pp_fill_stats(r, st);
    return BCPP_OK;
}

// Brandes++ (Alg. 1) for target set S: input checks, the target indicator, Build_SK and the
// host decisions (pp_top_prepare), then the per-source device work (pp_top_emit).
struct PpTop {
    bool trivial = false;
    int32_t n = 0;
    double* bc_out = nullptr;
    DBuf<uint8_t> in_s;
    DBuf<uint32_t> cnt;
    DBuf<int32_t> Sall;
    InCsr Tin;
    PpRun run;
};

int pp_top_prepare(bcpp_ctx* c, const bcpp_graph* g, const int32_t* S, int32_t nS, const int32_t* part, int32_t k,
                   const bcpp_opts& o, double* bc_out, PpTop& t, Timer* tb) {
    CK_RC(check_graph_struct(g));
    const int32_t n = g->n;
    if (nS < 0 || (nS > 0 && !S) || (n > 0 && (!bc_out || !part)) || k < 0 || (n > 0 && k == 0)) return BCPP_EINVAL;
    t.n = n;
    t.bc_out = bc_out;
    CK_RC(reset_flags(c));
    uint64_t wmax = 1;
    CK_RC(validate_csr(c, g, &wmax));
    const int64_t ns = nS > 0 ? nS : n;
    CK_ALLOC(t.in_s.alloc(c, n));
    const int32_t* Sp = S;
    if (nS > 0) {
        CK_ALLOC(t.cnt.alloc(c, n));
        CK_CUDA(cudaMemsetAsync(t.in_s.p, 0, (size_t)std::max(n, 1), c->stream));
        CK_CUDA(cudaMemsetAsync(t.cnt.p, 0, (size_t)std::max(n, 1) * 4, c->stream));
        targets_check(S, nS, n, t.in_s.p, t.cnt.p, c->flags, c->stream);
        c->launches++;
    } else {
        CK_CUDA(cudaMemsetAsync(t.in_s.p, 1, (size_t)std::max(n, 1), c->stream));
        CK_ALLOC(t.Sall.alloc(c, n));
        iota(t.Sall.p, n, c->stream);
        c->launches++;
        Sp = t.Sall.p;
    }
    CK_RC(sync_flags(c));
    if (c->hflags[FLAG_INVALID]) return BCPP_EINVAL;
    if (ns < 2 || n == 0) {
        t.trivial = true;
        return BCPP_OK;
    }
    if (g->directed) CK_RC(build_in_csr(c, g, t.Tin));
    const bool halve = !g->directed && o.halve_undirected != 0;
    return pp_prepare(c, g, wmax, &t.Tin, Sp, (int32_t)ns, Sp, (int32_t)ns, t.in_s.p, part, k, o, halve ? 0.5 : 1.0,
                      bc_out, t.run, tb);
}

int pp_top_emit(bcpp_ctx* c, PpTop& t, Timer* tbr, Timer* tce) {
    if (t.trivial) {
        if (t.n > 0) CK_CUDA(cudaMemsetAsync(t.bc_out, 0, (size_t)t.n * sizeof(double), c->stream));
        return BCPP_OK;
    }
    return pp_emit(c, t.run, tbr, tce);
}

int brandes_pp_dev(bcpp_ctx* c, const bcpp_graph* g, const int32_t* S, int32_t nS, const int32_t* part, int32_t k,
                   const bcpp_opts& o, double* bc_out, bcpp_stats* st) {
    Timer tt(c), tb(c), tbr(c), tce(c);
    tt.start();
    PpTop t;
    CK_RC(pp_top_prepare(c, g, S, nS, part, k, o, bc_out, t, &tb));
    CK_RC(pp_top_emit(c, t, &tbr, &tce));
    if (!t.trivial) pp_fill_stats(t.run, st);
    int rc = finish_status(c, st);
    tt.stop();
    if (st) {
        st->ms_build_sk = tb.acc;
        st->ms_brandes_sk = tbr.acc;
        st->ms_centrality = tce.acc;
        st->ms_total = tt.acc;
    }
    return rc;
}

// Brandes++ for separate source and destination sets (Alg. 3's Brandes_SK(G_sk, S_sc, S_dest)
// followed by Centrality): every node of S_sc and S_dest is a singleton part.
int brandes_pp_st_dev(bcpp_ctx* c, const bcpp_graph* g, const int32_t* Ssrc, int32_t nsrc, const int32_t* Sdst,
                      int32_t ndst, const int32_t* part, int32_t k, const bcpp_opts& o, double* bc_out,
                      bcpp_stats* st) {
    CK_RC(check_graph_struct(g));
    const int32_t n = g->n;
    if (nsrc < 0 || ndst < 0 || (nsrc > 0 && !Ssrc) || (ndst > 0 && !Sdst) || (n > 0 && (!bc_out || !part)) || k < 0 ||
        (n > 0 && k == 0))
        return BCPP_EINVAL;
    Timer tt(c);
    tt.start();
    CK_RC(reset_flags(c));
    uint64_t wmax = 1;
    CK_RC(validate_csr(c, g, &wmax));
    if (nsrc == 0 || ndst == 0 || n == 0) {
        if (n > 0) CK_CUDA(cudaMemsetAsync(bc_out, 0, (size_t)n * sizeof(double), c->stream));
        CK_CUDA(cudaStreamSynchronize(c->stream));
        return BCPP_OK;
    }
    DBuf<uint8_t> sflag(c, n), dflag(c, n);
    DBuf<uint32_t> cnt(c, n);
    CK_ALLOC(sflag); CK_ALLOC(dflag); CK_ALLOC(cnt);
    CK_CUDA(cudaMemsetAsync(sflag.p, 0, (size_t)n, c->stream));
    CK_CUDA(cudaMemsetAsync(dflag.p, 0, (size_t)n, c->stream));
    CK_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)n * 4, c->stream));
    targets_check(Ssrc, nsrc, n, sflag.p, cnt.p, c->flags, c->stream);
    CK_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)n * 4, c->stream));
    targets_check(Sdst, ndst, n, dflag.p, cnt.p, c->flags, c->stream);
    c->launches += 2;
    CK_RC(sync_flags(c));
    if (c->hflags[FLAG_INVALID]) return BCPP_EINVAL;
    // singletons: S_sc u S_dest, in node order
    DBuf<int32_t> f(c, n), uni(c, n);
    DBuf<int64_t> pos(c, (int64_t)n + 1), tmp(c, scan_tmp_elems((int64_t)n + 1));
    CK_ALLOC(f); CK_ALLOC(uni); CK_ALLOC(pos); CK_ALLOC(tmp);
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 8192);
    or_flags_kernel<<<blocks, 256, 0, c->stream>>>(sflag.p, dflag.p, n, f.p);
    exclusive_scan<int32_t>(f.p, pos.p, n, pos.p + n, tmp.p, c->stream, c->launches);
    compact_kernel<<<blocks, 256, 0, c->stream>>>(f.p, pos.p, n, uni.p);
    c->launches += 2;
    int64_t nuni = 0;
    CK_RC(to_host(c, &nuni, pos.p + n, 1));
    InCsr Tin;
    if (g->directed) CK_RC(build_in_csr(c, g, Tin));
    Timer tb(c), tbr(c), tce(c);
    const bool halve = !g->directed && o.halve_undirected != 0;
    int rc = brandes_pp_core(c, g, wmax, &Tin, uni.p, (int32_t)nuni, Ssrc, nsrc, dflag.p, part, k, o,
                             halve ? 0.5 : 1.0, bc_out, st, tb, tbr, tce);
    if (rc) return rc;
    rc = finish_status(c, st);
    tt.stop();
    if (st) {
        st->ms_build_sk = tb.acc;
        st->ms_brandes_sk = tbr.acc;
        st->ms_centrality = tce.acc;
        st->ms_total = tt.acc;
    }
    return rc;
}

// Brandes++All (Alg. 3): for every ordered pair of parts (i, j), Brandes_SK with S_sc = P_i
// and S_dest = P_j on the skeleton where both parts are expanded into singletons, then
// Centrality; C(v) is the sum of the k^2 partial results (Sec. 5).
// A context of its own (stream, workspace pool, status flags) for one lane of concurrent work.
struct SubCtx {
    bcpp_ctx* c = nullptr;
    cudaStream_t st = nullptr;
    SubCtx() = default;
    SubCtx(const SubCtx&) = delete;
    SubCtx& operator=(const SubCtx&) = delete;
    ~SubCtx() {
        if (c) bcpp_destroy(c);   // waits for the stream
        if (st) cudaStreamDestroy(st);
    }
    int open(const bcpp_ctx* parent) {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            st = nullptr;
            cudaGetLastError();
            return BCPP_ECUDA;
        }
        CK_RC(bcpp_create(&c, st));
        c->order_factor = parent->order_factor;
        return reset_flags(c);
    }
};

// One lane of Alg. 3's pair loop: its context, its pair buffers and its running sums.
struct PairLane {
    SubCtx sc;                      // destroyed last: the buffers below return to its pool first
    DBuf<int32_t> pair;
    DBuf<uint8_t> dflag;
    DBuf<double> tmp, sum, comp;
    std::unique_ptr<Timer> tb, tbr, tce;
    int64_t calls = 0;
};

// Brandes++All (Alg. 3): Build_SK once on P, then for every ordered pair (i, j) of non-empty
// parts Brandes_SK with S_sc = P_i and S_dest = P_j (both expanded into singletons) and
// Centrality, summed into C(v).  The pairs are independent: they run round-robin on
// ALL_LANES contexts of their own (streams, workspace), so that one pair's small Brandes_SK
// launch overlaps other pairs' work; each pair goes to a fixed lane, each lane keeps a
// compensated running sum and the lanes are added in a fixed order, so the combination does
// not depend on which pair finishes first.
constexpr int ALL_LANES = 4;

int brandes_pp_all_dev(bcpp_ctx* c, const bcpp_graph* g, const int32_t* part, int32_t k, const bcpp_opts& o,
                       double* bc_out, bcpp_stats* st) {
    CK_RC(check_graph_struct(g));
    const int32_t n = g->n;
    if ((n > 0 && (!bc_out || !part)) || k < 0 || (n > 0 && k == 0)) return BCPP_EINVAL;
    Timer tt(c);
    tt.start();
    CK_RC(reset_flags(c));
    uint64_t wmax = 1;
    CK_RC(validate_csr(c, g, &wmax));
    if (n == 0) return BCPP_OK;
    // nodes grouped by part on the device (a stable radix sort keyed by part, so each part keeps
    // increasing node ids) with the range check of the partition; the host reads only the k + 1
    // part offsets, which it needs to enumerate the pairs
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 8192);
    DBuf<uint64_t> gkeys(c, n), gkb(c, n);
    DBuf<uint32_t> gvals(c, n), gvb(c, n);
    DBuf<int64_t> gcnt(c, (int64_t)k + 1), goff(c, (int64_t)k + 1), ghist(c, radix_hist_elems(n)),
        gtmp(c, scan_tmp_elems(std::max<int64_t>(radix_hist_elems(n), (int64_t)k + 1)));
    CK_ALLOC(gkeys); CK_ALLOC(gkb); CK_ALLOC(gvals); CK_ALLOC(gvb);
    CK_ALLOC(gcnt); CK_ALLOC(goff); CK_ALLOC(ghist); CK_ALLOC(gtmp);
    CK_CUDA(cudaMemsetAsync(gcnt.p, 0, ((size_t)k + 1) * sizeof(int64_t), c->stream));
    group_by_part_kernel<<<blocks, 256, 0, c->stream>>>(part, n, k, gkeys.p, gvals.p, gcnt.p, c->flags);
    c->launches++;
    CK_RC(sync_flags(c));
    if (c->hflags[FLAG_INVALID]) return BCPP_EINVAL;
    radix_sort_pairs(gkeys.p, gvals.p, gkb.p, gvb.p, n, bits_for((uint64_t)k), ghist.p, gtmp.p, c->stream,
                     c->launches);
    exclusive_scan<int64_t>(gcnt.p, goff.p, (int64_t)k + 1, nullptr, gtmp.p, c->stream, c->launches);
    std::vector<int64_t> off((size_t)k + 1, 0);
    CK_RC(to_host(c, off.data(), goff.p, (int64_t)k + 1));
    const int32_t* dbyp = reinterpret_cast<const int32_t*>(gvals.p);   // node ids < 2^31
    DBuf<double> sum(c, n), comp(c, n);
    CK_ALLOC(sum); CK_ALLOC(comp);
    CK_CUDA(cudaMemsetAsync(sum.p, 0, (size_t)n * sizeof(double), c->stream));
    CK_CUDA(cudaMemsetAsync(comp.p, 0, (size_t)n * sizeof(double), c->stream));
    InCsr Tin;
    if (g->directed) CK_RC(build_in_csr(c, g, Tin));
    Timer tb(c);
    // Build_SK once on P: every pair reads the tables of the parts it keeps from it
    Skeleton K0;
    tb.start();
    CK_RC(build_sk(c, g, nullptr, 0, part, k, wmax, &Tin, o, K0));
    tb.stop();
    // the lanes start after everything above
    struct Ev {
        cudaEvent_t e = nullptr;
        ~Ev() { if (e) cudaEventDestroy(e); }
    } ready;
    CK_CUDA(cudaEventCreateWithFlags(&ready.e, cudaEventDisableTiming));
    CK_CUDA(cudaEventRecord(ready.e, c->stream));
    PairLane lanes[ALL_LANES];
    struct JoinMain {   // destroyed before the lanes: nothing queued here reads their buffers after
        cudaStream_t s;
        ~JoinMain() { cudaStreamSynchronize(s); }
    } join_main{c->stream};
    for (PairLane& L : lanes) {
        CK_RC(L.sc.open(c));
        bcpp_ctx* lc = L.sc.c;
        CK_CUDA(cudaStreamWaitEvent(lc->stream, ready.e, 0));
        CK_ALLOC(L.pair.alloc(lc, n)); CK_ALLOC(L.dflag.alloc(lc, n));
        CK_ALLOC(L.tmp.alloc(lc, n)); CK_ALLOC(L.sum.alloc(lc, n)); CK_ALLOC(L.comp.alloc(lc, n));
        CK_CUDA(cudaMemsetAsync(L.sum.p, 0, (size_t)n * sizeof(double), lc->stream));
        CK_CUDA(cudaMemsetAsync(L.comp.p, 0, (size_t)n * sizeof(double), lc->stream));
        L.tb.reset(new Timer(lc, true));
        L.tbr.reset(new Timer(lc, true));
        L.tce.reset(new Timer(lc, true));
    }
    int64_t p = 0;
    for (int32_t j = 0; j < k; j++) {
        const int32_t nj = (int32_t)(off[j + 1] - off[j]);
        if (nj == 0) continue;
        for (int32_t i = 0; i < k; i++) {
            const int32_t ni = (int32_t)(off[i + 1] - off[i]);
            if (ni == 0 || (i == j && ni < 2)) continue;
            PairLane& L = lanes[p++ % ALL_LANES];
            bcpp_ctx* lc = L.sc.c;
            part_flag_kernel<<<blocks, 256, 0, lc->stream>>>(part, n, j, L.dflag.p);
            lc->launches++;
            // singletons: P_i followed by P_j (P_i alone when i == j)
            CK_CUDA(cudaMemcpyAsync(L.pair.p, dbyp + off[i], (size_t)ni * 4, cudaMemcpyDeviceToDevice, lc->stream));
            int32_t nsing = ni;
            if (i != j) {
                CK_CUDA(cudaMemcpyAsync(L.pair.p + ni, dbyp + off[j], (size_t)nj * 4, cudaMemcpyDeviceToDevice,
                                        lc->stream));
                nsing += nj;
            }
            CK_RC(brandes_pp_core(lc, g, wmax, &Tin, L.pair.p, nsing, L.pair.p, ni, L.dflag.p, part, k, o, 1.0,
                                  L.tmp.p, nullptr, *L.tb, *L.tbr, *L.tce, &K0));
            accumulate_kernel<<<blocks, 256, 0, lc->stream>>>(L.tmp.p, n, L.sum.p, L.comp.p);
            lc->launches++;
            L.calls++;
        }
    }
    // join: the lanes' sums (and compensations) in lane order, and their status flags
    uint32_t merged[FLAG_COUNT] = {};
    float ms_b = tb.acc, ms_br = 0.f, ms_ce = 0.f;
    int64_t calls = 0;
    for (PairLane& L : lanes) {
        bcpp_ctx* lc = L.sc.c;
        CK_RC(sync_flags(lc));   // waits for the lane's stream
        for (int f = 0; f < FLAG_COUNT; f++) merged[f] |= lc->hflags[f];
        accumulate_kernel<<<blocks, 256, 0, c->stream>>>(L.sum.p, n, sum.p, comp.p);
        accumulate_kernel<<<blocks, 256, 0, c->stream>>>(L.comp.p, n, sum.p, comp.p);
        c->launches += 2 + lc->launches;
        ms_b += L.tb->resolve();
        ms_br += L.tbr->resolve();
        ms_ce += L.tce->resolve();
        calls += L.calls;
    }
    if (merged[FLAG_INVALID] | merged[FLAG_CAPACITY] | merged[FLAG_SIGMA_OVF] | merged[FLAG_DEPTH]) {
        CK_RC(sync_flags(c));
        for (int f = 0; f < FLAG_COUNT; f++) merged[f] |= c->hflags[f];
        CK_CUDA(cudaMemcpyAsync(c->flags, merged, sizeof(merged), cudaMemcpyHostToDevice, c->stream));
        CK_CUDA(cudaStreamSynchronize(c->stream));
    }
    const bool halve = !g->directed && o.halve_undirected != 0;
    finish_kernel<<<blocks, 256, 0, c->stream>>>(sum.p, comp.p, n, halve ? 0.5 : 1.0, bc_out);
    c->launches++;
    int rc = finish_status(c, st);
    tt.stop();
    if (st) {
        st->k = k;
        st->ms_build_sk = ms_b;
        st->ms_brandes_sk = ms_br;
        st->ms_centrality = ms_ce;
        st->ms_total = tt.acc;
        st->skel_edges = calls;   // number of (i, j) Brandes_SK runs
    }
    return rc;
}

// --------------------------------------------------------------------------- batched graphs
int batched_dev(bcpp_ctx* c, int32_t ngraphs, const int64_t* node_ptr_dev, const int64_t* node_ptr_host,
                const bcpp_graph* g, const bcpp_opts& o, double* bc_out, bcpp_stats* st) {
    CK_RC(check_graph_struct(g));
    if (ngraphs < 0 || (g->n > 0 && !bc_out) || g->directed) return BCPP_EINVAL;
    const int32_t n = g->n;
    const bool fp32 = o.precision == BCPP_FP32_DELTA;
    Timer tt(c), tb(c);
    tt.start();
    CK_RC(reset_flags(c));
    std::vector<int64_t> off((size_t)ngraphs + 1);
    std::memcpy(off.data(), node_ptr_host, off.size() * sizeof(int64_t));
    if (off[0] != 0 || off[ngraphs] != n) return BCPP_EINVAL;
    int64_t maxn = 0;
    for (int32_t i = 0; i < ngraphs; i++) {
        if (off[i + 1] < off[i]) return BCPP_EINVAL;
        maxn = std::max(maxn, off[i + 1] - off[i]);
    }
    uint64_t wmax = 1;
    CK_RC(validate_csr(c, g, &wmax));
    DBuf<int32_t> lcol(c, g->num_arcs);
    CK_ALLOC(lcol);
    csr_localize(n, g->row_ptr, g->col, node_ptr_dev, ngraphs, lcol.p, c->flags, c->stream);
    c->launches++;
    CK_RC(sync_flags(c));
    if (c->hflags[FLAG_INVALID]) return BCPP_EINVAL;
    if (n > 0) CK_CUDA(cudaMemsetAsync(bc_out, 0, (size_t)n * sizeof(double), c->stream));
    // largest graphs first (work grows about quadratically with the node count)
    std::vector<int32_t> gorder(ngraphs);
    std::iota(gorder.begin(), gorder.end(), 0);
    std::stable_sort(gorder.begin(), gorder.end(),
                     [&](int32_t a, int32_t b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
    int64_t total_sources = 0;
    for (int32_t gi = 0; gi < ngraphs; gi++) total_sources += off[gi + 1] - off[gi] >= 2 ? off[gi + 1] - off[gi] : 0;
    const int spl = choose_spl(c, total_sources, o);
    std::vector<LsItem> hitems;
    for (int32_t gi : gorder) {
        const int32_t ng = (int32_t)(off[gi + 1] - off[gi]);
        if (ng < 2) continue;
        const std::vector<LsItem> its = make_items(gi, 0, ng, 32 * spl);
        hitems.insert(hitems.end(), its.begin(), its.end());
    }
    const int nitems = (int)hitems.size();
    if (nitems == 0) {
        CK_CUDA(cudaStreamSynchronize(c->stream));
        return BCPP_OK;
    }
    DBuf<LsItem> items(c, nitems);
    DBuf<int32_t> srcs(c, maxn);
    CK_ALLOC(items); CK_ALLOC(srcs);
    CK_RC(to_dev(c, items.p, hitems.data(), nitems));
    iota(srcs.p, maxn, c->stream);
    c->launches++;
    const int nb = g->w ? (int)wmax + 1 : 2;
    const int slots =
        choose_slots(c, nitems, o.ctas_per_sm, slot_bytes(maxn, nb, fp32, entry_factor(c, g->w != nullptr, spl), spl),
                     (int64_t)n * 24);
    SlotWs ws;
    CK_RC(alloc_slots(c, ws, slots, maxn, nb, fp32, n, spl, entry_factor(c, g->w != nullptr, spl), false));
    ws.narrow = use_narrow(c, g->w != nullptr);
    CK_RC(init_slots(c, ws));
    LsArena A{};
    A.rp = g->row_ptr; A.col = lcol.p; A.w = (const int32_t*)g->w;
    A.irp = g->row_ptr; A.icol = lcol.p; A.iw = (const int32_t*)g->w;
    A.node_off = node_ptr_dev;
    LsParams P{};
    P.mode = LS_BRANDES;
    P.nb = nb;
    P.srcs = srcs.p;
    P.item_counter = ws.counter.p;
    P.flags = c->flags;
    P.phase_ns = c->phase;
    tb.start();
    ls_launch(fp32, true, A, P, ws.W, items.p, nitems, slots, c->stream, spl, 1, ws.narrow);
    c->launches++;
    CK_CUDA(cudaGetLastError());
    combine_launch(ws.W.bc_sum, ws.W.bc_cmp, slots, n, n, o.halve_undirected ? 0.5 : 1.0, bc_out, c->stream);
    c->launches++;
    tb.stop();
    int rc = finish_status(c, st);
    tt.stop();
    if (st) {
        st->ms_brandes_sk = tb.acc;
        st->ms_total = tt.acc;
    }
    return rc;
}

// --------------------------------------------------------------------------- partition
int partition_lp_dev(bcpp_ctx* c, const bcpp_graph* g, int32_t max_rounds, int32_t* part_out, int32_t* k_out,
                     int32_t* rounds_out) {
    CK_RC(check_graph_struct(g));
    const int32_t n = g->n;
    if (max_rounds < 1 || (n > 0 && !part_out) || !k_out) return BCPP_EINVAL;
    CK_RC(reset_flags(c));
    uint64_t wmax = 1;
    CK_RC(validate_csr(c, g, &wmax));
    *k_out = 0;
    if (rounds_out) *rounds_out = 0;
    if (n == 0) return BCPP_OK;
    InCsr T;
    if (g->directed) CK_RC(build_in_csr(c, g, T));
    DBuf<int32_t> l0(c, n), l1(c, n), used(c, n);
    DBuf<int64_t> rank(c, (int64_t)n + 1), tmp(c, scan_tmp_elems(n));
    DBuf<unsigned int> changes(c, 1);
    CK_ALLOC(l0); CK_ALLOC(l1); CK_ALLOC(used); CK_ALLOC(rank); CK_ALLOC(tmp); CK_ALLOC(changes);
    lp_init(n, l0.p, used.p, c->stream);
    c->launches++;
    const int64_t* irp = g->directed ? T.rp.p : nullptr;
    const int32_t* icol = g->directed ? T.col.p : nullptr;
    int32_t rounds = 0;
    for (int32_t r = 0; r < max_rounds; r++) {
        CK_CUDA(cudaMemsetAsync(changes.p, 0, sizeof(unsigned int), c->stream));
        lp_step(n, g->row_ptr, g->col, irp, icol, l0.p, l1.p, 0, changes.p, c->stream);
        lp_step(n, g->row_ptr, g->col, irp, icol, l1.p, l0.p, 1, changes.p, c->stream);
        c->launches += 2;
        rounds++;
        unsigned int hc = 0;
        CK_RC(to_host(c, &hc, changes.p, 1));
        if (hc == 0) break;
    }
    lp_mark(n, l0.p, used.p, c->stream);
    exclusive_scan<int32_t>(used.p, rank.p, n, rank.p + n, tmp.p, c->stream, c->launches);
    lp_number(n, l0.p, rank.p, part_out, c->stream);
    c->launches += 2;
    CK_CUDA(cudaGetLastError());
    int64_t k = 0;
    CK_RC(to_host(c, &k, rank.p + n, 1));
    *k_out = (int32_t)k;
    if (rounds_out) *rounds_out = rounds;
    return finish_status(c, nullptr);
}

// --------------------------------------------------------------------------- inspection
int sssp_dev(bcpp_ctx* c, const bcpp_graph* g, const int32_t* src, int32_t nsrc, int32_t* dist_out,
             uint64_t* sigma_out, const bcpp_opts& o) {
    CK_RC(check_graph_struct(g));
    if (nsrc < 0 || (nsrc > 0 && (!src || !dist_out || !sigma_out))) return BCPP_EINVAL;
    const int32_t n = g->n;
    CK_RC(reset_flags(c));
    uint64_t wmax = 1;
    CK_RC(validate_csr(c, g, &wmax));
    if (nsrc == 0 || n == 0) return BCPP_OK;
    {
        // sources must lie in range (repeats are fine here)
        std::vector<int32_t> hs(nsrc);
        CK_RC(to_host(c, hs.data(), src, nsrc));
        for (int32_t s : hs)
            if (s < 0 || s >= n) return BCPP_EINVAL;
    }
    InCsr T;
    if (g->directed) CK_RC(build_in_csr(c, g, T));
    const int nitems = (nsrc + LS_LANES - 1) / LS_LANES;
    std::vector<LsItem> hitems(nitems);
    for (int i = 0; i < nitems; i++) hitems[i] = LsItem{0, i * LS_LANES, std::min(LS_LANES, nsrc - i * LS_LANES), 0};
    DBuf<LsItem> items(c, nitems);
    DBuf<int64_t> node_off(c, 2);
    CK_ALLOC(items); CK_ALLOC(node_off);
    CK_RC(to_dev(c, items.p, hitems.data(), nitems));
    const int64_t hoff[2] = {0, n};
    CK_RC(to_dev(c, node_off.p, hoff, 2));
    // a batch holds each source at most once: split repeated sources across batches is not
    // needed because LS_SSSP lanes are independent rows (a repeat only repeats the row)
    const int nb = g->w ? (int)wmax + 1 : 2;
    const int ef = entry_factor(c, g->w != nullptr, 1);
    const int slots = choose_slots(c, nitems, o.ctas_per_sm, slot_bytes(n, nb, false, ef), 0);
    SlotWs ws;
    CK_RC(alloc_slots(c, ws, slots, n, nb, false, 0, 1, ef));
    LsArena A{};
    A.rp = g->row_ptr; A.col = g->col; A.w = (const int32_t*)g->w;
    if (g->directed) {
        A.irp = T.rp.p; A.icol = T.col.p; A.iw = g->w ? (const int32_t*)T.w.p : nullptr;
    } else {
        A.irp = g->row_ptr; A.icol = g->col; A.iw = (const int32_t*)g->w;
    }
    A.node_off = node_off.p;
    LsParams P{};
    P.mode = LS_SSSP;
    P.nb = nb;
    P.srcs = src;
    P.dbg_d = dist_out;
    P.dbg_s = sigma_out;
    P.dbg_n = n;
    P.item_counter = ws.counter.p;
    P.flags = c->flags;
    ls_launch(false, !g->directed, A, P, ws.W, items.p, nitems, slots, c->stream);
    c->launches++;
    CK_CUDA(cudaGetLastError());
    return finish_status(c, nullptr);
}

int skeleton_dev(bcpp_ctx* c, const bcpp_graph* g, const int32_t* S, int32_t nS, const int32_t* part, int32_t k,
                 int32_t* sk_nodes_out, int32_t* n_sk_out, int64_t cap_arcs, int32_t* au, int32_t* av, int32_t* aw,
                 uint64_t* amu, int64_t* n_arcs_out, const bcpp_opts& o, bool host_out) {
    CK_RC(check_graph_struct(g));
    const int32_t n = g->n;
    if (nS < 0 || (nS > 0 && !S) || (n > 0 && !part) || k < 0 || !n_sk_out || !n_arcs_out) return BCPP_EINVAL;
    CK_RC(reset_flags(c));
    uint64_t wmax = 1;
    CK_RC(validate_csr(c, g, &wmax));
    if (nS > 0) {
        DBuf<uint8_t> in_s(c, n);
        DBuf<uint32_t> cnt(c, n);
        CK_ALLOC(in_s); CK_ALLOC(cnt);
        CK_CUDA(cudaMemsetAsync(in_s.p, 0, (size_t)std::max(n, 1), c->stream));
        CK_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)std::max(n, 1) * 4, c->stream));
        targets_check(S, nS, n, in_s.p, cnt.p, c->flags, c->stream);
        c->launches++;
        CK_RC(sync_flags(c));
        if (c->hflags[FLAG_INVALID]) return BCPP_EINVAL;
    }
    InCsr Tin;
    if (g->directed) CK_RC(build_in_csr(c, g, Tin));
    Skeleton K;
    CK_RC(build_sk(c, g, S, nS, part, k, wmax, g->directed ? &Tin : nullptr, o, K));
    CK_RC(finish_status(c, nullptr));
    *n_sk_out = K.N;
    *n_arcs_out = K.arcs;
    std::vector<int32_t> sknode(K.N), col(K.arcs), w(K.arcs);
    std::vector<int64_t> rp((size_t)K.N + 1);
    std::vector<uint64_t> mu(K.arcs);
    CK_RC(to_host(c, sknode.data(), K.sknode.p, K.N));
    CK_RC(to_host(c, rp.data(), K.skrp.p, (int64_t)K.N + 1));
    CK_RC(to_host(c, col.data(), K.skcol.p, K.arcs));
    CK_RC(to_host(c, w.data(), K.skw.p, K.arcs));
    CK_RC(to_host(c, mu.data(), K.skmu.p, K.arcs));
    std::vector<int32_t> nodes(sknode);
    std::sort(nodes.begin(), nodes.end());
    if (K.arcs > cap_arcs) return BCPP_ECAPACITY;
    std::vector<int32_t> hu(K.arcs), hv(K.arcs);
    for (int32_t x = 0; x < K.N; x++)
        for (int64_t p = rp[x]; p < rp[x + 1]; p++) {
            hu[p] = sknode[x];
            hv[p] = sknode[col[p]];
        }
    auto put = [&](auto* dst, const auto* srcp, int64_t cnt) -> int {
        if (cnt <= 0) return BCPP_OK;
        if (host_out) {
            std::memcpy(dst, srcp, cnt * sizeof(*srcp));
            return BCPP_OK;
        }
        return to_dev(c, dst, srcp, cnt);
    };
    if (sk_nodes_out) CK_RC(put(sk_nodes_out, nodes.data(), K.N));
    if (au) CK_RC(put(au, hu.data(), K.arcs));
    if (av) CK_RC(put(av, hv.data(), K.arcs));
    if (aw) CK_RC(put(aw, w.data(), K.arcs));
    if (amu) CK_RC(put(amu, mu.data(), K.arcs));
    return BCPP_OK;
}

int csr_build_dev(bcpp_ctx* c, int32_t n, int64_t m, const int32_t* eu, const int32_t* ev, const uint32_t* ew,
                  int32_t directed, int64_t* rp, int32_t* col, uint32_t* w_out, int64_t* num_arcs_out) {
    if (n < 0 || m < 0 || !rp || !num_arcs_out || (m > 0 && (!eu || !ev || !col))) return BCPP_EINVAL;
    if (ew && !w_out && m > 0) return BCPP_EINVAL;
    CK_RC(reset_flags(c));
    const int64_t na = directed ? m : 2 * m;
    DBuf<uint64_t> keys(c, na), kb(c, na);
    DBuf<uint32_t> vals(c, na), vb(c, na);
    DBuf<int64_t> hist(c, radix_hist_elems(na)), tmp(c, scan_tmp_elems(radix_hist_elems(na)));
    CK_ALLOC(keys); CK_ALLOC(kb); CK_ALLOC(vals); CK_ALLOC(vb); CK_ALLOC(hist); CK_ALLOC(tmp);
    csr_expand(n, m, eu, ev, ew, directed, keys.p, vals.p, c->flags, c->stream);
    c->launches++;
    CK_RC(sync_flags(c));
    if (c->hflags[FLAG_INVALID]) return BCPP_EINVAL;
    radix_sort_pairs(keys.p, vals.p, kb.p, vb.p, na, bits_for((uint64_t)n * (uint64_t)n), hist.p, tmp.p, c->stream,
                     c->launches);
    csr_finish(keys.p, vals.p, na, n, rp, col, ew ? w_out : nullptr, c->flags, c->stream);
    c->launches += 2;
    CK_CUDA(cudaGetLastError());
    *num_arcs_out = na;
    return finish_status(c, nullptr);
}

// --------------------------------------------------------------------------- host-buffer staging
template <typename T>
int stage_in(bcpp_ctx* c, DBuf<T>& buf, const T* host, int64_t count, const T** dev) {
    if (!host) { *dev = nullptr; return BCPP_OK; }
    CK_ALLOC(buf.alloc(c, count));
    if (count > 0) CK_CUDA(cudaMemcpyAsync(buf.p, host, count * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    *dev = buf.p;
    return BCPP_OK;
}

struct StagedGraph {
    DBuf<int64_t> rp;
    DBuf<int32_t> col;
    DBuf<uint32_t> w;
    bcpp_graph g{};
};
int stage_graph(bcpp_ctx* c, const bcpp_graph* hg, StagedGraph& sg) {
    CK_RC(check_graph_struct(hg));
    sg.g = *hg;
    CK_RC(stage_in(c, sg.rp, hg->row_ptr, (int64_t)hg->n + 1, &sg.g.row_ptr));
    CK_RC(stage_in(c, sg.col, hg->col, hg->num_arcs, &sg.g.col));
    CK_RC(stage_in(c, sg.w, hg->w, hg->num_arcs, &sg.g.w));
    return BCPP_OK;
}

}  // namespace

// --------------------------------------------------------------------------- captured plans
// A plan is one evaluation whose host decisions were taken once (plain_prepare / pp_top_prepare)
// and whose device work was captured into CUDA graphs: `check` (plain Brandes only: the input
// checks) and `run` (the evaluation).  Replays launch the graphs on the context's stream.
struct bcpp_plan {
    bcpp_ctx* c = nullptr;
    int kind = 0;                        // 1: plain Brandes, 2: Brandes++
    bcpp_graph g{};
    const int32_t* S = nullptr;
    int32_t nS = 0;
    const int32_t* part = nullptr;
    int32_t k = 0;
    bcpp_opts o{};
    double* bc_out = nullptr;
    int order_factor = 8;
    PlainRun* plain = nullptr;
    PpTop* pp = nullptr;
    cudaStream_t cs = nullptr;           // capture stream (the context's may be the legacy stream)
    cudaGraphExec_t check = nullptr, run = nullptr;
    int64_t run_kernels = 0;
    bcpp_stats created{};                // skeleton sizes of creation (Brandes++)

    void release() {
        if (check) cudaGraphExecDestroy(check);
        if (run) cudaGraphExecDestroy(run);
        check = run = nullptr;
        delete plain;
        delete pp;
        plain = nullptr;
        pp = nullptr;
    }
};

namespace {

// Record the device work queued by f() on a private stream into an executable graph.
template <class F>
int capture_graph(bcpp_ctx* c, cudaStream_t cs, F&& f, cudaGraphExec_t* out, int64_t* nkernels) {
    CK_CUDA(cudaStreamSynchronize(c->stream));
    cudaStream_t saved = c->stream;
    c->stream = cs;
    const int64_t l0 = c->launches;
    cudaGraph_t gr = nullptr;
    int rc = BCPP_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = BCPP_ECUDA;
    } else {
        rc = f();
        const cudaError_t e = cudaStreamEndCapture(cs, &gr);
        if (rc == BCPP_OK && e != cudaSuccess) rc = BCPP_ECUDA;
    }
    c->stream = saved;
    if (rc == BCPP_OK && cudaGraphInstantiate(out, gr, 0) != cudaSuccess) rc = BCPP_ECUDA;
    if (gr) cudaGraphDestroy(gr);
    if (rc != BCPP_OK) cudaGetLastError();
    if (nkernels) *nkernels = c->launches - l0;
    return rc;
}

int plan_build(bcpp_plan* p) {
    bcpp_ctx* c = p->c;
    p->release();
    c->order_factor = p->order_factor;
    int rc = BCPP_OK;
    if (p->kind == 1) {
        p->plain = new (std::nothrow) PlainRun();
        if (!p->plain) rc = BCPP_ENOMEM;
        if (!rc) rc = plain_prepare(c, &p->g, p->S, p->nS, p->o, p->bc_out, *p->plain);
        if (!rc) rc = capture_graph(c, p->cs, [&] { return plain_emit_checks(c, *p->plain); }, &p->check, nullptr);
        if (!rc) rc = capture_graph(c, p->cs, [&] { return plain_emit(c, *p->plain, nullptr); }, &p->run,
                                    &p->run_kernels);
    } else {
        p->pp = new (std::nothrow) PpTop();
        if (!p->pp) rc = BCPP_ENOMEM;
        if (!rc) rc = pp_top_prepare(c, &p->g, p->S, p->nS, p->part, p->k, p->o, p->bc_out, *p->pp, nullptr);
        if (!rc && !p->pp->trivial) pp_fill_stats(p->pp->run, &p->created);
        if (!rc) rc = capture_graph(c, p->cs, [&] { return pp_top_emit(c, *p->pp, nullptr, nullptr); }, &p->run,
                                    &p->run_kernels);
    }
    c->order_factor = 8;
    return rc;
}

int plan_replay(bcpp_plan* p, bcpp_stats* st) {
    bcpp_ctx* c = p->c;
    if (p->check) {
        CK_CUDA(cudaGraphLaunch(p->check, c->stream));
        CK_RC(sync_flags(c));
        if (c->hflags[FLAG_INVALID]) return BCPP_EINVAL;
    } else {
        CK_RC(reset_flags(c));
    }
    CK_CUDA(cudaGraphLaunch(p->run, c->stream));
    return finish_status(c, st);
}

int plan_create(bcpp_ctx* c, int kind, const bcpp_graph* g, const int32_t* S, int32_t nS, const int32_t* part,
                int32_t k, const bcpp_opts* opts, double* bc_out, bcpp_plan** out) {
    if (!out) return BCPP_EINVAL;
    *out = nullptr;
    if (!c || !g) return BCPP_EINVAL;
    const bcpp_opts o = opts_or_default(opts);
    if (o.host_buffers) return BCPP_EINVAL;
    bcpp_plan* p = new (std::nothrow) bcpp_plan();
    if (!p) return BCPP_ENOMEM;
    p->c = c; p->kind = kind; p->g = *g; p->S = S; p->nS = nS; p->part = part; p->k = k; p->o = o; p->bc_out = bc_out;
    if (cudaStreamCreateWithFlags(&p->cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return BCPP_ECUDA;
    }
    int rc = plan_build(p);
    if (rc == BCPP_ECAPACITY) {   // Build_SK ran at creation and a batch outgrew its list
        p->order_factor = 64;
        rc = plan_build(p);
    }
    if (rc != BCPP_OK) {
        p->release();
        cudaStreamDestroy(p->cs);
        delete p;
        return rc;
    }
    *out = p;
    return BCPP_OK;
}

}  // namespace

// A call whose per-batch settle lists outgrew the default capacity is run once more with the
// worst-case capacity (one entry per node and source of a batch).
template <class F>
int with_capacity_retry(bcpp_ctx* c, F&& f) {
    c->order_factor = 8;
    int rc = f();
    if (rc == BCPP_ECAPACITY) {
        c->order_factor = 64;
        rc = f();
        c->order_factor = 8;
    }
    return rc;
}

// =========================================================================== C ABI
extern "C" {

void bcpp_default_opts(bcpp_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = BCPP_FP64;
    o->halve_undirected = 1;
    o->batch = 0;
    o->ctas_per_sm = 0;
    o->validate = 1;
    o->host_buffers = 0;
    o->order_sources = 1;
    o->cluster = 0;
    o->shard_index = 0;
    o->shard_count = 0;
    o->pp_chunks = 0;
}

int bcpp_shard_bounds(int64_t num_sources, int32_t index, int32_t count, int64_t* s0, int64_t* s1) {
    if (num_sources < 0 || !s0 || !s1) return BCPP_EINVAL;
    if (count > 1 && (index < 0 || index >= count)) return BCPP_EINVAL;
    shard_range(num_sources, index, count, *s0, *s1);
    return BCPP_OK;
}

const char* bcpp_strerror(int s) {
    switch (s) {
        case BCPP_OK: return "ok";
        case BCPP_EINVAL: return "invalid argument (graph, targets, partition or options)";
        case BCPP_ENOMEM: return "out of device or host memory";
        case BCPP_ECUDA: return "CUDA runtime error";
        case BCPP_ETIMEOUT: return "a bounded device wait expired";
        case BCPP_EOVERFLOW_SIGMA: return "a shortest-path count exceeded 2^64 (results written, not exact)";
        case BCPP_ECAPACITY: return "a per-batch device list or an output buffer is too small";
        default: return "unknown status";
    }
}

int bcpp_create(bcpp_ctx** out, void* stream) {
    if (!out) return BCPP_EINVAL;
    *out = nullptr;
    bcpp_ctx* c = new (std::nothrow) bcpp_ctx();
    if (!c) return BCPP_ENOMEM;
    c->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
        cudaMalloc(&c->flags, FLAG_BYTES) != cudaSuccess ||
        cudaMallocHost(&c->hflags, FLAG_BYTES) != cudaSuccess) {
        cudaGetLastError();
        if (c->flags) cudaFree(c->flags);
        delete c;
        return BCPP_ECUDA;
    }
    c->phase = reinterpret_cast<unsigned long long*>(c->flags + FLAG_COUNT);
    if (cudaMemset(c->flags, 0, FLAG_BYTES) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->flags);
        cudaFreeHost(c->hflags);
        delete c;
        return BCPP_ECUDA;
    }
    *out = c;
    return BCPP_OK;
}

void bcpp_destroy(bcpp_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (auto& b : c->pool) cudaFree(b.p);
    cudaFree(c->flags);
    cudaFreeHost(c->hflags);
    delete c;
}

int64_t bcpp_workspace_bytes(const bcpp_ctx* c) { return c ? c->held() : 0; }

int bcpp_csr_build(bcpp_ctx* c, int32_t n, int64_t m, const int32_t* eu, const int32_t* ev, const uint32_t* ew,
                   int32_t directed, int64_t* row_ptr_out, int32_t* col_out, uint32_t* w_out, int64_t* num_arcs_out) {
    if (!c) return BCPP_EINVAL;
    return csr_build_dev(c, n, m, eu, ev, ew, directed, row_ptr_out, col_out, w_out, num_arcs_out);
}

int bcpp_csr_validate(bcpp_ctx* c, const bcpp_graph* g) {
    if (!c) return BCPP_EINVAL;
    int rc = check_graph_struct(g);
    if (rc) return rc;
    if (reset_flags(c)) return BCPP_ECUDA;
    uint64_t wmax = 1;
    return validate_csr(c, g, &wmax);
}

int bcpp_brandes(bcpp_ctx* c, const bcpp_graph* g, const int32_t* S, int32_t nS, const bcpp_opts* opts, double* bc_out,
                 bcpp_stats* stats) {
    if (!c || !g) return BCPP_EINVAL;
    const bcpp_opts o = opts_or_default(opts);
    const int64_t l0 = c->launches;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    int rc;
    if (o.host_buffers) {
        StagedGraph sg;
        DBuf<int32_t> dS;
        DBuf<double> dbc;
        const int32_t* pS = nullptr;
        rc = stage_graph(c, g, sg);
        if (!rc) rc = stage_in(c, dS, S, nS, &pS);
        if (!rc && !dbc.alloc(c, g->n)) rc = BCPP_ENOMEM;
        if (!rc) rc = with_capacity_retry(c, [&] { return brandes_dev(c, &sg.g, pS, nS, o, dbc.p, stats); });
        if ((rc == BCPP_OK || rc == BCPP_EOVERFLOW_SIGMA) && g->n > 0 &&
            to_host(c, bc_out, dbc.p, g->n) != BCPP_OK)
            rc = BCPP_ECUDA;
    } else {
        rc = with_capacity_retry(c, [&] { return brandes_dev(c, g, S, nS, o, bc_out, stats); });
    }
    if (stats) stats->kernel_launches = c->launches - l0;
    return rc;
}

int bcpp_brandes_pp(bcpp_ctx* c, const bcpp_graph* g, const int32_t* S, int32_t nS, const int32_t* part, int32_t k,
                    const bcpp_opts* opts, double* bc_out, bcpp_stats* stats) {
    if (!c || !g) return BCPP_EINVAL;
    const bcpp_opts o = opts_or_default(opts);
    const int64_t l0 = c->launches;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    int rc;
    if (o.host_buffers) {
        StagedGraph sg;
        DBuf<int32_t> dS, dpart;
        DBuf<double> dbc;
        const int32_t *pS = nullptr, *pp = nullptr;
        rc = stage_graph(c, g, sg);
        if (!rc) rc = stage_in(c, dS, S, nS, &pS);
        if (!rc) rc = stage_in(c, dpart, part, g->n, &pp);
        if (!rc && !dbc.alloc(c, g->n)) rc = BCPP_ENOMEM;
        if (!rc) rc = with_capacity_retry(c, [&] { return brandes_pp_dev(c, &sg.g, pS, nS, pp, k, o, dbc.p, stats); });
        if ((rc == BCPP_OK || rc == BCPP_EOVERFLOW_SIGMA) && g->n > 0 &&
            to_host(c, bc_out, dbc.p, g->n) != BCPP_OK)
            rc = BCPP_ECUDA;
    } else {
        rc = with_capacity_retry(c, [&] { return brandes_pp_dev(c, g, S, nS, part, k, o, bc_out, stats); });
    }
    if (stats) stats->kernel_launches = c->launches - l0;
    return rc;
}

int bcpp_brandes_pp_st(bcpp_ctx* c, const bcpp_graph* g, const int32_t* Ssrc, int32_t nsrc, const int32_t* Sdst,
                       int32_t ndst, const int32_t* part, int32_t k, const bcpp_opts* opts, double* bc_out,
                       bcpp_stats* stats) {
    if (!c || !g) return BCPP_EINVAL;
    const bcpp_opts o = opts_or_default(opts);
    const int64_t l0 = c->launches;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    int rc;
    if (o.host_buffers) {
        StagedGraph sg;
        DBuf<int32_t> ds, dd, dpart;
        DBuf<double> dbc;
        const int32_t *ps = nullptr, *pd = nullptr, *pp = nullptr;
        rc = stage_graph(c, g, sg);
        if (!rc) rc = stage_in(c, ds, Ssrc, nsrc, &ps);
        if (!rc) rc = stage_in(c, dd, Sdst, ndst, &pd);
        if (!rc) rc = stage_in(c, dpart, part, g->n, &pp);
        if (!rc && !dbc.alloc(c, g->n)) rc = BCPP_ENOMEM;
        if (!rc)
            rc = with_capacity_retry(c, [&] { return brandes_pp_st_dev(c, &sg.g, ps, nsrc, pd, ndst, pp, k, o, dbc.p, stats); });
        if ((rc == BCPP_OK || rc == BCPP_EOVERFLOW_SIGMA) && g->n > 0 && to_host(c, bc_out, dbc.p, g->n) != BCPP_OK)
            rc = BCPP_ECUDA;
    } else {
        rc = with_capacity_retry(c, [&] { return brandes_pp_st_dev(c, g, Ssrc, nsrc, Sdst, ndst, part, k, o, bc_out, stats); });
    }
    if (stats) stats->kernel_launches = c->launches - l0;
    return rc;
}

int bcpp_brandes_pp_all(bcpp_ctx* c, const bcpp_graph* g, const int32_t* part, int32_t k, const bcpp_opts* opts,
                        double* bc_out, bcpp_stats* stats) {
    if (!c || !g) return BCPP_EINVAL;
    const bcpp_opts o = opts_or_default(opts);
    const int64_t l0 = c->launches;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    int rc;
    if (o.host_buffers) {
        StagedGraph sg;
        DBuf<int32_t> dpart;
        DBuf<double> dbc;
        const int32_t* pp = nullptr;
        rc = stage_graph(c, g, sg);
        if (!rc) rc = stage_in(c, dpart, part, g->n, &pp);
        if (!rc && !dbc.alloc(c, g->n)) rc = BCPP_ENOMEM;
        if (!rc) rc = with_capacity_retry(c, [&] { return brandes_pp_all_dev(c, &sg.g, pp, k, o, dbc.p, stats); });
        if ((rc == BCPP_OK || rc == BCPP_EOVERFLOW_SIGMA) && g->n > 0 && to_host(c, bc_out, dbc.p, g->n) != BCPP_OK)
            rc = BCPP_ECUDA;
    } else {
        rc = with_capacity_retry(c, [&] { return brandes_pp_all_dev(c, g, part, k, o, bc_out, stats); });
    }
    if (stats) stats->kernel_launches = c->launches - l0;
    return rc;
}

int bcpp_brandes_batched(bcpp_ctx* c, int32_t num_graphs, const int64_t* graph_node_ptr, const bcpp_graph* arena,
                         const bcpp_opts* opts, double* bc_out, bcpp_stats* stats) {
    if (!c || !arena || !graph_node_ptr || num_graphs < 0) return BCPP_EINVAL;
    const bcpp_opts o = opts_or_default(opts);
    const int64_t l0 = c->launches;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    int rc;
    std::vector<int64_t> hptr((size_t)num_graphs + 1);
    if (o.host_buffers) {
        std::memcpy(hptr.data(), graph_node_ptr, hptr.size() * sizeof(int64_t));
        StagedGraph sg;
        DBuf<int64_t> dptr;
        DBuf<double> dbc;
        const int64_t* pptr = nullptr;
        rc = stage_graph(c, arena, sg);
        if (!rc) rc = stage_in(c, dptr, graph_node_ptr, (int64_t)num_graphs + 1, &pptr);
        if (!rc && !dbc.alloc(c, arena->n)) rc = BCPP_ENOMEM;
        if (!rc)
            rc = with_capacity_retry(c, [&] { return batched_dev(c, num_graphs, pptr, hptr.data(), &sg.g, o, dbc.p, stats); });
        if ((rc == BCPP_OK || rc == BCPP_EOVERFLOW_SIGMA) && arena->n > 0 &&
            to_host(c, bc_out, dbc.p, arena->n) != BCPP_OK)
            rc = BCPP_ECUDA;
    } else {
        rc = to_host(c, hptr.data(), graph_node_ptr, (int64_t)num_graphs + 1);
        if (!rc)
            rc = with_capacity_retry(c, [&] { return batched_dev(c, num_graphs, graph_node_ptr, hptr.data(), arena, o, bc_out, stats); });
    }
    if (stats) stats->kernel_launches = c->launches - l0;
    return rc;
}

int bcpp_sssp(bcpp_ctx* c, const bcpp_graph* g, const int32_t* src, int32_t nsrc, int32_t* dist_out,
              uint64_t* sigma_out, const bcpp_opts* opts) {
    if (!c || !g) return BCPP_EINVAL;
    const bcpp_opts o = opts_or_default(opts);
    if (o.host_buffers) {
        StagedGraph sg;
        DBuf<int32_t> dsrc, dd;
        DBuf<uint64_t> ds;
        const int32_t* ps = nullptr;
        int rc = stage_graph(c, g, sg);
        if (!rc) rc = stage_in(c, dsrc, src, nsrc, &ps);
        const int64_t cnt = (int64_t)nsrc * g->n;
        if (!rc && (!dd.alloc(c, cnt) || !ds.alloc(c, cnt))) rc = BCPP_ENOMEM;
        if (!rc) rc = with_capacity_retry(c, [&] { return sssp_dev(c, &sg.g, ps, nsrc, dd.p, ds.p, o); });
        if ((rc == BCPP_OK || rc == BCPP_EOVERFLOW_SIGMA) && cnt > 0) {
            if (to_host(c, dist_out, dd.p, cnt) || to_host(c, sigma_out, ds.p, cnt)) rc = BCPP_ECUDA;
        }
        return rc;
    }
    return with_capacity_retry(c, [&] { return sssp_dev(c, g, src, nsrc, dist_out, sigma_out, o); });
}

int bcpp_skeleton(bcpp_ctx* c, const bcpp_graph* g, const int32_t* S, int32_t nS, const int32_t* part, int32_t k,
                  int32_t* sk_nodes_out, int32_t* n_sk_out, int64_t cap_arcs, int32_t* au, int32_t* av, int32_t* aw,
                  uint64_t* amu, int64_t* n_arcs_out, const bcpp_opts* opts) {
    if (!c || !g) return BCPP_EINVAL;
    const bcpp_opts o = opts_or_default(opts);
    if (o.host_buffers) {
        StagedGraph sg;
        DBuf<int32_t> dS, dpart;
        const int32_t *pS = nullptr, *pp = nullptr;
        int rc = stage_graph(c, g, sg);
        if (!rc) rc = stage_in(c, dS, S, nS, &pS);
        if (!rc) rc = stage_in(c, dpart, part, g->n, &pp);
        if (!rc)
            rc = with_capacity_retry(c, [&] {
                return skeleton_dev(c, &sg.g, pS, nS, pp, k, sk_nodes_out, n_sk_out, cap_arcs, au, av, aw, amu,
                                    n_arcs_out, o, true);
            });
        return rc;
    }
    return with_capacity_retry(c, [&] {
        return skeleton_dev(c, g, S, nS, part, k, sk_nodes_out, n_sk_out, cap_arcs, au, av, aw, amu, n_arcs_out, o,
                            false);
    });
}

int bcpp_plan_brandes(bcpp_ctx* c, const bcpp_graph* g, const int32_t* S, int32_t nS, const bcpp_opts* opts,
                      double* bc_out, bcpp_plan** plan) {
    return plan_create(c, 1, g, S, nS, nullptr, 0, opts, bc_out, plan);
}

int bcpp_plan_brandes_pp(bcpp_ctx* c, const bcpp_graph* g, const int32_t* S, int32_t nS, const int32_t* part,
                         int32_t k, const bcpp_opts* opts, double* bc_out, bcpp_plan** plan) {
    return plan_create(c, 2, g, S, nS, part, k, opts, bc_out, plan);
}

int bcpp_plan_launch(bcpp_plan* p, bcpp_stats* stats) {
    if (!p) return BCPP_EINVAL;
    bcpp_ctx* c = p->c;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    Timer tt(c);
    tt.start();
    int rc = plan_replay(p, stats);
    if (rc == BCPP_ECAPACITY && p->order_factor < 64) {
        // a batch outgrew the settled-entry list: rebuild once with the worst-case capacity
        p->order_factor = 64;
        rc = plan_build(p);
        if (rc == BCPP_OK) rc = plan_replay(p, stats);
    }
    tt.stop();
    if (stats) {
        const uint32_t ovf = stats->sigma_overflow;
        *stats = p->created;
        stats->sigma_overflow = ovf;
        stats->ms_total = tt.acc;
        stats->kernel_launches = p->run_kernels;
    }
    return rc;
}

void bcpp_plan_destroy(bcpp_plan* p) {
    if (!p) return;
    cudaStreamSynchronize(p->c->stream);
    p->release();
    cudaStreamDestroy(p->cs);
    delete p;
}

int bcpp_autotune(bcpp_ctx* c, const bcpp_graph* g, const int32_t* S, int32_t nS, const bcpp_opts* opts,
                  bcpp_opts* tuned, float* ms_out) {
    if (!c || !g || !tuned) return BCPP_EINVAL;
    const bcpp_opts base = opts_or_default(opts);
    if (base.host_buffers) return BCPP_EINVAL;
    int rc = check_graph_struct(g);
    if (rc) return rc;
    *tuned = base;
    const int64_t ns = nS > 0 ? nS : g->n;
    static const int cand[BCPP_AUTOTUNE_CANDIDATES][2] = {{32, 1}, {32, 2}, {32, 4}, {64, 1}};
    for (int i = 0; i < BCPP_AUTOTUNE_CANDIDATES; i++)
        if (ms_out) ms_out[i] = -1.f;
    if (ns < 2 || g->n == 0) return BCPP_OK;
    // sample: one shard of the sources holding at least two waves of resident 32-source batches
    const int64_t nitems = (ns + LS_LANES - 1) / LS_LANES;
    const int cps = base.ctas_per_sm > 0 ? base.ctas_per_sm : LS_MIN_CTAS;
    const int64_t wave = (int64_t)cps * c->num_sms;
    const int64_t shards = std::max<int64_t>(1, nitems / (2 * wave));
    DBuf<double> scratch(c, g->n);
    if (!scratch) return BCPP_ENOMEM;
    float best = -1.f;
    for (int i = 0; i < BCPP_AUTOTUNE_CANDIDATES; i++) {
        bcpp_opts o = base;
        o.batch = cand[i][0];
        o.cluster = cand[i][1];
        o.shard_index = 0;
        o.shard_count = (int32_t)shards;
        bcpp_stats st{};
        rc = with_capacity_retry(c, [&] { return brandes_dev(c, g, S, nS, o, scratch.p, &st); });
        if (rc != BCPP_OK && rc != BCPP_EOVERFLOW_SIGMA) return rc;
        if (ms_out) ms_out[i] = st.ms_brandes_sk;
        if (best < 0.f || st.ms_brandes_sk < best) {
            best = st.ms_brandes_sk;
            tuned->batch = cand[i][0];
            tuned->cluster = cand[i][1];
        }
    }
    return BCPP_OK;
}

int bcpp_autotune_batched(bcpp_ctx* c, int32_t num_graphs, const int64_t* graph_node_ptr, const bcpp_graph* arena,
                          const bcpp_opts* opts, bcpp_opts* tuned, float* ms_out) {
    if (!c || !arena || !graph_node_ptr || num_graphs < 0 || !tuned) return BCPP_EINVAL;
    const bcpp_opts base = opts_or_default(opts);
    if (base.host_buffers) return BCPP_EINVAL;
    int rc = check_graph_struct(arena);
    if (rc) return rc;
    *tuned = base;
    static const int cand[BCPP_AUTOTUNE_BATCHED_CANDIDATES][2] = {{32, 2}, {64, 2}, {32, 1}, {64, 1}};
    for (int i = 0; i < BCPP_AUTOTUNE_BATCHED_CANDIDATES; i++)
        if (ms_out) ms_out[i] = -1.f;
    if (arena->n == 0) return BCPP_OK;
    std::vector<int64_t> hptr((size_t)num_graphs + 1);
    rc = to_host(c, hptr.data(), graph_node_ptr, (int64_t)num_graphs + 1);
    if (rc) return rc;
    DBuf<double> scratch(c, arena->n);
    if (!scratch) return BCPP_ENOMEM;
    float best = -1.f;
    for (int i = 0; i < BCPP_AUTOTUNE_BATCHED_CANDIDATES; i++) {
        bcpp_opts o = base;
        o.batch = cand[i][0];
        o.ctas_per_sm = cand[i][1];
        bcpp_stats st{};
        rc = with_capacity_retry(c, [&] { return batched_dev(c, num_graphs, graph_node_ptr, hptr.data(), arena, o,
                                                             scratch.p, &st); });
        if (rc != BCPP_OK && rc != BCPP_EOVERFLOW_SIGMA) return rc;
        if (ms_out) ms_out[i] = st.ms_brandes_sk;
        if (best < 0.f || st.ms_brandes_sk < best) {
            best = st.ms_brandes_sk;
            tuned->batch = cand[i][0];
            tuned->ctas_per_sm = cand[i][1];
        }
    }
    return BCPP_OK;
}

int bcpp_partition_lp(bcpp_ctx* c, const bcpp_graph* g, int32_t max_rounds, const bcpp_opts* opts,
                      int32_t* part_out, int32_t* k_out, int32_t* rounds_out) {
    if (!c || !g) return BCPP_EINVAL;
    const bcpp_opts o = opts_or_default(opts);
    if (!o.host_buffers) return partition_lp_dev(c, g, max_rounds, part_out, k_out, rounds_out);
    StagedGraph sg;
    DBuf<int32_t> dp;
    int rc = stage_graph(c, g, sg);
    if (!rc && !dp.alloc(c, g->n)) rc = BCPP_ENOMEM;
    if (!rc) rc = partition_lp_dev(c, &sg.g, max_rounds, dp.p, k_out, rounds_out);
    if (rc == BCPP_OK && g->n > 0 && to_host(c, part_out, dp.p, g->n) != BCPP_OK) rc = BCPP_ECUDA;
    return rc;
}

}  // extern "C"

