// bcpp_brandes_noalloc: plain Brandes for small undirected graphs that allocates nothing.
//
// Some callers cannot call cudaMalloc: a host process whose own allocator owns all device
// memory (an allocation behind its back breaks its accounting, or fails because it has
// reserved the free memory), or a latency-critical path where an allocation, which may
// synchronize the device, is not acceptable.  This entry point keeps every byte of scratch
// it needs in one file-scope static device array of fixed size, so such callers only pass
// their inputs and output.
//
// The array belongs to the library's device code: every GPU on which the library's module is
// loaded holds it (about 43 MB) until the process exits.  CUDA loads modules lazily by
// default, so the array is placed on a device at the first call there (the address lookup
// loads the module), not when the library is opened; a host allocator that reserves the free
// memory must come after that first call, or the process must set CUDA_MODULE_LOADING=EAGER.
// All calls share the array and it keeps the last call's contents; each call clears what
// must start at zero.  Calls whose work overlaps on the GPU (other streams, other host
// threads) race on the array; serialize them.
#include "common.cuh"
#include "csr.cuh"
#include "lockstep.cuh"
#include "skeleton.cuh"

using namespace bcpp;

namespace {

constexpr int32_t NA_NODES = BCPP_NOALLOC_MAX_NODES;
constexpr int32_t NA_MAX_W = BCPP_NOALLOC_MAX_WEIGHT;
constexpr int NA_NB = NA_MAX_W + 1;
constexpr int NA_SLOTS = 8;
constexpr int64_t NA_CAP_ORDER = 32 * (int64_t)NA_NODES + 1024;
// steps of a batch: at most one per distinct distance 0 .. NA_MAX_W * (NA_NODES - 1)
constexpr int32_t NA_CAP_STEPS = NA_MAX_W * (NA_NODES - 1) + 2;
constexpr int64_t NA_BM_WORDS = (NA_NODES + 31) / 32;
constexpr int NA_MAX_ITEMS = (NA_NODES + LS_LANES - 1) / LS_LANES;

// Layout of the static scratch array.
struct NaScratch {
    int32_t d[NA_SLOTS][NA_NODES][LS_LANES];
    uint64_t sg[NA_SLOTS][NA_NODES][LS_LANES];
    double dl[NA_SLOTS][NA_NODES][LS_LANES];
    LsEnt order[NA_SLOTS][NA_CAP_ORDER];
    int32_t step_d[NA_SLOTS][NA_CAP_STEPS];
    int32_t step_beg[NA_SLOTS][NA_CAP_STEPS];
    uint32_t bm[NA_SLOTS][NA_NB][NA_BM_WORDS];
    double bc_sum[NA_SLOTS][NA_NODES];
    double bc_cmp[NA_SLOTS][NA_NODES];
    double bc_bat[NA_SLOTS][NA_NODES];
    int32_t hdr[NA_SLOTS][4];
    LsItem items[NA_MAX_ITEMS];
    int64_t node_off[2];
    int32_t srcs[NA_NODES];
    uint32_t tcnt[NA_NODES];
    uint8_t in_s[NA_NODES];
    uint8_t bflag[NA_SLOTS][NA_NB];
    uint32_t flags[FLAG_COUNT];
    unsigned long long wmax;
    int counter;
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NaScratch)];

// Device address of the array in the current context.  Host code may not use the symbol itself
// as an address (it names a host-side stand-in), so every call looks the address up; the lookup
// allocates nothing, and looking it up each time stays correct after a device reset or under
// another context, where the module (and the array) are loaded again at a new address.
int na_scratch(NaScratch** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return BCPP_ECUDA;
    }
    *out = reinterpret_cast<NaScratch*>(p);
    return BCPP_OK;
}

__global__ void na_prepare_kernel(NaScratch* s, int32_t n, int32_t ns, int nitems) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < (int64_t)NA_SLOTS * NA_NODES * LS_LANES; i += stride) (&s->d[0][0][0])[i] = DINF;
    for (int64_t i = tid; i < (int64_t)NA_SLOTS * NA_NB * NA_BM_WORDS; i += stride) (&s->bm[0][0][0])[i] = 0u;
    for (int64_t i = tid; i < (int64_t)NA_SLOTS * NA_NODES; i += stride) {
        (&s->bc_sum[0][0])[i] = 0.0;
        (&s->bc_cmp[0][0])[i] = 0.0;
        (&s->bc_bat[0][0])[i] = 0.0;
    }
    for (int64_t i = tid; i < (int64_t)NA_SLOTS * NA_NB; i += stride) (&s->bflag[0][0])[i] = 0;
    for (int64_t i = tid; i < NA_SLOTS * 4; i += stride) (&s->hdr[0][0])[i] = 0;
    for (int64_t i = tid; i < n; i += stride) {
        s->srcs[i] = (int32_t)i;
        s->tcnt[i] = 0u;
        s->in_s[i] = 0;
    }
    for (int64_t i = tid; i < nitems; i += stride)
        s->items[i] = LsItem{0, (int32_t)(i * LS_LANES), (int32_t)min((int64_t)LS_LANES, (int64_t)ns - i * LS_LANES), 0};
    if (tid == 0) {
        s->node_off[0] = 0;
        s->node_off[1] = n;
        s->wmax = 0ull;
        s->counter = 0;
    }
    for (int64_t i = tid; i < FLAG_COUNT; i += stride) s->flags[i] = 0u;
}

}  // namespace

extern "C" int bcpp_brandes_noalloc(const bcpp_graph* g, const int32_t* S, int32_t nS, int32_t halve,
                                    double* bc_out, void* cuda_stream) {
    if (!g || g->n < 0 || g->num_arcs < 0 || !g->row_ptr || (g->num_arcs > 0 && !g->col)) return BCPP_EINVAL;
    if (g->directed) return BCPP_EINVAL;                          // undirected graphs only
    if (g->n > NA_NODES) return BCPP_EINVAL;                      // beyond the static scratch
    if (nS < 0 || nS > g->n || (nS > 0 && !S) || (g->n > 0 && !bc_out)) return BCPP_EINVAL;
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    const int32_t n = g->n;
    NaScratch* s = nullptr;
    int rc = na_scratch(&s);
    if (rc) return rc;

    const int32_t ns = nS > 0 ? nS : n;
    const int nitems = (ns + LS_LANES - 1) / LS_LANES;
    na_prepare_kernel<<<256, 256, 0, st>>>(s, n, ns, nitems);
    csr_check(n, g->num_arcs, g->row_ptr, g->col, g->w, 0, s->flags, &s->wmax, st);
    if (nS > 0) targets_check(S, nS, n, s->in_s, s->tcnt, s->flags, st);
    uint32_t hflags[FLAG_COUNT];
    unsigned long long hw = 0;
    if (cudaMemcpyAsync(hflags, s->flags, sizeof(hflags), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&hw, &s->wmax, sizeof(hw), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return BCPP_ECUDA;
    }
    if (hflags[FLAG_INVALID]) return BCPP_EINVAL;
    if (hw > (unsigned long long)NA_MAX_W) return BCPP_EINVAL;   // bucket array holds weights <= 15
    if (ns < 2 || n == 0) {
        if (n > 0 && cudaMemsetAsync(bc_out, 0, (size_t)n * sizeof(double), st) != cudaSuccess) return BCPP_ECUDA;
        return cudaStreamSynchronize(st) == cudaSuccess ? BCPP_OK : BCPP_ECUDA;
    }

    LsArena A{};
    A.rp = g->row_ptr; A.col = g->col; A.w = (const int32_t*)g->w;
    A.irp = g->row_ptr; A.icol = g->col; A.iw = (const int32_t*)g->w;
    A.node_off = s->node_off;
    LsParams P{};
    P.mode = LS_BRANDES;
    P.nb = g->w ? NA_NB : 2;
    P.srcs = nS > 0 ? S : s->srcs;
    P.in_s = nS > 0 ? s->in_s : nullptr;
    P.item_counter = &s->counter;
    P.flags = s->flags;
    LsSlots W{};
    W.d = &s->d[0][0][0]; W.sg = &s->sg[0][0][0]; W.dl = &s->dl[0][0][0]; W.cap_n = NA_NODES;
    W.order = &s->order[0][0]; W.cap_order = NA_CAP_ORDER;
    W.step_d = &s->step_d[0][0]; W.step_beg = &s->step_beg[0][0]; W.cap_steps = NA_CAP_STEPS;
    // the kernel strides the bucket bitmaps by nb * bm_words per slot: with unit weights
    // (nb = 2) the slots use a packed prefix of the array, which the prepare kernel cleared
    W.bm = &s->bm[0][0][0]; W.bm_words = NA_BM_WORDS;
    W.bflag = &s->bflag[0][0];
    W.bc_sum = &s->bc_sum[0][0]; W.bc_cmp = &s->bc_cmp[0][0]; W.bc_bat = &s->bc_bat[0][0];
    W.cap_bc = NA_NODES;
    W.hdr = &s->hdr[0][0];
    const int slots = nitems < NA_SLOTS ? nitems : NA_SLOTS;
    ls_launch(false, true, A, P, W, s->items, nitems, slots, st);
    combine_launch(W.bc_sum, W.bc_cmp, slots, NA_NODES, n, halve ? 0.5 : 1.0, bc_out, st);
    if (cudaGetLastError() != cudaSuccess) return BCPP_ECUDA;
    if (cudaMemcpyAsync(hflags, s->flags, sizeof(hflags), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return BCPP_ECUDA;
    }
    if (hflags[FLAG_CAPACITY]) return BCPP_ECAPACITY;
    if (hflags[FLAG_SIGMA_OVF]) return BCPP_EOVERFLOW_SIGMA;
    return BCPP_OK;
}
