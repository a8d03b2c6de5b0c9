// Lockstep multi-source shortest paths with path counts and dependency accumulation.
//
// One CTA (or a cluster of 2 or 4 CTAs) owns a batch of up to 32 sources ("lanes") of one
// graph.  Its state lives in a private slot of device memory laid out node-major, lane-minor ([node][32]), so the 32
// sources of a node are one 128-byte line for distances and two for path counts: a warp
// reads one node's row for all its sources with a single coalesced access, and every lane
// follows the same adjacency list.  Settling proceeds in exact distance order with circular
// bucket bitmaps (unit weights: plain breadth-first levels; integer weights: buckets of
// width 1), which is what the path counts and the reverse-order dependency recursion need.
//
// Modes:
//   LS_BRANDES  forward (Eq. 2 / Eq. 11) then backward (Eq. 7 / Eq. 12); adds the
//               dependencies of every node into the slot's compensated FP64 partial sums
//   LS_SKEL     same, but the slot keeps d, sigma and (I_{v in S}+delta)/sigma after the
//               batch for the Centrality step; one batch per slot
//   LS_TABLE    forward only with the Dijkstra_SK parent rule (Eq. 10: a parent counts if it
//               is not a frontier or is the source); writes the node-major tables
//   LS_SSSP     forward only; writes d and sigma per source (inspection)
#pragma once
#include "common.cuh"

namespace bcpp {

constexpr int LS_LANES = 32;
#ifndef BCPP_LS_THREADS
#define BCPP_LS_THREADS 512
#endif
constexpr int LS_THREADS = BCPP_LS_THREADS;                 // threads per CTA
constexpr int LS_MIN_CTAS = 1024 / LS_THREADS;              // resident CTAs per SM (64 registers)

enum LsMode : int { LS_BRANDES = 0, LS_SKEL = 1, LS_TABLE = 2, LS_SSSP = 3 };

// A set of graphs stored back to back.  Node ids inside a graph's CSR are graph-local;
// graph g owns global nodes [node_off[g], node_off[g+1]).  rp has absolute arc offsets.
struct LsArena {
    const int64_t* rp;
    const int32_t* col;
    const int32_t* w;        // nullptr = unit weights
    const uint64_t* mu;      // nullptr = multiplicity 1
    const int64_t* irp;      // in-arcs (for the sigma pull of directed graphs)
    const int32_t* icol;
    const int32_t* iw;
    const uint64_t* imu;
    const int64_t* node_off;
    const void* mud;         // mu converted to the dependency type (the backward pass's products); nullptr = none
};

struct LsItem {
    int32_t g;        // graph
    int32_t src_off;  // sources are srcs[src_off, src_off + nsrc) (graph-local ids)
    int32_t nsrc;     // <= 32 * sources per lane
    int32_t aux;      // LS_TABLE: index of the batch's first frontier
};

struct LsParams {
    int mode;
    int nb;                      // circular buckets = max weight + 1
    const int32_t* srcs;
    const uint8_t* in_s;         // per global node: target flag; nullptr = every node
    const int32_t* nfront;       // per graph: locals < nfront are frontiers (LS_TABLE)
    const int32_t* bc_map;       // global node -> index into the partial sums (nullptr = same)
    const int64_t* toff;         // LS_TABLE: per graph table offset
    int32_t* td;                 // LS_TABLE: d_i[v][f]
    uint64_t* ts;                // LS_TABLE: sigma_i[v][f]
    int32_t* dbg_d;              // LS_SSSP: [source index][n]
    uint64_t* dbg_s;
    int64_t dbg_n;
    int items_static;            // 1: item index = slot
    int rows_by_item;            // LS_SKEL: distance / count / dependency rows of item i in row state i
                                 // (one per item), the rest of the slot state per slot
    int* item_counter;           // dynamic item counter (zeroed before launch)
    uint32_t* flags;
    unsigned long long* phase_ns;   // nullptr or [2]: summed forward / backward time of the batches (ns)
};

// One settled (node, step) entry: the node and its out-arc range, read with one 16-byte load.
struct __align__(16) LsEnt {
    int32_t u;
    int32_t deg;
    int64_t a0;
};

struct LsSlots {
    int32_t* d;                  // [slot][cap_n][32 * spl]
    uint64_t* sg;                // [slot][cap_n][32 * spl]
    void* dl;                    // [slot][cap_n][32 * spl] of DT: (I_{v in S} + delta) / sigma
    int64_t cap_n;
    LsEnt* order;                // [slot][cap_order] settled (node, step) entries, in step order
    int64_t cap_order;
    int32_t* step_d;             // [slot][cap_steps] distance of each non-empty step
    int32_t* step_beg;           // [slot][cap_steps] first entry of each step
    int32_t cap_steps;
    uint32_t* bm;                // [slot][nb][bm_words] bucket bitmaps
    int64_t bm_words;
    uint8_t* bflag;              // [slot][nb] bucket non-empty flags
    double* bc_sum;              // [slot][cap_bc] partial betweenness (Neumaier sum over the slot's batches)
    double* bc_cmp;              // [slot][cap_bc] its compensation
    double* bc_bat;              // [slot][cap_bc] the current batch's sums (zero between batches)
    int64_t cap_bc;
    int32_t* hdr;                // [slot][4]: order length, steps, item, -
};

// Launch the lockstep kernel over `nitems` items with `slots` batches in flight.  spl = sources
// per lane (1: 32-source batches, rows of 32; 2: 64-source batches, rows of 64, LS_BRANDES
// only).  cl = CTAs per batch (1, 2 or 4; with 2 or 4 they form a thread-block cluster that
// shares the batch's control state through distributed shared memory; spl = 1 only).
// narrow: one-byte distance rows and 32-bit path-count rows (unit weights, LS_BRANDES only;
// ignored otherwise), for slots whose distance rows start as 0xff bytes; a batch reaching
// distance 254 or a count of 2^32 or more aborts with FLAG_DEPTH and FLAG_CAPACITY, and the call
// reruns with int32 / uint64 rows.
void ls_launch(bool fp32_delta, bool fused, const LsArena& A, const LsParams& P, const LsSlots& W,
               const LsItem* items, int nitems, int slots, cudaStream_t st, int spl = 1, int cl = 1,
               bool narrow = false);

// Restore the distance rows of LS_SKEL slots to "unreached".
void ls_reset_launch(const LsSlots& W, int slots, cudaStream_t st);

// Fill helpers
void fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t st);
// out[i] = (double or float) mu[i], i < m
void convert_mult(const uint64_t* mu, int64_t m, bool fp32, void* out, cudaStream_t st);

}  // namespace bcpp
