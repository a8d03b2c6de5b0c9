/*
 * bcpp -- exact betweenness centrality on one GB300 (sm_103a): plain Brandes and Brandes++.
 *
 * C ABI of libbcpp.so.  The computation follows "A Divide-and-Conquer Algorithm for
 * Betweenness Centrality" (Erdos, Ishakian, Bestavros, Terzi): target-set betweenness
 * C^S(v) = sum over ordered pairs s != t in S of sigma(s,t|v)/sigma(s,t) (Sec. 3, Eq. 5),
 * computed either by Brandes' recursion on G (Eq. 6-7) or by Brandes++ (Sec. 4, Alg. 1):
 * Build_SK (Alg. 2, Dijkstra_SK of Eq. 10), Brandes_SK on the skeleton (Eq. 11-12) and the
 * Centrality step for non-frontier nodes (Eq. 13).
 *
 * Conventions shared by every call
 *   - Graphs are CSR: row_ptr[n+1] (int64), col[num_arcs] (int32).  Each row is strictly
 *     increasing (sorted, no repeated arc), no self-loops.  An undirected graph stores every
 *     edge as two arcs with equal weights.  w == NULL means unit weights; otherwise integer
 *     weights w >= 1 with max(w) * (n - 1) < 2^31 (weights are the edge lengths of Sec. 3;
 *     zero weights are rejected because they break the strict distance order the path
 *     counts rely on).
 *   - Unless opts->host_buffers is set, every pointer argument is a DEVICE pointer.  With
 *     host_buffers = 1 every array argument is a HOST pointer instead: the call copies the
 *     inputs to the device and the result back (end-to-end use).
 *   - The caller owns all argument buffers.  The context owns its workspace, which is kept
 *     between calls (grown on demand) and released by bcpp_destroy.
 *   - Work is queued on the context's stream; every call returns only after its results are
 *     written (it synchronizes the stream to read the status flags).
 *   - Distances are int32 (INT32_MAX = unreachable), path counts sigma are exact uint64;
 *     when a count exceeds 2^64 the results are still written and the call returns
 *     BCPP_EOVERFLOW_SIGMA (also reported in bcpp_stats.sigma_overflow).
 *   - Betweenness is FP64.  In BCPP_FP64 mode the per-source dependencies delta are FP64; in
 *     BCPP_FP32_DELTA mode they are FP32 (sigma stays exact) and only the sum over sources is
 *     FP64, compensated (Neumaier).
 *   - Undirected results are halved by default (each unordered pair once); directed results
 *     are never halved.  The paper assumes 2 <= |S| <= n (Sec. 3); |S| < 2 gives all zeros.
 */
#ifndef BCPP_H
#define BCPP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BCPP_OK 0
#define BCPP_EINVAL 1            /* malformed graph, targets, partition or options */
#define BCPP_ENOMEM 2            /* device or host allocation failed */
#define BCPP_ECUDA 3             /* a CUDA runtime call failed */
#define BCPP_ETIMEOUT 4          /* reserved: a bounded device wait expired */
#define BCPP_EOVERFLOW_SIGMA 5   /* results written, but some path count exceeded 2^64 */
#define BCPP_ECAPACITY 6         /* a per-batch device list outgrew its bound (see bcpp_strerror) */

/* precision modes */
#define BCPP_FP64 0
#define BCPP_FP32_DELTA 1

typedef struct bcpp_ctx bcpp_ctx;

typedef struct {
    int32_t n;                 /* nodes */
    int64_t num_arcs;          /* arcs (2 per undirected edge) */
    const int64_t *row_ptr;    /* [n+1] */
    const int32_t *col;        /* [num_arcs] */
    const uint32_t *w;         /* [num_arcs] or NULL (unit weights) */
    int32_t directed;          /* 0: undirected (symmetric arcs), 1: directed */
} bcpp_graph;

typedef struct {
    int32_t precision;         /* BCPP_FP64 (default) or BCPP_FP32_DELTA */
    int32_t halve_undirected;  /* 1 (default): halve undirected results; 0: ordered-pair sums */
    int32_t batch;             /* sources per batch: 0 = default (32), 32 or 64.  64 applies to plain
                                * Brandes passes (bcpp_brandes, bcpp_brandes_batched, Brandes++ without
                                * non-frontier nodes); Dijkstra_SK, Brandes_SK with Centrality and
                                * bcpp_sssp use 32. */
    int32_t ctas_per_sm;       /* resident source batches per SM: 0 = auto */
    int32_t validate;          /* reserved: the CSR, S and the partition are always checked */
    int32_t host_buffers;      /* 1: array arguments are host pointers (copied in and out) */
    int32_t order_sources;     /* 1 (default): batch the targets in order of their breadth-first level
                                * from the highest-degree node (plain Brandes: unit weights only;
                                * Brandes++: by part, then level), so that a batch's sources are close;
                                * 0: batch S in the given order.  Only the summation order changes. */
    int32_t cluster;           /* CTAs per source batch: 0 = auto (4 as a thread-block cluster when there
                                * are at most half as many batches as resident CTAs, 2 when fewer than
                                * resident CTAs, else 1), or 1, 2, 4 (32-source batches) */
    int32_t shard_index;       /* with shard_count > 1: use only this shard's targets as sources */
    int32_t shard_count;       /* 0 or 1: every target is a source.  Otherwise the targets, in the order
                                * used for batching, are split into shard_count contiguous shards
                                * (shard r: positions [|S| r / R, |S| (r+1) / R)); only shard_index's
                                * targets are sources and the result is that shard's partial sum
                                * (targets stay all of S), so the shards' results add up to the
                                * unsharded result (multi-GPU source sharding).  The order is the one
                                * of order_sources (with order_sources = 0: S as given). */
    int32_t pp_chunks;         /* Brandes++ with non-frontier nodes and more source batches than slots:
                                * 0 (default) = one Brandes_SK launch over all batches with a set of
                                * rows per batch for the Centrality step when device memory allows,
                                * else static chunks of batches; 1 = static chunks (less memory) */
} bcpp_opts;

typedef struct {
    uint32_t sigma_overflow;   /* 1 if some sigma exceeded 2^64 */
    int32_t skel_nodes;        /* N = |V_sk| (Brandes++), Table 2 */
    int64_t skel_edges;        /* M = |E_sk| (edges; arcs for directed graphs), Table 2 */
    int32_t k;                 /* non-empty parts of P' (Brandes++) */
    int32_t lcs;               /* largest part of P' */
    int64_t table_entries;     /* sum_i |F_i| |V_i| stored by Dijkstra_SK */
    float ms_build_sk;         /* Build_SK (frontiers, Dijkstra_SK, skeleton assembly) */
    float ms_brandes_sk;       /* Brandes_SK or plain Brandes passes */
    float ms_centrality;       /* Centrality step */
    float ms_total;            /* whole call, device time */
    int64_t kernel_launches;   /* kernels this call launched */
    float ms_batch_forward;    /* shortest-path batches (plain Brandes, Brandes_SK): the time each batch
                                * spent in its forward pass (Eq. 2 / Eq. 11), summed over the batches;
                                * batches run concurrently, so this exceeds the kernel time */
    float ms_batch_backward;   /* the same for the dependency pass (Eq. 7 / Eq. 12) */
} bcpp_stats;

/* Fill opts with the defaults listed above. */
void bcpp_default_opts(bcpp_opts *opts);

/* The source positions [*s0, *s1) of shard `index` of `count` over `num_sources` sources in
 * batch order: [num_sources * index / count, num_sources * (index + 1) / count), the rule that
 * opts.shard_index / shard_count apply (Alg. 1 sums over the sources s in S independently, so
 * the shards' partial sums add up to the full result).  count <= 1 gives [0, num_sources).
 * Host-only (no device work, no context).  BCPP_EINVAL for num_sources < 0, count > 1 with
 * index outside [0, count), or a NULL output pointer. */
int bcpp_shard_bounds(int64_t num_sources, int32_t index, int32_t count, int64_t *s0, int64_t *s1);

/* Message for a status code (static string). */
const char *bcpp_strerror(int status);

/* Create a context bound to a CUDA stream (NULL = legacy default stream) on the current
 * device.  Returns BCPP_OK and *ctx, or an error and *ctx = NULL. */
int bcpp_create(bcpp_ctx **ctx, void *cuda_stream);

/* Free the context and its workspace.  NULL is ignored. */
void bcpp_destroy(bcpp_ctx *ctx);

/* Workspace bytes currently held by the context (device). */
int64_t bcpp_workspace_bytes(const bcpp_ctx *ctx);

/* CSR build and validation (the input graph G(V,E,W) of Sec. 3).  From m edges
 * (eu[i], ev[i], weight ew[i] or unit if ew == NULL) build the CSR: row_ptr_out[n+1],
 * col_out and w_out (w_out may be NULL when ew is NULL) of capacity 2m (undirected: every
 * edge becomes two arcs) or m (directed); *num_arcs_out (host) receives the arc count.
 * Rows come out sorted.  BCPP_EINVAL for an endpoint outside [0,n), a self-loop, a repeated
 * edge (for undirected input also (u,v) given together with (v,u)), or a zero weight. */
int bcpp_csr_build(bcpp_ctx *ctx, int32_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                   const uint32_t *ew, int32_t directed, int64_t *row_ptr_out, int32_t *col_out,
                   uint32_t *w_out, int64_t *num_arcs_out);

/* Check a CSR against the conventions above (sorted strictly increasing rows, heads in
 * range, no self-loops, weights >= 1 and small enough, symmetric with equal weights when
 * undirected).  BCPP_OK or BCPP_EINVAL. */
int bcpp_csr_validate(bcpp_ctx *ctx, const bcpp_graph *g);

/* Plain Brandes with target set S (Sec. 3, Eq. 5-7): bc_out[n] (FP64) receives C^S(v).
 * S[nS] lists distinct targets in [0,n); nS == 0 (S may be NULL) means S = V.  Every target
 * is a source; the dependency recursion credits I_{v in S} (Eq. 7).  Unit weights run a
 * level-synchronous breadth-first search, integer weights an exact bucket order (Dial's
 * delta-stepping with bucket width 1).  stats may be NULL. */
int bcpp_brandes(bcpp_ctx *ctx, const bcpp_graph *g, const int32_t *S, int32_t nS,
                 const bcpp_opts *opts, double *bc_out, bcpp_stats *stats);

/* Brandes++ (Sec. 4, Alg. 1) for target set S with node partition part[n] (values in
 * [0,k)): targets become singleton parts (P'), Build_SK finds the frontiers and runs
 * Dijkstra_SK in every part (Alg. 2, Eq. 10), Brandes_SK runs from every target on the
 * weighted skeleton with multiplicities (Eq. 11-12), and the Centrality step gives the
 * dependencies of non-frontier nodes (Eq. 13, with the tight-frontier tests stated in the
 * text of Sec. 4).  Exact: bc_out equals bcpp_brandes on the same S for every partition.
 * nS == 0 means S = V.  stats (may be NULL) receives N, M, k, LCS of Table 2. */
int bcpp_brandes_pp(bcpp_ctx *ctx, const bcpp_graph *g, const int32_t *S, int32_t nS,
                    const int32_t *part, int32_t k, const bcpp_opts *opts, double *bc_out,
                    bcpp_stats *stats);

/* Brandes++ for separate source and destination sets: the step of Brandes++All (Sec. 5, Alg. 3)
 * written Brandes_SK(G_sk, S_sc, S_dest), followed by Centrality.  bc_out[n] receives
 * sum over s in Ssrc, t in Sdst, s != t, of sigma(s,t|v)/sigma(s,t) (halved for undirected graphs
 * when halve_undirected is set, as for the other calls).  Every node of Ssrc and Sdst is made a
 * singleton part (the expansion of Sec. 5), the sources are Ssrc, and the indicator of Eq. 7 /
 * Eq. 12 / Eq. 13 marks Sdst.  Each list must be distinct and in [0,n); the lists may overlap.
 * An empty list gives all zeros. */
int bcpp_brandes_pp_st(bcpp_ctx *ctx, const bcpp_graph *g, const int32_t *Ssrc, int32_t nsrc,
                       const int32_t *Sdst, int32_t ndst, const int32_t *part, int32_t k,
                       const bcpp_opts *opts, double *bc_out, bcpp_stats *stats);

/* Brandes++All (Sec. 5, Alg. 3): full betweenness (all ordered pairs, halved for undirected
 * graphs by default) as the sum over every ordered pair of parts (i, j) of the step above with
 * S_sc = P_i and S_dest = P_j (k^2 skeleton passes).  Exact: equals bcpp_brandes with S = V.
 * The skeleton of P is built once; the pairs run four at a time on streams and workspace of the
 * call's own (created and destroyed inside it, after the ctx stream's earlier work), and the
 * call returns when they are done.  stats->skel_edges receives the number of (i, j) passes run;
 * the phase times are summed over the pairs. */
int bcpp_brandes_pp_all(bcpp_ctx *ctx, const bcpp_graph *g, const int32_t *part, int32_t k,
                        const bcpp_opts *opts, double *bc_out, bcpp_stats *stats);

/* Full betweenness (S = V of each graph) of num_graphs independent undirected graphs in one
 * launch.  `arena` is their disjoint union as one CSR (global node ids); graph g owns the
 * nodes [graph_node_ptr[g], graph_node_ptr[g+1]) (int64, device; a host copy is taken), and
 * no arc may leave its graph (BCPP_EINVAL otherwise).  bc_out[arena->n] receives every
 * graph's betweenness in arena order.  With host_buffers, graph_node_ptr is a host array. */
int bcpp_brandes_batched(bcpp_ctx *ctx, int32_t num_graphs, const int64_t *graph_node_ptr,
                         const bcpp_graph *arena, const bcpp_opts *opts, double *bc_out,
                         bcpp_stats *stats);

/* Distances and path counts from nsrc sources (Eq. 2), for bit-exact checks:
 * dist_out[nsrc * n] (row i = source src[i]) and sigma_out[nsrc * n]. */
int bcpp_sssp(bcpp_ctx *ctx, const bcpp_graph *g, const int32_t *src, int32_t nsrc,
              int32_t *dist_out, uint64_t *sigma_out, const bcpp_opts *opts);

/* The skeleton of Build_SK (Sec. 3-4) for inspection, built on P' for the targets S[nS]
 * (nS == 0: no targets, the partition is used as given): sk_nodes_out[cap n] receives the
 * skeleton nodes (original ids, increasing), *n_sk_out (host) their count N; the arcs with
 * their characteristic tuples <weight, multiplicity> go to au/av/aw/amu (capacity cap_arcs,
 * original node ids; an undirected edge appears as two arcs); *n_arcs_out (host) receives
 * the arc count even when it exceeds cap_arcs (then BCPP_ECAPACITY and nothing is copied). */
int bcpp_skeleton(bcpp_ctx *ctx, const bcpp_graph *g, const int32_t *S, int32_t nS,
                  const int32_t *part, int32_t k, int32_t *sk_nodes_out, int32_t *n_sk_out,
                  int64_t cap_arcs, int32_t *au, int32_t *av, int32_t *aw, uint64_t *amu,
                  int64_t *n_arcs_out, const bcpp_opts *opts);

/* Autotuner for the launch shape of the shortest-path kernels (the paper has none: the source
 * batch width and the CTAs per batch are this implementation's knobs).  Runs plain Brandes on
 * (g, S) once per candidate shape -- 32-source batches on 1, 2 or 4 CTAs (a thread-block
 * cluster), and 64-source batches on 1 CTA, in this order -- over the same bounded sample of
 * the sources (the first of R source shards, R = max(1, batches / (2 x resident CTAs)), so the
 * sample fills the GPU at least twice over, or is all of S), and writes into *tuned a copy of
 * *opts (NULL: defaults) whose `batch` and `cluster` are the fastest candidate's.  ms_out
 * (host, may be NULL) receives the candidates' kernel times in milliseconds
 * [BCPP_AUTOTUNE_CANDIDATES] (-1 when |S| < 2).  The tuned options apply to bcpp_brandes,
 * bcpp_brandes_pp and the plans on the same graph.  Errors as for bcpp_brandes;
 * opts->host_buffers must be 0. */
#define BCPP_AUTOTUNE_CANDIDATES 4
int bcpp_autotune(bcpp_ctx *ctx, const bcpp_graph *g, const int32_t *S, int32_t nS,
                  const bcpp_opts *opts, bcpp_opts *tuned, float *ms_out);

/* Autotuner for bcpp_brandes_batched (many independent graphs in one launch): runs the batched
 * evaluation of the whole arena once per candidate -- source batches of 32 or 64 (`batch`) with
 * two or one resident batches per SM (`ctas_per_sm`), in the order (32, 2), (64, 2), (32, 1),
 * (64, 1) -- and writes into *tuned a copy of *opts (NULL: defaults) with the fastest candidate's
 * `batch` and `ctas_per_sm`.  A batched graph's batches are small and numerous, so every batch
 * runs on one CTA (no cluster candidates).  ms_out (host, may be NULL) receives the candidates'
 * kernel times in milliseconds [BCPP_AUTOTUNE_BATCHED_CANDIDATES] (-1 for an empty arena).
 * Arguments and errors as for bcpp_brandes_batched; opts->host_buffers must be 0. */
#define BCPP_AUTOTUNE_BATCHED_CANDIDATES 4
int bcpp_autotune_batched(bcpp_ctx *ctx, int32_t num_graphs, const int64_t *graph_node_ptr,
                          const bcpp_graph *arena, const bcpp_opts *opts, bcpp_opts *tuned, float *ms_out);

/* ---------------------------------------------------------------------------------------
 * Captured plans (CUDA graphs).  The paper has no counterpart: this is the repeated-evaluation
 * form of bcpp_brandes and bcpp_brandes_pp for a service that evaluates the same graph many
 * times.  Creating a plan takes every host decision of one evaluation once (input checks,
 * sizes, source batches and their order, workspace; for Brandes++ all of Build_SK) and records
 * the evaluation's device work as a CUDA graph; bcpp_plan_launch replays it with one graph
 * launch instead of one launch per kernel and no host decision in between.
 *
 * A plan keeps the pointers it was created with (g's arrays, S, part, bc_out) and the workspace
 * it sized (taken from the context's pool until bcpp_plan_destroy).  Destroy every plan before
 * its context.  opts->host_buffers must be 0 (device pointers only).
 * --------------------------------------------------------------------------------------- */
typedef struct bcpp_plan bcpp_plan;

/* Plain-Brandes plan: each launch computes what bcpp_brandes(ctx, g, S, nS, opts, bc_out)
 * computes from the CURRENT contents of g's arrays and of S.  Between launches the caller may
 * rewrite them (another target set of the same size; another graph with the same n, num_arcs,
 * directedness and weights present or absent, max weight not above the one at creation).
 * Every launch first re-checks the graph and S on the device (a separate small graph) and
 * returns BCPP_EINVAL without computing when they are invalid.  On success *plan receives the
 * plan; on error *plan = NULL and nothing is held. */
int bcpp_plan_brandes(bcpp_ctx *ctx, const bcpp_graph *g, const int32_t *S, int32_t nS,
                      const bcpp_opts *opts, double *bc_out, bcpp_plan **plan);

/* Brandes++ plan: Build_SK (Alg. 1 step 1) runs once at creation; each launch replays
 * Brandes_SK, Centrality and the combine on that skeleton and writes what bcpp_brandes_pp
 * would.  g, S and part must not change while the plan lives: the skeleton depends on all
 * three (a changed input needs a new plan). */
int bcpp_plan_brandes_pp(bcpp_ctx *ctx, const bcpp_graph *g, const int32_t *S, int32_t nS,
                         const int32_t *part, int32_t k, const bcpp_opts *opts, double *bc_out,
                         bcpp_plan **plan);

/* Replay the plan on the context's stream and wait for it.  Status as for the direct call
 * (a batch whose settled-entry list outgrows its bound makes the plan rebuild itself once
 * with the worst-case bound and replay, so BCPP_ECAPACITY is not returned for that).  stats
 * (may be NULL): ms_total = device time of the launch, kernel_launches = kernels in the
 * captured graph, and for Brandes++ the skeleton sizes of creation. */
int bcpp_plan_launch(bcpp_plan *plan, bcpp_stats *stats);

/* Free the plan's graphs and return its workspace to the context.  NULL is ignored. */
void bcpp_plan_destroy(bcpp_plan *plan);

/* A node partition for Brandes++ callers without one (the paper takes its partitions from
 * external tools, Sec. 6; Brandes++ is exact for every partition, Sec. 4, so only its speed
 * depends on this choice).  Deterministic label propagation (Raghavan, Albert and Kumara 2007):
 * labels start as the node ids; half-step t updates the nodes v with v mod 2 == t mod 2 from
 * the previous half-step's labels: v takes the label carried by most of its neighbours (for a
 * directed graph in- and out-arcs both count), keeps its own label when that one is among the
 * most frequent, else takes the smallest most frequent label; nodes without neighbours keep
 * theirs.  It stops after a round (two half-steps) without a change or after max_rounds >= 1
 * rounds.  part_out[n] (device; host with opts->host_buffers) receives the labels numbered
 * 0..k-1 in increasing label order, *k_out (host) the number of parts and *rounds_out (host,
 * may be NULL) the rounds run.  opts may be NULL.  Errors as for bcpp_csr_validate. */
int bcpp_partition_lp(bcpp_ctx *ctx, const bcpp_graph *g, int32_t max_rounds, const bcpp_opts *opts,
                      int32_t *part_out, int32_t *k_out, int32_t *rounds_out);

/* Limits of bcpp_brandes_noalloc (sizes of its static scratch array). */
#define BCPP_NOALLOC_MAX_NODES 4096
#define BCPP_NOALLOC_MAX_WEIGHT 15

/* Plain Brandes for small undirected graphs that allocates no memory at all.  The paper has
 * no counterpart: this is a deployment variant of bcpp_brandes for callers that cannot call
 * cudaMalloc -- a host whose own allocator owns all device memory (an allocation behind its
 * back breaks its accounting or fails against its reservation), or a latency-critical path
 * where an allocation, which can synchronize the device, is not acceptable.  No context is
 * needed: the call takes only inputs, the output and a stream.
 *
 * bc_out[n] (device, caller-owned) receives C^S(v) for the targets S[nS] (device; nS == 0
 * means S = V), halved when `halve` is non-zero, in FP64.  It runs the kernels of bcpp_brandes
 * with a fixed launch shape (eight batches of 32 sources in flight, sources in the given order),
 * so the FP64 sums are added in another order: results agree with bcpp_brandes to a relative
 * 1e-12, not bit for bit.  The graph (device CSR) must be undirected with
 * n <= BCPP_NOALLOC_MAX_NODES and unit weights or integer weights <= BCPP_NOALLOC_MAX_WEIGHT.
 *
 * Checks.  On the host, before any GPU work: null pointers, n above the limit, a directed
 * graph and nS outside [0, n] return BCPP_EINVAL.  On the device, before the betweenness
 * kernels run: an invalid CSR (as bcpp_csr_validate), a weight above the limit and repeated or
 * out-of-range targets return BCPP_EINVAL; such a refused call has already overwritten the
 * shared scratch array (never the output).  Other errors as for bcpp_brandes.
 *
 * Scratch lives in one file-scope static device array of about 43 MB.  Every GPU on which the
 * library's device code is loaded holds it until the process exits.  CUDA loads that code
 * lazily by default: the array is placed on a device by the first call there, which looks up
 * its device address (cudaGetSymbolAddress; every call looks it up again, which allocates
 * nothing); make that first call before a host allocator reserves the free device memory and
 * before any stream capture, or run the process with CUDA_MODULE_LOADING=EAGER.  All calls
 * share the array and it keeps the last call's contents (each call clears what must start at
 * zero), so calls whose GPU work overlaps -- on different streams or from different host
 * threads -- race on it: serialize them.  The call synchronizes `cuda_stream` (NULL = legacy
 * default stream) before it returns. */
int bcpp_brandes_noalloc(const bcpp_graph *g, const int32_t *S, int32_t nS, int32_t halve,
                         double *bc_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* BCPP_H */
