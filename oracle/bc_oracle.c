/*
 * CPU oracle for exact betweenness centrality: plain Brandes and Brandes++.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it; the library
 * never calls it and shares no code, header or table with it.
 *
 * Everything here is written for obviousness, not speed: adjacency lists built from the
 * edge list, a FIFO queue (unit weights) or a binary-heap Dijkstra (integer weights >= 1),
 * uint64 path counts with an overflow flag, FP64 dependencies, and FP64 betweenness summed
 * with Neumaier compensation.
 *
 * Definitions followed (paper: "A Divide-and-Conquer Algorithm for Betweenness Centrality"):
 *   Sec. 3, Eq. 2        sigma(s,v) = sum over shortest-path parents u of sigma(s,u)
 *   Sec. 3, Eq. 5-7      target-set betweenness and its Brandes recursion with I_{v in S}
 *   Sec. 3 (skeleton)    frontiers F_i, cross edges R, cliques X_i, tuples <d, sigma>
 *   Sec. 3, Eq. 10       Dijkstra_SK: sigma summed over non-frontier parents (and the source)
 *   Sec. 4, Alg. 1 and 2 Build_SK -> Brandes_SK -> Centrality, with the target singletons P'
 *   Sec. 4, Eq. 11-12    Brandes_SK with edge multiplicities
 *   Sec. 4, Eq. 13       Centrality of the non-frontier nodes, read as:
 *                          sigma(s,v) = sum over entry frontiers f with d(s,f)+d_i(f,v) = d(s,v)
 *                                       of sigma(s,f) * sigma_i(f,v),
 *                          delta(s|v) = sigma(s,v) * sum over exit frontiers f with
 *                                       d(s,v)+d_i(v,f) = d(s,f) of
 *                                       sigma_i(v,f) * (I_{f in S} + delta(s|f)) / sigma(s,f)
 *                        where d_i, sigma_i are the within-part, frontier-avoiding values of Eq. 10.
 * Readings taken where the paper is silent: ordered pairs s != t (Eq. 5) halved for undirected
 * graphs on request; endpoints are not credited; unreachable pairs contribute nothing;
 * directed graphs use directed paths, a frontier is a node with an arc to or from another
 * part, and exit tables come from the reversed part subgraph; weights are integers >= 1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define INF32 INT32_MAX

/* ------------------------------------------------------------------------- graph */
typedef struct {
    int32_t n;
    int64_t *off;     /* n+1 */
    int32_t *adj;     /* arc heads */
    int32_t *wt;      /* arc weights, NULL = all 1 */
    uint64_t *mu;     /* arc multiplicities, NULL = all 1 */
} graph_t;

static void graph_free(graph_t *g) {
    free(g->off); free(g->adj); free(g->wt); free(g->mu);
    memset(g, 0, sizeof(*g));
}

/* Build out-adjacency from arcs (a[i] -> b[i], weight w[i], multiplicity mu[i]).  When
 * `both` is set every arc is also added reversed (undirected graph). */
static int graph_build(graph_t *g, int32_t n, int64_t na, const int32_t *a, const int32_t *b,
                       const int32_t *w, const uint64_t *mu, int both) {
    memset(g, 0, sizeof(*g));
    g->n = n;
    int64_t tot = both ? 2 * na : na;
    g->off = calloc((size_t)n + 1, sizeof(int64_t));
    g->adj = malloc((size_t)(tot ? tot : 1) * sizeof(int32_t));
    if (w) g->wt = malloc((size_t)(tot ? tot : 1) * sizeof(int32_t));
    if (mu) g->mu = malloc((size_t)(tot ? tot : 1) * sizeof(uint64_t));
    int64_t *fill = calloc((size_t)n + 1, sizeof(int64_t));
    if (!g->off || !g->adj || (w && !g->wt) || (mu && !g->mu) || !fill) { free(fill); graph_free(g); return ORC_ENOMEM; }
    for (int64_t i = 0; i < na; i++) {
        g->off[a[i] + 1]++;
        if (both) g->off[b[i] + 1]++;
    }
    for (int32_t v = 0; v < n; v++) g->off[v + 1] += g->off[v];
    for (int64_t i = 0; i < na; i++) {
        int64_t p = g->off[a[i]] + fill[a[i]]++;
        g->adj[p] = b[i];
        if (w) g->wt[p] = w[i];
        if (mu) g->mu[p] = mu[i];
        if (both) {
            p = g->off[b[i]] + fill[b[i]]++;
            g->adj[p] = a[i];
            if (w) g->wt[p] = w[i];
            if (mu) g->mu[p] = mu[i];
        }
    }
    free(fill);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- helpers */
static inline int64_t arc_w(const graph_t *g, int64_t p) { return g->wt ? g->wt[p] : 1; }
static inline uint64_t arc_mu(const graph_t *g, int64_t p) { return g->mu ? g->mu[p] : 1; }

static inline uint64_t add_ck(uint64_t a, uint64_t b, uint32_t *ovf) {
    uint64_t r;
    if (__builtin_add_overflow(a, b, &r)) *ovf = 1;
    return r;
}
static inline uint64_t mul_ck(uint64_t a, uint64_t b, uint32_t *ovf) {
    uint64_t r;
    if (__builtin_mul_overflow(a, b, &r)) *ovf = 1;
    return r;
}

/* Neumaier (improved Kahan) summation */
static inline void neu_add(double *s, double *c, double x) {
    double t = *s + x;
    if (fabs(*s) >= fabs(x)) *c += (*s - t) + x; else *c += (x - t) + *s;
    *s = t;
}

/* binary min-heap of (key, node) with lazy deletion */
typedef struct { int64_t key; int32_t v; } hitem;
typedef struct { hitem *a; int64_t len, cap; } heap_t;
static int heap_push(heap_t *h, int64_t key, int32_t v) {
    if (h->len == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 64;
        hitem *na = realloc(h->a, (size_t)nc * sizeof(hitem));
        if (!na) return ORC_ENOMEM;
        h->a = na; h->cap = nc;
    }
    int64_t i = h->len++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h->a[p].key <= key) break;
        h->a[i] = h->a[p]; i = p;
    }
    h->a[i].key = key; h->a[i].v = v;
    return ORC_OK;
}
static hitem heap_pop(heap_t *h) {
    hitem top = h->a[0], last = h->a[--h->len];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        int64_t mk = last.key;
        if (l < h->len && h->a[l].key < mk) { m = l; mk = h->a[l].key; }
        if (r < h->len && h->a[r].key < mk) { m = r; }
        if (m == i) break;
        h->a[i] = h->a[m]; i = m;
    }
    if (h->len) h->a[i] = last;
    return top;
}

/* ------------------------------------------------------------------------- SSSP with path counts
 * Single-source shortest paths from s over g, restricted to nodes with keep[v] != 0 (keep
 * may be NULL = all).  dist[v] (INF32 if unreachable), sigma[v] = sum over parents u of
 * sigma[u]*mu(u,v) (Eq. 2 / Eq. 11).  When `frontier` is given, a parent u only contributes
 * if it is not a frontier or is the source itself (Eq. 10, Dijkstra_SK).  order[] receives
 * the settled nodes in non-decreasing distance; returns their count, or -1 on ENOMEM.
 * Unit weights use a FIFO queue (breadth-first search), otherwise a binary heap. */
static int64_t sssp(const graph_t *g, int32_t s, const uint8_t *keep, const uint8_t *frontier,
                    int32_t *dist, uint64_t *sigma, int32_t *order, uint32_t *ovf,
                    const int32_t *part_nodes, int32_t n_part) {
    int32_t n = g->n;
    /* with keep, only the part's own nodes can be reached, so only they are reset */
    if (part_nodes) {
        for (int32_t j = 0; j < n_part; j++) { dist[part_nodes[j]] = INF32; sigma[part_nodes[j]] = 0; }
    } else {
        for (int32_t v = 0; v < n; v++) { dist[v] = INF32; sigma[v] = 0; }
    }
    dist[s] = 0; sigma[s] = 1;
    int64_t cnt = 0;
    if (!g->wt) {
        int64_t head = 0;
        order[cnt++] = s;
        while (head < cnt) {
            int32_t u = order[head++];
            int parent_ok = !frontier || !frontier[u] || u == s;
            for (int64_t p = g->off[u]; p < g->off[u + 1]; p++) {
                int32_t v = g->adj[p];
                if (keep && !keep[v]) continue;
                if (dist[v] == INF32) { dist[v] = dist[u] + 1; order[cnt++] = v; }
                if (dist[v] == dist[u] + 1 && parent_ok)
                    sigma[v] = add_ck(sigma[v], mul_ck(sigma[u], arc_mu(g, p), ovf), ovf);
            }
        }
        return cnt;
    }
    heap_t h = {0};
    uint8_t *done = calloc((size_t)(n ? n : 1), 1);
    if (!done || heap_push(&h, 0, s)) { free(done); free(h.a); return -1; }
    while (h.len) {
        hitem it = heap_pop(&h);
        int32_t u = it.v;
        if (done[u] || it.key != dist[u]) continue;
        done[u] = 1;
        order[cnt++] = u;
        int parent_ok = !frontier || !frontier[u] || u == s;
        for (int64_t p = g->off[u]; p < g->off[u + 1]; p++) {
            int32_t v = g->adj[p];
            if (keep && !keep[v]) continue;
            int64_t nd = (int64_t)dist[u] + arc_w(g, p);
            if (nd < dist[v]) {
                dist[v] = (int32_t)nd;
                sigma[v] = parent_ok ? mul_ck(sigma[u], arc_mu(g, p), ovf) : 0;
                if (heap_push(&h, nd, v)) { free(done); free(h.a); return -1; }
            } else if (nd == dist[v] && parent_ok) {
                sigma[v] = add_ck(sigma[v], mul_ck(sigma[u], arc_mu(g, p), ovf), ovf);
            }
        }
    }
    free(done); free(h.a);
    return cnt;
}

/* Reverse-order dependency accumulation (Eq. 7, and Eq. 12 with multiplicities):
 * delta[u] = sum over arcs u->v with dist[v] = dist[u] + w of
 *            mu(u,v) * sigma[u] / sigma[v] * (I_{v in S} + delta[v]). */
static void accumulate(const graph_t *g, const int32_t *order, int64_t cnt, const int32_t *dist,
                       const uint64_t *sigma, const uint8_t *in_s, double *delta) {
    for (int64_t i = 0; i < cnt; i++) delta[order[i]] = 0.0;
    for (int64_t i = cnt - 1; i >= 0; i--) {
        int32_t u = order[i];
        double acc = 0.0;
        for (int64_t p = g->off[u]; p < g->off[u + 1]; p++) {
            int32_t v = g->adj[p];
            if (dist[v] == INF32 || (int64_t)dist[v] != (int64_t)dist[u] + arc_w(g, p)) continue;
            acc += (double)arc_mu(g, p) * ((double)(in_s[v] ? 1 : 0) + delta[v]) / (double)sigma[v];
        }
        delta[u] = (double)sigma[u] * acc;
    }
}

/* ------------------------------------------------------------------------- validation */
static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static int validate(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, const uint32_t *ew,
                    int32_t directed, const int32_t *S, int32_t nS) {
    if (n < 0 || m < 0) return ORC_EINVAL;
    uint64_t wmax = 1;
    for (int64_t i = 0; i < m; i++) {
        if (eu[i] < 0 || eu[i] >= n || ev[i] < 0 || ev[i] >= n || eu[i] == ev[i]) return ORC_EINVAL;
        if (ew && ew[i] == 0) return ORC_EINVAL;
        if (ew && ew[i] > wmax) wmax = ew[i];
    }
    if (n > 1 && wmax * (uint64_t)(n - 1) >= (1ull << 31)) return ORC_EINVAL;
    int64_t *keys = malloc((size_t)(m ? m : 1) * sizeof(int64_t));
    if (!keys) return ORC_ENOMEM;
    for (int64_t i = 0; i < m; i++) {
        int64_t a = eu[i], b = ev[i];
        if (!directed && a > b) { int64_t t = a; a = b; b = t; }
        keys[i] = a * (int64_t)n + b;
    }
    qsort(keys, (size_t)m, sizeof(int64_t), cmp_i64);
    for (int64_t i = 1; i < m; i++) if (keys[i] == keys[i - 1]) { free(keys); return ORC_EINVAL; }
    free(keys);
    if (S) {
        uint8_t *seen = calloc((size_t)(n ? n : 1), 1);
        if (!seen) return ORC_ENOMEM;
        for (int32_t i = 0; i < nS; i++) {
            if (S[i] < 0 || S[i] >= n || seen[S[i]]) { free(seen); return ORC_EINVAL; }
            seen[S[i]] = 1;
        }
        free(seen);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- public: SSSP */
/* Distances and path counts from one source (Eq. 2); for parity of d and sigma. */
int orc_sssp(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, const uint32_t *ew,
             int32_t directed, int32_t src, int32_t *dist, uint64_t *sigma, uint32_t *overflow) {
    int rc = validate(n, m, eu, ev, ew, directed, NULL, 0);
    if (rc) return rc;
    if (src < 0 || src >= n) return ORC_EINVAL;
    graph_t g;
    if (graph_build(&g, n, m, eu, ev, (const int32_t *)ew, NULL, !directed)) return ORC_ENOMEM;
    int32_t *order = malloc((size_t)n * sizeof(int32_t));
    uint32_t ovf = 0;
    int64_t c = order ? sssp(&g, src, NULL, NULL, dist, sigma, order, &ovf, NULL, 0) : -1;
    free(order); graph_free(&g);
    if (overflow) *overflow = ovf;
    return c < 0 ? ORC_ENOMEM : ORC_OK;
}

/* ------------------------------------------------------------------------- public: plain Brandes */
/* Target-set betweenness (Eq. 5) by Brandes' recursion (Eq. 7).  Sources are S[0..nsrc)
 * (nsrc < 0: all of S), targets are all of S; nS == 0 means S = V.  bc[n] receives the sum
 * over the sources; with `halve` it is multiplied by 1/2 (unordered pairs, undirected). */
int orc_brandes(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, const uint32_t *ew,
                int32_t directed, const int32_t *S, int32_t nS, int32_t nsrc, int32_t halve,
                double *bc, uint32_t *overflow) {
    int rc = validate(n, m, eu, ev, ew, directed, nS ? S : NULL, nS);
    if (rc) return rc;
    graph_t g;
    if (graph_build(&g, n, m, eu, ev, (const int32_t *)ew, NULL, !directed)) return ORC_ENOMEM;
    int32_t *dist = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    uint64_t *sigma = malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    int32_t *order = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    double *delta = malloc((size_t)(n ? n : 1) * sizeof(double));
    double *comp = calloc((size_t)(n ? n : 1), sizeof(double));
    uint8_t *in_s = calloc((size_t)(n ? n : 1), 1);
    if (!dist || !sigma || !order || !delta || !comp || !in_s) { rc = ORC_ENOMEM; goto out; }
    for (int32_t v = 0; v < n; v++) bc[v] = 0.0;
    int32_t ns_all = nS ? nS : n;
    for (int32_t i = 0; i < ns_all; i++) in_s[nS ? S[i] : i] = 1;
    int32_t ns = (nsrc < 0 || nsrc > ns_all) ? ns_all : nsrc;
    uint32_t ovf = 0;
    if (ns_all >= 2) {
        for (int32_t i = 0; i < ns; i++) {
            int32_t s = nS ? S[i] : i;
            int64_t cnt = sssp(&g, s, NULL, NULL, dist, sigma, order, &ovf, NULL, 0);
            if (cnt < 0) { rc = ORC_ENOMEM; goto out; }
            accumulate(&g, order, cnt, dist, sigma, in_s, delta);
            for (int64_t j = 0; j < cnt; j++) {
                int32_t v = order[j];
                if (v != s) neu_add(&bc[v], &comp[v], delta[v]);
            }
        }
    }
    for (int32_t v = 0; v < n; v++) {
        bc[v] += comp[v];
        if (halve) bc[v] *= 0.5;
    }
    if (overflow) *overflow = ovf;
out:
    free(dist); free(sigma); free(order); free(delta); free(comp); free(in_s);
    graph_free(&g);
    return rc;
}

/* ------------------------------------------------------------------------- Brandes++ */
typedef struct {
    int32_t n, kp;              /* nodes, parts in P' */
    int32_t *partp;             /* P' label of each node */
    uint8_t *frontier;          /* F = union of F_i */
    int32_t *pstart;            /* kp+1 offsets into pnodes */
    int32_t *pnodes;            /* nodes of each part: frontiers first, then interior */
    int32_t *nf;                /* |F_i| */
    int32_t *loc;               /* local index of each node inside its part */
    int64_t *toff;              /* kp+1 offsets of the per-part tables (|F_i| x |V_i|) */
    int32_t *td, *tdr;          /* d_i(f,v) and d_i(v,f) */
    uint64_t *ts, *tsr;         /* sigma_i(f,v) and sigma_i(v,f) (frontier-avoiding) */
    int32_t nsk;                /* skeleton nodes */
    int32_t *skid;              /* skeleton id of each node (-1 if not a frontier) */
    int32_t *sknode;            /* node of each skeleton id */
    graph_t sk;                 /* skeleton arcs with <weight, multiplicity> */
    int64_t sk_edges;           /* |E_sk| (edges for undirected, arcs for directed) */
    int32_t lcs;                /* largest part of P' */
} skel_t;

static void skel_free(skel_t *k) {
    free(k->partp); free(k->frontier); free(k->pstart); free(k->pnodes); free(k->nf); free(k->loc);
    free(k->toff); free(k->td); free(k->ts);
    if (k->tdr != k->td) free(k->tdr);
    if (k->tsr != k->ts) free(k->tsr);
    free(k->skid); free(k->sknode);
    graph_free(&k->sk);
    memset(k, 0, sizeof(*k));
}

/* Build_SK (Alg. 2) on the partition P' of Alg. 1: targets become singleton parts, frontiers
 * are found by one scan of the arcs, Dijkstra_SK runs from every frontier of every part
 * inside that part (Eq. 10), and the skeleton gets the cross arcs R with <w, 1> and the
 * clique arcs X_i with <d_i(f,q), sigma_i(f,q)> for sigma_i > 0. */
static int build_sk(skel_t *K, int32_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                    const uint32_t *ew, int32_t directed, const int32_t *S, int32_t nS,
                    const int32_t *part, int32_t k, uint32_t *ovf) {
    memset(K, 0, sizeof(*K));
    int rc = ORC_OK;
    K->n = n;
    K->kp = k + nS;
    int32_t kp = K->kp;
    K->partp = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    K->frontier = calloc((size_t)(n ? n : 1), 1);
    K->pstart = calloc((size_t)kp + 1, sizeof(int32_t));
    K->pnodes = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    K->nf = calloc((size_t)(kp ? kp : 1), sizeof(int32_t));
    K->loc = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    K->toff = calloc((size_t)kp + 1, sizeof(int64_t));
    K->skid = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    K->sknode = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    if (!K->partp || !K->frontier || !K->pstart || !K->pnodes || !K->nf || !K->loc || !K->toff ||
        !K->skid || !K->sknode) return ORC_ENOMEM;
    /* P' = {P_i \ S} u {{s} : s in S} */
    for (int32_t v = 0; v < n; v++) K->partp[v] = part[v];
    for (int32_t j = 0; j < nS; j++) K->partp[S[j]] = k + j;
    /* frontiers: an edge (arc in either direction) to another part */
    for (int64_t i = 0; i < m; i++)
        if (K->partp[eu[i]] != K->partp[ev[i]]) { K->frontier[eu[i]] = 1; K->frontier[ev[i]] = 1; }
    /* group nodes by part, frontiers first */
    int32_t *cnt = calloc((size_t)kp + 1, sizeof(int32_t));
    if (!cnt) return ORC_ENOMEM;
    for (int32_t v = 0; v < n; v++) { K->pstart[K->partp[v] + 1]++; if (K->frontier[v]) K->nf[K->partp[v]]++; }
    for (int32_t i = 0; i < kp; i++) K->pstart[i + 1] += K->pstart[i];
    for (int32_t pass = 0; pass < 2; pass++)
        for (int32_t v = 0; v < n; v++) {
            if ((pass == 0) != (K->frontier[v] != 0)) continue;
            int32_t i = K->partp[v];
            K->loc[v] = cnt[i];
            K->pnodes[K->pstart[i] + cnt[i]++] = v;
        }
    free(cnt);
    K->lcs = 0;
    for (int32_t i = 0; i < kp; i++) {
        int32_t sz = K->pstart[i + 1] - K->pstart[i];
        if (sz > K->lcs) K->lcs = sz;
        K->toff[i + 1] = K->toff[i] + (int64_t)K->nf[i] * sz;
    }
    int64_t tsz = K->toff[kp];
    K->td = malloc((size_t)(tsz ? tsz : 1) * sizeof(int32_t));
    K->ts = malloc((size_t)(tsz ? tsz : 1) * sizeof(uint64_t));
    if (directed) {
        K->tdr = malloc((size_t)(tsz ? tsz : 1) * sizeof(int32_t));
        K->tsr = malloc((size_t)(tsz ? tsz : 1) * sizeof(uint64_t));
    } else { K->tdr = K->td; K->tsr = K->ts; }
    if (!K->td || !K->ts || !K->tdr || !K->tsr) return ORC_ENOMEM;

    /* Dijkstra_SK in every part, from every frontier, on G_i (and on reversed G_i) */
    graph_t g, gr;
    if (graph_build(&g, n, m, eu, ev, (const int32_t *)ew, NULL, !directed)) return ORC_ENOMEM;
    if (directed) {
        if (graph_build(&gr, n, m, ev, eu, (const int32_t *)ew, NULL, 0)) { graph_free(&g); return ORC_ENOMEM; }
    }
    uint8_t *keep = calloc((size_t)(n ? n : 1), 1);
    int32_t *dist = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    uint64_t *sig = malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    int32_t *order = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    if (!keep || !dist || !sig || !order) { rc = ORC_ENOMEM; goto done; }
    for (int32_t v = 0; v < n; v++) { dist[v] = INF32; sig[v] = 0; }
    for (int32_t i = 0; i < kp; i++) {
        int32_t a = K->pstart[i], b = K->pstart[i + 1], sz = b - a;
        if (K->nf[i] == 0) continue;
        for (int32_t j = a; j < b; j++) keep[K->pnodes[j]] = 1;
        for (int32_t dir = 0; dir < (directed ? 2 : 1); dir++) {
            const graph_t *gg = dir ? &gr : &g;
            int32_t *T = dir ? K->tdr : K->td;
            uint64_t *TS = dir ? K->tsr : K->ts;
            for (int32_t fi = 0; fi < K->nf[i]; fi++) {
                int32_t f = K->pnodes[a + fi];
                if (sssp(gg, f, keep, K->frontier, dist, sig, order, ovf, K->pnodes + a, sz) < 0) {
                    rc = ORC_ENOMEM; goto done;
                }
                for (int32_t j = 0; j < sz; j++) {
                    int32_t v = K->pnodes[a + j];
                    T[K->toff[i] + (int64_t)fi * sz + j] = dist[v];
                    TS[K->toff[i] + (int64_t)fi * sz + j] = sig[v];
                }
            }
        }
        for (int32_t j = a; j < b; j++) keep[K->pnodes[j]] = 0;
    }
    /* skeleton nodes = union of frontiers; arcs = R (cross) u X_i (cliques) */
    K->nsk = 0;
    for (int32_t v = 0; v < n; v++) {
        K->skid[v] = -1;
        if (K->frontier[v]) { K->skid[v] = K->nsk; K->sknode[K->nsk++] = v; }
    }
    int64_t narcs = 0;
    for (int64_t i = 0; i < m; i++) if (K->partp[eu[i]] != K->partp[ev[i]]) narcs += directed ? 1 : 2;
    for (int32_t i = 0; i < kp; i++) narcs += (int64_t)K->nf[i] * (K->nf[i] - 1);
    int32_t *A = malloc((size_t)(narcs ? narcs : 1) * sizeof(int32_t));
    int32_t *B = malloc((size_t)(narcs ? narcs : 1) * sizeof(int32_t));
    int32_t *W = malloc((size_t)(narcs ? narcs : 1) * sizeof(int32_t));
    uint64_t *MU = malloc((size_t)(narcs ? narcs : 1) * sizeof(uint64_t));
    if (!A || !B || !W || !MU) { free(A); free(B); free(W); free(MU); rc = ORC_ENOMEM; goto done; }
    int64_t e = 0, und = 0;
    for (int64_t i = 0; i < m; i++) {
        if (K->partp[eu[i]] == K->partp[ev[i]]) continue;
        int32_t w = ew ? (int32_t)ew[i] : 1;
        A[e] = K->skid[eu[i]]; B[e] = K->skid[ev[i]]; W[e] = w; MU[e] = 1; e++;
        if (!directed) { A[e] = K->skid[ev[i]]; B[e] = K->skid[eu[i]]; W[e] = w; MU[e] = 1; e++; }
        und++;
    }
    for (int32_t i = 0; i < kp; i++) {
        int32_t a = K->pstart[i], sz = K->pstart[i + 1] - a;
        for (int32_t fi = 0; fi < K->nf[i]; fi++)
            for (int32_t qi = 0; qi < K->nf[i]; qi++) {
                if (fi == qi) continue;
                int64_t t = K->toff[i] + (int64_t)fi * sz + qi;
                if (K->td[t] == INF32 || K->ts[t] == 0) continue;
                A[e] = K->skid[K->pnodes[a + fi]]; B[e] = K->skid[K->pnodes[a + qi]];
                W[e] = K->td[t]; MU[e] = K->ts[t]; e++;
                if (directed || fi < qi) und++;
            }
    }
    K->sk_edges = und;
    rc = graph_build(&K->sk, K->nsk, e, A, B, W, MU, 0);
    free(A); free(B); free(W); free(MU);
done:
    free(keep); free(dist); free(sig); free(order);
    graph_free(&g);
    if (directed) graph_free(&gr);
    return rc;
}

/* Brandes++ (Alg. 1): Build_SK, then Brandes_SK from every target (Eq. 11, 12), then the
 * Centrality step for the non-frontier nodes of every part (Eq. 13 as read above).
 * Sources are S[0..nsrc) (nsrc < 0: all), targets are all of S; nS must be >= 1 (S = V is
 * passed explicitly).  stats (may be NULL) = {N, M, k', LCS}. */
int orc_brandes_pp(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, const uint32_t *ew,
                   int32_t directed, const int32_t *S, int32_t nS, int32_t nsrc, const int32_t *part,
                   int32_t k, int32_t halve, double *bc, uint32_t *overflow, int64_t *stats) {
    int rc = validate(n, m, eu, ev, ew, directed, S, nS);
    if (rc) return rc;
    if (k < 0) return ORC_EINVAL;
    for (int32_t v = 0; v < n; v++) if (part[v] < 0 || part[v] >= k) return ORC_EINVAL;
    for (int32_t v = 0; v < n; v++) bc[v] = 0.0;
    uint32_t ovf = 0;
    skel_t K;
    rc = build_sk(&K, n, m, eu, ev, ew, directed, S, nS, part, k, &ovf);
    if (rc) { skel_free(&K); return rc; }
    if (stats) {
        int32_t kp_nonempty = 0;
        for (int32_t i = 0; i < K.kp; i++) kp_nonempty += K.pstart[i + 1] > K.pstart[i];
        stats[0] = K.nsk; stats[1] = K.sk_edges; stats[2] = kp_nonempty; stats[3] = K.lcs;
    }
    int32_t N = K.nsk;
    double *comp = calloc((size_t)(n ? n : 1), sizeof(double));
    uint8_t *in_s = calloc((size_t)(n ? n : 1), 1);
    uint8_t *sk_in_s = calloc((size_t)(N ? N : 1), 1);
    int32_t *dist = malloc((size_t)(N ? N : 1) * sizeof(int32_t));
    uint64_t *sig = malloc((size_t)(N ? N : 1) * sizeof(uint64_t));
    int32_t *order = malloc((size_t)(N ? N : 1) * sizeof(int32_t));
    double *delta = malloc((size_t)(N ? N : 1) * sizeof(double));
    if (!comp || !in_s || !sk_in_s || !dist || !sig || !order || !delta) { rc = ORC_ENOMEM; goto out; }
    for (int32_t j = 0; j < nS; j++) {
        in_s[S[j]] = 1;
        if (K.skid[S[j]] >= 0) sk_in_s[K.skid[S[j]]] = 1;
    }
    int32_t ns = (nsrc < 0 || nsrc > nS) ? nS : nsrc;
    if (nS >= 2) {
        for (int32_t j = 0; j < ns; j++) {
            int32_t s = S[j], ss = K.skid[s];
            if (ss < 0) continue;               /* isolated target: no paths */
            /* Brandes_SK: SSSP with multiplicities (Eq. 11), dependencies (Eq. 12) */
            int64_t cnt = sssp(&K.sk, ss, NULL, NULL, dist, sig, order, &ovf, NULL, 0);
            if (cnt < 0) { rc = ORC_ENOMEM; goto out; }
            accumulate(&K.sk, order, cnt, dist, sig, sk_in_s, delta);
            for (int64_t x = 0; x < cnt; x++) {
                int32_t u = order[x];
                if (u != ss) neu_add(&bc[K.sknode[u]], &comp[K.sknode[u]], delta[u]);
            }
            for (int32_t v = 0; v < N; v++) if (dist[v] == INF32) delta[v] = 0.0;
            /* Centrality: non-frontier nodes of every part (Eq. 13) */
            for (int32_t i = 0; i < K.kp; i++) {
                int32_t a = K.pstart[i], sz = K.pstart[i + 1] - a, nf = K.nf[i];
                for (int32_t vi = nf; vi < sz; vi++) {
                    int32_t v = K.pnodes[a + vi];
                    int64_t dv = INF32;
                    uint64_t sv = 0;
                    for (int32_t fi = 0; fi < nf; fi++) {      /* entry frontiers */
                        int32_t f = K.skid[K.pnodes[a + fi]];
                        int64_t t = K.toff[i] + (int64_t)fi * sz + vi;
                        if (dist[f] == INF32 || K.td[t] == INF32) continue;
                        int64_t c = (int64_t)dist[f] + K.td[t];
                        if (c < dv) { dv = c; sv = 0; }
                        if (c == dv) sv = add_ck(sv, mul_ck(sig[f], K.ts[t], &ovf), &ovf);
                    }
                    if (sv == 0) continue;
                    double acc = 0.0;
                    for (int32_t fi = 0; fi < nf; fi++) {      /* exit frontiers */
                        int32_t f = K.skid[K.pnodes[a + fi]];
                        int64_t t = K.toff[i] + (int64_t)fi * sz + vi;
                        if (dist[f] == INF32 || K.tdr[t] == INF32 || K.tsr[t] == 0) continue;
                        if (dv + K.tdr[t] != (int64_t)dist[f]) continue;
                        acc += (double)K.tsr[t] * ((double)(sk_in_s[f] ? 1 : 0) + delta[f]) / (double)sig[f];
                    }
                    neu_add(&bc[v], &comp[v], (double)sv * acc);
                }
            }
        }
    }
    for (int32_t v = 0; v < n; v++) {
        bc[v] += comp[v];
        if (halve) bc[v] *= 0.5;
    }
    if (overflow) *overflow = ovf;
out:
    free(comp); free(in_s); free(sk_in_s); free(dist); free(sig); free(order); free(delta);
    skel_free(&K);
    return rc;
}

/* The skeleton of Build_SK for inspection: skeleton nodes (original ids, in increasing id
 * order) and its arcs with <weight, multiplicity> (undirected edges appear as two arcs).
 * Returns ORC_EINVAL if the caller's capacities are too small; counts are always written. */
int orc_skeleton(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, const uint32_t *ew,
                 int32_t directed, const int32_t *S, int32_t nS, const int32_t *part, int32_t k,
                 int32_t *sk_nodes, int32_t *n_sk, int64_t cap_arcs, int32_t *au, int32_t *av,
                 int32_t *aw, uint64_t *amu, int64_t *n_arcs, uint32_t *overflow) {
    int rc = validate(n, m, eu, ev, ew, directed, S, nS);
    if (rc) return rc;
    for (int32_t v = 0; v < n; v++) if (part[v] < 0 || part[v] >= k) return ORC_EINVAL;
    uint32_t ovf = 0;
    skel_t K;
    rc = build_sk(&K, n, m, eu, ev, ew, directed, S, nS, part, k, &ovf);
    if (rc) { skel_free(&K); return rc; }
    *n_sk = K.nsk;
    for (int32_t i = 0; i < K.nsk; i++) sk_nodes[i] = K.sknode[i];
    int64_t na = K.sk.off[K.nsk];
    *n_arcs = na;
    if (na > cap_arcs) { skel_free(&K); return ORC_EINVAL; }
    int64_t e = 0;
    for (int32_t u = 0; u < K.nsk; u++)
        for (int64_t p = K.sk.off[u]; p < K.sk.off[u + 1]; p++, e++) {
            au[e] = K.sknode[u]; av[e] = K.sknode[K.sk.adj[p]];
            aw[e] = K.sk.wt[p]; amu[e] = K.sk.mu[p];
        }
    if (overflow) *overflow = ovf;
    skel_free(&K);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- public: path lengths */
/* Sum over sources s = src[0..nsrc) and reachable t != s of (d(s,t) - 1), unit weights:
 * the right-hand side of the invariant sum_v C(v) = sum_{s != t} (d(s,t) - 1) of Eq. 1
 * (every shortest s-t path has d(s,t) - 1 interior nodes, each credited 1/sigma(s,t) per
 * path).  Breadth-first search only; no path counts. */
int orc_distance_sum(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, int32_t directed,
                     const int32_t *src, int32_t nsrc, int64_t *out) {
    if (n < 0 || m < 0 || !out) return ORC_EINVAL;
    graph_t g;
    if (graph_build(&g, n, m, eu, ev, NULL, NULL, !directed)) return ORC_ENOMEM;
    int32_t *dist = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    int32_t *queue = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    if (!dist || !queue) { free(dist); free(queue); graph_free(&g); return ORC_ENOMEM; }
    int64_t tot = 0;
    for (int32_t i = 0; i < nsrc; i++) {
        int32_t s = src[i];
        if (s < 0 || s >= n) { free(dist); free(queue); graph_free(&g); return ORC_EINVAL; }
        for (int32_t v = 0; v < n; v++) dist[v] = INF32;
        int64_t head = 0, cnt = 0;
        dist[s] = 0; queue[cnt++] = s;
        while (head < cnt) {
            int32_t u = queue[head++];
            if (u != s) tot += dist[u] - 1;
            for (int64_t p = g.off[u]; p < g.off[u + 1]; p++)
                if (dist[g.adj[p]] == INF32) { dist[g.adj[p]] = dist[u] + 1; queue[cnt++] = g.adj[p]; }
        }
    }
    *out = tot;
    free(dist); free(queue); graph_free(&g);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- public: sources -> destinations */
/* Plain Brandes with separate source and destination sets: bc[v] = sum over s in src, t in dst,
 * s != t, of sigma(s,t|v)/sigma(s,t) (Eq. 5 with the pair set S_sc x S_dest of Sec. 5; Eq. 7 with
 * the indicator of S_dest).  Halved on request. */
int orc_brandes_st(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, const uint32_t *ew,
                   int32_t directed, const int32_t *src, int32_t nsrc, const int32_t *dst, int32_t ndst,
                   int32_t halve, double *bc, uint32_t *overflow) {
    int rc = validate(n, m, eu, ev, ew, directed, src, nsrc);
    if (rc) return rc;
    rc = validate(n, 0, eu, ev, ew, directed, dst, ndst);
    if (rc) return rc;
    graph_t g;
    if (graph_build(&g, n, m, eu, ev, (const int32_t *)ew, NULL, !directed)) return ORC_ENOMEM;
    int32_t *dist = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    uint64_t *sigma = malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    int32_t *order = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    double *delta = malloc((size_t)(n ? n : 1) * sizeof(double));
    double *comp = calloc((size_t)(n ? n : 1), sizeof(double));
    uint8_t *in_d = calloc((size_t)(n ? n : 1), 1);
    if (!dist || !sigma || !order || !delta || !comp || !in_d) { rc = ORC_ENOMEM; goto out; }
    for (int32_t v = 0; v < n; v++) bc[v] = 0.0;
    for (int32_t i = 0; i < ndst; i++) in_d[dst[i]] = 1;
    uint32_t ovf = 0;
    for (int32_t i = 0; i < nsrc; i++) {
        int32_t s = src[i];
        int64_t cnt = sssp(&g, s, NULL, NULL, dist, sigma, order, &ovf, NULL, 0);
        if (cnt < 0) { rc = ORC_ENOMEM; goto out; }
        accumulate(&g, order, cnt, dist, sigma, in_d, delta);
        for (int64_t j = 0; j < cnt; j++) {
            int32_t v = order[j];
            if (v != s) neu_add(&bc[v], &comp[v], delta[v]);
        }
    }
    for (int32_t v = 0; v < n; v++) {
        bc[v] += comp[v];
        if (halve) bc[v] *= 0.5;
    }
    if (overflow) *overflow = ovf;
out:
    free(dist); free(sigma); free(order); free(delta); free(comp); free(in_d);
    graph_free(&g);
    return rc;
}

/* ------------------------------------------------------------------------- partition */
/* Label propagation, the partition input of Brandes++ for callers without one (not from the
 * paper, whose partitions come from external tools; Brandes++ is exact for any partition).
 * Deterministic rule (Raghavan, Albert and Kumara 2007, made deterministic):
 *   labels start as the node ids; half-step t updates the nodes v with v mod 2 == t mod 2 from
 *   the labels of half-step t-1: v takes the label carried by most of its neighbours (each arc
 *   counts for both of its endpoints, so a directed graph counts in- and out-arcs), keeps its
 *   own label when that one is among the most frequent, otherwise takes the smallest most
 *   frequent label; nodes without neighbours keep theirs.  Stop after a round of two
 *   half-steps without a change, or after max_rounds rounds.  part_out numbers the labels in
 *   use 0..k-1 in increasing order.  PARITY: this is a heuristic defined here, not by the
 *   paper; its pins are hand-derived small cases and properties (see the tests). */
static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int orc_label_propagation(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, int32_t directed,
                          int32_t max_rounds, int32_t *part_out, int32_t *k_out, int32_t *rounds_out) {
    (void)directed;   /* both orientations of every arc are neighbours either way */
    if (n < 0 || m < 0 || max_rounds < 1) return ORC_EINVAL;
    graph_t g;
    int rc = graph_build(&g, n, m, eu, ev, NULL, NULL, 1);
    if (rc) return rc;
    int32_t *lab = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    int32_t *nxt = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    int32_t maxdeg = 0;
    for (int32_t v = 0; v < n; v++)
        if (g.off[v + 1] - g.off[v] > maxdeg) maxdeg = (int32_t)(g.off[v + 1] - g.off[v]);
    int32_t *tmp = malloc((size_t)(maxdeg ? maxdeg : 1) * sizeof(int32_t));
    if (!lab || !nxt || !tmp) { free(lab); free(nxt); free(tmp); graph_free(&g); return ORC_ENOMEM; }
    for (int32_t v = 0; v < n; v++) lab[v] = v;
    int32_t rounds = 0;
    for (int32_t r = 0; r < max_rounds; r++) {
        int64_t changes = 0;
        for (int parity = 0; parity < 2; parity++) {
            memcpy(nxt, lab, (size_t)n * sizeof(int32_t));
            for (int32_t v = parity; v < n; v += 2) {
                const int64_t deg = g.off[v + 1] - g.off[v];
                if (deg == 0) continue;
                for (int64_t i = 0; i < deg; i++) tmp[i] = lab[g.adj[g.off[v] + i]];
                qsort(tmp, (size_t)deg, sizeof(int32_t), cmp_i32);
                int64_t best_cnt = 0, cur_cnt = 0;
                int32_t best_lab = 0;
                for (int64_t i = 0; i < deg;) {
                    int64_t j = i;
                    while (j < deg && tmp[j] == tmp[i]) j++;
                    if (j - i > best_cnt) { best_cnt = j - i; best_lab = tmp[i]; }   /* ascending: ties keep the smaller */
                    if (tmp[i] == lab[v]) cur_cnt = j - i;
                    i = j;
                }
                nxt[v] = cur_cnt == best_cnt ? lab[v] : best_lab;
                changes += nxt[v] != lab[v];
            }
            memcpy(lab, nxt, (size_t)n * sizeof(int32_t));
        }
        rounds++;
        if (changes == 0) break;
    }
    /* number the labels in use in increasing order */
    int32_t *rank = calloc((size_t)(n ? n : 1), sizeof(int32_t));
    if (!rank) { free(lab); free(nxt); free(tmp); graph_free(&g); return ORC_ENOMEM; }
    for (int32_t v = 0; v < n; v++) rank[lab[v]] = 1;
    int32_t k = 0;
    for (int32_t l = 0; l < n; l++) {
        const int32_t used = rank[l];
        rank[l] = k;
        k += used;
    }
    for (int32_t v = 0; v < n; v++) part_out[v] = rank[lab[v]];
    *k_out = k;
    if (rounds_out) *rounds_out = rounds;
    free(rank); free(lab); free(nxt); free(tmp);
    graph_free(&g);
    return ORC_OK;
}
