// Build_SK device steps (Sec. 3-4, Alg. 2), the Centrality step (Eq. 13) and the final
// combination of per-slot partial betweenness.
#pragma once
#include "common.cuh"

namespace bcpp {

// P' (Alg. 1): partp[v] = part[v], then partp[S[j]] = k + j.  Flags part values outside [0,k).
void sk_partition(int32_t n, const int32_t* part, int32_t k, const int32_t* S, int32_t nS, int32_t* partp,
                  uint32_t* flags, cudaStream_t st);
// frontier flags: an arc (either direction) whose ends lie in different parts of P'
void sk_frontiers(int32_t n, const int64_t* rp, const int32_t* col, const int32_t* partp, uint8_t* fr,
                  cudaStream_t st);
// grouping keys: 2 * partp[v] + (v is not a frontier); vals = v
void sk_group_keys(int32_t n, const int32_t* partp, const uint8_t* fr, uint64_t* keys, uint32_t* vals,
                   cudaStream_t st);
// from the sorted keys: pstart[kp+1] (first position of each part), nf[kp] (frontiers per part)
void sk_segments(const uint64_t* keys, int32_t n, int32_t kp, int32_t* pstart, int32_t* nf, cudaStream_t st);
// loc[v] (local index within its part), skid[v] / sknode[] (skeleton ids, part-major)
void sk_local_ids(int32_t n, const uint32_t* pnodes, const int32_t* partp, const int32_t* pstart,
                  const int32_t* nf, const int32_t* skbase, int32_t* loc, int32_t* skid, int32_t* sknode,
                  cudaStream_t st);
// part-local CSR in grouped order: count (lrp[j] = arcs of pnodes[j] inside its part) then fill
void sk_local_count(int32_t n, const uint32_t* pnodes, const int64_t* rp, const int32_t* col,
                    const int32_t* partp, int64_t* cnt, cudaStream_t st);
void sk_local_fill(int32_t n, const uint32_t* pnodes, const int64_t* rp, const int32_t* col, const uint32_t* w,
                   const int32_t* partp, const int32_t* loc, const int64_t* lrp, int32_t* lcol, int32_t* lw,
                   cudaStream_t st);

// skeleton arcs of every skeleton node: cross arcs R with <w, 1> and clique arcs X_i with
// <d_i(f,q), sigma_i(f,q)> read from the exit tables (row f); zero multiplicities dropped.
struct SkTables {
    const int32_t* pstart;   // [kp+1]
    const int32_t* nf;       // [kp]
    const int64_t* toff;     // [kp] table offset of each part
    const int32_t* tdr;      // exit tables: tdr[toff + v*nf + f] = d_i(v -> f)
    const uint64_t* tsr;
    const int32_t* td;       // entry tables: td[toff + v*nf + f] = d_i(f -> v)
    const uint64_t* ts;
};
void sk_arcs_count(int32_t N, const int32_t* sknode, const int64_t* rp, const int32_t* col, const int32_t* partp,
                   const int32_t* loc, SkTables T, int64_t* cnt, cudaStream_t st);
void sk_arcs_fill(int32_t N, const int32_t* sknode, const int64_t* rp, const int32_t* col, const uint32_t* w,
                  const int32_t* partp, const int32_t* loc, const int32_t* skid, SkTables T, const int64_t* skrp,
                  int32_t* skcol, int32_t* skw, uint64_t* skmu, unsigned long long* maxes, cudaStream_t st);
// skeleton transpose with multiplicities (directed graphs)
void sk_transpose(int32_t N, const int64_t* rp, const int32_t* col, const int32_t* w, const uint64_t* mu,
                  int64_t* cursor, int32_t* tcol, int32_t* tw, uint64_t* tmu, int pass, cudaStream_t st);
// gather: out[x] = in_s[sknode[x]]
void sk_gather_flags(int32_t N, const int32_t* sknode, const uint8_t* in_s, uint8_t* out, cudaStream_t st);
// out[j] = skeleton id of target S[j], or -1 when it is no skeleton node (isolated)
void sk_target_ids(const int32_t* S, int32_t nS, const int32_t* skid, int32_t* out, cudaStream_t st);

// Centrality (Eq. 13) for the slots of one Brandes_SK chunk.
struct CentralityUnit { int32_t part; int32_t v0; int32_t v1; int32_t pad; };
// h16: every finite table distance is at most CT_H16_MAX (the 16-bit distance path may run)
constexpr uint32_t CT_H16_MAX = 1023;
void centrality_launch(bool fp32_delta, bool h16, const CentralityUnit* units, int nunits, int nslots, SkTables T,
                       const uint32_t* pnodes, const int32_t* skbase, const int32_t* d, const uint64_t* sg,
                       const void* dl, int64_t cap_n, double* bc_sum, double* bc_cmp, int64_t cap_bc,
                       uint32_t* flags, cudaStream_t st);

// bc_out[v] = scale * sum over slots of (bc_sum + bc_cmp), Neumaier over slots
void combine_launch(const double* bc_sum, const double* bc_cmp, int nslots, int64_t cap_bc, int64_t n, double scale,
                    double* bc_out, cudaStream_t st);

}  // namespace bcpp
