// CSR construction, validation, transposition and target-set checks.
#pragma once
#include "common.cuh"

namespace bcpp {

// keys[i] = tail * n + head, vals[i] = weight (2 arcs per undirected edge); flags input errors
void csr_expand(int32_t n, int64_t m, const int32_t* eu, const int32_t* ev, const uint32_t* ew, int directed,
                uint64_t* keys, uint32_t* vals, uint32_t* flags, cudaStream_t st);
// from sorted keys: col, weights, row_ptr; flags repeated arcs
void csr_finish(const uint64_t* keys, const uint32_t* vals, int64_t na, int32_t n, int64_t* rp, int32_t* col,
                uint32_t* w_out, uint32_t* flags, cudaStream_t st);
void csr_check(int32_t n, int64_t na, const int64_t* rp, const int32_t* col, const uint32_t* w, int directed,
               uint32_t* flags, unsigned long long* wmax, cudaStream_t st, const int64_t* node_off = nullptr,
               int32_t ngraphs = 0);
// graph-local heads of a disjoint union (flags arcs that leave their graph)
void csr_localize(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* node_off, int32_t ngraphs,
                  int32_t* lcol, uint32_t* flags, cudaStream_t st);
void targets_check(const int32_t* S, int32_t nS, int32_t n, uint8_t* in_s, uint32_t* cnt, uint32_t* flags,
                   cudaStream_t st);
void csr_transpose_count(int32_t n, const int64_t* rp, const int32_t* col, int64_t* counts, cudaStream_t st);
void csr_transpose_fill(int32_t n, const int64_t* rp, const int32_t* col, const uint32_t* w, int64_t* cursor,
                        int32_t* tcol, uint32_t* tw, cudaStream_t st);

}  // namespace bcpp
