// Label-propagation partition kernels (see partition.cu for the rule).
#pragma once
#include "common.cuh"

namespace bcpp {

void lp_init(int32_t n, int32_t* lab, int32_t* used, cudaStream_t st);
// one half-step: nodes with v mod 2 == parity update from lin into lout, the others copy;
// changes (device) is incremented per changed label
void lp_step(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* irp, const int32_t* icol,
             const int32_t* lin, int32_t* lout, int parity, unsigned int* changes, cudaStream_t st);
void lp_mark(int32_t n, const int32_t* lab, int32_t* used, cudaStream_t st);
void lp_number(int32_t n, const int32_t* lab, const int64_t* rank, int32_t* part, cudaStream_t st);

}  // namespace bcpp
