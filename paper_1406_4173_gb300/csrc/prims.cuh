// Device primitives written for this library: exclusive scan and a stable LSD radix sort.
#pragma once
#include "common.cuh"

namespace bcpp {

struct Ctx;

// out[i] = sum_{j<i} in[j] (int64 result), *total_dev (device, may be null) = sum of all.
// in and out may alias.  tmp needs scan_tmp_elems(n) int64 elements.
int64_t scan_tmp_elems(int64_t n);
template <typename TI>
void exclusive_scan(const TI* in, int64_t* out, int64_t n, int64_t* total_dev, int64_t* tmp,
                    cudaStream_t st, int64_t& launches);

// Stable ascending sort of (keys, vals) by the low `bits` bits of the key.  The result lands
// in (keys, vals); kbuf/vbuf are scratch of n elements, hist needs radix_hist_elems(n).
int64_t radix_hist_elems(int64_t n);
void radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* kbuf, uint32_t* vbuf, int64_t n,
                      int bits, int64_t* hist, int64_t* scan_tmp, cudaStream_t st, int64_t& launches);

}  // namespace bcpp
