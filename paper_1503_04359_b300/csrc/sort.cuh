#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dobfs {

// Sorts n uint64 keys by their low `nbits` bits (LSD, stable), ping-ponging
// between a and b (each n keys). *result receives whichever of a, b holds
// the sorted keys. Synchronises `s` before returning.
int radix_sort_u64(uint64_t* a, uint64_t* b, int64_t n, int nbits, cudaStream_t s, uint64_t** result);

}  // namespace dobfs
