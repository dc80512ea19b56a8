// Radix sort and scans used by the deterministic scatter (detsort.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gde {

// scratch bytes for radix_sort / exclusive_scan_i64 of n elements
size_t sort_scratch_bytes(int64_t n);
size_t scan_scratch_bytes(int64_t n);

// Stable ascending sort of n 32-bit keys (only the low key_bits bits are compared) with their
// values (vals may be NULL).  Returns 0 if the result is in keys/vals, 1 if in the temporaries.
template <typename V>
int radix_sort(uint32_t *keys, V *vals, uint32_t *keys_tmp, V *vals_tmp, int64_t n, int key_bits,
               void *scratch, cudaStream_t s);

// out[i] = sum in[0..i); *total (device) = sum of all n
void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total, int64_t *scratch,
                        cudaStream_t s);

}  // namespace gde
