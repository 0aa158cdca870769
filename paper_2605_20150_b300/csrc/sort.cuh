// Device-wide exclusive scan and stable LSD radix sort (u32 keys, u32 values).
#pragma once
#include "common.cuh"

namespace tgs {

// Scratch sizes (bytes) for n elements.
size_t scan_scratch_bytes(uint64_t n);
size_t radix_scratch_bytes(uint64_t n);

// out[i] = sum_{j<i} in[j]; *total_dev (device, may be null) = sum of all.
// in and out may alias.
void exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint32_t* total_dev, uint64_t n, void* scratch,
                        cudaStream_t s);

// Stable sort of (keys, vals) by key bits [0, bits).  The result ends in
// keys/vals; keys_alt/vals_alt are same-sized ping-pong buffers.
void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, uint64_t n,
                      int bits, void* scratch, cudaStream_t s);

}  // namespace tgs
