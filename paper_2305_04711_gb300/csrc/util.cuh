// util.cuh -- small device primitives used at set-up time: an exclusive scan,
// a bitonic key/value sort and a brick hash table (open addressing).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define CPM_HASH_EMPTY 0xFFFFFFFFFFFFFFFFull

__host__ __device__ inline uint64_t cpm_hmix(uint64_t k) {
  k ^= k >> 33; k *= 0xff51afd7ed558ccdULL; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ULL; k ^= k >> 33;
  return k;
}

// insert key; returns the slot and sets *fresh if this call inserted it; -1 if full
__device__ inline int64_t cpm_hash_insert(unsigned long long *keys, int64_t cap, uint64_t key, bool *fresh) {
  uint64_t mask = (uint64_t)cap - 1, p = cpm_hmix(key) & mask;
  for (int64_t probe = 0; probe < cap; ++probe) {
    unsigned long long prev = atomicCAS(keys + p, (unsigned long long)CPM_HASH_EMPTY, (unsigned long long)key);
    if (prev == CPM_HASH_EMPTY) { *fresh = true; return (int64_t)p; }
    if (prev == key) { *fresh = false; return (int64_t)p; }
    p = (p + 1) & mask;
  }
  *fresh = false;
  return -1;
}

__device__ inline int64_t cpm_hash_find(const unsigned long long *keys, int64_t cap, uint64_t key) {
  uint64_t mask = (uint64_t)cap - 1, p = cpm_hmix(key) & mask;
  for (int64_t probe = 0; probe < cap; ++probe) {
    unsigned long long k = keys[p];
    if (k == key) return (int64_t)p;
    if (k == CPM_HASH_EMPTY) return -1;
    p = (p + 1) & mask;
  }
  return -1;
}

// exclusive scan of n int32 values (in place allowed: out may equal in);
// total written to *d_total if non-null.  Uses temporary device memory.
cudaError_t cpm_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, int32_t *d_total, cudaStream_t s);
// ascending sort of (key, value) pairs, n arbitrary (internally padded)
cudaError_t cpm_sort_pairs(int64_t *keys, int32_t *vals, int64_t n, cudaStream_t s);
