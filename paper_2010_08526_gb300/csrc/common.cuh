// Shared device helpers for the sm_103a SpGEMM kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define SPG_FULL 0xffffffffu

namespace spg {

// Hash-table key for an empty slot. Row indices are < 2^31 - 1, so every
// real key differs from it.
constexpr uint32_t kEmpty = 0xffffffffu;

// Error bits recorded by kernels in the plan's device error word.
enum : int {
    kErrProbe = 1,        // a hash probe sequence ran over the whole table
    kErrCount = 2,        // a column produced a different nnz than its symbolic count
    kErrIndex = 4,        // an index outside its array was met (corrupt input)
};

// Number of column tiers. Tier 0: empty column. Tiers 1..4: one warp per
// column with a 2*cap-slot table (cap 32, 128, 256, 512). Tiers 5..8: one CTA
// per column, table of 2*cap slots (cap 1024 .. 8192). Tiers 9..15: heavy
// columns (dense accumulators), split by log2 of their size so that the
// largest run first.
constexpr int kTiers = 16;
constexpr int kHeavyTier0 = 9;
// tiers 1..kWarpTiers run one warp per column (warp-private tables)
constexpr int kWarpTiers = 4;
__host__ __device__ constexpr int tier_cap(int t) {
    // capacity (max distinct rows) of hash tiers 1..8
    return t == 1 ? 32 : t == 2 ? 128 : (128 << (t - 2));
}

// Multiplicative (Fibonacci) hashing: the top log2(T) bits of key * 2^32/phi.
__device__ __forceinline__ uint32_t hash_slot(uint32_t key, int log2T) {
    return (key * 0x9E3779B1u) >> (32 - log2T);
}

template <class V> __device__ __forceinline__ void atomic_add_v(V *p, V v);
template <> __device__ __forceinline__ void atomic_add_v<float>(float *p, float v) { atomicAdd(p, v); }
template <> __device__ __forceinline__ void atomic_add_v<double>(double *p, double v) { atomicAdd(p, v); }
template <> __device__ __forceinline__ void atomic_add_v<int64_t>(int64_t *p, int64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

// Products of the semiring: float32 in float32, float64 in float64, int64 with
// two's-complement wrap-around (computed in uint64).
template <class V> __device__ __forceinline__ V mul_v(V a, V b) { return a * b; }
template <> __device__ __forceinline__ int64_t mul_v<int64_t>(int64_t a, int64_t b) {
    return static_cast<int64_t>(static_cast<uint64_t>(a) * static_cast<uint64_t>(b));
}

template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(SPG_FULL, v, o);
    return v;
}

// Inclusive prefix sum across the warp.
template <class T> __device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(SPG_FULL, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

__device__ __forceinline__ int ilog2_floor(uint64_t x) { return 63 - __clzll(x | 1); }

}  // namespace spg
