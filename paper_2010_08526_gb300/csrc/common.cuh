// Shared device helpers for the sm_103a SpGEMM kernels.
#pragma once

#include <cstdint>
#include <limits>
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

// ---- min-plus semiring values ----------------------------------------------
// The paper's algorithms hold over any semiring (Sec. II). MinPlus<F> stores
// the plain float / double bits; the type selects the operations: a (x) b =
// a + b, (+) = min, with NaN products ignored. Integer literals name the
// identities, so that the kernels' V(0) (a cleared accumulator) is +infinity
// and V(1) (the scale of a merged partial) is 0.
template <class F> struct MinPlus {
    F v;
    MinPlus() = default;
    __host__ __device__ constexpr MinPlus(int lit)
        : v(lit == 0 ? F(__builtin_huge_val()) : (lit == 1 ? F(0) : F(lit))) {}
    __host__ __device__ static constexpr MinPlus raw(F x) {
        MinPlus m(1);
        m.v = x;
        return m;
    }
    __host__ __device__ friend bool operator>=(MinPlus a, MinPlus b) { return a.v >= b.v; }
    __host__ __device__ friend bool operator==(MinPlus a, MinPlus b) { return a.v == b.v; }
};
template <class T> struct IsMinPlus { static constexpr bool v = false; };
template <class F> struct IsMinPlus<MinPlus<F>> { static constexpr bool v = true; };

template <> __device__ __forceinline__ MinPlus<float> mul_v<MinPlus<float>>(MinPlus<float> a, MinPlus<float> b) {
    return MinPlus<float>::raw(a.v + b.v);
}
template <> __device__ __forceinline__ MinPlus<double> mul_v<MinPlus<double>>(MinPlus<double> a, MinPlus<double> b) {
    return MinPlus<double>::raw(a.v + b.v);
}
// Atomic min of IEEE values through integer atomics: a non-negative value
// orders like its bits as a signed integer, a negative one inversely to its
// bits as an unsigned integer, so min is atomicMin on the signed view for
// x >= 0 and atomicMax on the unsigned view for x < 0 (whatever the stored
// value's sign). NaN is skipped.
template <> __device__ __forceinline__ void atomic_add_v<MinPlus<float>>(MinPlus<float> *p, MinPlus<float> x) {
    const float f = x.v;
    if (f != f) return;
    if (f >= 0.0f) atomicMin(reinterpret_cast<int *>(p), __float_as_int(f));
    else atomicMax(reinterpret_cast<unsigned int *>(p), __float_as_uint(f));
}
template <> __device__ __forceinline__ void atomic_add_v<MinPlus<double>>(MinPlus<double> *p, MinPlus<double> x) {
    const double f = x.v;
    if (f != f) return;
    if (f >= 0.0) atomicMin(reinterpret_cast<long long *>(p), __double_as_longlong(f));
    else atomicMax(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__double_as_longlong(f));
}

// ---- or-and (Boolean) semiring values -------------------------------------
// OrAnd<T> stores the plain float / double / int64 bits. A value is true when
// it is nonzero (-0.0 is false, NaN true); a (x) b = a AND b and (+) = OR,
// each written as 0 or 1 of type T. Integer literals name the identities:
// V(0) = false clears an accumulator, V(1) = true scales a merged partial.
template <class T> struct OrAnd {
    T v;
    OrAnd() = default;
    __host__ __device__ constexpr OrAnd(int lit) : v(lit != 0 ? T(1) : T(0)) {}
    __host__ __device__ static constexpr OrAnd raw(T x) {
        OrAnd o(0);
        o.v = x;
        return o;
    }
    __host__ __device__ friend bool operator>=(OrAnd a, OrAnd b) { return a.v >= b.v; }
    __host__ __device__ friend bool operator==(OrAnd a, OrAnd b) { return a.v == b.v; }
};
template <class T> struct IsOrAnd { static constexpr bool v = false; };
template <class T> struct IsOrAnd<OrAnd<T>> { static constexpr bool v = true; };

// the stored scalar of a value type (the wrapped one for semiring wrappers)
template <class V> struct Storage { using type = V; };
template <class F> struct Storage<MinPlus<F>> { using type = F; };
template <class T> struct Storage<OrAnd<T>> { using type = T; };

template <> __device__ __forceinline__ OrAnd<float> mul_v<OrAnd<float>>(OrAnd<float> a, OrAnd<float> b) {
    return OrAnd<float>::raw((a.v != 0.0f && b.v != 0.0f) ? 1.0f : 0.0f);
}
template <> __device__ __forceinline__ OrAnd<double> mul_v<OrAnd<double>>(OrAnd<double> a, OrAnd<double> b) {
    return OrAnd<double>::raw((a.v != 0.0 && b.v != 0.0) ? 1.0 : 0.0);
}
template <> __device__ __forceinline__ OrAnd<int64_t> mul_v<OrAnd<int64_t>>(OrAnd<int64_t> a, OrAnd<int64_t> b) {
    return OrAnd<int64_t>::raw((a.v != 0 && b.v != 0) ? 1 : 0);
}
// OR: a true operand sets the accumulator to the bits of 1 with an integer
// atomicOr; the accumulator starts as the bits of 0 and only ever receives
// the bits of 1, so it holds exactly 0 or 1. A false operand changes nothing.
template <> __device__ __forceinline__ void atomic_add_v<OrAnd<float>>(OrAnd<float> *p, OrAnd<float> x) {
    if (x.v != 0.0f) atomicOr(reinterpret_cast<unsigned int *>(p), __float_as_uint(1.0f));
}
template <> __device__ __forceinline__ void atomic_add_v<OrAnd<double>>(OrAnd<double> *p, OrAnd<double> x) {
    if (x.v != 0.0) atomicOr(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__double_as_longlong(1.0));
}
template <> __device__ __forceinline__ void atomic_add_v<OrAnd<int64_t>>(OrAnd<int64_t> *p, OrAnd<int64_t> x) {
    if (x.v != 0) atomicOr(reinterpret_cast<unsigned long long *>(p), 1ull);
}

// The semiring's sum of two values, for a sequential run (the sort-based
// accumulator): + for plus-times (int64 wrapping), min for min-plus with NaN
// operands skipped, OR for or-and. The same rules as atomic_add_v.
template <class V> __device__ __forceinline__ V add_v(V a, V b) { return a + b; }
template <> __device__ __forceinline__ int64_t add_v<int64_t>(int64_t a, int64_t b) {
    return static_cast<int64_t>(static_cast<uint64_t>(a) + static_cast<uint64_t>(b));
}
template <> __device__ __forceinline__ MinPlus<float> add_v<MinPlus<float>>(MinPlus<float> a, MinPlus<float> b) {
    return (b.v != b.v || !(b.v < a.v)) ? a : b;
}
template <> __device__ __forceinline__ MinPlus<double> add_v<MinPlus<double>>(MinPlus<double> a, MinPlus<double> b) {
    return (b.v != b.v || !(b.v < a.v)) ? a : b;
}
template <> __device__ __forceinline__ OrAnd<float> add_v<OrAnd<float>>(OrAnd<float> a, OrAnd<float> b) {
    return b.v != 0.0f ? OrAnd<float>(1) : a;
}
template <> __device__ __forceinline__ OrAnd<double> add_v<OrAnd<double>>(OrAnd<double> a, OrAnd<double> b) {
    return b.v != 0.0 ? OrAnd<double>(1) : a;
}
template <> __device__ __forceinline__ OrAnd<int64_t> add_v<OrAnd<int64_t>>(OrAnd<int64_t> a, OrAnd<int64_t> b) {
    return b.v != 0 ? OrAnd<int64_t>(1) : a;
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

// Loads and shuffles of min-plus values (the wrapped bits). Declared at global
// scope, next to the built-in overloads, so that unqualified calls inside the
// library's namespace still see those.
__device__ __forceinline__ spg::MinPlus<float> __ldg(const spg::MinPlus<float> *p) {
    return spg::MinPlus<float>::raw(__ldg(reinterpret_cast<const float *>(p)));
}
__device__ __forceinline__ spg::MinPlus<double> __ldg(const spg::MinPlus<double> *p) {
    return spg::MinPlus<double>::raw(__ldg(reinterpret_cast<const double *>(p)));
}
__device__ __forceinline__ spg::MinPlus<float> __shfl_sync(unsigned mask, spg::MinPlus<float> x, int src,
                                                           int width = 32) {
    return spg::MinPlus<float>::raw(__shfl_sync(mask, x.v, src, width));
}
__device__ __forceinline__ spg::MinPlus<double> __shfl_sync(unsigned mask, spg::MinPlus<double> x, int src,
                                                            int width = 32) {
    return spg::MinPlus<double>::raw(__shfl_sync(mask, x.v, src, width));
}
__device__ __forceinline__ spg::MinPlus<float> __shfl_xor_sync(unsigned mask, spg::MinPlus<float> x, int lane_mask,
                                                               int width = 32) {
    return spg::MinPlus<float>::raw(__shfl_xor_sync(mask, x.v, lane_mask, width));
}
__device__ __forceinline__ spg::MinPlus<double> __shfl_xor_sync(unsigned mask, spg::MinPlus<double> x,
                                                                int lane_mask, int width = 32) {
    return spg::MinPlus<double>::raw(__shfl_xor_sync(mask, x.v, lane_mask, width));
}
// Loads and shuffles of or-and values (the stored bits), as for min-plus.
#define SPG_ORAND_IO(T)                                                                           \
    __device__ __forceinline__ spg::OrAnd<T> __ldg(const spg::OrAnd<T> *p) {                     \
        return spg::OrAnd<T>::raw(__ldg(reinterpret_cast<const T *>(p)));                         \
    }                                                                                             \
    __device__ __forceinline__ spg::OrAnd<T> __shfl_sync(unsigned mask, spg::OrAnd<T> x, int src, \
                                                         int width = 32) {                        \
        return spg::OrAnd<T>::raw(__shfl_sync(mask, x.v, src, width));                            \
    }                                                                                             \
    __device__ __forceinline__ spg::OrAnd<T> __shfl_xor_sync(unsigned mask, spg::OrAnd<T> x,      \
                                                             int lane_mask, int width = 32) {     \
        return spg::OrAnd<T>::raw(__shfl_xor_sync(mask, x.v, lane_mask, width));                  \
    }
SPG_ORAND_IO(float)
SPG_ORAND_IO(double)
SPG_ORAND_IO(int64_t)
#undef SPG_ORAND_IO
