// Sorted final output and the column-wise prune of a result batch.
//
// Sorting: the paper keeps the final C sorted within each column (Sec. IV-D:
// only the intermediate products are left unsorted). The numeric pass leaves
// a column in one of three states: a light column (at most hash_cap_max rows,
// hash order), or a heavy column made of work items in panel order whose
// dense items are already in row order and whose hash-range items (at most
// kRangeCap rows each) are in hash order. So sorting the batch means sorting
// segments of at most 8192 entries: the light columns and the hash items.
//
// Prune: the consumer the column batches are shaped for keeps the largest
// entries of every column (Markov clustering, Sec. III; HipMCL prunes each
// batch, Sec. V-F). Per column: candidates are the entries with value >=
// threshold; if topk > 0 and more remain, the topk largest are kept, equal
// values going to the earlier stored entry; kept entries stay in their order.
#pragma once

#include "kernels.cuh"

namespace spg {

// ---- order-preserving keys ------------------------------------------------
// Unsigned keys whose order is the order of the values (IEEE floats: the sign
// bit flipped for positives, all bits flipped for negatives; int64: the sign
// bit flipped). NaN never reaches them: it fails every threshold test.
__device__ __forceinline__ uint64_t value_key(float v) {
    const uint32_t u = __float_as_uint(v);
    return (uint64_t)(u ^ ((u >> 31) ? 0xffffffffu : 0x80000000u));
}
__device__ __forceinline__ uint64_t value_key(double v) {
    const uint64_t u = (uint64_t)__double_as_longlong(v);
    return u ^ ((u >> 63) ? 0xffffffffffffffffull : 0x8000000000000000ull);
}
__device__ __forceinline__ uint64_t value_key(int64_t v) { return (uint64_t)v ^ 0x8000000000000000ull; }
template <class F> __device__ __forceinline__ uint64_t value_key(MinPlus<F> v) { return value_key(v.v); }
template <class T> __device__ __forceinline__ uint64_t value_key(OrAnd<T> v) { return value_key(v.v); }
template <class V> struct KeyBits { static constexpr int v = 64; };
template <> struct KeyBits<float> { static constexpr int v = 32; };
template <> struct KeyBits<MinPlus<float>> { static constexpr int v = 32; };
template <> struct KeyBits<OrAnd<float>> { static constexpr int v = 32; };

// ---- sort ------------------------------------------------------------------
// One warp per column of at most 32 entries: bitonic network over the lanes.
template <class I, class V>
__global__ void __launch_bounds__(256) k_sort_warp(const int64_t *colptr, int64_t base, int64_t c0,
                                                   int64_t c1, I *rows, V *vals) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = c0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); j < c1; j += nw) {
        const int64_t a = colptr[j] - base, n = colptr[j + 1] - colptr[j];
        if (n < 2 || n > 32) continue;
        uint32_t key = lane < n ? (uint32_t)rows[a + lane] : 0xffffffffu;
        V val = lane < n ? vals[a + lane] : V(0);
        // keys are distinct rows (the padding keys are all equal), so the order is total
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                const uint32_t ok = __shfl_xor_sync(SPG_FULL, key, jj);
                const V ov = __shfl_xor_sync(SPG_FULL, val, jj);
                const bool up = (lane & k) == 0;
                const bool lower = (lane & jj) == 0;
                const bool take = lower ? (up ? ok < key : ok > key) : (up ? ok > key : ok < key);
                if (take) { key = ok; val = ov; }
            }
        }
        if (lane < n) { rows[a + lane] = (I)key; vals[a + lane] = val; }
    }
}

// One CTA per light column with 32 < n <= CAP (and n <= cap_max, i.e. not a
// heavy column), columns [c0, c1).
template <class I, class V, int CAP>
__global__ void k_sort_block(const int64_t *colptr, int64_t base, int64_t c0, int64_t c1, int lo_excl,
                             int cap_max, I *rows, V *vals) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *sk = reinterpret_cast<uint32_t *>(smem);
    V *sv = reinterpret_cast<V *>(smem + sizeof(uint32_t) * CAP);
    for (int64_t j = c0 + blockIdx.x; j < c1; j += gridDim.x) {
        const int64_t a = colptr[j] - base;
        const int n = (int)(colptr[j + 1] - colptr[j]);
        if (n <= lo_excl || n > CAP || n > cap_max) continue;
        for (int i = threadIdx.x; i < n; i += blockDim.x) { sk[i] = (uint32_t)rows[a + i]; sv[i] = vals[a + i]; }
        block_bitonic<CAP>(sk, sv, n);
        for (int i = threadIdx.x; i < n; i += blockDim.x) { rows[a + i] = (I)sk[i]; vals[a + i] = sv[i]; }
        __syncthreads();
    }
}

// One CTA per hash-range item of a heavy column in [c0, c1). The item's
// rows are distinct and lie in its row range [p0 R, p1 R), so a bitmap over
// the range ranks them: set a bit per row, prefix the word popcounts, and an
// entry's position is the number of set bits below its row. O(n + range/32)
// per item. A range wider than the bitmap words given (wcap) falls back to
// the bitonic sort. Dense items are in row order already.
template <class I, class V, int CAP>
__global__ void __launch_bounds__(512, 2) k_sort_items(const HeavyItem *items, const int64_t *nitems_p, const int64_t *colptr,
                             int64_t base, int64_t c0, int64_t c1, int log2R, int wcap, I *rows, V *vals) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *sk = reinterpret_cast<uint32_t *>(smem);                       // CAP staged rows
    V *sv = reinterpret_cast<V *>(smem + sizeof(uint32_t) * CAP);            // CAP staged values
    uint32_t *bm = reinterpret_cast<uint32_t *>(smem + (sizeof(uint32_t) + sizeof(V)) * CAP);
    uint16_t *pre = reinterpret_cast<uint16_t *>(bm + wcap);                 // word prefix (< CAP <= 2^15)
    __shared__ uint32_t s_part[1024];
    const int64_t nitems = *nitems_p;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const HeavyItem item = items[it];
        if (item.cnt <= 1 || item.cnt > CAP || item.g < c0 || item.g >= c1) continue;   // dense (< 0) or trivial
        const int n = item.cnt;
        const int64_t a = colptr[item.g] - base + item.off;
        const int64_t r0 = (int64_t)item.p0 << log2R;
        const int W = (int)((((int64_t)(item.p1 - item.p0)) << log2R) >> 5);
        if (W > wcap) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) { sk[i] = (uint32_t)rows[a + i]; sv[i] = vals[a + i]; }
            block_bitonic<CAP>(sk, sv, n);
            for (int i = threadIdx.x; i < n; i += blockDim.x) { rows[a + i] = (I)sk[i]; vals[a + i] = sv[i]; }
            __syncthreads();
            continue;
        }
        for (int w = threadIdx.x; w < W; w += blockDim.x) bm[w] = 0u;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t r = (uint32_t)rows[a + i];
            sk[i] = r;
            sv[i] = vals[a + i];
            const uint32_t b = (uint32_t)((int64_t)r - r0);
            atomicOr(&bm[b >> 5], 1u << (b & 31));
        }
        __syncthreads();
        // exclusive prefix of the word popcounts: each thread a contiguous
        // run of words, then a scan over the threads' sums
        const int per = (W + (int)blockDim.x - 1) / (int)blockDim.x;
        const int w0 = threadIdx.x * per, w1 = min(W, w0 + per);
        uint32_t sum = 0;
        for (int w = w0; w < w1; ++w) sum += __popc(bm[w]);
        s_part[threadIdx.x] = sum;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const uint32_t t = threadIdx.x >= (unsigned)o ? s_part[threadIdx.x - o] : 0u;
            __syncthreads();
            s_part[threadIdx.x] += t;
            __syncthreads();
        }
        uint32_t run = s_part[threadIdx.x] - sum;
        for (int w = w0; w < w1; ++w) { pre[w] = (uint16_t)run; run += __popc(bm[w]); }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t b = (uint32_t)((int64_t)sk[i] - r0);
            const uint32_t pos = (uint32_t)pre[b >> 5] + __popc(bm[b >> 5] & ((1u << (b & 31)) - 1u));
            rows[a + pos] = (I)sk[i];
            vals[a + pos] = sv[i];
        }
        __syncthreads();
    }
}

// int32 colptr widened to int64
template <class T>
__global__ void k_widen(const T *src, int64_t n, int64_t *dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (int64_t)src[i];
}

// ---- prune -----------------------------------------------------------------
// Per column j of a batch (colptr relative offsets, ncols columns):
// keep[j] = kept count; for a column that needs a selection (more candidates
// than topk) its index goes to sel_list. mode[j]: 0 keep every candidate,
// 1 selection pending.
template <class V>
__global__ void __launch_bounds__(256) k_prune_count(const int64_t *colptr, const V *vals, int64_t ncols,
                                                     V thr, int64_t topk, int64_t *keep, int8_t *mode,
                                                     int64_t *sel_list, unsigned long long *nsel) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < ncols; j += nw) {
        const int64_t a = colptr[j] - colptr[0], b = colptr[j + 1] - colptr[0];
        int64_t c = 0;
        for (int64_t q = a + lane; q < b; q += 32) c += vals[q] >= thr;
        c = warp_sum(c);
        if (lane == 0) {
            if (topk > 0 && c > topk) {
                keep[j] = topk;
                mode[j] = 1;
                sel_list[atomicAdd(nsel, 1ull)] = j;
            } else {
                keep[j] = c;
                mode[j] = 0;
            }
        }
    }
}

// One CTA per listed column: radix select (8 bits a pass, most significant
// first) of the topk-th largest key among the candidates. Writes the key and
// the quota of entries equal to it that are kept (topk minus the candidates
// strictly above it). Each warp counts into its own 256-bin histogram (the
// values of a column crowd into few exponent bins, so one shared histogram
// would serialise the atomics); the warp histograms are then summed and a
// warp finds the digit with a suffix scan.
// tie_by_row != 0: when more candidates share the selected key than the quota
// keeps, a second radix pass over their rows (ascending) finds the largest
// row kept (sel_row), so that equal values go to the smaller rows whatever
// the storage order.
template <class I, class V>
__global__ void __launch_bounds__(512) k_prune_select(const int64_t *colptr, const I *rows, const V *vals,
                                                      V thr, int64_t topk, const int64_t *sel_list,
                                                      const unsigned long long *nsel, uint64_t *sel_key,
                                                      int64_t *sel_quota, int tie_by_row, uint32_t *sel_row) {
    __shared__ uint32_t hist[16][256];
    __shared__ uint32_t tot[256];
    __shared__ uint64_t s_prefix;
    __shared__ long long s_k;
    __shared__ long long s_cnt;   // candidates in the selected bin of the last pass
    __shared__ uint32_t s_rpre;   // row prefix of the tie pass
    constexpr int kBits = KeyBits<V>::v;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t ns = (int64_t)*nsel;
    for (int64_t s = blockIdx.x; s < ns; s += gridDim.x) {
        const int64_t j = sel_list[s];
        const int64_t a = colptr[j] - colptr[0], b = colptr[j + 1] - colptr[0];
        if (threadIdx.x == 0) { s_prefix = 0; s_k = topk; }   // want the s_k-th largest
        uint64_t mask = 0;   // bits of the key fixed so far
        for (int shift = kBits - 8; shift >= 0; shift -= 8) {
            for (int i = threadIdx.x; i < 16 * 256; i += blockDim.x) (&hist[0][0])[i] = 0u;
            __syncthreads();
            const uint64_t prefix = s_prefix;
            for (int64_t q = a + threadIdx.x; q < b; q += blockDim.x) {
                const V v = vals[q];
                if (!(v >= thr)) continue;
                const uint64_t key = value_key(v);
                if ((key & mask) != prefix) continue;
                atomicAdd(&hist[warp][(key >> shift) & 255u], 1u);
            }
            __syncthreads();
            for (int d = threadIdx.x; d < 256; d += blockDim.x) {
                uint32_t c = 0;
                for (int w = 0; w < nw; ++w) c += hist[w][d];
                tot[d] = c;
            }
            __syncthreads();
            if (warp == 0) {
                // lane l holds bins [8l, 8l+8); the digit is the highest bin
                // at which the count from the top reaches s_k
                const long long k = s_k;
                uint32_t c8[8];
                uint32_t mine = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) { c8[i] = tot[lane * 8 + i]; mine += c8[i]; }
                // counts of the lanes above this one (bins higher than 8l+7)
                uint32_t above = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_down_sync(SPG_FULL, above, o);
                    if (lane + o < 32) above += t;
                }
                above -= mine;   // exclusive suffix: bins above this lane's range
                int dsel = -1;
                long long kk = 0;
                long long acc = (long long)above;
                for (int i = 7; i >= 0; --i) {
                    if (dsel < 0 && acc + (long long)c8[i] >= k) { dsel = lane * 8 + i; kk = k - acc; }
                    acc += c8[i];
                }
                // the highest lane that found the digit wins
                const unsigned found = __ballot_sync(SPG_FULL, dsel >= 0);
                const int src = 31 - __clz(found);
                const int dg = __shfl_sync(SPG_FULL, dsel, src);
                const long long knew = __shfl_sync(SPG_FULL, kk, src);
                if (lane == 0) {
                    s_prefix = prefix | ((uint64_t)(dg < 0 ? 0 : dg) << shift);
                    s_k = knew;
                    s_cnt = dg < 0 ? 0 : (long long)tot[dg];
                }
            }
            __syncthreads();
            mask |= (uint64_t)255 << shift;
        }
        if (threadIdx.x == 0) {
            // s_k-th largest among the keys equal to s_prefix: those above it
            // number topk - s_k, so s_k equal keys are kept
            sel_key[j] = s_prefix;
            sel_quota[j] = s_k;
            if (tie_by_row) sel_row[j] = 0xffffffffu;   // every tie kept
            s_rpre = 0;
        }
        // read before the barrier: after it thread 0 may start the next column
        const bool row_pass = tie_by_row && s_cnt > s_k;
        const uint64_t kkey = s_prefix;
        __syncthreads();
        if (row_pass) {
            // the s_k-th smallest row among the s_cnt ties (rows are distinct)
            uint32_t rmask = 0;
            for (int shift = 24; shift >= 0; shift -= 8) {
                for (int i = threadIdx.x; i < 16 * 256; i += blockDim.x) (&hist[0][0])[i] = 0u;
                __syncthreads();
                const uint32_t rpre = s_rpre;
                for (int64_t q = a + threadIdx.x; q < b; q += blockDim.x) {
                    const V v = vals[q];
                    if (!(v >= thr) || value_key(v) != kkey) continue;
                    const uint32_t r = (uint32_t)rows[q];
                    if ((r & rmask) != rpre) continue;
                    atomicAdd(&hist[warp][(r >> shift) & 255u], 1u);
                }
                __syncthreads();
                for (int d = threadIdx.x; d < 256; d += blockDim.x) {
                    uint32_t c = 0;
                    for (int w = 0; w < nw; ++w) c += hist[w][d];
                    tot[d] = c;
                }
                __syncthreads();
                if (warp == 0) {
                    // lowest bin at which the count from the bottom reaches s_k
                    const long long k = s_k;
                    uint32_t c8[8];
                    uint32_t mine = 0;
#pragma unroll
                    for (int i = 0; i < 8; ++i) { c8[i] = tot[lane * 8 + i]; mine += c8[i]; }
                    const uint32_t incl = warp_incl_scan(mine);
                    long long acc = (long long)(incl - mine);   // bins below this lane's range
                    int dsel = -1;
                    long long kk = 0;
                    for (int i = 0; i < 8; ++i) {
                        if (dsel < 0 && acc + (long long)c8[i] >= k) { dsel = lane * 8 + i; kk = k - acc; }
                        acc += c8[i];
                    }
                    const unsigned found = __ballot_sync(SPG_FULL, dsel >= 0);
                    const int src = found ? __ffs(found) - 1 : 0;
                    const int dg = __shfl_sync(SPG_FULL, dsel, src);
                    const long long knew = __shfl_sync(SPG_FULL, kk, src);
                    if (lane == 0) {
                        s_rpre = rpre | ((uint32_t)(dg < 0 ? 0 : dg) << shift);
                        s_k = knew;
                    }
                }
                __syncthreads();
                rmask |= 255u << shift;
            }
            if (threadIdx.x == 0) sel_row[j] = s_rpre;
            __syncthreads();
        }
    }
}

// One warp per column: stable compaction of the kept entries into the
// output at out_colptr[j] (relative to out_colptr[0]).
template <class I, class V, class IO>
__global__ void __launch_bounds__(256) k_prune_compact(const int64_t *colptr, const I *rows, const V *vals,
                                                       int64_t ncols, V thr, const int8_t *mode,
                                                       const uint64_t *sel_key, const int64_t *sel_quota,
                                                       int tie_by_row, const uint32_t *sel_row,
                                                       const int64_t *out_colptr, IO *out_rows, V *out_vals) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t below = (1u << lane) - 1u;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < ncols; j += nw) {
        const int64_t a = colptr[j] - colptr[0], b = colptr[j + 1] - colptr[0];
        int64_t o = out_colptr[j] - out_colptr[0];
        const bool sel = mode[j] != 0;
        const uint64_t kk = sel ? sel_key[j] : 0;
        int64_t quota = sel ? sel_quota[j] : 0;
        const uint32_t rmax = (sel && tie_by_row) ? sel_row[j] : 0u;
        for (int64_t q0 = a; q0 < b; q0 += 32) {
            const int64_t q = q0 + lane;
            bool take = false, tie = false;
            V v = V(0);
            if (q < b) {
                v = vals[q];
                if (v >= thr) {
                    if (!sel) take = true;
                    else {
                        const uint64_t key = value_key(v);
                        take = key > kk;
                        tie = key == kk;
                    }
                }
            }
            if (sel && tie_by_row) {
                if (tie && (uint32_t)rows[q] <= rmax) take = true;
            } else if (sel) {
                const unsigned tb = __ballot_sync(SPG_FULL, tie);
                const int before = __popc(tb & below);
                if (tie && before < quota) take = true;
                quota -= __popc(tb);
                if (quota < 0) quota = 0;
            }
            const unsigned kb = __ballot_sync(SPG_FULL, take);
            if (take) {
                const int64_t d = o + __popc(kb & below);
                out_rows[d] = (IO)rows[q];
                out_vals[d] = v;
            }
            o += __popc(kb);
        }
    }
}

}  // namespace spg
