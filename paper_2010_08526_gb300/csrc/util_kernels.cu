// Non-templated helper kernels: numeric tiering, tier scatter, int64 scans,
// small copies.
#include "util.h"
#include "kernels.cuh"

namespace spg {

__device__ __forceinline__ int num_tier_of(int64_t n, int hash_cap_max) {
    if (n == 0) return 0;
    for (int t = 1; t <= 8; ++t) {
        const int cap = tier_cap(t);
        if (cap > hash_cap_max) break;
        if (n <= cap) return t;
    }
    return kHeavyTier0;
}

__global__ void k_numeric_tier(const int64_t *cnt, const int64_t *dense_sel, int64_t c_lo,
                               int64_t c_hi, int hash_cap_max, uint8_t *tier_out,
                               int32_t *tier_hist) {
    __shared__ int s_hist[kTiers];
    if (threadIdx.x < kTiers) s_hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t g = c_lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < c_hi) {
        int t = num_tier_of(cnt[g], hash_cap_max);
        if (dense_sel && dense_sel[g] > hash_cap_max) t = kHeavyTier0;
        tier_out[g] = (uint8_t)t;
        if (t) atomicAdd(&s_hist[t], 1);
    }
    __syncthreads();
    if (threadIdx.x < kTiers && s_hist[threadIdx.x]) atomicAdd(&tier_hist[threadIdx.x], s_hist[threadIdx.x]);
}

__global__ void k_bin_scatter(const uint8_t *tier, int64_t c_lo, int64_t c_hi,
                              const int32_t *tier_hist, int32_t *cursor, int32_t *list,
                              int32_t *list_off, int32_t *heavy_ord) {
    __shared__ int s_off[kTiers + 1];
    __shared__ int s_cnt[kTiers];
    __shared__ int s_base[kTiers];
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int t = 0; t < kTiers; ++t) { s_off[t] = acc; acc += (t == 0 ? 0 : tier_hist[t]); }
        s_off[kTiers] = acc;
        if (blockIdx.x == 0)
            for (int t = 0; t <= kTiers; ++t) list_off[t] = s_off[t];
    }
    if (threadIdx.x < kTiers) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t g = c_lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int t = 0, rank = 0;
    if (g < c_hi) {
        t = tier[g];
        if (t) rank = atomicAdd(&s_cnt[t], 1);
    }
    __syncthreads();
    if (threadIdx.x < kTiers && s_cnt[threadIdx.x])
        s_base[threadIdx.x] = atomicAdd(&cursor[threadIdx.x], s_cnt[threadIdx.x]);
    __syncthreads();
    if (g < c_hi && t) {
        const int pos = s_off[t] + s_base[t] + rank;
        list[pos] = (int32_t)g;
        if (heavy_ord && t >= kHeavyTier0) heavy_ord[g] = pos - s_off[kHeavyTier0];
    }
}

// mode 0: per-column item counts into ncount[h]; mode 1: write the items at
// item_off[h] (exclusive scan of the counts). One thread per heavy column runs
// the greedy cut over its P panel counts.
__global__ void k_heavy_items(const int32_t *list, const int32_t *list_off, const int64_t *sel,
                              int hash_cap_max, int64_t c_lo, int64_t c_hi, const int32_t *pcnt,
                              int P, int dense_min, int range_cap, int max_panels, int mode,
                              int64_t *ncount, const int64_t *item_off, HeavyItem *items) {
    const int lo = list_off[kHeavyTier0], hi = list_off[kTiers];
    const int nh = hi - lo;
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= nh) return;
    const int64_t g = list[lo + h];
    int64_t n_items = 0;
    if (g >= c_lo && g < c_hi && sel[g] > hash_cap_max) {
        const int32_t *pc = pcnt + h * P;
        int64_t w = mode ? item_off[h] : 0;
        int gp0 = -1, gcnt = 0, off = 0, goff = 0;
        auto flush = [&](int p_end) {
            if (gp0 >= 0 && gcnt > 0) {
                if (mode) items[w++] = HeavyItem{(int32_t)g, gp0, p_end, gcnt, goff, 0};
                ++n_items;
            }
            gp0 = -1; gcnt = 0;
        };
        for (int p = 0; p < P; ++p) {
            const int x = pc[p];
            if (x >= dense_min) {
                flush(p);
                if (mode) items[w++] = HeavyItem{(int32_t)g, p, p + 1, -x, off, 0};
                ++n_items;
                off += x;
                continue;
            }
            if (gp0 >= 0 && (gcnt + x > range_cap || p - gp0 >= max_panels)) flush(p);
            if (x == 0 && gp0 < 0) continue;      // no open group: skip empty panels
            if (gp0 < 0) { gp0 = p; goff = off; }
            gcnt += x;
            off += x;
        }
        flush(P);
    }
    if (!mode) ncount[h] = n_items;
}

// Offsets of the column-grouped copy of A (declared with its copy kernel).
__global__ void k_colpanel_offsets(const int64_t *ape, int64_t ka, int P, int32_t *apo) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ka;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t *o = apo + k * ((int64_t)P + 1);
        int32_t run = 0;
#pragma unroll 4
        for (int p = 0; p < P; ++p) {
            const int64_t idx = (int64_t)p * ka + k;
            const int64_t s = idx ? ape[idx - 1] : 0;
            o[p] = run;
            run += (int32_t)(ape[idx] - s);
        }
        o[P] = run;
    }
}

// Panel-major order of the heavy items (counting sort by first panel), so
// that the CTAs running at the same time read the same panel of A and of the
// panel offsets from L2. mode 0: histogram; mode 1: scatter.
__global__ void k_items_by_panel(const HeavyItem *items, const int64_t *n_items_p, int mode,
                                 int32_t *panel_cnt, int32_t *order) {
    const int64_t n = *n_items_p;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int p = items[i].p0;
        if (mode == 0) atomicAdd(&panel_cnt[p], 1);
        else order[atomicAdd(&panel_cnt[p], 1)] = (int32_t)i;
    }
}

__global__ void k_items_by_batch(const HeavyItem *items, int64_t n, const int64_t *bounds, int64_t nb,
                                 int pe, int mode, unsigned long long *cnt, int32_t *order) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const HeavyItem it = items[i];
        const int64_t g = it.g;
        // the batch t with bounds[t] <= g < bounds[t + 1]
        int64_t lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (bounds[mid] <= g) lo = mid; else hi = mid - 1;
        }
        // dense items (cnt < 0) before hash items inside a batch
        const int64_t key = (lo * 2 + (it.cnt < 0 ? 0 : 1)) * pe + (pe > 1 ? it.p0 : 0);
        if (mode == 0) atomicAdd(&cnt[key], 1ull);
        else order[atomicAdd(&cnt[key], 1ull)] = (int32_t)i;
    }
}

// After the scatter cnt[key] is the end of bucket key; a batch has 2 * pe
// buckets, so batch t starts at cnt[t * 2 * pe - 1] (0 for t = 0) and
// start[nb] = n.
__global__ void k_batch_item_starts(const unsigned long long *cnt, int64_t nb, int pe, int64_t n,
                                    int64_t *start) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > nb) return;
    start[t] = t == 0 ? 0 : t == nb ? n : (int64_t)cnt[t * 2 * pe - 1];
}

// exclusive scan of P ints in place (one CTA)
__global__ void k_small_excl_scan(int32_t *a, int P) {
    __shared__ int32_t s[1024];
    int carry = 0;
    for (int base = 0; base < P; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < P ? a[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < P) a[i] = carry + s[threadIdx.x] - v;
        const int tot = s[blockDim.x - 1];
        __syncthreads();
        carry += tot;
    }
}

// ---- exclusive scan of int64 (three phases, all on the device) ------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *s_warp, int64_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = warp_incl_scan(v);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
        int64_t wi = warp_incl_scan(w);
        s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    int64_t r = s_warp[warp] + incl - v;
    total = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int64_t *in, int64_t n,
                                                              int64_t *partials) {
    __shared__ int64_t s_warp[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    int64_t total;
    block_excl_scan(s, s_warp, total);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partials(int64_t *partials, int64_t np) {
    __shared__ int64_t s_warp[33];
    int64_t carry = 0;
    for (int64_t b = 0; b < np; b += kScanThreads) {
        const int64_t i = b + threadIdx.x;
        int64_t v = i < np ? partials[i] : 0;
        int64_t total;
        int64_t ex = block_excl_scan(v, s_warp, total);
        if (i < np) partials[i] = ex + carry;
        carry += total;
    }
    if (threadIdx.x == 0) partials[np] = carry;
}

// out[i] = sum_{j<i} in[j] for i in [0, n]; in and out may alias.
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int64_t *in, int64_t n,
                                                             const int64_t *partials,
                                                             int64_t *out, int write_total) {
    __shared__ int64_t s_warp[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        s += v[i];
    }
    int64_t total;
    int64_t ex = block_excl_scan(s, s_warp, total) + partials[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t idx = base + i;
        if (idx < n) out[idx] = ex;
        ex += v[i];
    }
    if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        out[n] = partials[gridDim.x];
}

int64_t scan_partials_len(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t exclusive_scan_i64(const int64_t *in, int64_t n, int64_t *out, int64_t *partials,
                               int write_total, cudaStream_t st) {
    const int64_t nb = n > 0 ? (n + kScanTile - 1) / kScanTile : 1;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, partials);
    k_scan_partials<<<1, kScanThreads, 0, st>>>(partials, nb);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, partials, out, write_total);
    return cudaGetLastError();
}

// ---- small kernels ----------------------------------------------------------

// dst[i] = src[i] - src[0] for i in [0, n], narrowed to the output pointer type.
__global__ void k_rebase_colptr_i64(const int64_t *src, int64_t n, int64_t *dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) dst[i] = src[i] - src[0];
}
__global__ void k_rebase_colptr_i32(const int64_t *src, int64_t n, int32_t *dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) dst[i] = (int32_t)(src[i] - src[0]);
}

cudaError_t rebase_colptr(const int64_t *src, int64_t n, void *dst, int dst_is_i64,
                          cudaStream_t st) {
    const unsigned nb = (unsigned)((n + 1 + 255) / 256);
    if (dst_is_i64) k_rebase_colptr_i64<<<nb, 256, 0, st>>>(src, n, (int64_t *)dst);
    else k_rebase_colptr_i32<<<nb, 256, 0, st>>>(src, n, (int32_t *)dst);
    return cudaGetLastError();
}

// Validation of a CSC: colptr monotone from 0 to nnz, rows in [0, nrows).
template <class I>
__global__ void k_validate(const I *colptr, const I *rowidx, int64_t ncols, int64_t nrows,
                           int64_t nnz, int *bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= ncols; i += stride) {
        const int64_t c = (int64_t)colptr[i];
        if (i == 0 && c != 0) atomicOr(bad, 1);
        if (i == ncols && c != nnz) atomicOr(bad, 1);
        if (i < ncols && (int64_t)colptr[i + 1] < c) atomicOr(bad, 1);
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride) {
        const int64_t r = (int64_t)rowidx[i];
        if (r < 0 || r >= nrows) atomicOr(bad, 2);
    }
}

cudaError_t validate_csc(const void *colptr, const void *rowidx, int idx64, int64_t ncols,
                         int64_t nrows, int64_t nnz, int *d_bad, cudaStream_t st) {
    const unsigned nb = 1024;
    if (idx64)
        k_validate<int64_t><<<nb, 256, 0, st>>>((const int64_t *)colptr, (const int64_t *)rowidx,
                                                ncols, nrows, nnz, d_bad);
    else
        k_validate<int32_t><<<nb, 256, 0, st>>>((const int32_t *)colptr, (const int32_t *)rowidx,
                                                ncols, nrows, nnz, d_bad);
    return cudaGetLastError();
}

// w[g] = bytes_per_nnz * (cnt[g] + extra[g]) + ptr_bytes, for g in [0, n).
__global__ void k_column_bytes(const int64_t *cnt, const int64_t *extra, int64_t n, int64_t r,
                               int64_t ptr_bytes, int64_t *w) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) w[g] = r * (cnt[g] + (extra ? extra[g] : 0)) + ptr_bytes;
}

cudaError_t column_bytes(const int64_t *cnt, const int64_t *extra, int64_t n, int64_t r,
                         int64_t ptr_bytes, int64_t *w, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_column_bytes<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cnt, extra, n, r, ptr_bytes, w);
    return cudaGetLastError();
}

__global__ void k_add_i64(int64_t *dst, const int64_t *src, int64_t n) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) dst[g] += src[g];
}

cudaError_t add_i64(int64_t *dst, const int64_t *src, int64_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_add_i64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dst, src, n);
    return cudaGetLastError();
}

}  // namespace spg
