// One persistent launch per pass of the multi-problem product (many
// independent C_i = A_i B_i, each column formed by Sec. II-C's column
// formula): the symbolic count and the numeric hash accumulation of every
// column of every problem run as work items of a single kernel.
//
// Work comes from the tier lists of k_bin_scatter (list, off[t]) through two
// device counters. First the CTA items: the columns above the largest
// shared-memory table (heaviest tier first), then the CTA-sized columns
// (largest first), one per item, taken by whole CTAs (atomicAdd on the first
// counter). Then the warp-sized columns: every warp takes a few columns at
// a time from the second counter, with no barrier between warps. Uneven
// problems so balance across SMs without a host round trip.
//
//   CTA item   : a hash table of 2 * cap(tier) slots in shared memory;
//   warp item  : a warp-private table of 2 * cap(tier) <= 2 * 512 slots;
//   heavy item : a hash table in global memory (2 * min(f_j, m) slots,
//                rounded up to a power of two), reached with global atomics.
#pragma once

namespace spg {

struct MultiQueue {
    const int32_t *list;            // global column ids grouped by tier
    const int32_t *off;             // [kTiers + 1] tier offsets in list
    unsigned long long *counter;    // [0] next CTA item, [1] next warp column (zeroed before each launch)
    const int64_t *gtab_off;        // heavy columns: first slot of the global table
    uint32_t *gkeys;                // global tables: keys
    void *gvals;                    // global tables: values
    int warp_tiers;                 // tiers 1..warp_tiers are warp items (<= kWarpTiers)
};

// Global-memory hash insert (linear probing); returns the slot, -1 when the
// table is full (records kErrProbe).
__device__ __forceinline__ int64_t ghash_insert(uint32_t *keys, int log2T, uint32_t key, bool &is_new,
                                                int *err) {
    const uint32_t mask = (1u << log2T) - 1u;
    uint32_t h = hash_slot(key, log2T);
    is_new = false;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint32_t cur = keys[h];
        if (cur == key) return h;
        if (cur == kEmpty) {
            const uint32_t old = atomicCAS(&keys[h], kEmpty, key);
            if (old == kEmpty) { is_new = true; return h; }
            if (old == key) return h;
        }
        h = (h + 1) & mask;
    }
    atomicOr(err, kErrProbe);
    return -1;
}

template <class V> __device__ __forceinline__ void gatomic_add_v(V *p, V v) { atomic_add_v(p, v); }

// MODE 0: symbolic (count distinct rows into c.cnt[g]); MODE 1: numeric
// (accumulate, write column g at c.colptr[g] - c.out_base, unsorted).
template <class Src, int NT, int MODE>
__global__ void __launch_bounds__(NT) k_multi_pass(typename Src::Args sa, TierCommon c, MultiQueue mq,
                                                   typename Src::Idx *out_rows, typename Src::Val *out_vals) {
    using V = typename Src::Val;
    using I = typename Src::Idx;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockShared<V, NT> sh;
    __shared__ long long s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wt = mq.warp_tiers;
    const int nbig = mq.off[kTiers] - mq.off[wt + 1];
    const int nwarp = mq.off[wt + 1] - mq.off[1];
    const int TW = 2 * tier_cap(wt);   // slots of the largest warp table
    if (threadIdx.x == 0) sh.pos = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(mq.counter, 1ull);
        __syncthreads();
        const long long item = s_item;
        __syncthreads();
        if (item >= nbig) break;
        {
            // one column per CTA, heaviest first (the list is ascending in tier)
            const int64_t g = mq.list[mq.off[kTiers] - 1 - item];
            Src src;
            src.open(sa, g);
            const int64_t m = src.m();
            // the tier's capacity bounds the column's distinct rows
            int64_t bound = 0;
            int t = kTiers - 1;
            while (t > wt + 1 && mq.off[t] > mq.off[kTiers] - 1 - item) --t;
            const bool heavy = t >= kHeavyTier0;
            if (!heavy) bound = tier_cap(t);
            int64_t out0 = 0, want = 0;
            if (MODE == 1) {
                out0 = c.colptr[g] - c.out_base;
                want = c.colptr[g + 1] - c.colptr[g];
            }
            if (!heavy) {
                int log2T = 1;
                while ((1ll << log2T) < 2 * bound) ++log2T;
                const int T = 1 << log2T;
                V *vals = reinterpret_cast<V *>(smem);
                uint32_t *keys = reinterpret_cast<uint32_t *>(smem + sizeof(V) * T);
                for (int s = threadIdx.x; s < T; s += NT) { keys[s] = kEmpty; if (MODE == 1) vals[s] = V(0); }
                __syncthreads();
                int mine = 0;
                auto emit = load_apply(
                    [&](int64_t q, V bv, int64_t) { return RowVal<V>{src.row(q), MODE == 1 ? src.val(q, bv) : V(0)}; },
                    [&](const RowVal<V> &e, bool valid) {
                        if (!valid) return;
                        bool nw;
                        const int h = hash_insert_dbl1(keys, log2T, e.r, c.err, nw);
                        if (MODE == 0) mine += nw;
                        else if (h >= 0) atomic_add_v(&vals[h], e.x);
                    });
                block_walk<kWalkBatch>(src, emit, c.short_seg, c.huge_seg, sh);
                if (MODE == 0) {
                    mine = warp_sum(mine);
                    if (lane == 0) sh.red[warp] = mine;
                    __syncthreads();
                    if (threadIdx.x < 32) {
                        int v = threadIdx.x < NW ? sh.red[threadIdx.x] : 0;
                        v = warp_sum(v);
                        if (threadIdx.x == 0) c.cnt[g] = v;
                    }
                } else {
                    for (int s0 = 0; s0 < T; s0 += NT) {
                        const int s = s0 + threadIdx.x;
                        const uint32_t key = s < T ? keys[s] : kEmpty;
                        const bool occ = key != kEmpty;
                        const unsigned bal = __ballot_sync(SPG_FULL, occ);
                        int wbase = 0;
                        if (lane == 0 && bal) wbase = atomicAdd(&sh.pos, __popc(bal));
                        wbase = __shfl_sync(SPG_FULL, wbase, 0);
                        if (occ) {
                            const int r = wbase + __popc(bal & ((1u << lane) - 1u));
                            if (r < want) {
                                out_rows[out0 + r] = (I)key;
                                out_vals[out0 + r] = vals[s];
                            }
                        }
                    }
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        if (sh.pos != want) atomicOr(c.err, kErrCount);
                        sh.pos = 0;
                    }
                }
                __syncthreads();
            } else {
                // the column's own table in global memory
                const int64_t f = src.flops();   // warp-wide: every warp computes it
                const int64_t rows = f < m ? f : m;
                int log2T = 1;
                while ((1ll << log2T) < 2 * rows) ++log2T;
                const int64_t T = 1ll << log2T;
                uint32_t *keys = mq.gkeys + mq.gtab_off[g];
                V *vals = reinterpret_cast<V *>(mq.gvals) + mq.gtab_off[g];
                for (int64_t s = threadIdx.x; s < T; s += NT) { keys[s] = kEmpty; if (MODE == 1) vals[s] = V(0); }
                __syncthreads();
                int mine = 0;
                auto emit = load_apply(
                    [&](int64_t q, V bv, int64_t) { return RowVal<V>{src.row(q), MODE == 1 ? src.val(q, bv) : V(0)}; },
                    [&](const RowVal<V> &e, bool valid) {
                        if (!valid) return;
                        bool nw;
                        const int64_t h = ghash_insert(keys, log2T, e.r, nw, c.err);
                        if (MODE == 0) mine += nw;
                        else if (h >= 0) gatomic_add_v(&vals[h], e.x);
                    });
                block_walk<kWalkBatch>(src, emit, c.short_seg, c.huge_seg, sh);
                __syncthreads();
                if (MODE == 0) {
                    mine = warp_sum(mine);
                    if (lane == 0) sh.red[warp] = mine;
                    __syncthreads();
                    if (threadIdx.x < 32) {
                        int v = threadIdx.x < NW ? sh.red[threadIdx.x] : 0;
                        v = warp_sum(v);
                        if (threadIdx.x == 0) c.cnt[g] = v;
                    }
                } else {
                    for (int64_t s0 = 0; s0 < T; s0 += NT) {
                        const int64_t s = s0 + threadIdx.x;
                        const uint32_t key = s < T ? keys[s] : kEmpty;
                        const bool occ = key != kEmpty;
                        const unsigned bal = __ballot_sync(SPG_FULL, occ);
                        int wbase = 0;
                        if (lane == 0 && bal) wbase = atomicAdd(&sh.pos, __popc(bal));
                        wbase = __shfl_sync(SPG_FULL, wbase, 0);
                        if (occ) {
                            const int r = wbase + __popc(bal & ((1u << lane) - 1u));
                            if (r < want) {
                                out_rows[out0 + r] = (I)key;
                                out_vals[out0 + r] = vals[s];
                            }
                        }
                    }
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        if (sh.pos != want) atomicOr(c.err, kErrCount);
                        sh.pos = 0;
                    }
                }
                __syncthreads();
            }
        }
    }
    // warp-sized columns: every warp takes kWarpGrab at a time (one counter
    // update per grab), each with a warp-private table. In the numeric pass the
    // table is cleared once and the compaction puts back the slots it reads
    // occupied; the symbolic pass clears it per column.
    constexpr int kWarpGrab = 8;
    if (MODE == 1) {
        V *vals = reinterpret_cast<V *>(smem) + warp * TW;
        uint32_t *keys = reinterpret_cast<uint32_t *>(smem + sizeof(V) * NW * TW) + warp * TW;
        for (int s = lane; s < TW; s += 32) { keys[s] = kEmpty; vals[s] = V(0); }
        __syncwarp();
    }
    for (;;) {
        long long wb = 0;
        if (lane == 0) wb = (long long)atomicAdd(mq.counter + 1, (unsigned long long)kWarpGrab);
        wb = __shfl_sync(SPG_FULL, wb, 0);
        if (wb >= nwarp) break;
        for (long long wi = wb; wi < wb + kWarpGrab && wi < nwarp; ++wi) {
            const int pos = mq.off[1] + (int)wi;
            const int64_t g = mq.list[pos];
            int t = 1;
            while (t < wt && mq.off[t + 1] <= pos) ++t;
            int log2T = 1;   // 2 * cap(t) slots
            while ((1 << log2T) < 2 * tier_cap(t)) ++log2T;
            const int T = 1 << log2T;
            V *vals = reinterpret_cast<V *>(smem) + warp * TW;
            uint32_t *keys = reinterpret_cast<uint32_t *>(smem + sizeof(V) * NW * TW) + warp * TW;
            Src src;
            src.open(sa, g);
            if (MODE == 0) {
                for (int s = lane; s < T; s += 32) keys[s] = kEmpty;
                __syncwarp();
            }
            int mine = 0;
            auto ld = [&](int64_t q, V bv) {
                return RowVal<V>{src.row(q), MODE == 1 ? src.val(q, bv) : V(0)};
            };
            auto ap = [&](const RowVal<V> &e) {
                bool nw;
                const int h = hash_insert_dbl1(keys, log2T, e.r, c.err, nw);
                if (MODE == 0) mine += nw;
                else if (h >= 0) atomic_add_v(&vals[h], e.x);
            };
            warp_walk_flat<4>(src, ld, ap);
            __syncwarp();
            if (MODE == 0) {
                mine = warp_sum(mine);
                if (lane == 0) c.cnt[g] = mine;
            } else {
                const int64_t out0 = c.colptr[g] - c.out_base;
                const int64_t want = c.colptr[g + 1] - c.colptr[g];
                int pos2 = 0;
                for (int s0 = 0; s0 < T; s0 += 32) {
                    const int s = s0 + lane;
                    const uint32_t key = keys[s];
                    const bool occ = key != kEmpty;
                    const unsigned bal = __ballot_sync(SPG_FULL, occ);
                    if (occ) {
                        const int r = pos2 + __popc(bal & ((1u << lane) - 1u));
                        if (r < want) {
                            out_rows[out0 + r] = (I)key;
                            out_vals[out0 + r] = vals[s];
                        }
                        keys[s] = kEmpty;
                        vals[s] = V(0);
                    }
                    pos2 += __popc(bal);
                }
                if (lane == 0 && pos2 != want) atomicOr(c.err, kErrCount);
            }
            __syncwarp();
        }
    }
}

// Table sizes of the heavy columns of the multi-problem product (2 * min(f_j,
// m) slots rounded up to a power of two; 0 for the other columns); their
// exclusive scan places each column's global table.
template <class Src>
__global__ void k_multi_gtab_sizes(typename Src::Args sa, const int64_t *f, const uint8_t *tier, int64_t n,
                                   int64_t *size) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    int64_t sz = 0;
    if (tier[g] >= kHeavyTier0) {
        Src src;
        src.open(sa, g);
        const int64_t m = src.m();
        const int64_t rows = f[g] < m ? f[g] : m;
        sz = 2;
        while (sz < 2 * rows) sz <<= 1;
    }
    size[g] = sz;
}

}  // namespace spg
