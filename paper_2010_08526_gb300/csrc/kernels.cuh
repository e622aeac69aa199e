// Device kernels of the SpGEMM hot path (templates; instantiated per index /
// value type in inst_*.cu).
//
// Work decomposition. Every output column j is formed independently (the
// column form of Gustavson's algorithm, Sec. II-C): C(:,j) = sum over
// B(k,j) != 0 of A(:,k) B(k,j). A "source" describes where the contributions
// (row, value) of column j come from:
//   SrcGemm       -- the products A(i,k) B(k,j), walking A(:,k) for every
//                    B(k,j) in a stage [k0, k1) of the inner dimension;
//   SrcPanel      -- the same products restricted to one row panel, walking
//                    a row-panelised copy of A;
//   SrcParts      -- the entries of column j of several partial results (the
//                    hash merge of Sec. IV-D);
//   SrcPartsPanel -- the same restricted to one row panel, through per-panel
//                    offsets of panel-grouped partial columns, or by filtering.
// Columns are put in tiers by the number of distinct rows they can hold:
//   warp tiers  : one warp per column, 2*cap-slot hash table (cap 32..512);
//   block tiers : one CTA per column, 2*cap-slot hash table (cap 1024..8192);
//   heavy tier  : symbolic -- a shared-memory bitmap over up to ~1.5M rows;
//                 numeric  -- dense accumulation of one row panel in shared
//                 memory per CTA.
// Hash tables are sort-free (Sec. IV-D): rows are emitted in table order.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace spg {

// ---------------------------------------------------------------------------
// Problem table (one entry for a single product; many for batched products)
// ---------------------------------------------------------------------------
template <class I, class V> struct ProbDev {
    const I *ap; const I *ai; const V *av;   // A: colptr, rowidx, vals
    const I *bp; const I *bi; const V *bv;   // B
    int64_t m;       // rows of A and C
    int64_t gcol0;   // first global column of this problem
    int64_t ncols;   // columns of this problem
    int64_t ka;      // columns of A (inner dimension)
};

template <class I, class V>
__device__ __forceinline__ int locate_prob(const ProbDev<I, V> *P, int nprob, int64_t g) {
    if (nprob == 1) return 0;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P[mid].gcol0 <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One partial result of a merge: column g occupies
// [colptr[g] - sub, colptr[g+1] - sub) of rows / vals.
template <class I, class V> struct PartDev {
    const void *colptr;
    int ptr64;
    int64_t sub;
    const I *rows;
    const V *vals;
    const int32_t *pcnt;   // per-panel counts [nheavy * P] when columns are panel-grouped
};

// Arguments shared by all tier kernels (independent of the source).
struct TierCommon {
    int *next_col;           // block-tier column counter (zero before the launch)
    const int32_t *list;     // global column ids, grouped by tier
    const int32_t *list_off; // [kTiers+1] tier offsets in list (device)
    int tier;
    int short_seg, huge_seg;
    int *err;
    int64_t *cnt;            // symbolic output: per global column
    const int64_t *colptr;   // numeric output offsets (global int64 colptr)
    int64_t out_base;        // subtracted from colptr to index the output arrays
    const int64_t *dense_sel;// dense numeric: columns with dense_sel[g] > hash_cap_max
    int hash_cap_max;
    const int32_t *heavy_ord;// heavy ordinal per global column
    int32_t *pcnt;           // symbolic heavy output: per-panel counts [nheavy*P]
    const int32_t *pcnt_in;  // dense numeric: per-panel counts of the output
    int P, log2R;            // numeric panels: count and log2(rows)
    int64_t Rs;              // symbolic bitmap rows per item
    int Q;                   // symbolic panels per column
    int64_t c_lo, c_hi;      // global column range (dense items)
    int item_counts_from_pcnt; // heavy items: take count / offset from pcnt_in (a k-stage)
    int range_cap;             // heavy hash items: at most this many output rows
    const int64_t *flops;      // flops per global column (hybrid accumulator), or null
    int hybrid_sort;           // CTA tiers: sort-accumulate columns with flops <= table size
};

template <class I, class V> struct GemmArgs {
    const ProbDev<I, V> *probs;
    int nprob;
    int64_t k0, k1;
    const int64_t *ap_end;   // row-panelised A: segment ends, index p*ka + c
    const uint16_t *ap_row;  // local rows
    const V *ap_val;
    // A grouped by panel within each column (column k starts at colptr[k] -
    // colptr[0]); apc_off[k*(P+1) + p] = entries of column k in panels < p
    const int32_t *apc_off;
    const uint32_t *apc_row;  // global rows
    const V *apc_val;
    int lean_dense;           // heavy items may use 32-bit entry offsets (nnz(A) < 2^31)
    int lean_sym;             // the heavy symbolic may use 32-bit stream positions too
};

template <class I, class V> struct PartsArgs {
    const PartDev<I, V> *parts;
    int nparts;
    int64_t m;
};

// ---------------------------------------------------------------------------
// Sources
// ---------------------------------------------------------------------------
template <class I, class V> struct SrcGemm {
    using Args = GemmArgs<I, V>;
    using Val = V;
    using Idx = I;
    const ProbDev<I, V> *p;
    int64_t b0, nb, k0, k1;
    __device__ __forceinline__ void open(const Args &a, int64_t g) {
        p = a.probs + locate_prob(a.probs, a.nprob, g);
        const int64_t bc = g - p->gcol0;
        b0 = (int64_t)p->bp[bc];
        nb = (int64_t)p->bp[bc + 1] - b0;
        k0 = a.k0; k1 = a.k1;
    }
    __device__ __forceinline__ int64_t nseg() const { return nb; }
    __device__ __forceinline__ int64_t m() const { return p->m; }
    __device__ __forceinline__ void seg(int64_t e, int64_t &beg, int &len, V &bv, int64_t &tag) const {
        const int64_t pe = b0 + e;
        const int64_t k = (int64_t)__ldg(&p->bi[pe]);
        if (k < k0 || k >= k1) { len = 0; return; }
        const int64_t a0 = (int64_t)__ldg(&p->ap[k]), a1 = (int64_t)__ldg(&p->ap[k + 1]);
        beg = a0; len = (int)(a1 - a0); bv = __ldg(&p->bv[pe]); tag = pe;
    }
    __device__ __forceinline__ uint32_t row(int64_t q) const { return (uint32_t)__ldg(&p->ai[q]); }
    __device__ __forceinline__ V val(int64_t q, V bv) const { return mul_v(__ldg(&p->av[q]), bv); }
    // number of contributions (multiplications) of the column; warp-wide
    __device__ __forceinline__ int64_t flops() const {
        const int lane = threadIdx.x & 31;
        int64_t s = 0;
        for (int64_t e = lane; e < nb; e += 32) {
            const int64_t k = (int64_t)p->bi[b0 + e];
            if (k >= k0 && k < k1) s += (int64_t)p->ap[k + 1] - (int64_t)p->ap[k];
        }
        return warp_sum(s);
    }
};

template <class I, class V> struct SrcParts {
    using Args = PartsArgs<I, V>;
    using Val = V;
    using Idx = I;
    static constexpr int kShift = 40;
    const PartDev<I, V> *parts;
    int nparts;
    int64_t g, mm;
    __device__ __forceinline__ void open(const Args &a, int64_t gg) {
        parts = a.parts; nparts = a.nparts; g = gg; mm = a.m;
    }
    __device__ __forceinline__ int64_t nseg() const { return nparts; }
    __device__ __forceinline__ int64_t m() const { return mm; }
    __device__ __forceinline__ void range(int e, int64_t &beg, int64_t &end) const {
        const PartDev<I, V> &pt = parts[e];
        if (pt.ptr64) {
            const int64_t *cp = (const int64_t *)pt.colptr;
            beg = cp[g] - pt.sub; end = cp[g + 1] - pt.sub;
        } else {
            const int32_t *cp = (const int32_t *)pt.colptr;
            beg = (int64_t)cp[g] - pt.sub; end = (int64_t)cp[g + 1] - pt.sub;
        }
    }
    // entries of part e are addressed as q = e << 40 | index in the part
    __device__ __forceinline__ void seg(int64_t e, int64_t &beg, int &len, V &bv, int64_t &tag) const {
        int64_t b, en;
        range((int)e, b, en);
        beg = (e << kShift) | b; len = (int)(en - b); bv = V(1); tag = e;
    }
    __device__ __forceinline__ uint32_t row(int64_t q) const {
        return (uint32_t)parts[q >> kShift].rows[q & ((1ll << kShift) - 1)];
    }
    __device__ __forceinline__ V val(int64_t q, V) const {
        return parts[q >> kShift].vals[q & ((1ll << kShift) - 1)];
    }
    __device__ __forceinline__ int64_t flops() const {
        const int lane = threadIdx.x & 31;
        int64_t s = 0;
        for (int e = lane; e < nparts; e += 32) {
            int64_t b, en;
            range(e, b, en);
            s += en - b;
        }
        return warp_sum(s);
    }
};

// Dense sources: contributions of column g restricted to row panel pnl;
// lrow(q) is the row local to the panel, or -1 when outside it.
template <class I, class V> struct SrcPanel {
    using Args = GemmArgs<I, V>;
    using Val = V;
    using Idx = I;
    const ProbDev<I, V> *p;
    const int64_t *ape;
    const uint16_t *apr;
    const V *apv;
    int64_t b0, nb, k0, k1, pk;
    __device__ __forceinline__ void open(const Args &a, const TierCommon &, int64_t g, int pnl, int) {
        p = a.probs;
        const int64_t bc = g - p->gcol0;
        b0 = (int64_t)p->bp[bc];
        nb = (int64_t)p->bp[bc + 1] - b0;
        k0 = a.k0; k1 = a.k1;
        pk = (int64_t)pnl * p->ka;
        ape = a.ap_end; apr = a.ap_row; apv = a.ap_val;
    }
    __device__ __forceinline__ int64_t nseg() const { return nb; }
    __device__ __forceinline__ void seg(int64_t e, int64_t &beg, int &len, V &bv, int64_t &tag) const {
        const int64_t pe = b0 + e;
        const int64_t k = (int64_t)__ldg(&p->bi[pe]);
        if (k < k0 || k >= k1) { len = 0; return; }
        const int64_t idx = pk + k;
        const int64_t s = idx ? __ldg(&ape[idx - 1]) : 0;
        beg = s; len = (int)(__ldg(&ape[idx]) - s); bv = __ldg(&p->bv[pe]); tag = pe;
    }
    __device__ __forceinline__ int lrow(int64_t q) const { return (int)__ldg(&apr[q]); }
    __device__ __forceinline__ V val(int64_t q, V bv) const { return mul_v(__ldg(&apv[q]), bv); }
};

template <class I, class V> struct SrcPartsPanel {
    using Args = PartsArgs<I, V>;
    using Val = V;
    using Idx = I;
    static constexpr int kShift = 40;
    SrcParts<I, V> base;
    int pnl, h, P;
    int64_t r0, R;
    __device__ __forceinline__ void open(const Args &a, const TierCommon &c, int64_t g, int pp, int hh) {
        base.open(a, g);
        pnl = pp; h = hh; P = c.P;
        R = 1ll << c.log2R;
        r0 = (int64_t)pp << c.log2R;
    }
    __device__ __forceinline__ int64_t nseg() const { return base.nparts; }
    __device__ __forceinline__ void seg(int64_t e, int64_t &beg, int &len, V &bv, int64_t &tag) const {
        int64_t b, en;
        base.range((int)e, b, en);
        const int32_t *pc = base.parts[e].pcnt;
        if (pc) {   // panel-grouped column: skip the lower panels
            const int32_t *row = pc + (int64_t)h * P;
            int64_t off = 0;
            for (int q = 0; q < pnl; ++q) off += row[q];
            b += off;
            en = b + row[pnl];
        }
        beg = (e << kShift) | b; len = (int)(en - b); bv = V(1); tag = e;
    }
    __device__ __forceinline__ int lrow(int64_t q) const {
        const int64_t r = (int64_t)base.row(q) - r0;
        return (r >= 0 && r < R) ? (int)r : -1;
    }
    __device__ __forceinline__ V val(int64_t q, V) const { return base.val(q, V(1)); }
};

// ---------------------------------------------------------------------------
// Segment walkers. A segment is a run [beg, beg+len) of source entries
// scaled by bv; tag names the B entry (or part) it came from.
// emit(q, bv, tag) handles one entry.
// ---------------------------------------------------------------------------

// Warp-level: every lane holds one segment. Segments of up to short_seg
// entries are walked by their lane; longer ones by the whole warp, one after
// another (coalesced reads). All 32 lanes must call it.
template <class V, class Emit>
__device__ __forceinline__ void warp_walk(int64_t beg, int len, V bv, int64_t tag, int short_seg,
                                          Emit &emit) {
    const int lane = threadIdx.x & 31;
    unsigned longmask = __ballot_sync(SPG_FULL, len > short_seg);
    if (len <= short_seg) {
        for (int i = 0; i < len; ++i) emit(beg + i, bv, tag);
    }
    while (longmask) {
        const int src = __ffs(longmask) - 1;
        longmask &= longmask - 1;
        const int64_t b = __shfl_sync(SPG_FULL, beg, src);
        const int l = __shfl_sync(SPG_FULL, len, src);
        const V v = __shfl_sync(SPG_FULL, bv, src);
        const int64_t tg = __shfl_sync(SPG_FULL, tag, src);
        for (int i = lane; i < l; i += 32) emit(b + i, v, tg);
    }
}

constexpr int kMaxBlock = 1024;

// Per-CTA scratch of the load-balanced walk: the non-empty segments of the
// current chunk, compacted, with their start in the flattened product stream.
template <class V, int MB = kMaxBlock> struct BlockShared {
    int64_t start[MB + 1];
    int64_t qb[MB];            // beg - start: entry index = qb[s] + stream position
    int64_t tag[MB];
    V bv[MB];
    int64_t red64[33];
    int nz;
    int pos;
    unsigned long long tot;
    int red[32];
};

// Block-level load-balanced walk over the segments of src. emit(q, bv, tag,
// valid) is called by all 32 lanes of a warp together (warp-synchronous
// emits may use warp intrinsics); lanes with valid == false carry no entry. Each chunk of
// blockDim segments is compacted to its non-empty segments and prefix-summed
// into a flattened product stream [0, T); every warp takes an equal
// contiguous share of the stream in 32-wide windows, and lane l of a window
// finds its segment from a bitmask of the segment starts inside the window.
// Consecutive lanes read consecutive entries of a segment (coalesced). All
// threads must call it; it ends with a __syncthreads.
//
// U > 0 selects the batched form, for emit = load_apply(load, apply):
// load(q, bv, tag) reads entry q (global loads only) and apply(loaded, valid)
// consumes it; the walker issues the loads of U windows before the first
// apply. An update in shared memory consumes its load and a warp issues in
// order, so this keeps U gathers in flight per warp instead of one.
template <class Load, class Apply> struct LoadApply {
    Load load;
    Apply apply;
    // the entries of the U windows of a batch, in order
    template <int U, class L>
    __device__ __forceinline__ void apply_all(const L (&l)[U], const bool (&ok)[U]) {
#pragma unroll
        for (int u = 0; u < U; ++u) apply(l[u], ok[u]);
    }
};
template <class Load, class Apply>
__device__ __forceinline__ LoadApply<Load, Apply> load_apply(Load l, Apply a) {
    return LoadApply<Load, Apply>{l, a};
}
// The same with one call for a whole batch: all(l, ok) takes the arrays of
// the U windows (a lane's U entries), so their updates can overlap.
template <class Load, class All> struct LoadApplyAll {
    Load load;
    All all;
    template <int U, class L>
    __device__ __forceinline__ void apply_all(const L (&l)[U], const bool (&ok)[U]) { all(l, ok); }
    template <class L> __device__ __forceinline__ void apply(const L &x, bool v) {
        const L a[1] = {x};
        const bool o[1] = {v};
        all(a, o);
    }
};
template <class Load, class All>
__device__ __forceinline__ LoadApplyAll<Load, All> load_apply_all(Load l, All a) {
    return LoadApplyAll<Load, All>{l, a};
}
// windows of gathers in flight per warp in the batched walks
constexpr int kWalkBatch = 4;

template <class V> struct RowVal {
    uint32_t r;
    V x;
};

template <int U = 0, class Src, class Emit, int MB>
__device__ __forceinline__ void block_walk(const Src &src, Emit &emit, int short_seg, int,
                                           BlockShared<typename Src::Val, MB> &sh) {
    using V = typename Src::Val;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int64_t nseg = src.nseg();
    for (int64_t base = 0; base < nseg; base += blockDim.x) {
        const int64_t e = base + threadIdx.x;
        int64_t beg = 0, tag = 0;
        int len = 0;
        V bv = V(0);
        if (e < nseg) src.seg(e, beg, len, bv, tag);
        // short segments: each lane walks its own, in a warp-uniform loop
        // bounded by the warp's longest short segment
        {
            const int mine = len <= short_seg ? len : 0;
            const int wmax = __reduce_max_sync(SPG_FULL, (unsigned)mine);
            for (int i = 0; i < wmax; ++i) {
                if constexpr (U == 0) {
                    emit(beg + i, bv, tag, i < mine);
                } else {
                    const bool v = i < mine;
                    decltype(emit.load(beg, bv, tag)) l{};
                    if (v) l = emit.load(beg + i, bv, tag);
                    emit.apply(l, v);
                }
            }
            if (len <= short_seg) len = 0;
        }
        // longer segments: block scan of (nonempty << 40 | len) gives the
        // compacted slot and the start in the flattened product stream
        const int64_t key = ((int64_t)(len > 0) << 40) | (int64_t)len;
        int64_t incl = warp_incl_scan(key);
        if (lane == 31) sh.red64[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t w = lane < nw ? sh.red64[lane] : 0;
            int64_t wi = warp_incl_scan(w);
            sh.red64[lane] = wi - w;
            if (lane == 31) sh.red64[32] = wi;
        }
        __syncthreads();
        const int64_t ex = sh.red64[warp] + incl - key;
        if (len > 0) {
            const int slot = (int)(ex >> 40);
            const int64_t st0 = ex & ((1ll << 40) - 1);
            sh.start[slot] = st0;
            sh.qb[slot] = beg - st0;
            sh.bv[slot] = bv;
            sh.tag[slot] = tag;
        }
        const int64_t tot = sh.red64[32];
        const int nz = (int)(tot >> 40);
        const int64_t T = tot & ((1ll << 40) - 1);
        __syncthreads();   // (start[nz] is never read: lookups stop at nz - 1)
        if (T > 0) {
            // this warp's share of [0, T), in whole windows
            const int64_t nwin = (T + 31) >> 5;
            const int64_t per = (nwin + nw - 1) / nw;
            const int64_t p0 = (int64_t)warp * per * 32;
            int64_t p1 = p0 + per * 32;
            if (p1 > T) p1 = T;
            if (p0 < p1) {
                // last segment starting at or before p0
                int lo = 0, hi = nz - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (sh.start[mid] <= p0) lo = mid; else hi = mid - 1;
                }
                int s_lo = lo;
                // cached state of segment s_lo: end of it in the stream, entry
                // index base, scale, tag
                int64_t seg_end = (s_lo + 1 < nz) ? sh.start[s_lo + 1] : T;
                int64_t qbase = sh.qb[s_lo];
                V bvc = sh.bv[s_lo];
                int64_t tagc = sh.tag[s_lo];
                // lane assignment of the window starting at wb; advances s_lo
                auto window = [&](int64_t wb, int64_t &q, V &bv, int64_t &tg, bool &valid) {
                    const int64_t t = wb + lane;
                    valid = t < p1;
                    if (wb + 32 <= seg_end) {          // the window lies in segment s_lo
                        q = qbase + t; bv = bvc; tg = tagc;
                        if (wb + 32 == seg_end && s_lo + 1 < nz) {
                            ++s_lo;
                            seg_end = (s_lo + 1 < nz) ? sh.start[s_lo + 1] : T;
                            qbase = sh.qb[s_lo]; bvc = sh.bv[s_lo]; tagc = sh.tag[s_lo];
                        }
                        return;
                    }
                    // the window crosses segment starts: lane l's segment is
                    // s_lo plus the number of starts at positions 1..l
                    const int j = s_lo + 1 + lane;
                    unsigned bit = 0u;
                    if (j < nz) {
                        const int64_t d = sh.start[j] - wb;
                        if (d < 32) bit = 1u << (int)d;
                    }
                    const unsigned M = __reduce_or_sync(SPG_FULL, bit);
                    const int sg = s_lo + __popc(M & (0xffffffffu >> (31 - lane)));
                    const int sgv = valid ? sg : s_lo;
                    q = sh.qb[sgv] + (valid ? t : sh.start[sgv]);
                    bv = sh.bv[sgv]; tg = sh.tag[sgv];
                    s_lo += __popc(M);
                    if (s_lo + 1 < nz && sh.start[s_lo + 1] == wb + 32) ++s_lo;
                    seg_end = (s_lo + 1 < nz) ? sh.start[s_lo + 1] : T;
                    qbase = sh.qb[s_lo]; bvc = sh.bv[s_lo]; tagc = sh.tag[s_lo];
                };
                if constexpr (U > 0) {
                  if (T < (1ll << 31) - 64) {
                    // 32-bit stream positions (T fits): the same walk with
                    // int arithmetic for the window bookkeeping
                    const int P1 = (int)p1, TT = (int)T;
                    int send = (int)seg_end;
                    auto window32 = [&](int wb, int64_t &q, V &bv, int64_t &tg, bool &valid) {
                        const int t = wb + lane;
                        valid = t < P1;
                        if (wb + 32 <= send) {
                            q = qbase + t; bv = bvc; tg = tagc;
                            if (wb + 32 == send && s_lo + 1 < nz) {
                                ++s_lo;
                                send = (s_lo + 1 < nz) ? (int)sh.start[s_lo + 1] : TT;
                                qbase = sh.qb[s_lo]; bvc = sh.bv[s_lo]; tagc = sh.tag[s_lo];
                            }
                            return;
                        }
                        const int j = s_lo + 1 + lane;
                        unsigned bit = 0u;
                        if (j < nz) {
                            const int d = (int)sh.start[j] - wb;
                            if (d < 32) bit = 1u << d;
                        }
                        const unsigned M = __reduce_or_sync(SPG_FULL, bit);
                        const int sg = s_lo + __popc(M & (0xffffffffu >> (31 - lane)));
                        q = sh.qb[sg] + t;
                        bv = sh.bv[sg]; tg = sh.tag[sg];
                        s_lo += __popc(M);
                        if (s_lo + 1 < nz && (int)sh.start[s_lo + 1] == wb + 32) ++s_lo;
                        send = (s_lo + 1 < nz) ? (int)sh.start[s_lo + 1] : TT;
                        qbase = sh.qb[s_lo]; bvc = sh.bv[s_lo]; tagc = sh.tag[s_lo];
                    };
                    for (int wb = (int)p0; wb < P1; wb += 32 * U) {
                        int64_t q[U], tg[U];
                        V b[U];
                        bool ok[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            if (wb + 32 * u < P1) {
                                window32(wb + 32 * u, q[u], b[u], tg[u], ok[u]);
                            } else {
                                q[u] = 0; tg[u] = 0; b[u] = V(0); ok[u] = false;
                            }
                        }
                        decltype(emit.load(q[0], b[0], tg[0])) l[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            l[u] = {};
                            if (ok[u]) l[u] = emit.load(q[u], b[u], tg[u]);
                        }
                        emit.apply_all(l, ok);
                    }
                  } else
                    for (int64_t wb = p0; wb < p1; wb += 32 * U) {
                        int64_t q[U], tg[U];
                        V b[U];
                        bool ok[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            if (wb + 32 * u < p1) {
                                window(wb + 32 * u, q[u], b[u], tg[u], ok[u]);
                            } else {
                                q[u] = 0; tg[u] = 0; b[u] = V(0); ok[u] = false;
                            }
                        }
                        decltype(emit.load(q[0], b[0], tg[0])) l[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            l[u] = {};
                            if (ok[u]) l[u] = emit.load(q[u], b[u], tg[u]);
                        }
                        emit.apply_all(l, ok);
                    }
                } else
                for (int64_t wb = p0; wb < p1;) {
                    if (wb + 128 <= seg_end && wb + 128 <= p1) {
                        // four whole windows inside segment s_lo: independent
                        // products back to back (their loads overlap)
                        const int64_t q0 = qbase + wb + lane;
                        emit(q0, bvc, tagc, true);
                        emit(q0 + 32, bvc, tagc, true);
                        emit(q0 + 64, bvc, tagc, true);
                        emit(q0 + 96, bvc, tagc, true);
                        wb += 128;
                        if (wb == seg_end && s_lo + 1 < nz) {
                            ++s_lo;
                            seg_end = (s_lo + 1 < nz) ? sh.start[s_lo + 1] : T;
                            qbase = sh.qb[s_lo]; bvc = sh.bv[s_lo]; tagc = sh.tag[s_lo];
                        }
                        continue;
                    }
                    int64_t q;
                    V v;
                    int64_t tg;
                    bool ok;
                    window(wb, q, v, tg, ok);
                    emit(q, v, tg, ok);
                    wb += 32;
                }
            }
        }
        __syncthreads();
    }
}

// Warp walk over all segments of src (one warp per column).
template <class Src, class Emit>
__device__ __forceinline__ void warp_walk_all(const Src &src, Emit &emit, int short_seg) {
    using V = typename Src::Val;
    const int lane = threadIdx.x & 31;
    const int64_t nb = src.nseg();
    for (int64_t base = 0; base < nb; base += 32) {
        int64_t beg = 0, tag = 0;
        int len = 0;
        V bv = V(0);
        if (base + lane < nb) src.seg(base + lane, beg, len, bv, tag);
        warp_walk(beg, len, bv, tag, short_seg, emit);
    }
}

// A value's bits through a warp shuffle (any 4- or 8-byte value type).
template <class V> __device__ __forceinline__ V shfl_bits(V v, int src) {
    static_assert(sizeof(V) == 4 || sizeof(V) == 8, "4- or 8-byte values");
    if constexpr (sizeof(V) == 4) {
        uint32_t b;
        memcpy(&b, &v, 4);
        b = __shfl_sync(SPG_FULL, b, src);
        memcpy(&v, &b, 4);
    } else {
        unsigned long long b;
        memcpy(&b, &v, 8);
        b = __shfl_sync(SPG_FULL, b, src);
        memcpy(&v, &b, 8);
    }
    return v;
}

// Warp-level load-balanced walk over src's segments, for one warp per column:
// per round of 32 B entries (one per lane) the products form a flattened
// stream [0, T), walked in 32-wide windows; lane j of a window takes position
// p, whose segment is the last lane with stream start <= p (a 5-step shuffle
// search over the lanes' exclusive prefix). load(q, bv) reads entry q (global
// loads only) and apply(loaded) consumes it; the loads of U windows are
// issued before the first apply, so a lane keeps U gathers in flight rather
// than walking its own segment one entry at a time.
template <int U, class Src, class Load, class Apply>
__device__ __forceinline__ void warp_walk_flat(const Src &src, Load &load, Apply &apply) {
    using V = typename Src::Val;
    using L = decltype(load(int64_t(0), V(0)));
    const int lane = threadIdx.x & 31;
    const int64_t nb = src.nseg();
    for (int64_t base = 0; base < nb; base += 32) {
        int64_t beg = 0, tag = 0;
        int len = 0;
        V bv = V(0);
        if (base + lane < nb) src.seg(base + lane, beg, len, bv, tag);
        const int incl = warp_incl_scan(len);
        const int excl = incl - len;
        const int T = __shfl_sync(SPG_FULL, incl, 31);
        for (int w = 0; w < T; w += 32 * U) {
            L x[U];
            bool ok[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = w + 32 * u + lane;
                ok[u] = p < T;
                int sl = 0;
#pragma unroll
                for (int b = 16; b > 0; b >>= 1) {
                    const int e = __shfl_sync(SPG_FULL, excl, sl + b);
                    if (e <= p) sl += b;
                }
                const int64_t bs = __shfl_sync(SPG_FULL, beg, sl);
                const int es = __shfl_sync(SPG_FULL, excl, sl);
                const V vs = shfl_bits(bv, sl);
                if (ok[u]) x[u] = load(bs + (p - es), vs);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (ok[u]) apply(x[u]);
        }
    }
}

// ---------------------------------------------------------------------------
// Shared-memory hash tables (linear probing, 32-bit keys)
// ---------------------------------------------------------------------------

// Insert key; returns its slot and sets is_new when this call claimed it.
// Returns -1 (and records kErrProbe) if the table is full -- impossible when
// the table has more slots than the column has distinct rows.
__device__ __forceinline__ int hash_insert(uint32_t *keys, int log2T, uint32_t key, bool &is_new,
                                           int *err) {
    const uint32_t mask = (1u << log2T) - 1u;
    uint32_t h = hash_slot(key, log2T);
    is_new = false;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint32_t cur = keys[h];
        if (cur == key) return (int)h;
        if (cur == kEmpty) {
            const uint32_t old = atomicCAS(&keys[h], kEmpty, key);
            if (old == kEmpty) { is_new = true; return (int)h; }
            if (old == key) return (int)h;
        }
        h = (h + 1) & mask;
    }
    atomicOr(err, kErrProbe);
    return -1;
}

// Insert key with double hashing (an odd step from a second multiplicative
// hash, so the probe sequence visits every slot); each probe is one
// compare-and-swap, the cheap form when most keys are new. Returns the slot,
// or -1 (recording kErrProbe) for a full table.
__device__ __forceinline__ int hash_insert_dbl1(uint32_t *keys, int log2T, uint32_t key, int *err,
                                                bool &is_new) {
    const uint32_t mask = (1u << log2T) - 1u;
    uint32_t h = hash_slot(key, log2T);
    const uint32_t step = ((key * 0x85EBCA6Bu) >> (32 - log2T)) | 1u;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint32_t cur = atomicCAS(&keys[h], kEmpty, key);
        if (cur == kEmpty || cur == key) {
            is_new = cur == kEmpty;
            return (int)h;
        }
        h = (h + step) & mask;
    }
    is_new = false;
    atomicOr(err, kErrProbe);
    return -1;
}
__device__ __forceinline__ int hash_insert_dbl1(uint32_t *keys, int log2T, uint32_t key, int *err) {
    bool is_new;
    return hash_insert_dbl1(keys, log2T, key, err, is_new);
}

// hash_insert for a lane's U keys at once (kEmpty = no key): every round
// issues the probe loads of all pending keys, then the CAS of those that met
// an empty slot, then resolves them, so the U probe chains overlap instead of
// running one after another. slot[u] = the key's slot, -1 for no key (or a
// full table, which sets kErrProbe).
template <int U>
__device__ __forceinline__ void hash_insert_all(uint32_t *keys, int log2T, const uint32_t (&key)[U],
                                                int (&slot)[U], int *err) {
    const uint32_t mask = (1u << log2T) - 1u;
    uint32_t h[U];
    unsigned pending = 0u;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        slot[u] = -1;
        h[u] = hash_slot(key[u], log2T);
        if (key[u] != kEmpty) pending |= 1u << u;
    }
    for (uint32_t probe = 0; pending && probe <= mask; ++probe) {
        uint32_t cur[U];
#pragma unroll
        for (int u = 0; u < U; ++u) cur[u] = ((pending >> u) & 1u) ? keys[h[u]] : 0u;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (((pending >> u) & 1u) && cur[u] == kEmpty) cur[u] = atomicCAS(&keys[h[u]], kEmpty, key[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!((pending >> u) & 1u)) continue;
            if (cur[u] == kEmpty || cur[u] == key[u]) {
                slot[u] = (int)h[u];
                pending &= ~(1u << u);
            } else {
                h[u] = (h[u] + 1u) & mask;
            }
        }
    }
    if (pending) atomicOr(err, kErrProbe);
}

// Exclusive prefix of the per-warp values n over the block's warps (all
// threads call it; red holds >= nw ints). Contains one __syncthreads, and
// red may be reused after the next one.
__device__ __forceinline__ int warp_offset(int n, int *red, int warp, int nw, int lane) {
    if (lane == 0) red[warp] = n;
    __syncthreads();
    const int v = lane < nw ? red[lane] : 0;
    const int incl = warp_incl_scan(v);
    return __shfl_sync(SPG_FULL, incl - v, warp & 31);
}

// Lookup only; -1 when absent.
__device__ __forceinline__ int hash_find(const uint32_t *keys, int log2T, uint32_t key) {
    const uint32_t mask = (1u << log2T) - 1u;
    uint32_t h = hash_slot(key, log2T);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint32_t cur = keys[h];
        if (cur == key) return (int)h;
        if (cur == kEmpty) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

template <int T> struct Log2 { static constexpr int v = 1 + Log2<T / 2>::v; };
template <> struct Log2<1> { static constexpr int v = 0; };

// ---------------------------------------------------------------------------
// K1: contributions per column (flops for a product) and tier binning
// ---------------------------------------------------------------------------
__device__ __forceinline__ int heavy_subtier(int64_t u) {
    const int lg = 63 - __clzll((unsigned long long)(u | 1));
    const int h = kHeavyTier0 + (lg - 13 < 0 ? 0 : lg - 13);
    return h > kTiers - 1 ? kTiers - 1 : h;
}

__device__ __forceinline__ int hash_tier_of(int64_t u, int hash_cap_max) {
    if (u == 0) return 0;
    for (int t = 1; t <= 8; ++t) {
        const int cap = tier_cap(t);
        if (cap > hash_cap_max) break;
        if (u <= cap) return t;
    }
    return -1;
}

// One warp per column computes f_j, the number of contributions; the CTA
// keeps a tier histogram. bound (optional) is the exact count of the unsplit
// product when a k-stage is binned: columns with bound > hash_cap_max go to
// the heavy tier (their stage output must be panel-grouped), others use
// min(f, bound) as their size.
template <class Src>
__global__ void __launch_bounds__(256) k_flops_bin(typename Src::Args sa, int64_t c_lo,
                                                   int64_t c_hi, int hash_cap_max,
                                                   const int64_t *bound, int64_t *f_out,
                                                   uint8_t *tier_out, int64_t *cnt_out,
                                                   int32_t *tier_hist) {
    __shared__ int s_hist[kTiers];
    if (threadIdx.x < kTiers) s_hist[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t cbase = c_lo + (int64_t)blockIdx.x * 256;
    for (int c = 0; c < 32; ++c) {
        const int64_t g = cbase + warp * 32 + c;
        if (g >= c_hi) break;
        Src src;
        src.open(sa, g);
        const int64_t f = src.flops();
        if (lane == 0) {
            int64_t u = f < src.m() ? f : src.m();
            int t;
            if (bound && bound[g] > hash_cap_max) {
                t = heavy_subtier(f);
            } else {
                if (bound && bound[g] < u) u = bound[g];
                t = hash_tier_of(u, hash_cap_max);
                if (t < 0) t = heavy_subtier(u);
            }
            if (f_out) f_out[g] = f;
            tier_out[g] = (uint8_t)t;
            if (cnt_out) cnt_out[g] = 0;
            if (t) atomicAdd(&s_hist[t], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x < kTiers && s_hist[threadIdx.x])
        atomicAdd(&tier_hist[threadIdx.x], s_hist[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// K2: symbolic hash tiers (count distinct rows per column)
// ---------------------------------------------------------------------------
template <class Src, int T>
__global__ void __launch_bounds__(256) k_sym_warp(typename Src::Args sa, TierCommon c) {
    constexpr int LOG2T = Log2<T>::v;
    using V = typename Src::Val;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *keys = reinterpret_cast<uint32_t *>(smem) + warp * T;
    const int lo = c.list_off[c.tier], hi = c.list_off[c.tier + 1];
    const int nwarps = gridDim.x * 8;
    for (int it = lo + blockIdx.x * 8 + warp; it < hi; it += nwarps) {
        const int64_t g = c.list[it];
        Src src;
        src.open(sa, g);
        for (int s = lane; s < T; s += 32) keys[s] = kEmpty;
        __syncwarp();
        int mine = 0;
        auto ld = [&](int64_t q, V) { return src.row(q); };
        auto ap = [&](uint32_t r) {
            bool nw;
            hash_insert_dbl1(keys, LOG2T, r, c.err, nw);
            mine += nw;
        };
        warp_walk_flat<4>(src, ld, ap);
        mine = warp_sum(mine);
        if (lane == 0) c.cnt[g] = mine;
        __syncwarp();
    }
}

template <class Src, int T>
__global__ void k_sym_block(typename Src::Args sa, TierCommon c) {
    constexpr int LOG2T = Log2<T>::v;
    using V = typename Src::Val;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *keys = reinterpret_cast<uint32_t *>(smem);
    __shared__ BlockShared<V> sh;
    __shared__ int s_it;
    const int lo = c.list_off[c.tier], hi = c.list_off[c.tier + 1];
    // columns are taken in list order from a device counter, one per CTA at a
    // time; thread 0 reserves the next one when it starts a column
    int ahead = 0;
    if (threadIdx.x == 0) ahead = atomicAdd(c.next_col, 1);
    auto fetch = [&]() -> int {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_it = lo + ahead;
            ahead = atomicAdd(c.next_col, 1);
        }
        __syncthreads();
        return s_it;
    };
    for (int it = fetch(); it < hi; it = fetch()) {
        const int64_t g = c.list[it];
        Src src;
        src.open(sa, g);
        for (int s = threadIdx.x; s < T; s += blockDim.x) keys[s] = kEmpty;
        __syncthreads();
        int mine = 0;
        auto emit = load_apply([&](int64_t q, V, int64_t) { return src.row(q); },
                               [&](uint32_t r, bool valid) {
                                   if (!valid) return;
                                   bool nw;
                                   hash_insert_dbl1(keys, LOG2T, r, c.err, nw);
                                   mine += nw;
                               });
        block_walk<kWalkBatch>(src, emit, c.short_seg, c.huge_seg, sh);
        mine = warp_sum(mine);
        if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = mine;
        __syncthreads();
        if (threadIdx.x < 32) {
            int v = threadIdx.x < (int)(blockDim.x >> 5) ? sh.red[threadIdx.x] : 0;
            v = warp_sum(v);
            if (threadIdx.x == 0) c.cnt[g] = v;
        }
    }
}

// Heavy symbolic: a shared-memory bitmap over Rs rows. Items are (symbolic
// panel q, heavy column), largest heavy sub-tier first. Writes per numeric
// panel counts pcnt[h*P + p] and adds the column total to cnt[g].
template <class Src>
__global__ void __launch_bounds__(1024, 1) k_sym_bitmap(typename Src::Args sa, TierCommon c) {
    using V = typename Src::Val;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *bm = reinterpret_cast<uint32_t *>(smem);
    __shared__ BlockShared<V> sh;
    const int nwords_max = (int)((c.Rs + 31) >> 5);
    for (int w = threadIdx.x; w < nwords_max; w += blockDim.x) bm[w] = 0u;
    if (threadIdx.x == 0) { sh.tot = 0; }
    __syncthreads();
    const int lo = c.list_off[kHeavyTier0], hi = c.list_off[kTiers];
    const int64_t nitems = (int64_t)(hi - lo) * c.Q;
    const int wordsR = 1 << (c.log2R - 5);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // items are taken from a device counter, one per CTA at a time
    __shared__ int s_item;
    auto fetch = [&]() -> int64_t {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(c.next_col, 1);
        __syncthreads();
        return s_item;
    };
    for (int64_t item = fetch(); item < nitems; item = fetch()) {
        const int64_t ri = nitems - 1 - item;   // list is ascending in sub-tier
        const int hpos = (int)(ri / c.Q);
        const int q = (int)(ri % c.Q);
        const int64_t g = c.list[lo + hpos];
        Src src;
        src.open(sa, g);
        const int64_t r0 = (int64_t)q * c.Rs;
        const int64_t mrows = src.m();
        const int64_t rows = (mrows - r0) < c.Rs ? (mrows - r0) : c.Rs;
        const int nwords = (int)((rows + 31) >> 5);
        const bool filt = c.Q > 1;
        auto emit = load_apply([&](int64_t qq, V, int64_t) { return src.row(qq); },
                               [&](uint32_t rr, bool valid) {
                                   if (!valid) return;
                                   int64_t r = (int64_t)rr;
                                   if (filt) {
                                       r -= r0;
                                       if (r < 0 || r >= rows) return;
                                   }
                                   atomicOr(&bm[r >> 5], 1u << (r & 31));
                               });
        block_walk<kWalkBatch>(src, emit, c.short_seg, c.huge_seg, sh);
        const int h = c.heavy_ord[g];
        const int p0 = (int)(r0 >> c.log2R);
        const int np = (nwords + wordsR - 1) / wordsR;
        for (int pp = warp; pp < np; pp += nw) {
            const int w0 = pp * wordsR;
            const int w1 = (w0 + wordsR) < nwords ? (w0 + wordsR) : nwords;
            int cntp = 0;
            for (int w = w0 + lane; w < w1; w += 32) { cntp += __popc(bm[w]); bm[w] = 0u; }
            cntp = warp_sum(cntp);
            if (lane == 0) {
                c.pcnt[(int64_t)h * c.P + p0 + pp] = cntp;
                if (cntp) atomicAdd(&sh.tot, (unsigned long long)cntp);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (c.Q == 1) c.cnt[g] = (int64_t)sh.tot;
            else atomicAdd(reinterpret_cast<unsigned long long *>(&c.cnt[g]), sh.tot);
            sh.tot = 0;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// K3 / K4: numeric hash tiers (products or merge), unsorted output
// ---------------------------------------------------------------------------
template <class Src, int T>
__global__ void __launch_bounds__(256) k_num_warp(typename Src::Args sa, TierCommon c,
                                                  typename Src::Idx *out_rows,
                                                  typename Src::Val *out_vals) {
    constexpr int LOG2T = Log2<T>::v;
    using V = typename Src::Val;
    using I = typename Src::Idx;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    V *vals = reinterpret_cast<V *>(smem) + warp * T;
    uint32_t *keys = reinterpret_cast<uint32_t *>(smem + sizeof(V) * 8 * T) + warp * T;
    const int lo = c.list_off[c.tier], hi = c.list_off[c.tier + 1];
    const int nwarps = gridDim.x * 8;
    // the table is cleared once; the compaction puts back the slots it reads
    // occupied, so it is clean again for the warp's next column
    for (int s = lane; s < T; s += 32) { keys[s] = kEmpty; vals[s] = V(0); }
    __syncwarp();
    for (int it = lo + blockIdx.x * 8 + warp; it < hi; it += nwarps) {
        const int64_t g = c.list[it];
        Src src;
        src.open(sa, g);
        auto ld = [&](int64_t q, V bv) { return RowVal<V>{src.row(q), src.val(q, bv)}; };
        auto ap = [&](const RowVal<V> &e) {
            const int h = hash_insert_dbl1(keys, LOG2T, e.r, c.err);
            if (h >= 0) atomic_add_v(&vals[h], e.x);
        };
        warp_walk_flat<4>(src, ld, ap);
        __syncwarp();
        const int64_t out0 = c.colptr[g] - c.out_base;
        const int64_t want = c.colptr[g + 1] - c.colptr[g];
        int pos = 0;
        for (int s0 = 0; s0 < T; s0 += 32) {
            const int s = s0 + lane;
            const uint32_t key = keys[s];
            const bool occ = key != kEmpty;
            const unsigned bal = __ballot_sync(SPG_FULL, occ);
            if (occ) {
                const int r = pos + __popc(bal & ((1u << lane) - 1u));
                if (r < want) {
                    out_rows[out0 + r] = (I)key;
                    out_vals[out0 + r] = vals[s];
                }
                keys[s] = kEmpty;
                vals[s] = V(0);
            }
            pos += __popc(bal);
        }
        if (lane == 0 && pos != want) atomicOr(c.err, kErrCount);
        __syncwarp();
    }
}

// Bitonic sort of one segment of n <= CAP entries in shared memory (keys
// padded with 0xffffffff to the next power of two). All threads call it.
template <int CAP, class V>
__device__ __forceinline__ void block_bitonic(uint32_t *sk, V *sv, int n) {
    int np2 = 1;
    while (np2 < n) np2 <<= 1;
    for (int i = n + threadIdx.x; i < np2; i += blockDim.x) { sk[i] = 0xffffffffu; sv[i] = V(0); }
    __syncthreads();
    for (int k = 2; k <= np2; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < np2; i += blockDim.x) {
                const int l = i ^ jj;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const uint32_t a = sk[i], b = sk[l];
                    if (up ? a > b : a < b) {
                        sk[i] = b; sk[l] = a;
                        const V t = sv[i]; sv[i] = sv[l]; sv[l] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Sort-based accumulation of one column, the hybrid accumulator's other
// half: with few products per distinct row (low compression), appending the
// products and sorting them by row can replace the hash. The products are
// appended to keys / vals (T slots; the caller checked flops <= T) with one
// shared counter bump per warp window, sorted by row (block bitonic), and
// each run of equal rows is summed in sorted order with the semiring's sum.
// The column is written in ascending row order. sh.pos is 0 on entry and on
// return; all threads call it; it ends with a barrier.
template <class Src, int T>
__device__ __forceinline__ void num_block_sorted(const Src &src, const TierCommon &c, uint32_t *keys,
                                                 typename Src::Val *vals, BlockShared<typename Src::Val> &sh,
                                                 int64_t out0, int64_t want, typename Src::Idx *out_rows,
                                                 typename Src::Val *out_vals) {
    using V = typename Src::Val;
    using I = typename Src::Idx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    auto emit = load_apply(
        [&](int64_t q, V bv, int64_t) { return RowVal<V>{src.row(q), src.val(q, bv)}; },
        [&](const RowVal<V> &e, bool valid) {
            const bool ok = valid && e.r != kEmpty;
            const unsigned bal = __ballot_sync(SPG_FULL, ok);
            int base = 0;
            if (lane == 0 && bal) base = atomicAdd(&sh.pos, __popc(bal));
            base = __shfl_sync(SPG_FULL, base, 0);
            if (ok) {
                const int at = base + __popc(bal & below);
                if (at < T) { keys[at] = e.r; vals[at] = e.x; }
                else atomicOr(c.err, kErrCount);
            }
        });
    block_walk<kWalkBatch>(src, emit, c.short_seg, c.huge_seg, sh);
    const int n = sh.pos < T ? sh.pos : T;
    block_bitonic<T>(keys, vals, n);
    // runs of equal rows: a run's first entry sums it and writes it at the
    // number of runs before it
    int base = 0;
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const bool head = i < n && (i == 0 || keys[i] != keys[i - 1]);
        const unsigned bal = __ballot_sync(SPG_FULL, head);
        if (lane == 0) sh.red[warp] = __popc(bal);
        __syncthreads();
        int woff = 0, tot = 0;
        for (int w = 0; w < nw; ++w) {
            const int x = sh.red[w];
            woff += w < warp ? x : 0;
            tot += x;
        }
        if (head) {
            V acc = V(0);
            for (int k = i; k < n && keys[k] == keys[i]; ++k) acc = add_v(acc, vals[k]);
            const int64_t r = base + woff + __popc(bal & below);
            if (r < want) {
                out_rows[out0 + r] = (I)keys[i];
                out_vals[out0 + r] = acc;
            }
        }
        base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (base != want) atomicOr(c.err, kErrCount);
        sh.pos = 0;
    }
    __syncthreads();
}

template <class Src, int T>
__global__ void k_num_block(typename Src::Args sa, TierCommon c, typename Src::Idx *out_rows,
                            typename Src::Val *out_vals) {
    constexpr int LOG2T = Log2<T>::v;
    using V = typename Src::Val;
    using I = typename Src::Idx;
    extern __shared__ __align__(16) unsigned char smem[];
    V *vals = reinterpret_cast<V *>(smem);
    uint32_t *keys = reinterpret_cast<uint32_t *>(smem + sizeof(V) * T);
    __shared__ BlockShared<V> sh;
    __shared__ int s_it;
    if (threadIdx.x == 0) { sh.pos = 0; }
    const int lo = c.list_off[c.tier], hi = c.list_off[c.tier + 1];
    const int lane = threadIdx.x & 31;
    // The table is cleared once; the compaction puts back every slot it
    // reads occupied, so it is clean again for the next column.
    auto clear = [&]() {
        for (int s = threadIdx.x; s < T; s += blockDim.x) { keys[s] = kEmpty; vals[s] = V(0); }
    };
    clear();
    // columns are taken in list order from a device counter, one per CTA at a
    // time; thread 0 reserves the next one when it starts a column
    int ahead = 0;
    if (threadIdx.x == 0) ahead = atomicAdd(c.next_col, 1);
    auto fetch = [&]() -> int {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_it = lo + ahead;
            ahead = atomicAdd(c.next_col, 1);
        }
        __syncthreads();
        return s_it;
    };
    for (int it = fetch(); it < hi; it = fetch()) {
        const int64_t g = c.list[it];
        Src src;
        src.open(sa, g);
        const int64_t out0 = c.colptr[g] - c.out_base;
        const int64_t want = c.colptr[g + 1] - c.colptr[g];
        if (c.hybrid_sort && c.flops && c.flops[g] <= T) {   // the same branch for the whole CTA
            num_block_sorted<Src, T>(src, c, keys, vals, sh, out0, want, out_rows, out_vals);
            __syncthreads();
            clear();
            continue;
        }
        auto emit = load_apply(
            [&](int64_t q, V bv, int64_t) { return RowVal<V>{src.row(q), src.val(q, bv)}; },
            [&](const RowVal<V> &e, bool valid) {
                if (!valid) return;
                const int h = hash_insert_dbl1(keys, LOG2T, e.r, c.err);
                if (h >= 0) atomic_add_v(&vals[h], e.x);
            });
        block_walk<kWalkBatch>(src, emit, c.short_seg, c.huge_seg, sh);
        for (int s0 = 0; s0 < T; s0 += blockDim.x) {
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
                keys[s] = kEmpty;
                vals[s] = V(0);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (sh.pos != want) atomicOr(c.err, kErrCount);
            sh.pos = 0;
        }
    }
}

// Heavy numeric: dense accumulation of one row panel of one column in shared
// memory (values + a presence bitmap). Items (p, h) are panel-major so that
// the CTAs running at the same time share one panel of A in L2. An item writes
// pcnt_in[h*P+p] entries at the column's offset plus the counts of the lower
// panels (rows grouped by panel, ascending within the panel).
template <class DSrc>
__global__ void __launch_bounds__(512, 2) k_num_dense(typename DSrc::Args sa, TierCommon c,
                                                    typename DSrc::Idx *out_rows,
                                                    typename DSrc::Val *out_vals) {
    using V = typename DSrc::Val;
    using I = typename DSrc::Idx;
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = 1 << c.log2R;
    V *acc = reinterpret_cast<V *>(smem);
    // presence flags: one byte per row, set with plain stores (no read-modify-write)
    unsigned char *flg = smem + sizeof(V) * R;
    uint32_t *flg4 = reinterpret_cast<uint32_t *>(flg);
    __shared__ BlockShared<V> sh;
    for (int r = threadIdx.x; r < R; r += blockDim.x) { acc[r] = V(0); flg[r] = 0; }
    if (threadIdx.x == 0) sh.pos = 0;
    __syncthreads();
    const int lo = c.list_off[kHeavyTier0], hi = c.list_off[kTiers];
    const int nh = hi - lo;
    const int64_t nitems = (int64_t)nh * c.P;
    const int lane = threadIdx.x & 31;
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int p = (int)(item / nh);
        const int hl = (int)(item % nh);
        const int64_t g = c.list[lo + hl];
        if (g < c.c_lo || g >= c.c_hi) continue;
        if (c.dense_sel[g] <= c.hash_cap_max) continue;   // a hash tier has it
        const int h = c.heavy_ord[g];
        const int32_t *pc = c.pcnt_in + (int64_t)h * c.P;
        const int mycnt = pc[p];
        if (mycnt == 0) continue;
        int below = 0;
        for (int pp = lane; pp < p; pp += 32) below += pc[pp];
        below = warp_sum(below);
        const int64_t out0 = c.colptr[g] - c.out_base + below;
        DSrc src;
        src.open(sa, c, g, p, h);
        auto emit = load_apply(
            [&](int64_t q, V bv, int64_t) { return RowVal<V>{(uint32_t)src.lrow(q), src.val(q, bv)}; },
            [&](const RowVal<V> &e, bool valid) {
                const int r = (int)e.r;
                if (!valid || r < 0) return;
                atomic_add_v(&acc[r], e.x);
                flg[r] = 1;
            });
        block_walk<kWalkBatch>(src, emit, c.short_seg, c.huge_seg, sh);
        // compaction: each thread takes 4-row flag words; warp-aggregated slots
        const int64_t rbase = (int64_t)p << c.log2R;
        for (int w0 = 0; w0 < (R >> 2); w0 += blockDim.x) {
            const int w = w0 + threadIdx.x;
            const uint32_t x = w < (R >> 2) ? flg4[w] : 0u;
            const int n1 = __popc(x);   // flags are 0 or 1 per byte
            const int incl = warp_incl_scan(n1);
            const int tot = __shfl_sync(SPG_FULL, incl, 31);
            int wb = 0;
            if (lane == 31 && tot) wb = atomicAdd(&sh.pos, tot);
            wb = __shfl_sync(SPG_FULL, wb, 31);
            if (x) {
                flg4[w] = 0u;
                int o = wb + incl - n1;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    if ((x >> (8 * b)) & 1u) {
                        const int r = w * 4 + b;
                        if (o < mycnt) {
                            out_rows[out0 + o] = (I)(rbase + r);
                            out_vals[out0 + o] = acc[r];
                        }
                        acc[r] = V(0);
                        ++o;
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (sh.pos != mycnt) atomicOr(c.err, kErrCount);
            sh.pos = 0;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Heavy numeric by work items. For every heavy column the per-panel output
// counts are cut, in panel order, into items: a panel holding at least
// dense_min rows becomes a dense item (shared-memory accumulator over its
// 2^log2R rows); runs of lighter panels are grouped into hash items of at most
// kRangeCap output rows and a bounded number of panels (shared-memory hash table
// keyed by the global row). Items of one column write consecutive, disjoint
// ranges of the column's output, in panel order.
// ---------------------------------------------------------------------------
constexpr int kRangeCap = 8192;
constexpr int kRangeMaxPanels = 16;   // panels per hash item when the items are sorted or merged
constexpr int kRangeLog2T = 14;   // 16384 slots = 2 * kRangeCap

struct HeavyItem {
    int32_t g;      // global column
    int32_t p0, p1; // panel range [p0, p1)
    int32_t cnt;    // output rows of the item; negative: dense item
    int32_t off;    // offset of the item's rows inside the column
    int32_t pad;
};

// Cut heavy columns into work items (defined in util_kernels.cu).
// mode 0: per-column item counts into ncount[h]; mode 1: write the items at
// item_off[h] (exclusive scan of the counts).
__global__ void k_heavy_items(const int32_t *list, const int32_t *list_off, const int64_t *sel,
                              int hash_cap_max, int64_t c_lo, int64_t c_hi, const int32_t *pcnt,
                              int P, int dense_min, int range_cap, int max_panels, int mode,
                              int64_t *ncount, const int64_t *item_off, HeavyItem *items);

// Panel-major item order (defined in util_kernels.cu).
__global__ void k_items_by_panel(const HeavyItem *items, const int64_t *n_items_p, int mode,
                                 int32_t *panel_cnt, int32_t *order);
__global__ void k_small_excl_scan(int32_t *a, int P);
// Batch-major item order: by batch (the contiguous column ranges
// bounds[0..nb]), then dense items before hash items, then by first panel
// when pe > 1 (mode 0: histogram of the keys; mode 1: scatter at the scanned
// offsets), then each batch's first position (defined in util_kernels.cu).
__global__ void k_items_by_batch(const HeavyItem *items, int64_t n, const int64_t *bounds, int64_t nb,
                                 int pe, int mode, unsigned long long *cnt, int32_t *order);
__global__ void k_batch_item_starts(const unsigned long long *cnt, int64_t nb, int pe, int64_t n,
                                    int64_t *start);

// Range sources: the contributions of column g restricted to panels
// [p0, p1). seg() yields segments; row(q, tag) is the global row.
template <class I, class V> struct SrcPanelRange {
    using Args = GemmArgs<I, V>;
    using Val = V;
    using Idx = I;
    const ProbDev<I, V> *p;
    const int64_t *ape;
    const uint16_t *apr;
    const V *apv;
    int64_t b0, nb, k0, k1, ka;
    int p0, np, log2R;
    __device__ __forceinline__ void open(const Args &a, const TierCommon &c, int64_t g, int pp0,
                                         int pp1, int) {
        p = a.probs;
        const int64_t bc = g - p->gcol0;
        b0 = (int64_t)p->bp[bc];
        nb = (int64_t)p->bp[bc + 1] - b0;
        k0 = a.k0; k1 = a.k1; ka = p->ka;
        p0 = pp0; np = pp1 - pp0; log2R = c.log2R;
        ape = a.ap_end; apr = a.ap_row; apv = a.ap_val;
    }
    __device__ __forceinline__ int64_t nseg() const { return nb * np; }
    __device__ __forceinline__ void seg(int64_t e2, int64_t &beg, int &len, V &bv, int64_t &tag) const {
        const int64_t e = e2 / np;
        const int pp = p0 + (int)(e2 - e * np);
        const int64_t pe = b0 + e;
        const int64_t k = (int64_t)__ldg(&p->bi[pe]);
        if (k < k0 || k >= k1) { len = 0; return; }
        const int64_t idx = (int64_t)pp * ka + k;
        const int64_t s = idx ? __ldg(&ape[idx - 1]) : 0;
        beg = s; len = (int)(__ldg(&ape[idx]) - s); bv = __ldg(&p->bv[pe]);
        tag = (int64_t)pp << log2R;      // row base of the panel
    }
    __device__ __forceinline__ uint32_t row(int64_t q, int64_t tag) const {
        return (uint32_t)(tag + __ldg(&apr[q]));
    }
    __device__ __forceinline__ V val(int64_t q, V bv) const { return mul_v(__ldg(&apv[q]), bv); }
};

// Hash-range items over the column-grouped copy of A: the entries of column
// k in panels [p0, p1) are one contiguous run, so a B entry is one segment
// whatever the number of panels (SrcPanelRange needs one per panel).
template <class I, class V> struct SrcColRange {
    using Args = GemmArgs<I, V>;
    using Val = V;
    using Idx = I;
    const ProbDev<I, V> *p;
    const int32_t *apo;
    const uint32_t *cr;
    const V *cv;
    int64_t b0, nb, k0, k1, a0, P1;
    int p0, p1;
    __device__ __forceinline__ void open(const Args &a, const TierCommon &c, int64_t g, int pp0,
                                         int pp1, int) {
        p = a.probs;
        const int64_t bc = g - p->gcol0;
        b0 = (int64_t)p->bp[bc];
        nb = (int64_t)p->bp[bc + 1] - b0;
        k0 = a.k0; k1 = a.k1;
        a0 = (int64_t)p->ap[0];
        P1 = (int64_t)c.P + 1;
        p0 = pp0; p1 = pp1;
        apo = a.apc_off; cr = a.apc_row; cv = a.apc_val;
    }
    __device__ __forceinline__ int64_t nseg() const { return nb; }
    __device__ __forceinline__ void seg(int64_t e, int64_t &beg, int &len, V &bv, int64_t &tag) const {
        const int64_t pe = b0 + e;
        const int64_t k = (int64_t)__ldg(&p->bi[pe]);
        if (k < k0 || k >= k1) { len = 0; return; }
        const int32_t *o = apo + k * P1;
        const int o0 = __ldg(&o[p0]), o1 = __ldg(&o[p1]);
        beg = (int64_t)__ldg(&p->ap[k]) - a0 + o0;
        len = o1 - o0;
        bv = __ldg(&p->bv[pe]);
        tag = 0;
    }
    __device__ __forceinline__ uint32_t row(int64_t q, int64_t) const { return __ldg(&cr[q]); }
    __device__ __forceinline__ V val(int64_t q, V bv) const { return mul_v(__ldg(&cv[q]), bv); }
};

template <class I, class V> struct SrcPartsRange {
    using Args = PartsArgs<I, V>;
    using Val = V;
    using Idx = I;
    static constexpr int kShift = 40;
    SrcParts<I, V> base;
    int p0, p1, h, P;
    int64_t r0, r1;
    __device__ __forceinline__ void open(const Args &a, const TierCommon &c, int64_t g, int pp0,
                                         int pp1, int hh) {
        base.open(a, g);
        p0 = pp0; p1 = pp1; h = hh; P = c.P;
        r0 = (int64_t)pp0 << c.log2R;
        r1 = (int64_t)pp1 << c.log2R;
    }
    __device__ __forceinline__ int64_t nseg() const { return base.nparts; }
    __device__ __forceinline__ void seg(int64_t e, int64_t &beg, int &len, V &bv, int64_t &tag) const {
        int64_t b, en;
        base.range((int)e, b, en);
        const int32_t *pc = base.parts[e].pcnt;
        if (pc) {   // panel-grouped column: the range [p0, p1) is one run
            const int32_t *rowc = pc + (int64_t)h * P;
            int64_t off = 0, len2 = 0;
            for (int q = 0; q < p0; ++q) off += rowc[q];
            for (int q = p0; q < p1; ++q) len2 += rowc[q];
            b += off;
            en = b + len2;
        }
        beg = (e << kShift) | b; len = (int)(en - b); bv = V(1); tag = 0;
    }
    // rows outside the range (filter mode) map to kEmpty and are skipped
    __device__ __forceinline__ uint32_t row(int64_t q, int64_t) const {
        const int64_t r = (int64_t)base.row(q);
        return (r >= r0 && r < r1) ? (uint32_t)r : kEmpty;
    }
    __device__ __forceinline__ V val(int64_t q, V) const { return base.val(q, V(1)); }
};

// windows whose gathers a warp of the heavy kernel keeps in flight
constexpr int kHeavyBatch = 4;

// the source a heavy kernel uses for hash-range items, given its panel source
template <class RSrc> struct HashSrcOf { using type = RSrc; };
template <class I, class V> struct HashSrcOf<SrcPanelRange<I, V>> { using type = SrcColRange<I, V>; };

template <class DSrc, class HSrc, int MINB>
__global__ void __launch_bounds__(512, MINB) k_num_heavy(typename DSrc::Args sa, TierCommon c,
                                                      const HeavyItem *items, const int32_t *order,
                                                      int64_t nitems,
                                                      typename DSrc::Idx *out_rows,
                                                      typename DSrc::Val *out_vals) {
    using V = typename DSrc::Val;
    using I = typename DSrc::Idx;
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = 1 << c.log2R;
    // dense view: acc[R] values + flg[R] bytes; hash view (same memory):
    // vals[Ti] + keys[Ti] with Ti <= 2^kRangeLog2T sized per item
    V *acc = reinterpret_cast<V *>(smem);
    unsigned char *flg = smem + sizeof(V) * R;
    uint32_t *flg4 = reinterpret_cast<uint32_t *>(flg);
    __shared__ BlockShared<V, 512> sh;
    for (int r = threadIdx.x; r < R; r += blockDim.x) { acc[r] = V(0); flg[r] = 0; }
    if (threadIdx.x == 0) sh.pos = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const HeavyItem item = items[order[it]];
        const int64_t g = item.g;
        if (g < c.c_lo || g >= c.c_hi) continue;
        bool dense = item.cnt < 0;
        const int p0 = item.p0;
        const int p1 = item.p1;
        int mycnt = dense ? -item.cnt : item.cnt;
        int64_t ioff = item.off;
        const int h = c.heavy_ord[g];
        if (c.item_counts_from_pcnt) {
            // a k-stage: the same panel ranges, this stage's counts
            const int32_t *pc = c.pcnt_in + (int64_t)h * c.P;
            int below = 0, in = 0;
            for (int pp = lane; pp < p1; pp += 32) {
                const int x = pc[pp];
                if (pp < p0) below += x; else in += x;
            }
            below = warp_sum(below);
            in = warp_sum(in);
            mycnt = in;
            ioff = below;
            dense = (p1 - p0 == 1);
            if (mycnt == 0) continue;
        }
        const int64_t out0 = c.colptr[g] - c.out_base + ioff;
        if (dense) {
            DSrc src;
            src.open(sa, c, g, p0, p1, h);
            const int64_t rbase = (int64_t)p0 << c.log2R;
            auto emit = load_apply(
                [&](int64_t q, V bv, int64_t tag) { return RowVal<V>{src.row(q, tag), src.val(q, bv)}; },
                [&](const RowVal<V> &e, bool valid) {
                    if (!valid || e.r == kEmpty) return;
                    const int r = (int)((int64_t)e.r - rbase);
                    atomic_add_v(&acc[r], e.x);
                    flg[r] = 1;
                });
            block_walk<kHeavyBatch>(src, emit, c.short_seg, c.huge_seg, sh);
            // compaction in row order: warp w owns flag words [w*per, (w+1)*per)
            // (4 rows each); it counts them, one barrier gives each warp its
            // offset, then it writes its rows with a running base
            const int nwf = R >> 2;
            const int per = (nwf + nw - 1) / nw;
            const int wlo = warp * per, whi = min(nwf, wlo + per);
            int n = 0;
            for (int w = wlo + lane; w < whi; w += 32) n += __popc(flg4[w]);
            n = warp_sum(n);
            int o = warp_offset(n, sh.red, warp, nw, lane);
            for (int w0 = wlo; w0 < whi; w0 += 32) {
                const int w = w0 + lane;
                const uint32_t x = w < whi ? flg4[w] : 0u;
                const int n1 = __popc(x);
                const int incl = warp_incl_scan(n1);
                if (x) {
                    flg4[w] = 0u;
                    int oo = o + incl - n1;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        if ((x >> (8 * b)) & 1u) {
                            const int r = w * 4 + b;
                            if (oo < mycnt) {
                                out_rows[out0 + oo] = (I)(rbase + r);
                                out_vals[out0 + oo] = acc[r];
                            }
                            acc[r] = V(0);
                            ++oo;
                        }
                    }
                }
                o += __shfl_sync(SPG_FULL, incl, 31);
            }
            if (warp == nw - 1 && lane == 0) sh.pos = o;
        } else {
            // table sized to the item: the next power of two >= 2 * count
            int lt = 6;
            while ((1 << lt) < 2 * mycnt && (1 << lt) < 2 * c.range_cap) ++lt;
            const int Ti = 1 << lt;
            V *tv = reinterpret_cast<V *>(smem);
            uint32_t *tk = reinterpret_cast<uint32_t *>(smem + sizeof(V) * Ti);
            for (int s = threadIdx.x; s < Ti; s += blockDim.x) { tk[s] = kEmpty; tv[s] = V(0); }
            __syncthreads();
            HSrc src;
            src.open(sa, c, g, p0, p1, h);
            auto emit = load_apply_all(
                [&](int64_t q, V bv, int64_t tag) { return RowVal<V>{src.row(q, tag), src.val(q, bv)}; },
                [&](const auto &e, const auto &ok) {
                    constexpr int UU = sizeof(ok) / sizeof(ok[0]);
                    uint32_t key[UU];
#pragma unroll
                    for (int u = 0; u < UU; ++u) key[u] = ok[u] ? e[u].r : kEmpty;
                    int hs[UU];
                    hash_insert_all<UU>(tk, lt, key, hs, c.err);
#pragma unroll
                    for (int u = 0; u < UU; ++u)
                        if (hs[u] >= 0) atomic_add_v(&tv[hs[u]], e[u].x);
                });
            block_walk<kHeavyBatch>(src, emit, c.short_seg, c.huge_seg, sh);
            // compaction: warp w owns slots [w*per, (w+1)*per); counts, one
            // barrier for the offsets, then writes with a running base
            const int per = (Ti + nw - 1) / nw;
            const int slo = warp * per, shi = min(Ti, slo + per);
            int n = 0;
            for (int s = slo + lane; s < shi; s += 32) n += tk[s] != kEmpty;
            n = warp_sum(n);
            int o = warp_offset(n, sh.red, warp, nw, lane);
            for (int s0 = slo; s0 < shi; s0 += 32) {
                const int s = s0 + lane;
                const uint32_t key = s < shi ? tk[s] : kEmpty;
                const bool occ = key != kEmpty;
                const unsigned bal = __ballot_sync(SPG_FULL, occ);
                if (occ) {
                    const int oo = o + __popc(bal & ((1u << lane) - 1u));
                    if (oo < mycnt) {
                        out_rows[out0 + oo] = (I)key;
                        out_vals[out0 + oo] = tv[s];
                    }
                }
                o += __popc(bal);
            }
            if (warp == nw - 1 && lane == 0) sh.pos = o;
            __syncthreads();
            // the dense view shares this memory: put back the empty accumulator
            // (V(0), the semiring's identity: +inf for min-plus) and cleared
            // flags over the bytes the table used
            const int64_t used = (int64_t)(sizeof(V) + 4) * Ti;
            const int64_t nacc_all = (used + (int64_t)sizeof(V) - 1) / (int64_t)sizeof(V);
            const int nacc = (int)(nacc_all < R ? nacc_all : R);
            for (int r = threadIdx.x; r < nacc; r += blockDim.x) acc[r] = V(0);
            const int64_t fl = used - (int64_t)sizeof(V) * R;   // table bytes over the flags
            for (int r = threadIdx.x; r < fl && r < R; r += blockDim.x) flg[r] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (sh.pos != mycnt) atomicOr(c.err, kErrCount);
            sh.pos = 0;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Row panels of A for the dense numeric tier
// ---------------------------------------------------------------------------

// count[p*ka + c] += entries of A(:, c) in row panel p (one warp per column).
template <class I>
__global__ void k_panel_count(const I *ap, const I *ai, int64_t ka, int log2R,
                              unsigned long long *count) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t col = wid; col < ka; col += nw) {
        const int64_t a0 = (int64_t)ap[col], a1 = (int64_t)ap[col + 1];
        for (int64_t q = a0 + lane; q < a1; q += 32) {
            const int64_t p = (int64_t)ai[q] >> log2R;
            atomicAdd(&count[p * ka + col], 1ull);
        }
    }
}

// cursor[idx] starts at the segment start (exclusive scan of the counts);
// every entry takes a slot with atomicAdd, which leaves cursor[idx] at the
// segment end.
template <class I, class V>
__global__ void k_panel_scatter(const I *ap, const I *ai, const V *av, int64_t ka, int log2R,
                                unsigned long long *cursor, uint16_t *out_row, V *out_val) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t mask = (1ll << log2R) - 1;
    for (int64_t col = wid; col < ka; col += nw) {
        const int64_t a0 = (int64_t)ap[col], a1 = (int64_t)ap[col + 1];
        for (int64_t q = a0 + lane; q < a1; q += 32) {
            const int64_t r = (int64_t)ai[q];
            const int64_t p = r >> log2R;
            const unsigned long long pos = atomicAdd(&cursor[p * ka + col], 1ull);
            out_row[pos] = (uint16_t)(r & mask);
            out_val[pos] = av[q];
        }
    }
}

// The column-grouped copy of A, from the panel-major one. Offsets: one
// thread per column writes apo[k*(P+1) + p] = entries of column k in panels
// < p (the panel lengths are read coalesced across the threads of a panel).
__global__ void k_colpanel_offsets(const int64_t *ape, int64_t ka, int P, int32_t *apo);

// Copy: one thread per (panel, column) segment (blockIdx.y strides the
// panels), moving it with global rows to colptr[k] - colptr[0] + offset.
template <class I, class V>
__global__ void k_colpanel_copy(const I *ap, const int64_t *ape, const uint16_t *apr, const V *apv,
                                int64_t ka, int P, int log2R, const int32_t *apo, uint32_t *cr, V *cv) {
    const int64_t a0 = (int64_t)ap[0];
    for (int p = blockIdx.y; p < P; p += gridDim.y) {
        const uint32_t base = (uint32_t)p << log2R;
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ka;
             k += (int64_t)gridDim.x * blockDim.x) {
            const int64_t idx = (int64_t)p * ka + k;
            const int64_t s = idx ? ape[idx - 1] : 0;
            const int64_t e = ape[idx];
            if (s == e) continue;
            const int64_t d0 = (int64_t)ap[k] - a0 + apo[k * ((int64_t)P + 1) + p] - s;
            for (int64_t q = s; q < e; ++q) {
                cr[d0 + q] = base + apr[q];
                cv[d0 + q] = apv[q];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K5: masked-SpGEMM backward. For every product A(i,k) B(k,j) of column j:
//   dA(i,k) += G(i,j) B(k,j),  dB(k,j) += A(i,k) G(i,j),
// with G(:,j) loaded into a shared-memory hash table (key row -> value).
// Columns are tiered by nnz(G(:,j)); columns above the largest table use a
// dense per-panel copy of G(:,j), one item per (panel, column), filtering
// the products by row.
// ---------------------------------------------------------------------------
template <class I, class V> struct GradArgs {
    GemmArgs<I, V> gemm;
    const void *gcolptr;
    int gptr64;
    const I *grows;
    const V *gvals;
    V *dA;
    V *dB;
};

template <class I, class V>
__device__ __forceinline__ void g_range(const GradArgs<I, V> &a, int64_t g, int64_t &b, int64_t &e) {
    if (a.gptr64) {
        b = ((const int64_t *)a.gcolptr)[g]; e = ((const int64_t *)a.gcolptr)[g + 1];
    } else {
        b = ((const int32_t *)a.gcolptr)[g]; e = ((const int32_t *)a.gcolptr)[g + 1];
    }
}

template <class I, class V, int T>
__global__ void k_bwd_block(GradArgs<I, V> a, TierCommon c) {
    constexpr int LOG2T = Log2<T>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    V *gv = reinterpret_cast<V *>(smem);
    uint32_t *keys = reinterpret_cast<uint32_t *>(smem + sizeof(V) * T);
    __shared__ BlockShared<V> sh;
    const int lo = c.list_off[c.tier], hi = c.list_off[c.tier + 1];
    for (int it = lo + blockIdx.x; it < hi; it += gridDim.x) {
        const int64_t g = c.list[it];
        for (int s = threadIdx.x; s < T; s += blockDim.x) keys[s] = kEmpty;
        __syncthreads();
        int64_t gb, ge;
        g_range(a, g, gb, ge);
        for (int64_t q = gb + threadIdx.x; q < ge; q += blockDim.x) {
            bool nw;
            const int h = hash_insert(keys, LOG2T, (uint32_t)a.grows[q], nw, c.err);
            if (h >= 0) gv[h] = a.gvals[q];
        }
        __syncthreads();
        SrcGemm<I, V> src;
        src.open(a.gemm, g);
        auto emit = [&](int64_t q, V bv, int64_t pe, bool valid) {
            if (!valid) return;
            const int h = hash_find(keys, LOG2T, src.row(q));
            if (h < 0) return;
            const V gval = gv[h];
            atomic_add_v(&a.dA[q], mul_v(gval, bv));
            atomic_add_v(&a.dB[pe], mul_v(src.p->av[q], gval));
        };
        block_walk(src, emit, c.short_seg, c.huge_seg, sh);
    }
}

template <class I, class V, int T>
__global__ void __launch_bounds__(256) k_bwd_warp(GradArgs<I, V> a, TierCommon c) {
    constexpr int LOG2T = Log2<T>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    V *gv = reinterpret_cast<V *>(smem) + warp * T;
    uint32_t *keys = reinterpret_cast<uint32_t *>(smem + sizeof(V) * 8 * T) + warp * T;
    const int lo = c.list_off[c.tier], hi = c.list_off[c.tier + 1];
    const int nwarps = gridDim.x * 8;
    for (int it = lo + blockIdx.x * 8 + warp; it < hi; it += nwarps) {
        const int64_t g = c.list[it];
        for (int s = lane; s < T; s += 32) keys[s] = kEmpty;
        __syncwarp();
        int64_t gb, ge;
        g_range(a, g, gb, ge);
        for (int64_t q = gb + lane; q < ge; q += 32) {
            bool nw;
            const int h = hash_insert(keys, LOG2T, (uint32_t)a.grows[q], nw, c.err);
            if (h >= 0) gv[h] = a.gvals[q];
        }
        __syncwarp();
        SrcGemm<I, V> src;
        src.open(a.gemm, g);
        auto emit = [&](int64_t q, V bv, int64_t pe) {
            const int h = hash_find(keys, LOG2T, src.row(q));
            if (h < 0) return;
            const V gval = gv[h];
            atomic_add_v(&a.dA[q], mul_v(gval, bv));
            atomic_add_v(&a.dB[pe], mul_v(src.p->av[q], gval));
        };
        warp_walk_all(src, emit, c.short_seg);
        __syncwarp();
    }
}

// Heavy backward: dense panel of G(:,j) in shared memory; the products of the
// column are filtered to the panel's rows. Items (p, column) over the heavy
// list; an item with no G entries in its panel is skipped.
template <class I, class V>
__global__ void __launch_bounds__(1024) k_bwd_dense(GradArgs<I, V> a, TierCommon c) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = 1 << c.log2R;
    V *gd = reinterpret_cast<V *>(smem);
    uint32_t *bm = reinterpret_cast<uint32_t *>(smem + sizeof(V) * R);
    __shared__ BlockShared<V> sh;
    __shared__ int s_any;
    for (int w = threadIdx.x; w < (R >> 5); w += blockDim.x) bm[w] = 0u;
    if (threadIdx.x == 0) { s_any = 0; }
    __syncthreads();
    const int lo = c.list_off[kHeavyTier0], hi = c.list_off[kTiers];
    const int nh = hi - lo;
    const int64_t nitems = (int64_t)nh * c.P;
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int p = (int)(item / nh);
        const int64_t g = c.list[lo + (int)(item % nh)];
        const int64_t r0 = (int64_t)p << c.log2R;
        int64_t gb, ge;
        g_range(a, g, gb, ge);
        for (int64_t q = gb + threadIdx.x; q < ge; q += blockDim.x) {
            const int64_t r = (int64_t)a.grows[q] - r0;
            if (r >= 0 && r < R) {
                gd[r] = a.gvals[q];
                atomicOr(&bm[r >> 5], 1u << (r & 31));
                s_any = 1;
            }
        }
        __syncthreads();
        if (s_any) {
            SrcGemm<I, V> src;
            src.open(a.gemm, g);
            auto emit = [&](int64_t q, V bv, int64_t pe, bool valid) {
                if (!valid) return;
                const int64_t r = (int64_t)src.row(q) - r0;
                if (r < 0 || r >= R) return;
                if (!((bm[r >> 5] >> (r & 31)) & 1u)) return;
                const V gval = gd[r];
                atomic_add_v(&a.dA[q], mul_v(gval, bv));
                atomic_add_v(&a.dB[pe], mul_v(src.p->av[q], gval));
            };
            block_walk(src, emit, c.short_seg, c.huge_seg, sh);
        }
        for (int w = threadIdx.x; w < (R >> 5); w += blockDim.x) bm[w] = 0u;
        __syncthreads();
        if (threadIdx.x == 0) s_any = 0;
        __syncthreads();
    }
}

// Tiering of the backward columns by nnz(G(:, j)).
template <class I, class V>
__global__ void k_bwd_tier(GradArgs<I, V> a, int64_t n, int hash_cap_max, uint8_t *tier_out,
                           int32_t *tier_hist) {
    __shared__ int s_hist[kTiers];
    if (threadIdx.x < kTiers) s_hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) {
        int64_t b, e;
        g_range(a, g, b, e);
        const int64_t cnt = e - b;
        int t = hash_tier_of(cnt, hash_cap_max);
        if (t < 0) t = kHeavyTier0;
        if (cnt == 0) t = 0;
        tier_out[g] = (uint8_t)t;
        if (t) atomicAdd(&s_hist[t], 1);
    }
    __syncthreads();
    if (threadIdx.x < kTiers && s_hist[threadIdx.x])
        atomicAdd(&tier_hist[threadIdx.x], s_hist[threadIdx.x]);
}

template <class V> __global__ void k_fill_zero(V *p, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = V(0);
}

}  // namespace spg

#include "dense_items.cuh"
#include "sym_heavy32.cuh"
#include "multi_persistent.cuh"
