// Typed host driver of the kernels: symbolic step, batch plan, numeric step
// (plain or k-split + hash merge), standalone merge, backward.
#pragma once

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "sort_prune.cuh"
#include "plan.h"
#include "util.h"

namespace spg {

#define SPG_CK(call)                                                   \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);            \
    } while (0)

#define SPG_ST(...)                                                    \
    do {                                                               \
        spgemm_status s_ = (__VA_ARGS__);                              \
        if (s_ != SPGEMM_OK) return s_;                                \
    } while (0)

inline int block_tier_threads(int T, const Tuning &tun) {
    if (tun.block_threads) return tun.block_threads;
    if (T <= 1024) return 128;
    if (T <= 4096) return 256;
    if (T <= 8192) return 512;
    return 1024;
}

// Scratch shared by one symbolic / numeric pass.
struct Ctx {
    int nsm;
    Tuning tun;
    int *err;
    int32_t *hist;       // 64 ints
    int32_t *cursor;     // 64 ints
    int32_t *h_small;    // pinned host, >= 64 ints
    int P, Q;
    int64_t Rs;
    PhaseTimer *tm = nullptr;   // optional phase timing and launch counting
    int ph_hash = kPhNumHash, ph_dense = kPhNumDense;
    bool stage_items = false;   // heavy items take their counts from pcnt_in
    const int64_t *f = nullptr; // flops per column of the full product (hybrid accumulator)
    int tbegin(int phase, cudaStream_t st) const { return tm ? tm->begin(phase, st) : -1; }
    void tend(int idx, cudaStream_t st) const { if (tm) tm->end(idx, st); }
    void launched(int n = 1) const { if (tm) tm->launches += n; }
};

inline Ctx make_ctx(PlanState &ps) {
    Ctx c;
    c.tm = &ps.timer;
    c.nsm = ps.nsm; c.tun = ps.tun; c.err = ps.err.as<int>();
    c.hist = ps.hist.as<int32_t>(); c.cursor = ps.cursor.as<int32_t>();
    c.h_small = ps.h_small.as<int32_t>();
    c.P = ps.P; c.Q = ps.Q; c.Rs = ps.Rs;
    c.f = ps.f.as<int64_t>();
    return c;
}

inline TierCommon common_of(const Ctx &c) {
    TierCommon t{};
    t.short_seg = c.tun.short_seg;
    t.huge_seg = c.tun.huge_seg;
    t.err = c.err;
    t.hash_cap_max = c.tun.hash_cap_max;
    t.P = c.P; t.log2R = c.tun.log2R; t.Rs = c.Rs; t.Q = c.Q;
    t.flops = c.f;
    t.hybrid_sort = c.tun.hybrid_sort;
    return t;
}

// Allow a kernel the largest dynamic shared memory the device permits next to
// its static shared memory (opt-in maximum minus static size).
template <class K> static void set_smem(K kern, int) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess && optin > (int)fa.sharedSizeBytes)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
    cudaGetLastError();   // attribute calls must not leave a sticky error behind
}

// Output of a numeric pass.
template <class I, class V> struct NumOut {
    const int64_t *colptr;
    int64_t out_base;
    I *rows;
    V *vals;
};

template <class I, class V> struct Engine : EngineBase {
    using PD = ProbDev<I, V>;
    using GA = GemmArgs<I, V>;
    using PA = PartsArgs<I, V>;

    // ---- one-time attributes ----------------------------------------------
    static void attrs() {
        static bool done = false;
        if (done) return;
        const int sv = (int)(sizeof(V) + 4);
        const int mx = 220 * 1024;
        set_smem(k_sym_block<SrcGemm<I, V>, 512>, mx);
        set_smem(k_sym_block<SrcGemm<I, V>, 1024>, mx);
        set_smem(k_sym_block<SrcGemm<I, V>, 2048>, mx);
        set_smem(k_sym_block<SrcGemm<I, V>, 4096>, mx);
        set_smem(k_sym_block<SrcGemm<I, V>, 8192>, mx);
        set_smem(k_sym_block<SrcGemm<I, V>, 16384>, mx);
        set_smem(k_sym_block<SrcParts<I, V>, 512>, mx);
        set_smem(k_sym_block<SrcParts<I, V>, 1024>, mx);
        set_smem(k_sym_block<SrcParts<I, V>, 2048>, mx);
        set_smem(k_sym_block<SrcParts<I, V>, 4096>, mx);
        set_smem(k_sym_block<SrcParts<I, V>, 8192>, mx);
        set_smem(k_sym_block<SrcParts<I, V>, 16384>, mx);
        set_smem(k_num_block<SrcGemm<I, V>, 512>, mx);
        set_smem(k_num_block<SrcGemm<I, V>, 1024>, mx);
        set_smem(k_num_block<SrcGemm<I, V>, 2048>, mx);
        set_smem(k_num_block<SrcGemm<I, V>, 4096>, mx);
        set_smem(k_num_block<SrcGemm<I, V>, 8192>, mx);
        set_smem(k_num_block<SrcGemm<I, V>, 16384>, mx);
        set_smem(k_num_block<SrcParts<I, V>, 512>, mx);
        set_smem(k_num_block<SrcParts<I, V>, 1024>, mx);
        set_smem(k_num_block<SrcParts<I, V>, 2048>, mx);
        set_smem(k_num_block<SrcParts<I, V>, 4096>, mx);
        set_smem(k_num_block<SrcParts<I, V>, 8192>, mx);
        set_smem(k_num_block<SrcParts<I, V>, 16384>, mx);
        set_smem(k_bwd_block<I, V, 512>, mx);
        set_smem(k_bwd_block<I, V, 1024>, mx);
        set_smem(k_bwd_block<I, V, 2048>, mx);
        set_smem(k_bwd_block<I, V, 4096>, mx);
        set_smem(k_bwd_block<I, V, 8192>, mx);
        set_smem(k_bwd_block<I, V, 16384>, mx);
        set_smem(k_sym_bitmap<SrcGemm<I, V>>, mx);
        set_smem(k_sym_heavy32<I, V>, mx);
        set_smem(k_sym_bitmap<SrcParts<I, V>>, mx);
        set_smem(k_num_dense<SrcPanel<I, V>>, mx);
        set_smem(k_num_dense<SrcPartsPanel<I, V>>, mx);
        set_smem(k_bwd_dense<I, V>, mx);
        set_smem(k_sym_warp<SrcGemm<I, V>, 1024>, mx);
        set_smem(k_sym_warp<SrcParts<I, V>, 1024>, mx);
        set_smem(k_num_warp<SrcGemm<I, V>, 512>, mx);
        set_smem(k_num_warp<SrcGemm<I, V>, 1024>, mx);
        set_smem(k_num_warp<SrcParts<I, V>, 512>, mx);
        set_smem(k_num_warp<SrcParts<I, V>, 1024>, mx);
        set_smem(k_bwd_warp<I, V, 512>, mx);
        set_smem(k_bwd_warp<I, V, 1024>, mx);
        set_smem(k_num_heavy<SrcPanelRange<I, V>, SrcColRange<I, V>, 2>, mx);
        set_smem(k_num_heavy<SrcPartsRange<I, V>, SrcPartsRange<I, V>, 2>, mx);
        set_smem(k_num_heavy<SrcPanelRange<I, V>, SrcColRange<I, V>, 3>, mx);
        set_smem(k_num_heavy<SrcPartsRange<I, V>, SrcPartsRange<I, V>, 3>, mx);
        set_smem(k_multi_pass<SrcGemm<I, V>, 512, 0>, mx);
        set_smem(k_multi_pass<SrcGemm<I, V>, 512, 1>, mx);
        set_smem(k_multi_pass<SrcGemm<I, V>, 256, 0>, mx);
        set_smem(k_multi_pass<SrcGemm<I, V>, 256, 1>, mx);
        set_smem(k_multi_pass<SrcGemm<I, V>, 128, 0>, mx);
        set_smem(k_multi_pass<SrcGemm<I, V>, 128, 1>, mx);
        set_smem(k_num_heavy32<I, V, 1>, mx);
        set_smem(k_num_heavy32<I, V, 2>, mx);
        set_smem(k_num_heavy32<I, V, 3>, mx);
        set_smem(k_sort_block<I, V, 1024>, mx);
        set_smem(k_sort_block<I, V, 8192>, mx);
        set_smem(k_sort_items<I, V, 8192>, mx);
        set_smem(k_sort_items<I, V, 4096>, mx);
        (void)sv;
        done = true;
    }

    // ---- tier launches -----------------------------------------------------
    // count < 0: population unknown on the host (device-driven persistent grid)
    template <class Src>
    static void launch_sym_tier(const Ctx &cx, const typename Src::Args &sa, TierCommon c, int t,
                                int count, cudaStream_t st) {
        c.tier = t;
        const int T = 2 * tier_cap(t);
        if (t <= kWarpTiers) {
            // one warp per column, 8 warps per CTA, warp-private tables
            const int smem = 8 * T * 4;
            const int per_sm = std::max(1, std::min(8, (228 * 1024) / (smem + 1024)));
            const int want = count < 0 ? cx.nsm * per_sm : (count + 7) / 8;
            const int blocks = std::max(1, std::min(want, cx.nsm * per_sm));
            switch (T) {
                case 64: k_sym_warp<Src, 64><<<blocks, 256, smem, st>>>(sa, c); break;
                case 256: k_sym_warp<Src, 256><<<blocks, 256, smem, st>>>(sa, c); break;
                case 512: k_sym_warp<Src, 512><<<blocks, 256, smem, st>>>(sa, c); break;
                default: k_sym_warp<Src, 1024><<<blocks, 256, smem, st>>>(sa, c); break;
            }
            return;
        }
        const int thr = block_tier_threads(T, cx.tun);
        const int smem = T * 4;
        const int per_sm = std::max(1, std::min(2048 / thr, (228 * 1024) / (smem + 34 * 1024)));
        c.next_col = cx.cursor + 32 + t;   // zeroed with the cursors at the start of the pass
        const int want = count < 0 ? cx.nsm * per_sm : count;
        const int blocks = std::max(1, std::min(want, cx.nsm * per_sm));
        switch (T) {
            case 512: k_sym_block<Src, 512><<<blocks, thr, smem, st>>>(sa, c); break;
            case 1024: k_sym_block<Src, 1024><<<blocks, thr, smem, st>>>(sa, c); break;
            case 2048: k_sym_block<Src, 2048><<<blocks, thr, smem, st>>>(sa, c); break;
            case 4096: k_sym_block<Src, 4096><<<blocks, thr, smem, st>>>(sa, c); break;
            case 8192: k_sym_block<Src, 8192><<<blocks, thr, smem, st>>>(sa, c); break;
            default: k_sym_block<Src, 16384><<<blocks, thr, smem, st>>>(sa, c); break;
        }
    }

    template <class Src>
    static void launch_num_tier(const Ctx &cx, const typename Src::Args &sa, TierCommon c, int t,
                                int count, I *rows, V *vals, cudaStream_t st) {
        c.tier = t;
        const int T = 2 * tier_cap(t);
        if (t <= kWarpTiers) {
            const int smem = 8 * T * (int)(4 + sizeof(V));
            const int per_sm = std::max(1, std::min(8, (228 * 1024) / (smem + 1024)));
            const int want = count < 0 ? cx.nsm * per_sm : (count + 7) / 8;
            const int blocks = std::max(1, std::min(want, cx.nsm * per_sm));
            switch (T) {
                case 64: k_num_warp<Src, 64><<<blocks, 256, smem, st>>>(sa, c, rows, vals); break;
                case 256: k_num_warp<Src, 256><<<blocks, 256, smem, st>>>(sa, c, rows, vals); break;
                case 512: k_num_warp<Src, 512><<<blocks, 256, smem, st>>>(sa, c, rows, vals); break;
                default: k_num_warp<Src, 1024><<<blocks, 256, smem, st>>>(sa, c, rows, vals); break;
            }
            return;
        }
        const int thr = block_tier_threads(T, cx.tun);
        const int smem = T * (int)(4 + sizeof(V));
        const int per_sm = std::max(1, std::min(2048 / thr, (228 * 1024) / (smem + 34 * 1024)));
        const int want = count < 0 ? cx.nsm * per_sm : count;
        const int blocks = std::max(1, std::min(want, cx.nsm * per_sm));
        // the tier's column counter: binning cursors 32 + t, zeroed with the
        // cursors at the start of the pass
        c.next_col = cx.cursor + 32 + t;
        switch (T) {
            case 512: k_num_block<Src, 512><<<blocks, thr, smem, st>>>(sa, c, rows, vals); break;
            case 1024: k_num_block<Src, 1024><<<blocks, thr, smem, st>>>(sa, c, rows, vals); break;
            case 2048: k_num_block<Src, 2048><<<blocks, thr, smem, st>>>(sa, c, rows, vals); break;
            case 4096: k_num_block<Src, 4096><<<blocks, thr, smem, st>>>(sa, c, rows, vals); break;
            case 8192: k_num_block<Src, 8192><<<blocks, thr, smem, st>>>(sa, c, rows, vals); break;
            default: k_num_block<Src, 16384><<<blocks, thr, smem, st>>>(sa, c, rows, vals); break;
        }
    }

    static int dense_smem(const Ctx &cx) {
        const int R = 1 << cx.tun.log2R;
        return R * (int)sizeof(V) + R;
    }

    // k_num_heavy32: the accumulator and a presence bitmap
    static int heavy32_smem(const Ctx &cx) {
        const int R = 1 << cx.tun.log2R;
        return R * (int)sizeof(V) + R / 8;
    }

    // largest hash-range item (output rows) whose table (2x slots) fits the
    // memory of a dense item
    static int range_cap(const Ctx &cx) {
        const int R = 1 << cx.tun.log2R;
        const int fit = (int)((int64_t)R * (sizeof(V) + 1) / (sizeof(V) + 4) / 2);
        int cap = 64;
        while (cap * 2 <= fit && cap * 2 <= kRangeCap) cap *= 2;
        return cap;
    }

    static int heavy_smem(const Ctx &cx) {
        const int hs = 2 * range_cap(cx) * (int)(sizeof(V) + 4);
        return std::max(dense_smem(cx), hs);
    }

    // Cut the heavy columns of the symbolic list into work items (dense
    // panels and hash ranges) from their per-panel output counts; reads the
    // item total back (one small synchronisation).
    // max_panels: panels one hash item may span (any number for the products;
    // kRangeMaxPanels when the items are later sorted, or merged part by part)
    static spgemm_status build_items(const Ctx &cx, int nheavy, const int32_t *sym_list,
                                     const int32_t *sym_off, const int64_t *sel,
                                     const int32_t *pcnt, int64_t n, DevBuf &items, DevBuf &icnt,
                                     DevBuf &ioff, DevBuf &scan_part, DevBuf &order,
                                     int64_t *n_items, cudaStream_t st, int max_panels = kRangeMaxPanels) {
        *n_items = 0;
        if (!nheavy) return SPGEMM_OK;
        SPG_CK(icnt.ensure(sizeof(int64_t) * (nheavy + 1)));
        SPG_CK(ioff.ensure(sizeof(int64_t) * (nheavy + 1)));
        SPG_CK(scan_part.ensure(sizeof(int64_t) * scan_partials_len(std::max<int64_t>(n, nheavy) + 1)));
        const int R = 1 << cx.tun.log2R;
        // a panel with at least R/8 output rows is a dense item; the rest are
        // grouped into hash items of at most range_cap rows, so a lone panel
        // below the dense threshold must fit one (dense_min - 1 <= range_cap)
        const int rcap = range_cap(cx);
        const int dmin = std::max(1, std::min(R / 8, rcap));
        const unsigned nb = (unsigned)((nheavy + 255) / 256);
        k_heavy_items<<<nb, 256, 0, st>>>(sym_list, sym_off, sel, cx.tun.hash_cap_max, 0, n, pcnt, cx.P,
                                          dmin, rcap, max_panels, 0, icnt.as<int64_t>(), nullptr, nullptr);
        SPG_CK(exclusive_scan_i64(icnt.as<int64_t>(), nheavy, ioff.as<int64_t>(),
                                  scan_part.as<int64_t>(), 1, st));
        int64_t total = 0;
        SPG_CK(cudaMemcpyAsync(cx.h_small + 256, ioff.as<int64_t>() + nheavy, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, st));
        SPG_CK(cudaStreamSynchronize(st));
        std::memcpy(&total, cx.h_small + 256, sizeof(int64_t));
        SPG_CK(items.ensure(sizeof(HeavyItem) * (size_t)(total + 1)));
        k_heavy_items<<<nb, 256, 0, st>>>(sym_list, sym_off, sel, cx.tun.hash_cap_max, 0, n, pcnt, cx.P,
                                          dmin, rcap, max_panels, 1, nullptr, ioff.as<int64_t>(), items.as<HeavyItem>());
        // panel-major processing order: item indices sorted by first panel,
        // stored after the items (icnt is reused for the panel histogram)
        SPG_CK(order.ensure(sizeof(int32_t) * (size_t)(total + 1)));
        SPG_CK(icnt.ensure(sizeof(int64_t) * (size_t)(std::max(nheavy, cx.P) + 1)));
        int32_t *pc = reinterpret_cast<int32_t *>(icnt.p);
        SPG_CK(cudaMemsetAsync(pc, 0, sizeof(int32_t) * (cx.P + 1), st));
        const int64_t *tot_d = ioff.as<int64_t>() + nheavy;
        const unsigned ob = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4096));
        k_items_by_panel<<<ob, 256, 0, st>>>(items.as<HeavyItem>(), tot_d, 0, pc, nullptr);
        k_small_excl_scan<<<1, 1024, 0, st>>>(pc, cx.P);
        k_items_by_panel<<<ob, 256, 0, st>>>(items.as<HeavyItem>(), tot_d, 1, pc, order.as<int32_t>());
        cx.launched(8);
        SPG_CK(cudaGetLastError());
        *n_items = total;
        return SPGEMM_OK;
    }

    // ---- symbolic pass -------------------------------------------------------
    // Bins columns [c_lo, c_hi) of the source, counts distinct rows into
    // cnt_out, fills list/off; heavy columns get per-panel counts in pcnt.
    // heavy_ord_w (optional) receives the heavy ordinals (full pass only).
    template <class Src>
    static spgemm_status sym_pass(const Ctx &cx, const typename Src::Args &sa, int64_t c_lo, int64_t c_hi,
                           const int64_t *bound, int64_t *f_out, uint8_t *tier, int64_t *cnt_out,
                           int32_t *list, int32_t *off, int32_t *heavy_ord_w,
                           const int32_t *heavy_ord_r, DevBuf *pcnt_grow, int32_t *pcnt_ptr,
                           int *hist_out, cudaStream_t st, bool allow_heavy = true) {
        const int64_t nc = c_hi - c_lo;
        SPG_CK(cudaMemsetAsync(cx.hist, 0, sizeof(int32_t) * 64, st));
        SPG_CK(cudaMemsetAsync(cx.cursor, 0, sizeof(int32_t) * 64, st));
        if (nc > 0) {
            const int tb = cx.tbegin(kPhFlopsBin, st);
            k_flops_bin<Src><<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(
                sa, c_lo, c_hi, cx.tun.hash_cap_max, bound, f_out, tier, cnt_out, cx.hist);
            k_bin_scatter<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(tier, c_lo, c_hi, cx.hist,
                                                                       cx.cursor, list, off,
                                                                       heavy_ord_w);
            cx.tend(tb, st);
            cx.launched(2);
            SPG_CK(cudaGetLastError());
        }
        SPG_CK(cudaMemcpyAsync(cx.h_small, cx.hist, sizeof(int32_t) * 16, cudaMemcpyDeviceToHost, st));
        SPG_CK(cudaStreamSynchronize(st));
        int hist[16];
        std::memcpy(hist, cx.h_small, sizeof(hist));
        if (nc <= 0) std::memset(hist, 0, sizeof(hist));
        if (hist_out) std::memcpy(hist_out, hist, sizeof(hist));
        int nheavy = 0;
        for (int t = kHeavyTier0; t < kTiers; ++t) nheavy += hist[t];
        if (nheavy && !allow_heavy) {
            set_error("a column's entries summed over its sources (capped at the row count) exceed " +
                      std::to_string(cx.tun.hash_cap_max) +
                      ", the largest shared-memory hash table this call may use");
            return SPGEMM_ERR_INVALID;
        }
        TierCommon c = common_of(cx);
        c.list = list; c.list_off = off; c.cnt = cnt_out;
        const int th = cx.tbegin(kPhSymHash, st);
        for (int t = 1; t <= 8; ++t)
            if (hist[t]) { launch_sym_tier<Src>(cx, sa, c, t, hist[t], st); cx.launched(); }
        cx.tend(th, st);
        if (nheavy) {
            if (pcnt_grow) {
                SPG_CK(pcnt_grow->ensure(sizeof(int32_t) * (size_t)nheavy * cx.P));
                pcnt_ptr = pcnt_grow->as<int32_t>();
            }
            c.pcnt = pcnt_ptr;
            c.heavy_ord = heavy_ord_r;
            const int64_t items = (int64_t)nheavy * cx.Q;
            const int smem = (int)(((cx.Rs + 31) / 32) * 4);
            const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(items, cx.nsm));
            const int tb = cx.tbegin(kPhSymHeavy, st);
            c.next_col = cx.cursor + 63;   // zeroed with the cursors above
            bool lean = false;
            if constexpr (std::is_same<Src, SrcGemm<I, V>>::value) {
                if (sa.lean_sym) {
                    k_sym_heavy32<I, V><<<blocks, kSymChunk, smem, st>>>(sa, c);
                    lean = true;
                }
            }
            if (!lean) k_sym_bitmap<Src><<<blocks, 1024, smem, st>>>(sa, c);
            cx.tend(tb, st);
            cx.launched();
        }
        SPG_CK(cudaGetLastError());
        return SPGEMM_OK;
    }

    // ---- numeric pass --------------------------------------------------------
    // tc: host tier populations (nullptr: device-driven grids). heavy: whether
    // dense items exist. sym_list/sym_off: the symbolic heavy list.
    template <class Src, class DSrc, class RSrc = DSrc>
    static spgemm_status num_pass(const Ctx &cx, const typename Src::Args &sa,
                           const typename DSrc::Args &da, int64_t c_lo, int64_t c_hi,
                           const int64_t *cnt, const int64_t *dense_sel, const NumOut<I, V> &o,
                           const int *tc, bool heavy, const int32_t *sym_list,
                           const int32_t *sym_off, const int32_t *heavy_ord,
                           const int32_t *pcnt_in, uint8_t *tier, int32_t *list, int32_t *off,
                           cudaStream_t st, const HeavyItem *items = nullptr, int64_t n_items = 0,
                           const int32_t *item_order = nullptr) {
        const int64_t nc = c_hi - c_lo;
        bool any_hash = tc == nullptr;
        if (tc) for (int t = 1; t <= 8; ++t) any_hash |= tc[t] > 0;
        TierCommon c = common_of(cx);
        c.colptr = o.colptr;
        c.out_base = o.out_base;
        if (any_hash && nc > 0) {
            const int th = cx.tbegin(cx.ph_hash, st);
            SPG_CK(cudaMemsetAsync(cx.hist, 0, sizeof(int32_t) * 64, st));
            SPG_CK(cudaMemsetAsync(cx.cursor, 0, sizeof(int32_t) * 64, st));
            k_numeric_tier<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(
                cnt, dense_sel, c_lo, c_hi, cx.tun.hash_cap_max, tier, cx.hist);
            k_bin_scatter<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(
                tier, c_lo, c_hi, cx.hist, cx.cursor, list, off, nullptr);
            SPG_CK(cudaGetLastError());
            c.list = list; c.list_off = off;
            for (int t = 1; t <= 8; ++t) {
                if (tier_cap(t) > cx.tun.hash_cap_max) break;
                const int cntt = tc ? tc[t] : -1;
                if (cntt != 0) { launch_num_tier<Src>(cx, sa, c, t, cntt, o.rows, o.vals, st); cx.launched(); }
            }
            cx.launched(2);
            cx.tend(th, st);
        }
        if (heavy) {
            c.list = sym_list; c.list_off = sym_off;
            c.dense_sel = dense_sel;
            c.heavy_ord = heavy_ord;
            c.pcnt_in = pcnt_in;
            c.c_lo = c_lo; c.c_hi = c_hi;
            c.item_counts_from_pcnt = cx.stage_items ? 1 : 0;
            c.range_cap = range_cap(cx);
            if constexpr (!std::is_same<RSrc, DSrc>::value) {
              if (items) {
                // 512-thread CTAs; 3 per SM when the item memory allows it
                // (registers are then capped at 40 per thread), else 2
                using HS = typename HashSrcOf<RSrc>::type;
                const int smem = heavy_smem(cx);
                const int stat = (int)sizeof(BlockShared<V, 512>) + 256;
                const int per_sm = (3 * (smem + stat) <= 227 * 1024) ? 3 : 2;
                const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(n_items, (int64_t)cx.nsm * per_sm));
                if constexpr (std::is_same<RSrc, SrcPanelRange<I, V>>::value) {
                    // products: all heavy items in the kernel with 32-bit
                    // offsets (every entry index < nnz(A) < 2^31), whose
                    // largest hash table lies inside the accumulator
                    const bool table_fits =
                        2 * range_cap(cx) * (int)(sizeof(V) + 4) <= (1 << cx.tun.log2R) * (int)sizeof(V);
                    if (da.lean_dense && table_fits) {
                        // three CTAs per SM when their shared memory allows it
                        // (registers are then capped at 40 per thread), else two
                        const int dsm = heavy32_smem(cx);
                        const int dstat = (int)sizeof(DenseShared<V>) + 512;
                        const int dper = std::max(1, std::min(3, (227 * 1024) / (dsm + dstat)));
                        const int dblocks = (int)std::max<int64_t>(1, std::min<int64_t>(n_items, (int64_t)cx.nsm * dper));
                        const int tdd = cx.tbegin(cx.ph_dense, st);
                        // the item counter (the last int of the binning cursors)
                        int *next_item = cx.cursor + 63;
                        SPG_CK(cudaMemsetAsync(next_item, 0, sizeof(int), st));
                        if (dper >= 3)
                            k_num_heavy32<I, V, 3><<<dblocks, kDenseChunk, dsm, st>>>(da, c, items, item_order,
                                                                                     n_items, next_item, o.rows, o.vals);
                        else if (dper == 2)
                            k_num_heavy32<I, V, 2><<<dblocks, kDenseChunk, dsm, st>>>(da, c, items, item_order,
                                                                                     n_items, next_item, o.rows, o.vals);
                        else
                            k_num_heavy32<I, V, 1><<<dblocks, kDenseChunk, dsm, st>>>(da, c, items, item_order,
                                                                                     n_items, next_item, o.rows, o.vals);
                        cx.tend(tdd, st);
                        cx.launched();
                        SPG_CK(cudaGetLastError());
                        return SPGEMM_OK;
                    }
                }
                const int td = cx.tbegin(cx.ph_dense, st);
                if (per_sm == 3)
                    k_num_heavy<RSrc, HS, 3><<<blocks, 512, smem, st>>>(da, c, items, item_order, n_items,
                                                                        o.rows, o.vals);
                else
                    k_num_heavy<RSrc, HS, 2><<<blocks, 512, smem, st>>>(da, c, items, item_order, n_items,
                                                                        o.rows, o.vals);
                cx.tend(td, st);
                cx.launched();
                SPG_CK(cudaGetLastError());
                return SPGEMM_OK;
              }
            }
            {
                const int smem = dense_smem(cx);
                const int per_sm = std::max(1, std::min(2, (228 * 1024) / (smem + 34 * 1024)));
                const int td = cx.tbegin(cx.ph_dense, st);
                k_num_dense<DSrc><<<cx.nsm * per_sm, 512, smem, st>>>(da, c, o.rows, o.vals);
                cx.tend(td, st);
            }
            cx.launched();
        }
        SPG_CK(cudaGetLastError());
        return SPGEMM_OK;
    }

    // ---- plan ----------------------------------------------------------------
    GA gemm_args(PlanState &ps, int64_t k0, int64_t k1) {
        GA a{};
        a.probs = ps.probs.as<PD>();
        a.nprob = 1;
        a.k0 = k0; a.k1 = k1;
        a.ap_end = ps.ap_end.as<int64_t>();
        a.ap_row = ps.ap_row.as<uint16_t>();
        a.ap_val = ps.ap_val.as<V>();
        a.apc_off = ps.apc_off.as<int32_t>();
        a.apc_row = ps.apc_row.as<uint32_t>();
        a.apc_val = ps.apc_val.as<V>();
        a.lean_dense = ps.A.nnz < (int64_t(1) << 31) ? 1 : 0;
        // a chunk's stream is at most kSymChunk columns of A, each of at most
        // min(m, nnz(A)) entries
        a.lean_sym = a.lean_dense && std::min<int64_t>(ps.A.nrows, ps.A.nnz) * kSymChunk < (int64_t(1) << 31);
        return a;
    }

    static bool incremental(const PlanState &ps) {
        return ps.s > 1 && ps.opts.merge_mode == SPGEMM_MERGE_INCREMENTAL;
    }

    spgemm_status setup(PlanState &ps, cudaStream_t st) override {
        attrs();
        PD pd{};
        pd.ap = (const I *)ps.A.colptr; pd.ai = (const I *)ps.A.rowidx; pd.av = (const V *)ps.A.vals;
        pd.bp = (const I *)ps.B.colptr; pd.bi = (const I *)ps.B.rowidx; pd.bv = (const V *)ps.B.vals;
        pd.m = ps.m; pd.gcol0 = 0; pd.ncols = ps.n; pd.ka = ps.k;
        SPG_CK(ps.probs.ensure(sizeof(PD)));
        SPG_CK(cudaMemcpyAsync(ps.probs.p, &pd, sizeof(PD), cudaMemcpyHostToDevice, st));
        const int64_t n = ps.n;
        SPG_CK(ps.f.ensure(sizeof(int64_t) * (n + 1)));
        SPG_CK(ps.cnt.ensure(sizeof(int64_t) * (n + 1)));
        SPG_CK(ps.colptr.ensure(sizeof(int64_t) * (n + 1)));
        SPG_CK(ps.wbytes.ensure(sizeof(int64_t) * (n + 1)));
        SPG_CK(ps.tier.ensure(n + 16));
        SPG_CK(ps.list_sym.ensure(sizeof(int32_t) * (n + 1)));
        SPG_CK(ps.list_num.ensure(sizeof(int32_t) * (n + 1)));
        SPG_CK(ps.heavy_ord.ensure(sizeof(int32_t) * (n + 1)));
        SPG_CK(ps.hist.ensure(sizeof(int32_t) * 64));
        SPG_CK(ps.cursor.ensure(sizeof(int32_t) * 64));
        SPG_CK(ps.off_sym.ensure(sizeof(int32_t) * 64));
        SPG_CK(ps.off_num.ensure(sizeof(int32_t) * 64));
        SPG_CK(ps.err.ensure(sizeof(int) * 4));
        SPG_CK(ps.scan_part.ensure(sizeof(int64_t) * scan_partials_len(n + 1)));
        SPG_CK(ps.h_colptr.ensure(sizeof(int64_t) * (n + 1)));
        SPG_CK(ps.h_small.ensure(4096));
        SPG_CK(cudaMemsetAsync(ps.err.p, 0, sizeof(int) * 4, st));
        if (ps.s > 1) {
            SPG_CK(ps.stage_cnt.ensure(sizeof(int64_t) * (size_t)ps.s * (n + 1)));
            SPG_CK(ps.stage_colptr.ensure(sizeof(int64_t) * (size_t)ps.s * (n + 1)));
            SPG_CK(ps.h_stage_colptr.ensure(sizeof(int64_t) * (size_t)ps.s * (n + 1)));
        }
        return SPGEMM_OK;
    }

    spgemm_status symbolic(PlanState &ps, cudaStream_t st) override {
        const int64_t n = ps.n;
        ps.have_symbolic = false;
        ps.panels_built = false;
        Ctx cx = make_ctx(ps);
        SPG_CK(cudaMemsetAsync(ps.err.p, 0, sizeof(int) * 4, st));
        // full product: flops, counts, heavy list
        SPG_ST(sym_pass<SrcGemm<I, V>>(cx, gemm_args(ps, 0, ps.k), 0, n, nullptr, ps.f.as<int64_t>(),
                                       ps.tier.as<uint8_t>(), ps.cnt.as<int64_t>(),
                                       ps.list_sym.as<int32_t>(), ps.off_sym.as<int32_t>(),
                                       ps.heavy_ord.as<int32_t>(), ps.heavy_ord.as<int32_t>(),
                                       &ps.pcnt, nullptr, ps.sym_hist, st));
        ps.nheavy = 0;
        for (int t = kHeavyTier0; t < kTiers; ++t) ps.nheavy += ps.sym_hist[t];
        int tsc = cx.tbegin(kPhScan, st);
        SPG_CK(exclusive_scan_i64(ps.cnt.as<int64_t>(), n, ps.colptr.as<int64_t>(),
                                  ps.scan_part.as<int64_t>(), 1, st));
        cx.tend(tsc, st);
        cx.launched(3);
        // k-split stages: per-stage counts nnz(D_t(:, j)) (LocalSymbolic per stage,
        // Algorithm 3), panel counts for the heavy columns
        if (ps.s > 1) {
            if (ps.nheavy)
                SPG_CK(ps.stage_pcnt.ensure(sizeof(int32_t) * (size_t)ps.s * ps.nheavy * ps.P));
            for (int t = 0; t < ps.s; ++t) {
                const int64_t k0 = (int64_t)t * ps.k / ps.s, k1 = (int64_t)(t + 1) * ps.k / ps.s;
                int64_t *scnt = ps.stage_cnt.as<int64_t>() + (size_t)t * (n + 1);
                int32_t *spc = ps.nheavy ? ps.stage_pcnt.as<int32_t>() + (size_t)t * ps.nheavy * ps.P
                                         : nullptr;
                SPG_ST(sym_pass<SrcGemm<I, V>>(cx, gemm_args(ps, k0, k1), 0, n, ps.cnt.as<int64_t>(),
                                               nullptr, ps.tier.as<uint8_t>(), scnt,
                                               ps.list_num.as<int32_t>(), ps.off_num.as<int32_t>(),
                                               nullptr, ps.heavy_ord.as<int32_t>(), nullptr, spc,
                                               nullptr, st));
                SPG_CK(exclusive_scan_i64(scnt, n, ps.stage_colptr.as<int64_t>() + (size_t)t * (n + 1),
                                          ps.scan_part.as<int64_t>(), 1, st));
                cx.launched(3);
            }
            SPG_CK(cudaMemcpyAsync(ps.h_stage_colptr.p, ps.stage_colptr.p,
                                   sizeof(int64_t) * (size_t)ps.s * (n + 1), cudaMemcpyDeviceToHost, st));
            // incremental merge: counts of the running sums M_u = D_0 + ... + D_u,
            // i.e. the product over k in [0, k1_u), for u = 1..s-2 (M_0 is D_0,
            // M_{s-1} is C), with panel counts for the heavy columns
            if (incremental(ps) && ps.s > 2) {
                const int nu = ps.s - 2;
                SPG_CK(ps.pref_cnt.ensure(sizeof(int64_t) * (size_t)nu * (n + 1)));
                SPG_CK(ps.pref_colptr.ensure(sizeof(int64_t) * (size_t)nu * (n + 1)));
                SPG_CK(ps.h_pref_colptr.ensure(sizeof(int64_t) * (size_t)nu * (n + 1)));
                if (ps.nheavy)
                    SPG_CK(ps.pref_pcnt.ensure(sizeof(int32_t) * (size_t)nu * ps.nheavy * ps.P));
                for (int u = 1; u <= nu; ++u) {
                    const int64_t k1 = (int64_t)(u + 1) * ps.k / ps.s;
                    int64_t *pc = ps.pref_cnt.as<int64_t>() + (size_t)(u - 1) * (n + 1);
                    int32_t *pp = ps.nheavy ? ps.pref_pcnt.as<int32_t>() + (size_t)(u - 1) * ps.nheavy * ps.P
                                            : nullptr;
                    SPG_ST(sym_pass<SrcGemm<I, V>>(cx, gemm_args(ps, 0, k1), 0, n, ps.cnt.as<int64_t>(),
                                                   nullptr, ps.tier.as<uint8_t>(), pc,
                                                   ps.list_num.as<int32_t>(), ps.off_num.as<int32_t>(),
                                                   nullptr, ps.heavy_ord.as<int32_t>(), nullptr, pp,
                                                   nullptr, st));
                    SPG_CK(exclusive_scan_i64(pc, n, ps.pref_colptr.as<int64_t>() + (size_t)(u - 1) * (n + 1),
                                              ps.scan_part.as<int64_t>(), 1, st));
                    cx.launched(3);
                }
                SPG_CK(cudaMemcpyAsync(ps.h_pref_colptr.p, ps.pref_colptr.p,
                                       sizeof(int64_t) * (size_t)nu * (n + 1), cudaMemcpyDeviceToHost, st));
            }
        }
        SPG_CK(cudaMemcpyAsync(ps.h_colptr.p, ps.colptr.p, sizeof(int64_t) * (n + 1),
                               cudaMemcpyDeviceToHost, st));
        SPG_CK(cudaMemcpyAsync(ps.h_small.as<char>() + 256, ps.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        tsc = cx.tbegin(kPhScan, st);
        SPG_CK(exclusive_scan_i64(ps.f.as<int64_t>(), n, ps.wbytes.as<int64_t>(),
                                  ps.scan_part.as<int64_t>(), 1, st));
        cx.tend(tsc, st);
        cx.launched(3);
        SPG_CK(cudaMemcpyAsync(ps.h_small.as<char>() + 512, ps.wbytes.as<int64_t>() + n, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, st));
        if (ps.nheavy) SPG_ST(build_panels(ps, st));
        // products alone: a hash item may span any number of panels (one run
        // of the column-grouped copy of A); sorted output and the k-split's
        // part-by-part merges keep the narrower items
        const int max_panels = (ps.opts.sort_output || ps.s > 1 || !ps.A.nnz || ps.A.nnz >= (int64_t(1) << 31))
                                   ? kRangeMaxPanels : std::max(kRangeMaxPanels, ps.P);
        SPG_ST(build_items(cx, ps.nheavy, ps.list_sym.as<int32_t>(), ps.off_sym.as<int32_t>(),
                           ps.cnt.as<int64_t>(), ps.pcnt.as<int32_t>(), n, ps.items, ps.item_cnt,
                           ps.item_off, ps.scan_part, ps.item_order, &ps.n_items, st, max_panels));
        SPG_CK(cudaStreamSynchronize(st));
        const int errw = *(int *)(ps.h_small.as<char>() + 256);
        if (errw) {
            set_error("symbolic: device error flags " + std::to_string(errw));
            return SPGEMM_ERR_OVERFLOW;
        }
        ps.flops = *(int64_t *)(ps.h_small.as<char>() + 512);
        ps.nnz_c = ps.h_colptr.as<int64_t>()[n];
        SPG_ST(plan_batches(ps));
        SPG_ST(order_items_by_batch(ps, st));
        if (ps.s > 1) SPG_ST(setup_stage_buffers(ps, st));
        ps.have_symbolic = true;
        return SPGEMM_OK;
    }

    // Order the heavy items batch-major, so that a batch's numeric launch
    // walks its own items only (not every item of the product with a
    // column-range test); inside a batch dense items come first, then hash
    // items, each panel-major. batch_item_off records each batch's run. The
    // item-count buffer is the scratch: without room for the panel histogram
    // the order inside a (batch, kind) is arbitrary, and without room for
    // that the panel-major order of all items stays.
    spgemm_status order_items_by_batch(PlanState &ps, cudaStream_t st) {
        ps.batch_item_off.clear();
        const int64_t nb = (int64_t)ps.batches.size();
        if (!ps.nheavy || ps.n_items <= 0 || nb < 1) return SPGEMM_OK;
        const int64_t capw = (int64_t)(ps.item_cnt.bytes / sizeof(int64_t));
        const int64_t caps = (int64_t)(ps.scan_part.bytes / sizeof(int64_t));
        auto fits = [&](int64_t pe) {
            const int64_t nbins = nb * 2 * pe;
            return nbins + 1 + nb + 1 <= capw && scan_partials_len(nbins + 1) <= caps;
        };
        const int pe = fits(ps.P) ? ps.P : 1;
        if (!fits(pe)) return SPGEMM_OK;
        const int64_t nbins = nb * 2 * pe;
        unsigned long long *cnt = ps.item_cnt.as<unsigned long long>();
        int64_t *bounds = reinterpret_cast<int64_t *>(cnt + nbins + 1);
        std::vector<int64_t> hb((size_t)nb + 1);
        for (int64_t t = 0; t < nb; ++t) hb[(size_t)t] = ps.batches[(size_t)t].c0;
        hb[(size_t)nb] = ps.batches[(size_t)nb - 1].c1;
        SPG_CK(cudaMemcpyAsync(bounds, hb.data(), sizeof(int64_t) * (size_t)(nb + 1), cudaMemcpyHostToDevice, st));
        SPG_CK(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (size_t)(nbins + 1), st));
        const unsigned ob = (unsigned)std::max<int64_t>(1, std::min<int64_t>((ps.n_items + 255) / 256, 4096));
        const HeavyItem *items = ps.items.as<HeavyItem>();
        k_items_by_batch<<<ob, 256, 0, st>>>(items, ps.n_items, bounds, nb, pe, 0, cnt, nullptr);
        SPG_CK(exclusive_scan_i64(reinterpret_cast<int64_t *>(cnt), nbins, reinterpret_cast<int64_t *>(cnt),
                                  ps.scan_part.as<int64_t>(), 0, st));
        k_items_by_batch<<<ob, 256, 0, st>>>(items, ps.n_items, bounds, nb, pe, 1, cnt,
                                             ps.item_order.as<int32_t>());
        k_batch_item_starts<<<(unsigned)((nb + 1 + 255) / 256), 256, 0, st>>>(cnt, nb, pe, ps.n_items, bounds);
        ps.timer.launches += 6;
        SPG_CK(cudaGetLastError());
        std::vector<int64_t> off((size_t)nb + 1);
        SPG_CK(cudaMemcpyAsync(off.data(), bounds, sizeof(int64_t) * (size_t)(nb + 1), cudaMemcpyDeviceToHost, st));
        SPG_CK(cudaStreamSynchronize(st));
        ps.batch_item_off.swap(off);
        return SPGEMM_OK;
    }

    // The heavy items of batch t: its run of item_order when the items are
    // ordered batch-major, else all of them (the kernels skip other columns).
    struct BatchItems {
        int64_t n;
        const int32_t *order;
    };
    static BatchItems batch_items(const PlanState &ps, int64_t t) {
        if (ps.batch_item_off.size() == ps.batches.size() + 1) {
            const int64_t a = ps.batch_item_off[(size_t)t];
            return {ps.batch_item_off[(size_t)t + 1] - a, ps.item_order.as<int32_t>() + a};
        }
        return {ps.n_items, ps.item_order.as<int32_t>()};
    }

    spgemm_status build_panels(PlanState &ps, cudaStream_t st) {
        const int64_t ka = ps.k;
        const int64_t N = (int64_t)ps.P * ka;
        const int64_t nnzA = ps.A.nnz;
        SPG_CK(ps.ap_end.ensure(sizeof(int64_t) * (N + 1)));
        SPG_CK(ps.ap_row.ensure(sizeof(uint16_t) * (nnzA + 8)));
        SPG_CK(ps.ap_val.ensure(sizeof(V) * (nnzA + 8)));
        SPG_CK(ps.merge_tmp.ensure(sizeof(int64_t) * scan_partials_len(N + 1)));
        const int tp = ps.timer.begin(kPhPanels, st);
        SPG_CK(cudaMemsetAsync(ps.ap_end.p, 0, sizeof(int64_t) * (N + 1), st));
        const int blocks = ps.nsm * 8;
        k_panel_count<I><<<blocks, 256, 0, st>>>((const I *)ps.A.colptr, (const I *)ps.A.rowidx, ka,
                                                 ps.tun.log2R, ps.ap_end.as<unsigned long long>());
        SPG_CK(exclusive_scan_i64(ps.ap_end.as<int64_t>(), N, ps.ap_end.as<int64_t>(),
                                  ps.merge_tmp.as<int64_t>(), 0, st));
        k_panel_scatter<I, V><<<blocks, 256, 0, st>>>((const I *)ps.A.colptr, (const I *)ps.A.rowidx,
                                                      (const V *)ps.A.vals, ka, ps.tun.log2R,
                                                      ps.ap_end.as<unsigned long long>(),
                                                      ps.ap_row.as<uint16_t>(), ps.ap_val.as<V>());
        // the column-grouped copy read by hash-range items
        SPG_CK(ps.apc_off.ensure(sizeof(int32_t) * (size_t)(ka * ((int64_t)ps.P + 1))));
        SPG_CK(ps.apc_row.ensure(sizeof(uint32_t) * (nnzA + 8)));
        SPG_CK(ps.apc_val.ensure(sizeof(V) * (nnzA + 8)));
        const unsigned kb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((ka + 255) / 256, 1 << 20));
        k_colpanel_offsets<<<kb, 256, 0, st>>>(ps.ap_end.as<int64_t>(), ka, ps.P, ps.apc_off.as<int32_t>());
        k_colpanel_copy<I, V><<<dim3(kb, (unsigned)std::min(ps.P, 65535)), 256, 0, st>>>(
            (const I *)ps.A.colptr, ps.ap_end.as<int64_t>(), ps.ap_row.as<uint16_t>(), ps.ap_val.as<V>(), ka,
            ps.P, ps.tun.log2R, ps.apc_off.as<int32_t>(), ps.apc_row.as<uint32_t>(), ps.apc_val.as<V>());
        ps.timer.end(tp, st);
        ps.timer.launches += 7;
        SPG_CK(cudaGetLastError());
        ps.panels_built = true;
        return SPGEMM_OK;
    }

    static void tier_counts(const int64_t *cp, const int64_t *sel, int64_t c0, int64_t c1, int capmax,
                            std::array<int, 16> &tc, int64_t *heavy) {
        tc.fill(0);
        int64_t hv = 0;
        for (int64_t j = c0; j < c1; ++j) {
            const int64_t x = cp[j + 1] - cp[j];
            const int64_t s = sel ? sel[j + 1] - sel[j] : x;
            if (s > capmax) { ++hv; continue; }
            if (x == 0) continue;
            for (int t = 1; t <= 8; ++t) {
                if (tier_cap(t) > capmax) break;
                if (x <= tier_cap(t)) { tc[t]++; break; }
            }
        }
        if (heavy) *heavy = hv;
    }

    // Greedy contiguous column ranges under the per-batch cap, from the exact
    // per-column counts (Eq. (2)'s smallest b for contiguous ranges).
    spgemm_status plan_batches(PlanState &ps) {
        const int64_t n = ps.n;
        const int64_t *hc = ps.h_colptr.as<int64_t>();
        const int64_t *hs = ps.s > 1 ? ps.h_stage_colptr.as<int64_t>() : nullptr;
        const int64_t r = (ps.idx64 ? 8 : 4) + (ps.vtype == SPGEMM_F32 ? 4 : 8);
        ps.bytes_per_nnz = r;
        const int64_t ptr_bytes = 8;
        const int64_t inputs = (int64_t)(ps.A.nnz + ps.B.nnz) * r +
                               (ps.A.ncols + 1 + ps.B.ncols + 1) * (ps.idx64 ? 8 : 4);
        // the stage partial buffers are part of each batch's bytes (w_j counts
        // the unmerged entries), so they are not workspace here; this keeps the
        // plan identical across repeated symbolic calls on one plan
        const int64_t ws = (int64_t)ps.workspace_bytes() - (int64_t)ps.drows.bytes -
                           (int64_t)ps.dvals.bytes - (int64_t)ps.parts_tab.bytes;
        const int64_t avail = (int64_t)ps.budget - inputs - ws;
        const int ring = ps.opts.ring_depth > 0 ? ps.opts.ring_depth : 2;
        if (avail <= 0) {
            set_error("budget " + std::to_string(ps.budget) + " B does not cover the inputs (" +
                      std::to_string(inputs) + " B) and the workspace (" + std::to_string(ws) + " B)");
            return SPGEMM_ERR_BUDGET;
        }
        const int64_t cap = avail / ring;
        ps.batch_cap = cap;
        ps.batches.clear();
        // unmerged entries up to column j: sum over stages of the stage colptrs
        auto unm = [&](int64_t j) {
            if (!hs) return (int64_t)0;
            int64_t u = 0;
            for (int t = 0; t < ps.s; ++t) u += hs[(size_t)t * (n + 1) + j];
            return u;
        };
        // with opts.prune a batch also holds its pruned copy (at most
        // min(nnz_j, topk) entries per column), its colptr and the prune
        // workspace
        const bool prune = ps.opts.prune != 0;
        if (prune) {
            ps.prune_prefix.assign((size_t)n + 1, 0);
            const int64_t k = ps.opts.prune_topk;
            for (int64_t j = 0; j < n; ++j) {
                const int64_t c = hc[j + 1] - hc[j];
                ps.prune_prefix[(size_t)j + 1] = ps.prune_prefix[(size_t)j] + (k > 0 && c > k ? k : c);
            }
        }
        // incremental merge: the stage buffers of columns [c, x) hold the
        // largest stage partial D_t (t >= 1) and nm running sums, each sized
        // by the largest M_u (u <= s-2; M_0 = D_0)
        const bool inc = incremental(ps);
        const int64_t *hp = (inc && ps.s > 2) ? ps.h_pref_colptr.as<int64_t>() : nullptr;
        const int nm = ps.s > 2 ? 2 : 1;
        auto inc_sizes = [&](int64_t c0, int64_t x, int64_t &dsz, int64_t &msz) {
            dsz = 0;
            for (int t = 1; t < ps.s; ++t)
                dsz = std::max(dsz, hs[(size_t)t * (n + 1) + x] - hs[(size_t)t * (n + 1) + c0]);
            msz = hs[x] - hs[c0];
            for (int u = 1; u <= ps.s - 2; ++u)
                msz = std::max(msz, hp[(size_t)(u - 1) * (n + 1) + x] - hp[(size_t)(u - 1) * (n + 1) + c0]);
        };
        auto wprefix = [&](int64_t j) {
            int64_t w = r * (hc[j] + (inc ? 0 : unm(j))) + ptr_bytes * j;
            if (prune) w += r * ps.prune_prefix[(size_t)j] + (ptr_bytes + kPruneWsPerCol) * j;
            return w;
        };
        // bytes of a batch over columns [c0, x)
        auto wrange = [&](int64_t c0, int64_t x) {
            int64_t w = wprefix(x) - wprefix(c0);
            if (inc) {
                int64_t d, m;
                inc_sizes(c0, x, d, m);
                w += r * (d + nm * m);
            }
            return w;
        };
        int64_t c = 0;
        if (n == 0) {
            Batch b;
            b.tc.resize(ps.s > 1 ? ps.s + 1 : 1);
            for (auto &x : b.tc) x.fill(0);
            ps.batches.push_back(b);
        }
        while (c < n) {
            int64_t lo = c, hi = n;
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo + 1) / 2;
                if (wrange(c, mid) <= cap) lo = mid; else hi = mid - 1;
            }
            if (lo == c) {
                set_error("column " + std::to_string(c) + " needs " + std::to_string(wrange(c, c + 1)) +
                          " B, more than one batch may hold (" + std::to_string(cap) + " B)");
                return SPGEMM_ERR_BUDGET;
            }
            Batch b;
            b.c0 = c; b.c1 = lo; b.nnz = hc[lo] - hc[c];
            b.unmerged = hs ? unm(lo) - unm(c) : b.nnz;
            if (inc) inc_sizes(c, lo, b.dsz, b.msz);
            b.pnnz = prune ? ps.prune_prefix[(size_t)lo] - ps.prune_prefix[(size_t)c] : b.nnz;
            ps.batches.push_back(b);
            c = lo;
        }
        const int capmax = ps.tun.hash_cap_max;
        int64_t total_unm = 0;
        for (auto &b : ps.batches) {
            if (ps.s == 1) {
                b.tc.resize(1);
                tier_counts(hc, nullptr, b.c0, b.c1, capmax, b.tc[0], &b.heavy);
            } else {
                // [0] the final merge, [1 + t] stage t, [s + u] the merge into
                // the running sum M_u (incremental, u = 1..s-2)
                b.tc.resize(ps.s + 1 + (inc ? ps.s - 2 : 0));
                tier_counts(hc, nullptr, b.c0, b.c1, capmax, b.tc[0], &b.heavy);
                b.doff.resize(ps.s);
                int64_t off = 0;
                for (int t = 0; t < ps.s; ++t) {
                    const int64_t *sc = hs + (size_t)t * (n + 1);
                    tier_counts(sc, hc, b.c0, b.c1, capmax, b.tc[1 + t], nullptr);
                    b.doff[t] = off;
                    off += sc[b.c1] - sc[b.c0];
                }
                if (inc)
                    for (int u = 1; u <= ps.s - 2; ++u)
                        tier_counts(hp + (size_t)(u - 1) * (n + 1), hc, b.c0, b.c1, capmax, b.tc[ps.s + u],
                                    nullptr);
            }
            total_unm += b.unmerged;
        }
        ps.unmerged = ps.s > 1 ? total_unm : ps.nnz_c;
        ps.stage_buffer_nnz = 0;
        if (ps.s > 1)
            for (auto &b : ps.batches)
                ps.stage_buffer_nnz = std::max(ps.stage_buffer_nnz, inc ? b.dsz + nm * b.msz : b.unmerged);
        return SPGEMM_OK;
    }

    // Partial buffers and per-batch part tables for the k-split merge.
    spgemm_status setup_stage_buffers(PlanState &ps, cudaStream_t st) {
        if (incremental(ps)) return setup_incremental_buffers(ps, st);
        int64_t mx = 0;
        for (auto &b : ps.batches) mx = std::max(mx, b.unmerged);
        SPG_CK(ps.drows.ensure(sizeof(I) * (size_t)(mx + 1)));
        SPG_CK(ps.dvals.ensure(sizeof(V) * (size_t)(mx + 1)));
        const size_t nb = ps.batches.size();
        const size_t bytes = sizeof(PartDev<I, V>) * nb * ps.s;
        SPG_CK(ps.parts_tab.ensure(bytes));
        SPG_CK(ps.h_parts.ensure(bytes));
        auto *tab = ps.h_parts.as<PartDev<I, V>>();
        const int64_t *hs = ps.h_stage_colptr.as<int64_t>();
        for (size_t bi = 0; bi < nb; ++bi) {
            const Batch &b = ps.batches[bi];
            for (int t = 0; t < ps.s; ++t) {
                PartDev<I, V> &p = tab[bi * ps.s + t];
                p.colptr = ps.stage_colptr.as<int64_t>() + (size_t)t * (ps.n + 1);
                p.ptr64 = 1;
                p.sub = hs[(size_t)t * (ps.n + 1) + b.c0] - b.doff[t];
                p.rows = ps.drows.as<I>();
                p.vals = ps.dvals.as<V>();
                p.pcnt = ps.nheavy ? ps.stage_pcnt.as<int32_t>() + (size_t)t * ps.nheavy * ps.P : nullptr;
            }
        }
        SPG_CK(cudaMemcpyAsync(ps.parts_tab.p, ps.h_parts.p, bytes, cudaMemcpyHostToDevice, st));
        SPG_CK(cudaStreamSynchronize(st));
        return SPGEMM_OK;
    }

    // Incremental merge: per batch, the stage buffer holds [D | M_a | M_b]:
    // D (dsz entries) takes stage t >= 1, the running sums alternate between
    // M_a and M_b (msz entries each; M_u lives in region u % 2). The part
    // table has two parts per merge step t = 1..s-1: M_{t-1} and D_t.
    spgemm_status setup_incremental_buffers(PlanState &ps, cudaStream_t st) {
        SPG_CK(ps.drows.ensure(sizeof(I) * (size_t)(ps.stage_buffer_nnz + 1)));
        SPG_CK(ps.dvals.ensure(sizeof(V) * (size_t)(ps.stage_buffer_nnz + 1)));
        const size_t nb = ps.batches.size();
        const int ns = ps.s - 1;
        const size_t bytes = sizeof(PartDev<I, V>) * nb * ns * 2;
        SPG_CK(ps.parts_tab.ensure(bytes));
        SPG_CK(ps.h_parts.ensure(bytes));
        auto *tab = ps.h_parts.as<PartDev<I, V>>();
        for (size_t bi = 0; bi < nb; ++bi) {
            const Batch &b = ps.batches[bi];
            for (int t = 1; t <= ns; ++t) {
                const int u = t - 1;
                PartDev<I, V> &pm = tab[(bi * ns + (size_t)u) * 2];
                PartDev<I, V> &pd = tab[(bi * ns + (size_t)u) * 2 + 1];
                pm.colptr = run_colptr(ps, u);
                pm.ptr64 = 1;
                pm.sub = run_hcolptr(ps, u)[b.c0] - run_offset(b, u);
                pm.rows = ps.drows.as<I>();
                pm.vals = ps.dvals.as<V>();
                pm.pcnt = run_pcnt(ps, u);
                pd.colptr = ps.stage_colptr.as<int64_t>() + (size_t)t * (ps.n + 1);
                pd.ptr64 = 1;
                pd.sub = ps.h_stage_colptr.as<int64_t>()[(size_t)t * (ps.n + 1) + b.c0];
                pd.rows = ps.drows.as<I>();
                pd.vals = ps.dvals.as<V>();
                pd.pcnt = ps.nheavy ? ps.stage_pcnt.as<int32_t>() + (size_t)t * ps.nheavy * ps.P : nullptr;
            }
        }
        SPG_CK(cudaMemcpyAsync(ps.parts_tab.p, ps.h_parts.p, bytes, cudaMemcpyHostToDevice, st));
        SPG_CK(cudaStreamSynchronize(st));
        return SPGEMM_OK;
    }
    // the running sum M_u (u <= s-2): device and host colptr, panel counts,
    // and its offset in a batch's stage buffer
    static const int64_t *run_colptr(const PlanState &ps, int u) {
        return u == 0 ? ps.stage_colptr.as<int64_t>()
                      : ps.pref_colptr.as<int64_t>() + (size_t)(u - 1) * (ps.n + 1);
    }
    static const int64_t *run_hcolptr(const PlanState &ps, int u) {
        return u == 0 ? ps.h_stage_colptr.as<int64_t>()
                      : ps.h_pref_colptr.as<int64_t>() + (size_t)(u - 1) * (ps.n + 1);
    }
    static const int32_t *run_pcnt(const PlanState &ps, int u) {
        if (!ps.nheavy) return nullptr;
        return u == 0 ? ps.stage_pcnt.as<int32_t>()
                      : ps.pref_pcnt.as<int32_t>() + (size_t)(u - 1) * ps.nheavy * ps.P;
    }
    static int64_t run_offset(const Batch &b, int u) { return b.dsz + (int64_t)(u & 1) * b.msz; }

    // ---- numeric -------------------------------------------------------------
    spgemm_status numeric(PlanState &ps, int64_t t, spgemm_csc *C, cudaStream_t st) override {
        const Batch &b = ps.batches[(size_t)t];
        const BatchItems bitems = batch_items(ps, t);
        Ctx cx = make_ctx(ps);
        const int64_t n = ps.n;
        const int64_t *hc = ps.h_colptr.as<int64_t>();
        if (ps.s == 1) {
            NumOut<I, V> o{ps.colptr.as<int64_t>(), hc[b.c0], (I *)C->rowidx, (V *)C->vals};
            GA ga = gemm_args(ps, 0, ps.k);
            SPG_ST((num_pass<SrcGemm<I, V>, SrcPanel<I, V>, SrcPanelRange<I, V>>(
                cx, ga, ga, b.c0, b.c1, ps.cnt.as<int64_t>(), ps.cnt.as<int64_t>(), o, b.tc[0].data(),
                b.heavy > 0, ps.list_sym.as<int32_t>(), ps.off_sym.as<int32_t>(),
                ps.heavy_ord.as<int32_t>(), ps.pcnt.as<int32_t>(), ps.tier.as<uint8_t>(),
                ps.list_num.as<int32_t>(), ps.off_num.as<int32_t>(), st, ps.items.as<HeavyItem>(),
                bitems.n, bitems.order)));
        } else if (incremental(ps)) {
            SPG_ST(numeric_incremental(ps, cx, t, C, st));
        } else {
            const int64_t *hs = ps.h_stage_colptr.as<int64_t>();
            for (int s = 0; s < ps.s; ++s) {
                const int64_t k0 = (int64_t)s * ps.k / ps.s, k1 = (int64_t)(s + 1) * ps.k / ps.s;
                const int64_t *scp = ps.stage_colptr.as<int64_t>() + (size_t)s * (n + 1);
                const int64_t *scnt = ps.stage_cnt.as<int64_t>() + (size_t)s * (n + 1);
                NumOut<I, V> o{scp, hs[(size_t)s * (n + 1) + b.c0] - b.doff[s], ps.drows.as<I>(),
                               ps.dvals.as<V>()};
                GA ga = gemm_args(ps, k0, k1);
                const int32_t *spc = ps.nheavy ? ps.stage_pcnt.as<int32_t>() + (size_t)s * ps.nheavy * ps.P
                                               : nullptr;
                // heavy columns: the merge's work items with this stage's counts,
                // so each stage column is grouped by the ranges the merge reads
                cx.stage_items = true;
                SPG_ST((num_pass<SrcGemm<I, V>, SrcPanel<I, V>, SrcPanelRange<I, V>>(
                    cx, ga, ga, b.c0, b.c1, scnt, ps.cnt.as<int64_t>(), o, b.tc[1 + s].data(),
                    b.heavy > 0, ps.list_sym.as<int32_t>(), ps.off_sym.as<int32_t>(),
                    ps.heavy_ord.as<int32_t>(), spc, ps.tier.as<uint8_t>(), ps.list_num.as<int32_t>(),
                    ps.off_num.as<int32_t>(), st, ps.items.as<HeavyItem>(),
                    bitems.n, bitems.order)));
                cx.stage_items = false;
            }
            // sort-free hash merge of the stage partials (Sec. IV-D)
            cx.ph_hash = kPhMerge;
            cx.ph_dense = kPhMerge;
            PA pa{ps.parts_tab.as<PartDev<I, V>>() + (size_t)t * ps.s, ps.s, ps.m};
            NumOut<I, V> o{ps.colptr.as<int64_t>(), hc[b.c0], (I *)C->rowidx, (V *)C->vals};
            SPG_ST((num_pass<SrcParts<I, V>, SrcPartsPanel<I, V>, SrcPartsRange<I, V>>(
                cx, pa, pa, b.c0, b.c1, ps.cnt.as<int64_t>(), ps.cnt.as<int64_t>(), o, b.tc[0].data(),
                b.heavy > 0, ps.list_sym.as<int32_t>(), ps.off_sym.as<int32_t>(),
                ps.heavy_ord.as<int32_t>(), ps.pcnt.as<int32_t>(), ps.tier.as<uint8_t>(),
                ps.list_num.as<int32_t>(), ps.off_num.as<int32_t>(), st, ps.items.as<HeavyItem>(),
                bitems.n, bitems.order)));
        }
        if (ps.opts.sort_output && !ps.defer_sort)
            SPG_ST(sort_batch(cx, ps.colptr.as<int64_t>(), hc[b.c0], b.c0, b.c1, (I *)C->rowidx, (V *)C->vals,
                              b.heavy > 0 ? ps.items.as<HeavyItem>() : nullptr,
                              ps.item_off.as<int64_t>() + ps.nheavy, ps.n_items, st));
        SPG_CK(rebase_colptr(ps.colptr.as<int64_t>() + b.c0, b.c1 - b.c0, C->colptr,
                             C->ptr_type == SPGEMM_I64, st));
        cx.launched();
        return SPGEMM_OK;
    }

    // Incremental k-split of batch bi: stage 0 goes to the running sum M_0;
    // every later stage t goes to D and is hash-merged with M_{t-1} into M_t
    // (into C for the last stage). Each merge is the same two-part merge as
    // the final one, with the counts and panel counts of M_t.
    spgemm_status numeric_incremental(PlanState &ps, Ctx &cx, int64_t bi, spgemm_csc *C, cudaStream_t st) {
        const Batch &b = ps.batches[(size_t)bi];
        const BatchItems bitems = batch_items(ps, bi);
        const int64_t n = ps.n;
        const int64_t *hc = ps.h_colptr.as<int64_t>();
        const int64_t *hs = ps.h_stage_colptr.as<int64_t>();
        const int ph_hash = cx.ph_hash, ph_dense = cx.ph_dense;
        for (int s = 0; s < ps.s; ++s) {
            const int64_t k0 = (int64_t)s * ps.k / ps.s, k1 = (int64_t)(s + 1) * ps.k / ps.s;
            const int64_t *scp = ps.stage_colptr.as<int64_t>() + (size_t)s * (n + 1);
            const int64_t *scnt = ps.stage_cnt.as<int64_t>() + (size_t)s * (n + 1);
            // stage 0 straight into M_0's region, later stages into D (offset 0)
            const int64_t at = s == 0 ? run_offset(b, 0) : 0;
            NumOut<I, V> o{scp, hs[(size_t)s * (n + 1) + b.c0] - at, ps.drows.as<I>(), ps.dvals.as<V>()};
            GA ga = gemm_args(ps, k0, k1);
            const int32_t *spc = ps.nheavy ? ps.stage_pcnt.as<int32_t>() + (size_t)s * ps.nheavy * ps.P
                                           : nullptr;
            cx.ph_hash = ph_hash;
            cx.ph_dense = ph_dense;
            cx.stage_items = true;
            SPG_ST((num_pass<SrcGemm<I, V>, SrcPanel<I, V>, SrcPanelRange<I, V>>(
                cx, ga, ga, b.c0, b.c1, scnt, ps.cnt.as<int64_t>(), o, b.tc[1 + s].data(), b.heavy > 0,
                ps.list_sym.as<int32_t>(), ps.off_sym.as<int32_t>(), ps.heavy_ord.as<int32_t>(), spc,
                ps.tier.as<uint8_t>(), ps.list_num.as<int32_t>(), ps.off_num.as<int32_t>(), st,
                ps.items.as<HeavyItem>(), bitems.n, bitems.order)));
            if (s == 0) continue;
            // M_s = M_{s-1} + D_s (sort-free hash merge, Sec. IV-D)
            cx.ph_hash = kPhMerge;
            cx.ph_dense = kPhMerge;
            PA pa{ps.parts_tab.as<PartDev<I, V>>() + ((size_t)bi * (ps.s - 1) + (size_t)(s - 1)) * 2, 2, ps.m};
            if (s < ps.s - 1) {
                const int64_t *mcp = run_colptr(ps, s);
                const int64_t *mcnt = ps.pref_cnt.as<int64_t>() + (size_t)(s - 1) * (n + 1);
                NumOut<I, V> om{mcp, run_hcolptr(ps, s)[b.c0] - run_offset(b, s), ps.drows.as<I>(),
                                ps.dvals.as<V>()};
                cx.stage_items = true;
                SPG_ST((num_pass<SrcParts<I, V>, SrcPartsPanel<I, V>, SrcPartsRange<I, V>>(
                    cx, pa, pa, b.c0, b.c1, mcnt, ps.cnt.as<int64_t>(), om, b.tc[ps.s + s].data(),
                    b.heavy > 0, ps.list_sym.as<int32_t>(), ps.off_sym.as<int32_t>(),
                    ps.heavy_ord.as<int32_t>(), run_pcnt(ps, s), ps.tier.as<uint8_t>(),
                    ps.list_num.as<int32_t>(), ps.off_num.as<int32_t>(), st, ps.items.as<HeavyItem>(),
                    bitems.n, bitems.order)));
            } else {
                NumOut<I, V> oc{ps.colptr.as<int64_t>(), hc[b.c0], (I *)C->rowidx, (V *)C->vals};
                cx.stage_items = false;
                SPG_ST((num_pass<SrcParts<I, V>, SrcPartsPanel<I, V>, SrcPartsRange<I, V>>(
                    cx, pa, pa, b.c0, b.c1, ps.cnt.as<int64_t>(), ps.cnt.as<int64_t>(), oc, b.tc[0].data(),
                    b.heavy > 0, ps.list_sym.as<int32_t>(), ps.off_sym.as<int32_t>(),
                    ps.heavy_ord.as<int32_t>(), ps.pcnt.as<int32_t>(), ps.tier.as<uint8_t>(),
                    ps.list_num.as<int32_t>(), ps.off_num.as<int32_t>(), st, ps.items.as<HeavyItem>(),
                    bitems.n, bitems.order)));
            }
        }
        cx.stage_items = false;
        return SPGEMM_OK;
    }

    // ---- sorted output and prune ---------------------------------------------
    // Sort the rows of columns [c0, c1) of a batch in place: the light columns
    // (warp bitonic up to 32 entries, shared-memory bitonic up to 8192) and the
    // hash-range items of the heavy columns; dense items are in row order.
    // colptr: the plan's global offsets, base = offset of column c0.
    static spgemm_status sort_batch(const Ctx &cx, const int64_t *colptr, int64_t base, int64_t c0,
                                    int64_t c1, I *rows, V *vals, const HeavyItem *items,
                                    const int64_t *nitems_dev, int64_t n_items, cudaStream_t st) {
        const int64_t nc = c1 - c0;
        if (nc <= 0) return SPGEMM_OK;
        const unsigned wb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nc + 7) / 8, 1 << 20));
        k_sort_warp<I, V><<<wb, 256, 0, st>>>(colptr, base, c0, c1, rows, vals);
        const int cap = cx.tun.hash_cap_max;
        const unsigned bb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nc, (int64_t)cx.nsm * 8));
        k_sort_block<I, V, 1024><<<bb, 256, (int)(1024 * (4 + sizeof(V))), st>>>(colptr, base, c0, c1, 32,
                                                                                 cap, rows, vals);
        if (cap > 1024)
            k_sort_block<I, V, 8192><<<bb, 512, (int)(8192 * (4 + sizeof(V))), st>>>(colptr, base, c0, c1,
                                                                                   1024, cap, rows, vals);
        if (items && n_items > 0) {
            // staging for the largest hash item (range_cap rows), a bitmap
            // over item row ranges of up to 16 panels and its 16-bit word
            // prefix (wider ranges fall back to the bitonic sort); two CTAs
            // per SM when that fits
            const int64_t want = (int64_t)kRangeMaxPanels << cx.tun.log2R >> 5;
            auto launch = [&](auto cap_tag) -> void {
                constexpr int CAP = decltype(cap_tag)::value;
                const int stage = (int)(CAP * (4 + sizeof(V)));
                const int fit2 = 110 * 1024;   // bytes per CTA for two CTAs per SM
                const int64_t room = std::max<int64_t>(fit2 - stage, 64 * 1024 - stage);
                const int wcap = (int)std::max<int64_t>(32, std::min<int64_t>(want, room / 6));
                const unsigned ib = (unsigned)std::max<int64_t>(1, std::min<int64_t>(n_items, (int64_t)cx.nsm * 2));
                k_sort_items<I, V, CAP><<<ib, 512, stage + 6 * wcap, st>>>(items, nitems_dev, colptr, base, c0,
                                                                            c1, cx.tun.log2R, wcap, rows, vals);
            };
            if (range_cap(cx) <= 4096) launch(std::integral_constant<int, 4096>{});
            else launch(std::integral_constant<int, 8192>{});
        }
        cx.launched(items ? 4 : 3);
        SPG_CK(cudaGetLastError());
        return SPGEMM_OK;
    }

    // The smallest value of type V that is >= thr (so that "v >= it" in V is
    // exactly "v >= thr" in double).
    static V typed_threshold(double thr) {
        using S = typename Storage<V>::type;
        S t;
        if constexpr (std::is_same<S, float>::value) {
            t = (float)thr;
            if (std::isfinite(thr) && (double)t < thr) t = std::nextafterf(t, INFINITY);
        } else if constexpr (std::is_same<S, double>::value) {
            t = thr;
        } else {
            if (thr <= -9.2233720368547758e18) t = INT64_MIN;
            else if (thr > 9.2233720368547748e18) t = INT64_MAX;
            else t = (int64_t)std::ceil(thr);
        }
        if constexpr (std::is_same<V, S>::value) return t;
        else return V::raw(t);
    }

    // prune workspace bytes per column (PruneWs: keep, sel, key, quota 8 B, row
    // 4 B, mode 1 B, and the scan partials)
    static constexpr int64_t kPruneWsPerCol = 40;

    // Prune step 1: kept count per column, the selections, and out_colptr =
    // exclusive scan of the counts (ncols + 1 entries, total last).
    static spgemm_status prune_plan(const int64_t *colptr, const I *rows, const V *vals, int64_t ncols, V thr,
                                    int64_t topk, int tie_by_row, PruneWs &ws, int64_t *out_colptr, int nsm,
                                    cudaStream_t st) {
        SPG_CK(ws.ensure(ncols));
        SPG_CK(cudaMemsetAsync(ws.nsel.p, 0, sizeof(unsigned long long), st));
        if (ncols > 0) {
            const unsigned wb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((ncols + 7) / 8, 1 << 20));
            k_prune_count<V><<<wb, 256, 0, st>>>(colptr, vals, ncols, thr, topk, ws.keep.as<int64_t>(),
                                                 ws.mode.as<int8_t>(), ws.sel.as<int64_t>(),
                                                 ws.nsel.as<unsigned long long>());
            k_prune_select<I, V><<<(unsigned)nsm * 4, 512, 0, st>>>(
                colptr, rows, vals, thr, topk, ws.sel.as<int64_t>(), ws.nsel.as<unsigned long long>(),
                ws.key.as<uint64_t>(), ws.quota.as<int64_t>(), tie_by_row, ws.row.as<uint32_t>());
        }
        SPG_CK(exclusive_scan_i64(ws.keep.as<int64_t>(), ncols, out_colptr, ws.part.as<int64_t>(), 1, st));
        SPG_CK(cudaGetLastError());
        return SPGEMM_OK;
    }

    // Prune step 2: the kept entries, in input order, at out_colptr.
    template <class IO>
    static spgemm_status prune_fill(const int64_t *colptr, const I *rows, const V *vals, int64_t ncols, V thr,
                                    int tie_by_row, PruneWs &ws, const int64_t *out_colptr, IO *orows, V *ovals,
                                    cudaStream_t st) {
        if (ncols <= 0) return SPGEMM_OK;
        const unsigned wb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((ncols + 7) / 8, 1 << 20));
        k_prune_compact<I, V, IO><<<wb, 256, 0, st>>>(colptr, rows, vals, ncols, thr, ws.mode.as<int8_t>(),
                                                      ws.key.as<uint64_t>(), ws.quota.as<int64_t>(), tie_by_row,
                                                      ws.row.as<uint32_t>(), out_colptr, orows, ovals);
        SPG_CK(cudaGetLastError());
        return SPGEMM_OK;
    }

    // spgemm_prune on a caller's CSC (two-call protocol).
    static spgemm_status prune(const spgemm_csc *in, double thr_d, int64_t topk, spgemm_csc *out,
                               cudaStream_t st) {
        int dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int64_t n = in->ncols;
        const V thr = typed_threshold(thr_d);
        DevBuf cp64;
        const int64_t *cp = (const int64_t *)in->colptr;
        if (in->ptr_type == SPGEMM_I32) {
            SPG_CK(cp64.ensure(sizeof(int64_t) * (size_t)(n + 1)));
            k_widen<int32_t><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 256) / 256, 1 << 20)), 256, 0, st>>>(
                (const int32_t *)in->colptr, n + 1, cp64.as<int64_t>());
            cp = cp64.as<int64_t>();
        }
        PruneWs ws;
        DevBuf tmp;
        const bool count_only = out->rowidx == nullptr;
        int64_t *ocp = (int64_t *)out->colptr;
        if (!count_only) {   // recount into scratch; out->colptr holds the first call's offsets
            SPG_CK(tmp.ensure(sizeof(int64_t) * (size_t)(n + 1)));
            ocp = tmp.as<int64_t>();
        }
        SPG_ST(prune_plan(cp, (const I *)in->rowidx, (const V *)in->vals, n, thr, topk, 0, ws, ocp, nsm, st));
        if (count_only) {
            int64_t total = 0;
            SPG_CK(cudaMemcpyAsync(&total, ocp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            SPG_CK(cudaStreamSynchronize(st));
            out->nnz = total;
            return SPGEMM_OK;
        }
        const int64_t *fin = (const int64_t *)out->colptr;
        SPG_ST(prune_fill<I>(cp, (const I *)in->rowidx, (const V *)in->vals, n, thr, 0, ws, fin, (I *)out->rowidx,
                             (V *)out->vals, st));
        SPG_CK(cudaStreamSynchronize(st));   // the scratch buffers go out of scope
        return SPGEMM_OK;
    }

    spgemm_status prune_batch(PlanState &ps, int64_t ncols, const int64_t *colptr, const void *rows,
                              const void *vals, int64_t *ocolptr, void *orows, void *ovals, PruneWs &ws,
                              cudaStream_t st) override {
        const V thr = typed_threshold(ps.opts.prune_threshold);
        // sorted output with a small topk: prune the unsorted batch (ties to
        // the smaller rows, the order sorting would give), then sort only
        // the kept entries
        const int tie_by_row = ps.defer_sort ? 1 : 0;
        SPG_ST(prune_plan(colptr, (const I *)rows, (const V *)vals, ncols, thr, ps.opts.prune_topk, tie_by_row, ws,
                          ocolptr, ps.nsm, st));
        SPG_ST(prune_fill<I>(colptr, (const I *)rows, (const V *)vals, ncols, thr, tie_by_row, ws, ocolptr,
                             (I *)orows, (V *)ovals, st));
        ps.timer.launches += 6;
        if (ps.defer_sort) {
            const int cap = (int)std::min<int64_t>(ps.opts.prune_topk, 8192);
            const unsigned wbk = (unsigned)std::max<int64_t>(1, std::min<int64_t>((ncols + 7) / 8, 1 << 20));
            const unsigned bb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ncols, (int64_t)ps.nsm * 8));
            k_sort_warp<I, V><<<wbk, 256, 0, st>>>(ocolptr, 0, 0, ncols, (I *)orows, (V *)ovals);
            if (cap > 32)
                k_sort_block<I, V, 1024><<<bb, 256, (int)(1024 * (4 + sizeof(V))), st>>>(
                    ocolptr, 0, 0, ncols, 32, cap, (I *)orows, (V *)ovals);
            if (cap > 1024)
                k_sort_block<I, V, 8192><<<bb, 512, (int)(8192 * (4 + sizeof(V))), st>>>(
                    ocolptr, 0, 0, ncols, 1024, cap, (I *)orows, (V *)ovals);
            ps.timer.launches += 3;
            SPG_CK(cudaGetLastError());
        }
        return SPGEMM_OK;
    }

    // ---- backward ------------------------------------------------------------
    spgemm_status backward(PlanState &ps, const spgemm_csc *G, void *dA, void *dB,
                           cudaStream_t st) override {
        if (ps.vtype == SPGEMM_INT64) {
            set_error("backward needs floating-point values");
            return SPGEMM_ERR_INVALID;
        }
        if (IsMinPlus<V>::v || IsOrAnd<V>::v) {
            set_error("backward is defined for the plus-times semiring only");
            return SPGEMM_ERR_INVALID;
        }
        Ctx cx = make_ctx(ps);
        const int64_t n = ps.n;
        GradArgs<I, V> ga{};
        ga.gemm = gemm_args(ps, 0, ps.k);
        ga.gcolptr = G->colptr;
        ga.gptr64 = G->ptr_type == SPGEMM_I64;
        ga.grows = (const I *)G->rowidx;
        ga.gvals = (const V *)G->vals;
        ga.dA = (V *)dA;
        ga.dB = (V *)dB;
        const int tbw = cx.tbegin(kPhBackward, st);
        if (ps.A.nnz)
            k_fill_zero<V><<<(unsigned)((ps.A.nnz + 255) / 256), 256, 0, st>>>((V *)dA, ps.A.nnz);
        if (ps.B.nnz)
            k_fill_zero<V><<<(unsigned)((ps.B.nnz + 255) / 256), 256, 0, st>>>((V *)dB, ps.B.nnz);
        cx.launched(2);
        if (n == 0) { cx.tend(tbw, st); return SPGEMM_OK; }
        SPG_CK(cudaMemsetAsync(cx.hist, 0, sizeof(int32_t) * 64, st));
        SPG_CK(cudaMemsetAsync(cx.cursor, 0, sizeof(int32_t) * 64, st));
        k_bwd_tier<I, V><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ga, n, cx.tun.hash_cap_max,
                                                                       ps.tier.as<uint8_t>(), cx.hist);
        k_bin_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            ps.tier.as<uint8_t>(), 0, n, cx.hist, cx.cursor, ps.list_num.as<int32_t>(),
            ps.off_num.as<int32_t>(), nullptr);
        SPG_CK(cudaMemcpyAsync(cx.h_small, cx.hist, sizeof(int32_t) * 16, cudaMemcpyDeviceToHost, st));
        SPG_CK(cudaStreamSynchronize(st));
        int hist[16];
        std::memcpy(hist, cx.h_small, sizeof(hist));
        TierCommon c = common_of(cx);
        c.list = ps.list_num.as<int32_t>();
        c.list_off = ps.off_num.as<int32_t>();
        for (int t = 1; t <= 8; ++t) {
            if (!hist[t]) continue;
            c.tier = t;
            const int T = 2 * tier_cap(t);
            if (t <= kWarpTiers) {
                const int smem = 8 * T * (int)(4 + sizeof(V));
                const int per_sm = std::max(1, std::min(8, (228 * 1024) / (smem + 1024)));
                const int blocks = std::max(1, std::min((hist[t] + 7) / 8, cx.nsm * per_sm));
                switch (T) {
                    case 64: k_bwd_warp<I, V, 64><<<blocks, 256, smem, st>>>(ga, c); break;
                    case 256: k_bwd_warp<I, V, 256><<<blocks, 256, smem, st>>>(ga, c); break;
                    case 512: k_bwd_warp<I, V, 512><<<blocks, 256, smem, st>>>(ga, c); break;
                    default: k_bwd_warp<I, V, 1024><<<blocks, 256, smem, st>>>(ga, c); break;
                }
                continue;
            }
            const int thr = block_tier_threads(T, cx.tun);
            const int smem = T * (int)(4 + sizeof(V));
            const int per_sm = std::max(1, std::min(2048 / thr, (228 * 1024) / (smem + 34 * 1024)));
            const int blocks = std::max(1, std::min(hist[t], cx.nsm * per_sm));
            switch (T) {
                case 512: k_bwd_block<I, V, 512><<<blocks, thr, smem, st>>>(ga, c); break;
                case 1024: k_bwd_block<I, V, 1024><<<blocks, thr, smem, st>>>(ga, c); break;
                case 2048: k_bwd_block<I, V, 2048><<<blocks, thr, smem, st>>>(ga, c); break;
                case 4096: k_bwd_block<I, V, 4096><<<blocks, thr, smem, st>>>(ga, c); break;
                case 8192: k_bwd_block<I, V, 8192><<<blocks, thr, smem, st>>>(ga, c); break;
                default: k_bwd_block<I, V, 16384><<<blocks, thr, smem, st>>>(ga, c); break;
            }
        }
        int nheavy = 0;
        for (int t = kHeavyTier0; t < kTiers; ++t) nheavy += hist[t];
        if (nheavy) {
            const int smem = dense_smem(cx);
            k_bwd_dense<I, V><<<cx.nsm, 1024, smem, st>>>(ga, c);
            cx.launched();
        }
        for (int t = 1; t <= 8; ++t) if (hist[t]) cx.launched();
        cx.launched(2);
        cx.tend(tbw, st);
        SPG_CK(cudaGetLastError());
        return SPGEMM_OK;
    }

    // ---- standalone merge (spgemm_merge) ---------------------------------------
    static spgemm_status merge(const spgemm_csc *parts, int nparts, spgemm_csc *out, cudaStream_t st) {
        attrs();
        const int64_t n = parts[0].ncols, m = parts[0].nrows;
        int dev = 0;
        cudaDeviceProp prop;
        SPG_CK(cudaGetDevice(&dev));
        SPG_CK(cudaGetDeviceProperties(&prop, dev));
        PlanState tmp;   // scratch only
        tmp.nsm = prop.multiProcessorCount;
        tmp.tun.log2R = sizeof(V) == 4 ? 14 : 13;
        const int64_t R = 1ll << tmp.tun.log2R;
        tmp.P = (int)std::max<int64_t>(1, (m + R - 1) / R);
        const int64_t maxbm = (int64_t)(160 * 1024) * 8;
        const int64_t mpad = ((m + R - 1) / R) * R;
        tmp.Rs = mpad <= maxbm ? (mpad > 0 ? mpad : R) : (maxbm / R) * R;
        tmp.Q = (int)std::max<int64_t>(1, (m + tmp.Rs - 1) / tmp.Rs);
        struct Guard { PlanState &p; ~Guard() { p.release_all(); } } guard{tmp};
        std::vector<PartDev<I, V>> tab(nparts);
        for (int i = 0; i < nparts; ++i) {
            tab[i].colptr = parts[i].colptr;
            tab[i].ptr64 = parts[i].ptr_type == SPGEMM_I64;
            tab[i].sub = 0;
            tab[i].rows = (const I *)parts[i].rowidx;
            tab[i].vals = (const V *)parts[i].vals;
            tab[i].pcnt = nullptr;
        }
        SPG_CK(tmp.parts_tab.ensure(sizeof(PartDev<I, V>) * nparts));
        SPG_CK(tmp.cnt.ensure(sizeof(int64_t) * (n + 1)));
        SPG_CK(tmp.colptr.ensure(sizeof(int64_t) * (n + 1)));
        SPG_CK(tmp.tier.ensure(n + 16));
        SPG_CK(tmp.list_sym.ensure(sizeof(int32_t) * (n + 1)));
        SPG_CK(tmp.list_num.ensure(sizeof(int32_t) * (n + 1)));
        SPG_CK(tmp.heavy_ord.ensure(sizeof(int32_t) * (n + 1)));
        SPG_CK(tmp.hist.ensure(sizeof(int32_t) * 64));
        SPG_CK(tmp.cursor.ensure(sizeof(int32_t) * 64));
        SPG_CK(tmp.off_sym.ensure(sizeof(int32_t) * 64));
        SPG_CK(tmp.off_num.ensure(sizeof(int32_t) * 64));
        SPG_CK(tmp.err.ensure(sizeof(int) * 4));
        SPG_CK(tmp.scan_part.ensure(sizeof(int64_t) * scan_partials_len(n + 1)));
        SPG_CK(tmp.h_small.ensure(4096));
        SPG_CK(cudaMemcpyAsync(tmp.parts_tab.p, tab.data(), sizeof(PartDev<I, V>) * nparts,
                               cudaMemcpyHostToDevice, st));
        SPG_CK(cudaMemsetAsync(tmp.err.p, 0, sizeof(int) * 4, st));
        Ctx cx = make_ctx(tmp);
        PA pa{tmp.parts_tab.as<PartDev<I, V>>(), nparts, m};
        int hist[16];
        SPG_ST(sym_pass<SrcParts<I, V>>(cx, pa, 0, n, nullptr, nullptr, tmp.tier.as<uint8_t>(),
                                        tmp.cnt.as<int64_t>(), tmp.list_sym.as<int32_t>(),
                                        tmp.off_sym.as<int32_t>(), tmp.heavy_ord.as<int32_t>(),
                                        tmp.heavy_ord.as<int32_t>(), &tmp.pcnt, nullptr, hist, st));
        SPG_CK(exclusive_scan_i64(tmp.cnt.as<int64_t>(), n, tmp.colptr.as<int64_t>(),
                                  tmp.scan_part.as<int64_t>(), 1, st));
        int64_t nnz = 0;
        SPG_CK(cudaMemcpyAsync(&nnz, tmp.colptr.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        SPG_CK(cudaStreamSynchronize(st));
        if (out->ptr_type == SPGEMM_I32 && nnz > 0x7fffffffLL) {
            set_error("merged nnz does not fit a 32-bit colptr");
            return SPGEMM_ERR_INDEX_OVERFLOW;
        }
        if (!out->rowidx) {
            SPG_CK(rebase_colptr(tmp.colptr.as<int64_t>(), n, out->colptr, out->ptr_type == SPGEMM_I64, st));
            out->nnz = nnz;
            SPG_CK(cudaStreamSynchronize(st));
            return SPGEMM_OK;
        }
        if (out->nnz != nnz) {
            set_error("out->nnz does not match the merged size");
            return SPGEMM_ERR_INVALID;
        }
        int nheavy = 0;
        for (int t = kHeavyTier0; t < kTiers; ++t) nheavy += hist[t];
        int64_t n_items = 0;
        SPG_ST(build_items(cx, nheavy, tmp.list_sym.as<int32_t>(), tmp.off_sym.as<int32_t>(),
                           tmp.cnt.as<int64_t>(), tmp.pcnt.as<int32_t>(), n, tmp.items, tmp.item_cnt,
                           tmp.item_off, tmp.scan_part, tmp.item_order, &n_items, st));
        NumOut<I, V> o{tmp.colptr.as<int64_t>(), 0, (I *)out->rowidx, (V *)out->vals};
        SPG_ST((num_pass<SrcParts<I, V>, SrcPartsPanel<I, V>, SrcPartsRange<I, V>>(
            cx, pa, pa, 0, n, tmp.cnt.as<int64_t>(), tmp.cnt.as<int64_t>(), o, nullptr, nheavy > 0,
            tmp.list_sym.as<int32_t>(), tmp.off_sym.as<int32_t>(), tmp.heavy_ord.as<int32_t>(),
            tmp.pcnt.as<int32_t>(), tmp.tier.as<uint8_t>(), tmp.list_num.as<int32_t>(),
            tmp.off_num.as<int32_t>(), st, tmp.items.as<HeavyItem>(),
            n_items, tmp.item_order.as<int32_t>())));
        int errw = 0;
        SPG_CK(cudaMemcpyAsync(&errw, tmp.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        SPG_CK(cudaStreamSynchronize(st));
        if (errw) {
            set_error("merge: device error flags " + std::to_string(errw));
            return SPGEMM_ERR_OVERFLOW;
        }
        return SPGEMM_OK;
    }

    // ---- merge into caller-free scratch (spgemm_merge_noalloc) ----------------
    // Same two-call protocol and kernels as merge(), with every work buffer
    // carved from the given device scratch and host staging in static memory;
    // no allocation of any kind. Columns must fit the shared-memory hash tiers.
    static size_t merge_noalloc_bytes(int64_t n, int nparts) {
        auto al = [](size_t x) { return (x + 255) / 256 * 256; };
        return al(sizeof(int64_t) * (n + 1)) * 2 + al(n + 16) + al(sizeof(int32_t) * (n + 1)) * 3 +
               al(sizeof(int32_t) * 64) * 4 + al(sizeof(int) * 4) +
               al(sizeof(int64_t) * scan_partials_len(n + 1)) + al(sizeof(PartDev<I, V>) * nparts);
    }

    static spgemm_status merge_noalloc(const spgemm_csc *parts, int nparts, spgemm_csc *out,
                                       cudaStream_t st, unsigned char *scratch, size_t cap,
                                       int32_t *h_stage, int nsm) {
        const int64_t n = parts[0].ncols, m = parts[0].nrows;
        const size_t need = merge_noalloc_bytes(n, nparts);
        attrs();
        if (need > cap) {
            set_error("merge_noalloc: " + std::to_string(n) + " columns and " + std::to_string(nparts) +
                      " parts need " + std::to_string(need) + " B of scratch; the static scratch holds " +
                      std::to_string(cap) + " B");
            return SPGEMM_ERR_INVALID;
        }
        auto al = [](size_t x) { return (x + 255) / 256 * 256; };
        unsigned char *p = scratch;
        auto take = [&](size_t bytes) { unsigned char *q = p; p += al(bytes); return q; };
        int64_t *cnt = (int64_t *)take(sizeof(int64_t) * (n + 1));
        int64_t *colptr = (int64_t *)take(sizeof(int64_t) * (n + 1));
        uint8_t *tier = (uint8_t *)take(n + 16);
        int32_t *list_sym = (int32_t *)take(sizeof(int32_t) * (n + 1));
        int32_t *list_num = (int32_t *)take(sizeof(int32_t) * (n + 1));
        int32_t *heavy_ord = (int32_t *)take(sizeof(int32_t) * (n + 1));
        int32_t *hist = (int32_t *)take(sizeof(int32_t) * 64);
        int32_t *cursor = (int32_t *)take(sizeof(int32_t) * 64);
        int32_t *off_sym = (int32_t *)take(sizeof(int32_t) * 64);
        int32_t *off_num = (int32_t *)take(sizeof(int32_t) * 64);
        int *err = (int *)take(sizeof(int) * 4);
        int64_t *part_sc = (int64_t *)take(sizeof(int64_t) * scan_partials_len(n + 1));
        PartDev<I, V> *tab_d = (PartDev<I, V> *)take(sizeof(PartDev<I, V>) * nparts);
        PartDev<I, V> tab[64];
        for (int i = 0; i < nparts; ++i) {
            tab[i].colptr = parts[i].colptr;
            tab[i].ptr64 = parts[i].ptr_type == SPGEMM_I64;
            tab[i].sub = 0;
            tab[i].rows = (const I *)parts[i].rowidx;
            tab[i].vals = (const V *)parts[i].vals;
            tab[i].pcnt = nullptr;
        }
        // the scratch keeps the previous call's contents: clear what is read
        // before it is written (error word; tier histogram and cursors are
        // cleared inside the passes)
        SPG_CK(cudaMemcpyAsync(tab_d, tab, sizeof(PartDev<I, V>) * nparts, cudaMemcpyHostToDevice, st));
        SPG_CK(cudaMemsetAsync(err, 0, sizeof(int) * 4, st));
        Ctx cx;
        cx.nsm = nsm;
        cx.err = err; cx.hist = hist; cx.cursor = cursor; cx.h_small = h_stage;
        cx.tun.log2R = sizeof(V) == 4 ? 14 : 13;
        cx.P = 1; cx.Q = 1; cx.Rs = 32;
        PA pa{tab_d, nparts, m};
        int hist_h[16];
        // columns above the largest hash table would need the dense path's
        // per-panel workspace: sym_pass rejects them before any launch
        SPG_ST(sym_pass<SrcParts<I, V>>(cx, pa, 0, n, nullptr, nullptr, tier, cnt, list_sym, off_sym,
                                        heavy_ord, heavy_ord, nullptr, nullptr, hist_h, st, false));
        SPG_CK(exclusive_scan_i64(cnt, n, colptr, part_sc, 1, st));
        int64_t nnz = 0;
        SPG_CK(cudaMemcpyAsync(&nnz, colptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        SPG_CK(cudaStreamSynchronize(st));
        if (out->ptr_type == SPGEMM_I32 && nnz > 0x7fffffffLL) {
            set_error("merged nnz does not fit a 32-bit colptr");
            return SPGEMM_ERR_INDEX_OVERFLOW;
        }
        if (!out->rowidx) {
            SPG_CK(rebase_colptr(colptr, n, out->colptr, out->ptr_type == SPGEMM_I64, st));
            out->nnz = nnz;
            SPG_CK(cudaStreamSynchronize(st));
            return SPGEMM_OK;
        }
        if (out->nnz != nnz) {
            set_error("out->nnz does not match the merged size");
            return SPGEMM_ERR_INVALID;
        }
        NumOut<I, V> o{colptr, 0, (I *)out->rowidx, (V *)out->vals};
        SPG_ST((num_pass<SrcParts<I, V>, SrcPartsPanel<I, V>>(
            cx, pa, pa, 0, n, cnt, cnt, o, nullptr, false, list_sym, off_sym, heavy_ord, nullptr, tier,
            list_num, off_num, st)));
        int errw = 0;
        SPG_CK(cudaMemcpyAsync(&errw, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        SPG_CK(cudaStreamSynchronize(st));
        if (errw) {
            set_error("merge_noalloc: device error flags " + std::to_string(errw));
            return SPGEMM_ERR_OVERFLOW;
        }
        return SPGEMM_OK;
    }

    // ---- many independent products (spgemm_multi) ------------------------------
    static Ctx multi_ctx(MultiState &ms) {
        Ctx c;
        c.nsm = ms.nsm; c.tun = ms.tun; c.err = ms.err.as<int>();
        c.hist = ms.hist.as<int32_t>(); c.cursor = ms.cursor.as<int32_t>();
        c.h_small = ms.h_small.as<int32_t>();
        c.P = 1; c.Q = 1; c.Rs = 32;
        return c;
    }

    static GA multi_args(MultiState &ms) {
        GA a{};
        a.probs = ms.probs.as<PD>();
        a.nprob = ms.nprob;
        a.k0 = 0; a.k1 = INT64_MAX;
        return a;
    }

    static spgemm_status multi_create(MultiState &ms, const spgemm_csc *As, const spgemm_csc *Bs,
                                      cudaStream_t st) {
        attrs();
        std::vector<PD> tab(ms.nprob);
        int64_t g = 0;
        for (int i = 0; i < ms.nprob; ++i) {
            PD &p = tab[i];
            p.ap = (const I *)As[i].colptr; p.ai = (const I *)As[i].rowidx; p.av = (const V *)As[i].vals;
            p.bp = (const I *)Bs[i].colptr; p.bi = (const I *)Bs[i].rowidx; p.bv = (const V *)Bs[i].vals;
            p.m = As[i].nrows; p.gcol0 = g; p.ncols = Bs[i].ncols; p.ka = As[i].ncols;
            g += Bs[i].ncols;
        }
        ms.total_cols = g;
        const int64_t n = g;
        SPG_CK(ms.probs.ensure(sizeof(PD) * ms.nprob));
        SPG_CK(cudaMemcpyAsync(ms.probs.p, tab.data(), sizeof(PD) * ms.nprob, cudaMemcpyHostToDevice, st));
        SPG_CK(ms.f.ensure(sizeof(int64_t) * (n + 1)));
        SPG_CK(ms.cnt.ensure(sizeof(int64_t) * (n + 1)));
        SPG_CK(ms.colptr.ensure(sizeof(int64_t) * (n + 1)));
        SPG_CK(ms.tier.ensure(n + 16));
        SPG_CK(ms.list.ensure(sizeof(int32_t) * (n + 1)));
        SPG_CK(ms.off.ensure(sizeof(int32_t) * 64));
        SPG_CK(ms.hist.ensure(sizeof(int32_t) * 64));
        SPG_CK(ms.cursor.ensure(sizeof(int32_t) * 64));
        SPG_CK(ms.err.ensure(sizeof(int) * 4));
        SPG_CK(ms.scan_part.ensure(sizeof(int64_t) * scan_partials_len(n + 1)));
        SPG_CK(ms.h_small.ensure(4096));
        SPG_CK(cudaMemsetAsync(ms.err.p, 0, sizeof(int) * 4, st));
        // flops of every column: arena capacity (nnz <= flops) and tier check
        Ctx cx = multi_ctx(ms);
        SPG_CK(cudaMemsetAsync(cx.hist, 0, sizeof(int32_t) * 64, st));
        if (n > 0)
            k_flops_bin<SrcGemm<I, V>><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                multi_args(ms), 0, n, cx.tun.hash_cap_max, nullptr, ms.f.as<int64_t>(),
                ms.tier.as<uint8_t>(), ms.cnt.as<int64_t>(), cx.hist);
        SPG_CK(cudaGetLastError());
        SPG_CK(exclusive_scan_i64(ms.f.as<int64_t>(), n, ms.colptr.as<int64_t>(),
                                  ms.scan_part.as<int64_t>(), 1, st));
        SPG_CK(cudaMemcpyAsync(ms.h_small.p, cx.hist, sizeof(int32_t) * 16, cudaMemcpyDeviceToHost, st));
        SPG_CK(cudaMemcpyAsync(ms.h_small.as<char>() + 256, ms.colptr.as<int64_t>() + n, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, st));
        SPG_CK(cudaStreamSynchronize(st));
        int hist[16];
        std::memcpy(hist, ms.h_small.p, sizeof(hist));
        ms.total_flops = *(int64_t *)(ms.h_small.as<char>() + 256);
        ms.capacity = ms.total_flops;
        SPG_CK(ms.rows.ensure(sizeof(I) * (size_t)(ms.capacity + 1)));
        SPG_CK(ms.vals.ensure(sizeof(V) * (size_t)(ms.capacity + 1)));
        // columns above the largest shared-memory table: one global-memory
        // hash table each (2 * min(f_j, m) slots, a power of two)
        ms.heavy_cols = 0;
        for (int t = kHeavyTier0; t < kTiers; ++t) ms.heavy_cols += n > 0 ? hist[t] : 0;
        SPG_CK(ms.gtab_off.ensure(sizeof(int64_t) * (n + 1)));
        if (ms.heavy_cols) {
            SPG_CK(ms.gsize.ensure(sizeof(int64_t) * (n + 1)));
            k_multi_gtab_sizes<SrcGemm<I, V>><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                multi_args(ms), ms.f.as<int64_t>(), ms.tier.as<uint8_t>(), n, ms.gsize.as<int64_t>());
            SPG_CK(cudaGetLastError());
            SPG_CK(exclusive_scan_i64(ms.gsize.as<int64_t>(), n, ms.gtab_off.as<int64_t>(),
                                      ms.scan_part.as<int64_t>(), 1, st));
            int64_t gslots = 0;
            SPG_CK(cudaMemcpyAsync(&gslots, ms.gtab_off.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            SPG_CK(cudaStreamSynchronize(st));
            SPG_CK(ms.gkeys.ensure(sizeof(uint32_t) * (size_t)(gslots + 1)));
            SPG_CK(ms.gvals.ensure(sizeof(V) * (size_t)(gslots + 1)));
        }
        SPG_CK(ms.counter.ensure(sizeof(unsigned long long) * 4));
        // shared memory of the persistent passes: the largest CTA table or
        // the warps' private tables, whichever is larger
        const size_t sv = sizeof(V) + 4;
        const size_t nw = (size_t)ms.threads / 32;
        ms.smem = std::max((size_t)2 * ms.tun.hash_cap_max * sv, nw * 2 * tier_cap(ms.warp_tiers) * sv);
        int per_sm = 0;
        cudaError_t oe = ms.threads == 512
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi_pass<SrcGemm<I, V>, 512, 1>, 512, ms.smem)
            : ms.threads == 256
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi_pass<SrcGemm<I, V>, 256, 1>, 256, ms.smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi_pass<SrcGemm<I, V>, 128, 1>, 128, ms.smem);
        SPG_CK(oe);
        if (per_sm < 1) {
            set_error("the batched tables do not fit shared memory: lower hash_max_cap or warp_max_cap");
            return SPGEMM_ERR_INVALID;
        }
        ms.grid = ms.nsm * per_sm;
        ms.enqueue = &multi_enqueue;
        return SPGEMM_OK;
    }

    // flops, symbolic, scan and numeric for all problems; no host
    // synchronisation (device-driven tier grids), so it can be captured.
    static spgemm_status multi_enqueue(MultiState &ms, cudaStream_t st) {
        Ctx cx = multi_ctx(ms);
        const int64_t n = ms.total_cols;
        GA ga = multi_args(ms);
        SPG_CK(cudaMemsetAsync(cx.hist, 0, sizeof(int32_t) * 64, st));
        SPG_CK(cudaMemsetAsync(cx.cursor, 0, sizeof(int32_t) * 64, st));
        SPG_CK(cudaMemsetAsync(ms.counter.p, 0, sizeof(unsigned long long) * 4, st));
        if (n > 0) {
            // tiers by the flop bound min(f_j, m), the same as at creation
            k_flops_bin<SrcGemm<I, V>><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                ga, 0, n, cx.tun.hash_cap_max, nullptr, nullptr, ms.tier.as<uint8_t>(),
                ms.cnt.as<int64_t>(), cx.hist);
            k_bin_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                ms.tier.as<uint8_t>(), 0, n, cx.hist, cx.cursor, ms.list.as<int32_t>(),
                ms.off.as<int32_t>(), nullptr);
        }
        TierCommon c = common_of(cx);
        c.cnt = ms.cnt.as<int64_t>();
        MultiQueue mq{ms.list.as<int32_t>(), ms.off.as<int32_t>(), ms.counter.as<unsigned long long>(),
                      ms.gtab_off.as<int64_t>(), ms.gkeys.as<uint32_t>(), ms.gvals.p, ms.warp_tiers};
        // one persistent launch counts every column of every problem ...
        if (n > 0) {
            if (ms.threads == 512)
                k_multi_pass<SrcGemm<I, V>, 512, 0><<<ms.grid, 512, ms.smem, st>>>(ga, c, mq, nullptr, nullptr);
            else if (ms.threads == 256)
                k_multi_pass<SrcGemm<I, V>, 256, 0><<<ms.grid, 256, ms.smem, st>>>(ga, c, mq, nullptr, nullptr);
            else
                k_multi_pass<SrcGemm<I, V>, 128, 0><<<ms.grid, 128, ms.smem, st>>>(ga, c, mq, nullptr, nullptr);
        }
        SPG_CK(cudaGetLastError());
        SPG_CK(exclusive_scan_i64(ms.cnt.as<int64_t>(), n, ms.colptr.as<int64_t>(),
                                  ms.scan_part.as<int64_t>(), 1, st));
        // ... and one forms them, into the output arena at the scanned offsets
        c.colptr = ms.colptr.as<int64_t>();
        c.out_base = 0;
        mq.counter = ms.counter.as<unsigned long long>() + 2;
        if (n > 0) {
            if (ms.threads == 512)
                k_multi_pass<SrcGemm<I, V>, 512, 1><<<ms.grid, 512, ms.smem, st>>>(ga, c, mq, ms.rows.as<I>(),
                                                                                    ms.vals.as<V>());
            else if (ms.threads == 256)
                k_multi_pass<SrcGemm<I, V>, 256, 1><<<ms.grid, 256, ms.smem, st>>>(ga, c, mq, ms.rows.as<I>(),
                                                                                    ms.vals.as<V>());
            else
                k_multi_pass<SrcGemm<I, V>, 128, 1><<<ms.grid, 128, ms.smem, st>>>(ga, c, mq, ms.rows.as<I>(),
                                                                                    ms.vals.as<V>());
        }
        SPG_CK(cudaGetLastError());
        return SPGEMM_OK;
    }
};

}  // namespace spg
