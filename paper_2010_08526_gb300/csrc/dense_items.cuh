// Work items of the heavy-column numeric (products of one column of C
// restricted to a range of row panels, Sec. II-C's column formula), with
// 32-bit offsets throughout.
//
// A dense item (column j, panel p) accumulates C(p*R : (p+1)*R, j) in shared
// memory. A hash-range item (column j, panels [p0, p1) holding few output
// rows) accumulates them in a shared-memory hash table keyed by the global
// row, reading each B entry's run of A over all its panels at once from the
// column-grouped copy of A. The contributions of a dense item are the segments
// A_p(:, k) * B(k, j) for k in B(:, j), read from the row-panelised copy of A
// (panel-major: the entries of panel p are one contiguous block, local rows
// as 16-bit integers). Per chunk of B entries (one per thread) the CTA
//   1. looks up every segment and compacts the non-empty ones into a table
//      of 32-bit stream starts, entry offsets and B values (one block scan);
//   2. walks the flattened product stream [0, T) in 32-wide windows, each
//      warp a contiguous share: a window inside one segment needs no lookup;
//      a window crossing segment starts finds every lane's segment with one
//      shared load per lane and one OR-reduce of the start bits;
//   3. keeps the gathers of kDenseBatch windows in flight before applying them.
// Offsets inside a panel are 32-bit (the caller guarantees nnz(A) < 2^31), so
// the walk's bookkeeping is plain int arithmetic.
//
// Presence without a per-product flag: a row is taken as present when its
// accumulator differs from the identity V(0). The item's exact row count (the
// symbolic step's per-panel count) checks this: if fewer rows qualify (a sum
// that cancelled back to the identity, or products equal to it), a second
// walk marks the rows reached in a bitmap and the bits decide. The
// output is written one row per lane, rows ascending within the panel.
#pragma once

namespace spg {

constexpr int kDenseChunk = 512;   // B entries per chunk (= threads per CTA)
constexpr int kDenseBatch = 4;     // windows whose gathers a warp keeps in flight

template <class V> struct DenseShared {
    int start[kDenseChunk + 1];    // stream start of compacted segment s; start[nz] = T
    int qb[kDenseChunk];           // segment begin (panel-relative entry) minus stream start
    V bv[kDenseChunk];             // B(k, j) of the segment
    int red_len[32];
    int red_cnt[32];
    int tot_len, tot_cnt;
};

// Bits of an accumulator equal to the semiring's identity V(0) (never
// touched, or summed back to exactly the identity).
template <class V> __device__ __forceinline__ bool is_identity(const V &a) {
    const V z = V(0);
    if constexpr (sizeof(V) == 4) {
        return *reinterpret_cast<const uint32_t *>(&a) == *reinterpret_cast<const uint32_t *>(&z);
    } else {
        return *reinterpret_cast<const uint64_t *>(&a) == *reinterpret_cast<const uint64_t *>(&z);
    }
}

// Count of accumulators in acc[lo, lo + n) (n a multiple of 32 / sizeof(V)
// * 4 words) that left the identity, read 16 bytes per lane; warp-wide.
template <class V> __device__ __forceinline__ int count_touched(const V *acc, int lo, int n) {
    const int lane = threadIdx.x & 31;
    const V z = V(0);
    const uint4 *a4 = reinterpret_cast<const uint4 *>(acc + lo);
    const int n4 = n * (int)sizeof(V) / 16;
    int cnt = 0;
    if constexpr (sizeof(V) == 4) {
        const uint32_t id = *reinterpret_cast<const uint32_t *>(&z);
        for (int i = lane; i < n4; i += 32) {
            const uint4 w = a4[i];
            cnt += (w.x != id) + (w.y != id) + (w.z != id) + (w.w != id);
        }
    } else {
        const uint64_t id = *reinterpret_cast<const uint64_t *>(&z);
        const uint32_t lo32 = (uint32_t)id, hi32 = (uint32_t)(id >> 32);
        for (int i = lane; i < n4; i += 32) {
            const uint4 w = a4[i];
            cnt += (w.x != lo32 || w.y != hi32) + (w.z != lo32 || w.w != hi32);
        }
    }
    return warp_sum(cnt);
}

// Exclusive offset of this warp's count among the CTA's warps, and the CTA
// total (all threads call it; two barriers; red holds nw ints).
__device__ __forceinline__ int warp_offset_total(int n, int *red, int warp, int nw, int lane, int &tot) {
    if (lane == 0) red[warp] = n;
    __syncthreads();
    const int v = lane < nw ? red[lane] : 0;
    const int incl = warp_incl_scan(v);
    const int off = __shfl_sync(SPG_FULL, incl - v, warp & 31);
    tot = __shfl_sync(SPG_FULL, incl, 31);
    __syncthreads();
    return off;
}

// Inserts a lane's U keys (kEmpty = no key) into a table of 2^log2T slots
// and returns their slots in slot[u] (-1: no key, or a full table, which sets
// kErrProbe). Double hashing (an odd step from a second multiplicative hash,
// so a probe sequence visits every slot) keeps the probe chains short, and a
// probe is a single compare-and-swap: most keys of a hash-range item are new.
template <int U>
__device__ __forceinline__ void hash_insert_dbl(uint32_t *keys, int log2T, const uint32_t (&key)[U],
                                                int (&slot)[U], int *err) {
    const uint32_t mask = (1u << log2T) - 1u;
    uint32_t h[U], step[U];
    unsigned pending = 0u;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        slot[u] = -1;
        h[u] = hash_slot(key[u], log2T);
        step[u] = ((key[u] * 0x85EBCA6Bu) >> (32 - log2T)) | 1u;
        if (key[u] != kEmpty) pending |= 1u << u;
    }
    for (uint32_t probe = 0; pending && probe <= mask; ++probe) {
        uint32_t cur[U];
#pragma unroll
        for (int u = 0; u < U; ++u) cur[u] = ((pending >> u) & 1u) ? atomicCAS(&keys[h[u]], kEmpty, key[u]) : 0u;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!((pending >> u) & 1u)) continue;
            if (cur[u] == kEmpty || cur[u] == key[u]) {
                slot[u] = (int)h[u];
                pending &= ~(1u << u);
            } else {
                h[u] = (h[u] + step[u]) & mask;
            }
        }
    }
    if (pending) atomicOr(err, kErrProbe);
}

template <class I, class V, int MINB>
__global__ void __launch_bounds__(kDenseChunk, MINB)
    k_num_heavy32(GemmArgs<I, V> ga, TierCommon c, const HeavyItem *items, const int32_t *order,
                  int64_t nitems, int *next_item, I *out_rows, V *out_vals) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = 1 << c.log2R;
    // dense view: acc[R] + a presence bitmap fb[R/32] (used only when the
    // values cannot tell presence); hash view (inside acc, fixed layout for
    // every table size Ti <= Tmax): tv[Tmax] values, then tk[Tmax] keys.
    // Between items the memory is clean for the current view (acc all V(0);
    // or tv all V(0) and tk all kEmpty), so an item clears nothing: a hash
    // item resets the slots it filled, a dense item the rows it wrote, and
    // the key words are rewritten only when the item kind changes (the items
    // come ordered dense first, then hash, within each batch).
    V *acc = reinterpret_cast<V *>(smem);
    uint32_t *fb = reinterpret_cast<uint32_t *>(smem + sizeof(V) * R);
    const int Tmax = 2 * c.range_cap;
    V *tv = reinterpret_cast<V *>(smem);
    uint32_t *tk = reinterpret_cast<uint32_t *>(smem + sizeof(V) * Tmax);
    bool hash_view = false;   // the same in every thread
    __shared__ DenseShared<V> sh;
    for (int r = threadIdx.x; r < R; r += blockDim.x) acc[r] = V(0);
    for (int w = threadIdx.x; w < (R >> 5); w += blockDim.x) fb[w] = 0u;
    __syncthreads();
    const ProbDev<I, V> *pd = ga.probs;
    const I *bp = pd->bp;
    const I *bi = pd->bi;
    const I *ap = pd->ap;
    const V *bvp = pd->bv;
    const int64_t ka = pd->ka, k0 = ga.k0, k1 = ga.k1;
    const int64_t a0 = (int64_t)ap[0];
    const int64_t P1s = (int64_t)c.P + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned below_mask = (1u << lane) - 1u;
    const unsigned upto_mask = 0xffffffffu >> (31 - lane);
    // rows owned by each warp in the count and write passes of a dense item
    // (R / nw, a multiple of 32 for R >= 2^10)
    const int rpw = R / nw;
    const int rlo = warp * rpw;
    // items are taken in order from a device counter, one at a time per CTA
    // (reserving the next item early, as the symbolic kernels do, measured 1%
    // slower here: the reserved items unbalance the tail)
    __shared__ int s_item;
    auto fetch = [&]() -> int64_t {
        __syncthreads();   // every thread is past the previous item
        if (threadIdx.x == 0) s_item = atomicAdd(next_item, 1);
        __syncthreads();
        return s_item;
    };
    for (int64_t it = fetch(); it < nitems; it = fetch()) {
        const HeavyItem item = items[order[it]];
        const int64_t g = item.g;
        if (g < c.c_lo || g >= c.c_hi) continue;
        const int p0 = item.p0, p1 = item.p1;
        bool dense = item.cnt < 0;
        int mycnt;
        int64_t ioff;
        if (c.item_counts_from_pcnt) {
            // a k-stage: the same panel ranges, this stage's counts
            const int32_t *pc = c.pcnt_in + (int64_t)c.heavy_ord[g] * c.P;
            int below = 0, in = 0;
            for (int pp = lane; pp < p1; pp += 32) {
                const int x = pc[pp];
                if (pp < p0) below += x; else in += x;
            }
            mycnt = warp_sum(in);
            ioff = warp_sum(below);
            dense = (p1 - p0 == 1);
            if (mycnt == 0) continue;
        } else {
            mycnt = dense ? -item.cnt : item.cnt;
            ioff = item.off;
        }
        const int64_t out0 = c.colptr[g] - c.out_base + ioff;
        const int64_t bc = g - pd->gcol0;
        const int64_t b0 = (int64_t)bp[bc];
        const int nb = (int)((int64_t)bp[bc + 1] - b0);
        const int64_t pk = (int64_t)p0 * ka;
        const int64_t pbase = pk ? ga.ap_end[pk - 1] : 0;
        // dense items read the panel-major copy (16-bit rows local to panel
        // p0, entries relative to the panel's first); hash-range items read the
        // column-grouped copy (global rows, entries relative to column 0)
        const uint16_t *prow = ga.ap_row + pbase;
        const V *pval = ga.ap_val + pbase;
        const uint32_t *crow = ga.apc_row;
        const V *cval = ga.apc_val;
        // hash view: the next power of two >= 2 * count slots
        int lt = 6;
        while ((1 << lt) < 2 * mycnt && (1 << lt) < Tmax) ++lt;
        const int Ti = 1 << lt;
        if (dense == hash_view) {
            // switch views: the key words become kEmpty (to hash) or V(0)
            // (to dense); the value words are V(0) in both
            uint32_t *kw = reinterpret_cast<uint32_t *>(tk);
            if (dense) {
                V *a = reinterpret_cast<V *>(kw);
                const int nv = Tmax * 4 / (int)sizeof(V);
                for (int r = threadIdx.x; r < nv; r += blockDim.x) a[r] = V(0);
            } else {
                uint4 *k4 = reinterpret_cast<uint4 *>(kw);
                for (int w = threadIdx.x; w < Tmax / 4; w += blockDim.x)
                    k4[w] = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
            }
            hash_view = !dense;
            __syncthreads();
        }
        // all chunks of the item; mode 0: accumulate the values (dense or
        // hash by the item's kind); mode 1: mark the rows of a dense item
        auto walk_item = [&](const int mode) {
            for (int base = 0; base < nb; base += kDenseChunk) {
                // 1. segments of this chunk's B entries
                const int e = base + (int)threadIdx.x;
                int len = 0, qrel = 0;
                V bvv = V(0);
                if (e < nb) {
                    const int64_t k = (int64_t)__ldg(&bi[b0 + e]);
                    if (k >= k0 && k < k1) {
                        if (dense) {
                            const int64_t idx = pk + k;
                            const int64_t s = idx ? __ldg(&ga.ap_end[idx - 1]) : 0;
                            len = (int)(__ldg(&ga.ap_end[idx]) - s);
                            qrel = (int)(s - pbase);
                        } else {
                            const int32_t *o = ga.apc_off + k * P1s;
                            const int o0 = __ldg(&o[p0]);
                            len = __ldg(&o[p1]) - o0;
                            qrel = (int)((int64_t)__ldg(&ap[k]) - a0) + o0;
                        }
                        bvv = __ldg(&bvp[b0 + e]);
                    }
                }
                const unsigned nzm = __ballot_sync(SPG_FULL, len > 0);
                const int incl = warp_incl_scan(len);
                if (lane == 31) { sh.red_len[warp] = incl; sh.red_cnt[warp] = __popc(nzm); }
                __syncthreads();
                if (warp == 0) {
                    const int vl = lane < nw ? sh.red_len[lane] : 0;
                    const int vc = lane < nw ? sh.red_cnt[lane] : 0;
                    const int il = warp_incl_scan(vl), ic = warp_incl_scan(vc);
                    sh.red_len[lane] = il - vl;
                    sh.red_cnt[lane] = ic - vc;
                    if (lane == 31) { sh.tot_len = il; sh.tot_cnt = ic; }
                }
                __syncthreads();
                const int T = sh.tot_len, nz = sh.tot_cnt;
                if (len > 0) {
                    const int slot = sh.red_cnt[warp] + __popc(nzm & below_mask);
                    const int st0 = sh.red_len[warp] + incl - len;
                    sh.start[slot] = st0;
                    sh.qb[slot] = qrel - st0;
                    sh.bv[slot] = bvv;
                }
                if (threadIdx.x == 0) sh.start[nz] = T;
                __syncthreads();
                // 2-3. the flattened stream, a contiguous share of windows per warp
                const int nwin = (T + 31) >> 5;
                const int per = (nwin + nw - 1) / nw;
                const int w0 = warp * per * 32;
                const int W1 = min(T, w0 + per * 32);
                if (w0 < W1) {
                    // the segment holding position w0
                    int lo = 0, hi = nz - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (sh.start[mid] <= w0) lo = mid; else hi = mid - 1;
                    }
                    // invariant: start[s] <= w <= send for the next window w
                    int s = lo;
                    int send = sh.start[s + 1];
                    int qb = sh.qb[s];
                    V bvc = sh.bv[s];
                    for (int wb = w0; wb < W1; wb += 32 * kDenseBatch) {
                        int q[kDenseBatch];
                        V b[kDenseBatch];
                        bool ok[kDenseBatch];
#pragma unroll
                        for (int u = 0; u < kDenseBatch; ++u) {
                            const int w = wb + 32 * u;
                            const int t = w + lane;
                            ok[u] = t < W1;
                            q[u] = 0;
                            b[u] = V(0);
                            if (w >= W1) continue;   // warp-uniform
                            if (w + 32 <= send) {
                                q[u] = qb + t;
                                b[u] = bvc;
                            } else {
                                // segment starts at window offsets d in [0, 32)
                                const int j = s + 1 + lane;
                                unsigned bit = 0u;
                                if (j < nz) {
                                    const int d = sh.start[j] - w;
                                    if (d < 32) bit = 1u << d;
                                }
                                const unsigned M = __reduce_or_sync(SPG_FULL, bit);
                                const int sg = s + __popc(M & upto_mask);
                                if (ok[u]) {
                                    q[u] = sh.qb[sg] + t;
                                    b[u] = sh.bv[sg];
                                }
                                s += __popc(M);
                                send = sh.start[s + 1];
                                qb = sh.qb[s];
                                bvc = sh.bv[s];
                            }
                        }
                        if (mode == 1) {
#pragma unroll
                            for (int u = 0; u < kDenseBatch; ++u)
                                if (ok[u]) {
                                    const uint32_t r = __ldg(&prow[q[u]]);
                                    atomicOr(&fb[r >> 5], 1u << (r & 31));
                                }
                        } else if (dense) {
                            uint32_t r[kDenseBatch];
                            V x[kDenseBatch];
#pragma unroll
                            for (int u = 0; u < kDenseBatch; ++u) {
                                r[u] = 0;
                                x[u] = V(0);
                                if (ok[u]) {
                                    r[u] = __ldg(&prow[q[u]]);
                                    x[u] = mul_v(__ldg(&pval[q[u]]), b[u]);
                                }
                            }
#pragma unroll
                            for (int u = 0; u < kDenseBatch; ++u)
                                if (ok[u]) atomic_add_v(&acc[r[u]], x[u]);
                        } else {
                            uint32_t key[kDenseBatch];
                            V x[kDenseBatch];
#pragma unroll
                            for (int u = 0; u < kDenseBatch; ++u) {
                                key[u] = kEmpty;
                                x[u] = V(0);
                                if (ok[u]) {
                                    key[u] = __ldg(&crow[q[u]]);
                                    x[u] = mul_v(__ldg(&cval[q[u]]), b[u]);
                                }
                            }
                            int hs[kDenseBatch];
                            hash_insert_dbl<kDenseBatch>(tk, lt, key, hs, c.err);
#pragma unroll
                            for (int u = 0; u < kDenseBatch; ++u)
                                if (hs[u] >= 0) atomic_add_v(&tv[hs[u]], x[u]);
                        }
                    }
                }
                __syncthreads();
            }
        };
        walk_item(0);
        if (!dense) {
            // slots split among the warps; the keys mark the rows exactly
            const int spw = (Ti + nw - 1) / nw;
            const int slo = min(Ti, warp * spw), shi = min(Ti, slo + spw);
            int n = 0;
            for (int s = slo + lane; s < shi; s += 32) n += tk[s] != kEmpty;
            n = warp_sum(n);
            int tot;
            int o = warp_offset_total(n, sh.red_cnt, warp, nw, lane, tot);
            if (threadIdx.x == 0 && tot != mycnt) atomicOr(c.err, kErrCount);
            for (int s0 = slo; s0 < shi; s0 += 32) {
                const int s = s0 + lane;
                const uint32_t key = s < shi ? tk[s] : kEmpty;
                const bool occ = key != kEmpty;
                const unsigned bal = __ballot_sync(SPG_FULL, occ);
                if (occ) {
                    const int oo = o + __popc(bal & below_mask);
                    if (oo < mycnt) {
                        out_rows[out0 + oo] = (I)key;
                        out_vals[out0 + oo] = tv[s];
                    }
                    tk[s] = kEmpty;
                    tv[s] = V(0);
                }
                o += __popc(bal);
            }
            __syncthreads();
            continue;
        }
        // A row is present when its accumulator left the identity. The
        // symbolic count of the item is exact: when fewer rows qualify (a
        // sum that cancelled to the identity, or products equal to it), the
        // rows reached are marked in a second walk and the bits decide.
        int tot;
        int o = warp_offset_total(count_touched(acc, rlo, rpw), sh.red_cnt, warp, nw, lane, tot);
        const bool by_flags = tot != mycnt;   // the same for the whole CTA
        if (by_flags) {
            walk_item(1);
            int n = 0;
            for (int w = (rlo >> 5) + lane; w < ((rlo + rpw) >> 5); w += 32) n += __popc(fb[w]);
            n = warp_sum(n);
            o = warp_offset_total(n, sh.red_cnt, warp, nw, lane, tot);
            if (threadIdx.x == 0 && tot != mycnt) atomicOr(c.err, kErrCount);
        }
        // write pass: one row per lane, rows ascending, coalesced stores
        const int64_t rbase = (int64_t)p0 << c.log2R;
        for (int r0 = rlo; r0 < rlo + rpw; r0 += 32) {
            const int rr = r0 + lane;
            const V a = acc[rr];
            const bool pr = by_flags ? ((fb[rr >> 5] >> (rr & 31)) & 1u) != 0 : !is_identity(a);
            const unsigned bal = __ballot_sync(SPG_FULL, pr);
            if (pr) {
                const int oo = o + __popc(bal & below_mask);
                if (oo < mycnt) {
                    out_rows[out0 + oo] = (I)(rbase + rr);
                    out_vals[out0 + oo] = a;
                }
                acc[rr] = V(0);
            }
            o += __popc(bal);
        }
        if (by_flags) {
            __syncwarp();
            for (int w = (rlo >> 5) + lane; w < ((rlo + rpw) >> 5); w += 32) fb[w] = 0u;
        }
        __syncthreads();
    }
}

}  // namespace spg
