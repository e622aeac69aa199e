// Heavy-column symbolic step with 32-bit offsets: the distinct rows of
// C(:, j) = A * B(:, j) (Sec. II-C's column formula), counted per row panel,
// for the columns above the hash tiers. A CTA takes a (row range q, column)
// item from a device counter, marks every contribution's row in a
// shared-memory bitmap over the range, then popcounts it panel by panel.
// The walk is the flattened-stream walk of the heavy numeric: per chunk of
// B entries (one per thread) the non-empty columns of A are compacted into a
// table of 32-bit stream starts, and warps take contiguous 32-wide windows of
// the stream, resolving windows that cross segment starts with one OR-reduce.
// The caller guarantees nnz(A) < 2^31 and min(m, nnz(A)) * kSymChunk < 2^31,
// so entry offsets and stream positions fit in 32 bits.
#pragma once

namespace spg {

constexpr int kSymChunk = 1024;   // B entries per chunk (= threads per CTA)
constexpr int kSymBatch = 4;      // windows whose row loads a warp keeps in flight

struct SymShared {
    int start[kSymChunk + 1];     // stream start of compacted segment s; start[nz] = T
    int qb[kSymChunk];            // segment begin (entry offset from colptr[0]) minus stream start
    int red_len[32];
    int red_cnt[32];
    int tot_len, tot_cnt;
    unsigned long long tot;
};

template <class I, class V>
__global__ void __launch_bounds__(kSymChunk, 1) k_sym_heavy32(GemmArgs<I, V> ga, TierCommon c) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *bm = reinterpret_cast<uint32_t *>(smem);
    __shared__ SymShared sh;
    const int nwords_max = (int)((c.Rs + 31) >> 5);
    for (int w = threadIdx.x; w < nwords_max; w += blockDim.x) bm[w] = 0u;
    if (threadIdx.x == 0) sh.tot = 0;
    const int lo = c.list_off[kHeavyTier0], hi = c.list_off[kTiers];
    const int64_t nitems = (int64_t)(hi - lo) * c.Q;
    const int wordsR = 1 << (c.log2R - 5);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned below_mask = (1u << lane) - 1u;
    const unsigned upto_mask = 0xffffffffu >> (31 - lane);
    const int64_t k0 = ga.k0, k1 = ga.k1;
    // items come from a device counter; thread 0 reserves the next item when
    // it starts one, so the counter's round trip overlaps the item's work
    __shared__ int s_item;
    int ahead = 0;
    if (threadIdx.x == 0) ahead = atomicAdd(c.next_col, 1);
    auto fetch = [&]() -> int64_t {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_item = ahead;
            ahead = atomicAdd(c.next_col, 1);
        }
        __syncthreads();
        return s_item;
    };
    for (int64_t item = fetch(); item < nitems; item = fetch()) {
        const int64_t ri = nitems - 1 - item;   // the list ascends in sub-tier: largest first
        const int hpos = (int)(ri / c.Q);
        const int q = (int)(ri % c.Q);
        const int64_t g = c.list[lo + hpos];
        const ProbDev<I, V> *pd = ga.probs + locate_prob(ga.probs, ga.nprob, g);
        const I *ap = pd->ap;
        const int64_t a0 = (int64_t)ap[0];
        const I *arow = pd->ai + a0;
        const int64_t bc = g - pd->gcol0;
        const int64_t b0 = (int64_t)pd->bp[bc];
        const int nb = (int)((int64_t)pd->bp[bc + 1] - b0);
        const int64_t r0 = (int64_t)q * c.Rs;
        const int64_t rows = (pd->m - r0) < c.Rs ? (pd->m - r0) : c.Rs;
        const bool filt = c.Q > 1;
        for (int base = 0; base < nb; base += kSymChunk) {
            // 1. segments of this chunk's B entries
            const int e = base + (int)threadIdx.x;
            int len = 0, qrel = 0;
            if (e < nb) {
                const int64_t k = (int64_t)__ldg(&pd->bi[b0 + e]);
                if (k >= k0 && k < k1) {
                    const int64_t s = (int64_t)__ldg(&ap[k]);
                    len = (int)((int64_t)__ldg(&ap[k + 1]) - s);
                    qrel = (int)(s - a0);
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
            }
            if (threadIdx.x == 0) sh.start[nz] = T;
            __syncthreads();
            // 2. the flattened stream, a contiguous share of windows per warp
            const int nwin = (T + 31) >> 5;
            const int per = (nwin + nw - 1) / nw;
            const int w0 = warp * per * 32;
            const int W1 = min(T, w0 + per * 32);
            if (w0 < W1) {
                int lo_s = 0, hi_s = nz - 1;
                while (lo_s < hi_s) {
                    const int mid = (lo_s + hi_s + 1) >> 1;
                    if (sh.start[mid] <= w0) lo_s = mid; else hi_s = mid - 1;
                }
                int s = lo_s;
                int send = sh.start[s + 1];
                int qb = sh.qb[s];
                for (int wb = w0; wb < W1; wb += 32 * kSymBatch) {
                    int qq[kSymBatch];
                    bool ok[kSymBatch];
#pragma unroll
                    for (int u = 0; u < kSymBatch; ++u) {
                        const int w = wb + 32 * u;
                        const int t = w + lane;
                        ok[u] = t < W1;
                        qq[u] = 0;
                        if (w >= W1) continue;   // warp-uniform
                        if (w + 32 <= send) {
                            qq[u] = qb + t;
                        } else {
                            const int j = s + 1 + lane;
                            unsigned bit = 0u;
                            if (j < nz) {
                                const int d = sh.start[j] - w;
                                if (d < 32) bit = 1u << d;
                            }
                            const unsigned M = __reduce_or_sync(SPG_FULL, bit);
                            const int sg = s + __popc(M & upto_mask);
                            if (ok[u]) qq[u] = sh.qb[sg] + t;
                            s += __popc(M);
                            send = sh.start[s + 1];
                            qb = sh.qb[s];
                        }
                    }
                    int64_t rr[kSymBatch];
#pragma unroll
                    for (int u = 0; u < kSymBatch; ++u) rr[u] = ok[u] ? (int64_t)__ldg(&arow[qq[u]]) - r0 : -1;
#pragma unroll
                    for (int u = 0; u < kSymBatch; ++u) {
                        const int64_t r = rr[u];
                        if (ok[u] && (!filt || (r >= 0 && r < rows)))
                            atomicOr(&bm[r >> 5], 1u << (r & 31));
                    }
                }
            }
            __syncthreads();
        }
        // 3. per-panel popcounts (clearing the words), the column total
        const int nwords = (int)((rows + 31) >> 5);
        const int h = c.heavy_ord[g];
        const int p0 = (int)(r0 >> c.log2R);
        const int np = (nwords + wordsR - 1) / wordsR;
        for (int pp = warp; pp < np; pp += nw) {
            const int wlo = pp * wordsR;
            const int whi = (wlo + wordsR) < nwords ? (wlo + wordsR) : nwords;
            int cntp = 0;
            for (int w = wlo + lane; w < whi; w += 32) { cntp += __popc(bm[w]); bm[w] = 0u; }
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
    }
}

}  // namespace spg
