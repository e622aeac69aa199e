// The memory-constrained batch loop (Algorithm 4 on one device): batch t+1 is
// multiplied on the compute stream while batch t is copied, piece by piece,
// into pinned host slots on the copy stream and handed to the sink.
#include <algorithm>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "../../include/spgemm.h"
#include "plan.h"

using namespace spg;

namespace {

struct Piece {
    int64_t batch, c0, c1;   // global column range
    int slot;
    cudaEvent_t done;
    int64_t nnz;
};

}  // namespace

extern "C" spgemm_status spgemm_run_batched(spgemm_plan *plan, spgemm_sink_fn sink, void *ctx,
                                            cudaStream_t compute, cudaStream_t copy) {
    if (!plan || !sink) { set_error("NULL argument"); return SPGEMM_ERR_INVALID; }
    PlanState &ps = plan->ps;
    AllocScope scope(ps.alloc);
    if (!ps.have_symbolic) { set_error("call spgemm_symbolic first"); return SPGEMM_ERR_STATE; }
    const int R = ps.opts.ring_depth > 0 ? ps.opts.ring_depth : 2;
    const int H = ps.opts.host_slots >= 2 ? ps.opts.host_slots : 3;
    const size_t slot_req = ps.opts.host_slot_bytes ? ps.opts.host_slot_bytes : ((size_t)256 << 20);
    const int64_t si = ps.idx64 ? 8 : 4;
    const int64_t sv = ps.vtype == SPGEMM_F32 ? 4 : 8;
    const int64_t *hc = ps.h_colptr.as<int64_t>();
    const int64_t nb = (int64_t)ps.batches.size();

    // with opts.prune every batch is pruned on the device (into a second
    // ring) before its copy; the host reads the pruned colptr to cut pieces
    const bool prune = ps.opts.prune != 0;
    // sorted output with 0 < topk <= 8192: the prune runs on the unsorted batch
    // and only the kept entries are sorted (restored on every return path)
    struct DeferSort {
        PlanState &p;
        ~DeferSort() { p.defer_sort = false; }
    } defer_guard{ps};
    ps.defer_sort = prune && ps.opts.sort_output && ps.opts.prune_topk > 0 && ps.opts.prune_topk <= 8192;
    // pieces: column ranges whose rows + values + colptr fit one host slot
    int64_t max_nnz = 0, max_cols = 0, max_col_bytes = 0, max_pnnz = 0;
    for (auto &b : ps.batches) {
        max_nnz = std::max(max_nnz, b.nnz);
        max_cols = std::max(max_cols, b.c1 - b.c0);
        max_pnnz = std::max(max_pnnz, b.pnnz);
    }
    for (int64_t j = 0; j < ps.n; ++j)
        max_col_bytes = std::max(max_col_bytes, (hc[j + 1] - hc[j]) * (si + sv) + 16);
    const size_t slot_bytes = std::max<size_t>(slot_req, (size_t)max_col_bytes + 64);

    // device ring and pinned host slots (kept by the plan across runs)
    if ((int)ps.ring_col.size() < R) {
        ps.ring_col.resize(R); ps.ring_row.resize(R); ps.ring_val.resize(R);
    }
    if ((int)ps.host_slots.size() < H) ps.host_slots.resize(H);
    std::vector<DevBuf> &dcol = ps.ring_col, &drow = ps.ring_row, &dval = ps.ring_val;
    std::vector<HostBuf> &hslot = ps.host_slots;
    std::vector<cudaEvent_t> ready(R, nullptr), freed(R, nullptr);
    auto cleanup = [&]() {
        for (auto ev : ready) if (ev) cudaEventDestroy(ev);
        for (auto ev : freed) if (ev) cudaEventDestroy(ev);
    };
    cudaError_t e = cudaSuccess;
    if (prune) {
        if ((int)ps.ring_pcol.size() < R) {
            ps.ring_pcol.resize(R); ps.ring_prow.resize(R); ps.ring_pval.resize(R);
            ps.ring_hpc.resize(R); ps.ring_pws.resize(R);
        }
        for (int i = 0; i < R && e == cudaSuccess; ++i) {
            if ((e = ps.ring_pcol[i].ensure(sizeof(int64_t) * (max_cols + 1))) != cudaSuccess) break;
            if ((e = ps.ring_prow[i].ensure((size_t)si * (max_pnnz + 1))) != cudaSuccess) break;
            if ((e = ps.ring_pval[i].ensure((size_t)sv * (max_pnnz + 1))) != cudaSuccess) break;
            if ((e = ps.ring_hpc[i].ensure(sizeof(int64_t) * (max_cols + 1))) != cudaSuccess) break;
            if ((e = ps.ring_pws[i].ensure(max_cols)) != cudaSuccess) break;
        }
    }
    for (int i = 0; i < R && e == cudaSuccess; ++i) {
        if ((e = dcol[i].ensure(sizeof(int64_t) * (max_cols + 1))) != cudaSuccess) break;
        if ((e = drow[i].ensure((size_t)si * (max_nnz + 1))) != cudaSuccess) break;
        if ((e = dval[i].ensure((size_t)sv * (max_nnz + 1))) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&ready[i], cudaEventDisableTiming)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&freed[i], cudaEventDisableTiming)) != cudaSuccess) break;
    }
    for (int i = 0; i < H && e == cudaSuccess; ++i) e = hslot[i].ensure(slot_bytes);
    if (e != cudaSuccess) {
        cleanup();
        set_error(std::string("run_batched: allocation failed: ") + cudaGetErrorString(e));
        return SPGEMM_ERR_OOM;
    }
    std::vector<cudaEvent_t> slot_evt(H, nullptr);
    for (int i = 0; i < H; ++i) cudaEventCreateWithFlags(&slot_evt[i], cudaEventDisableTiming);

    auto launch = [&](int64_t t) -> spgemm_status {
        const int i = (int)(t % R);
        const Batch &b = ps.batches[(size_t)t];
        if (t >= R) {
            cudaError_t ee = cudaStreamWaitEvent(compute, freed[i], 0);
            if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamWaitEvent");
        }
        spgemm_csc C{};
        C.nrows = ps.m; C.ncols = b.c1 - b.c0; C.nnz = b.nnz;
        C.colptr = dcol[i].p; C.rowidx = drow[i].p; C.vals = dval[i].p;
        C.ptr_type = SPGEMM_I64;
        C.idx_type = ps.idx64 ? SPGEMM_I64 : SPGEMM_I32;
        C.val_type = (spgemm_value_t)ps.vtype;
        spgemm_status s = ps.eng->numeric(ps, t, &C, compute);
        if (s != SPGEMM_OK) return s;
        if (prune) {
            const int64_t nc = b.c1 - b.c0;
            s = ps.eng->prune_batch(ps, nc, (const int64_t *)dcol[i].p, drow[i].p, dval[i].p,
                                    ps.ring_pcol[i].as<int64_t>(), ps.ring_prow[i].p, ps.ring_pval[i].p,
                                    ps.ring_pws[i], compute);
            if (s != SPGEMM_OK) return s;
            cudaError_t ce = cudaMemcpyAsync(ps.ring_hpc[i].p, ps.ring_pcol[i].p, sizeof(int64_t) * (size_t)(nc + 1),
                                             cudaMemcpyDeviceToHost, compute);
            if (ce != cudaSuccess) return cuda_fail(ce, "pruned colptr copy");
        }
        cudaError_t ee = cudaEventRecord(ready[i], compute);
        return ee == cudaSuccess ? SPGEMM_OK : cuda_fail(ee, "cudaEventRecord");
    };

    std::deque<Piece> inflight;
    int64_t piece_no = 0;
    spgemm_status status = SPGEMM_OK;
    bool stop = false;

    auto deliver = [&](Piece &p) -> spgemm_status {
        cudaError_t ee = cudaEventSynchronize(p.done);
        if (ee != cudaSuccess) return cuda_fail(ee, "cudaEventSynchronize");
        char *base = (char *)hslot[p.slot].p;
        int64_t *cp = (int64_t *)base;
        const int64_t nc = p.c1 - p.c0;
        const int64_t first = cp[0];
        for (int64_t j = 0; j <= nc; ++j) cp[j] -= first;   // relative to the piece
        spgemm_csc piece{};
        piece.nrows = ps.m; piece.ncols = nc; piece.nnz = p.nnz;
        piece.colptr = cp;
        const size_t cp_bytes = (size_t)((nc + 1) * 8 + 15) / 16 * 16;
        piece.rowidx = base + cp_bytes;
        piece.vals = base + cp_bytes + (size_t)(((p.nnz * si) + 15) / 16 * 16);
        piece.ptr_type = SPGEMM_I64;
        piece.idx_type = ps.idx64 ? SPGEMM_I64 : SPGEMM_I32;
        piece.val_type = (spgemm_value_t)ps.vtype;
        const int r = sink(ctx, p.batch, p.c0, p.c1, &piece);
        if (r != 0) {
            set_error("sink returned " + std::to_string(r));
            return SPGEMM_ERR_SINK;
        }
        return SPGEMM_OK;
    };

    if (nb > 0) status = launch(0);
    for (int64_t t = 0; t < nb && status == SPGEMM_OK && !stop; ++t) {
        if (t + 1 < nb) {
            status = launch(t + 1);
            if (status != SPGEMM_OK) break;
        }
        const int i = (int)(t % R);
        const Batch &b = ps.batches[(size_t)t];
        if ((e = cudaStreamWaitEvent(copy, ready[i], 0)) != cudaSuccess) { status = cuda_fail(e, "wait"); break; }
        // offsets of the batch's output (pruned: read back after the prune)
        const int64_t *pc = nullptr;
        if (prune) {
            if ((e = cudaEventSynchronize(ready[i])) != cudaSuccess) { status = cuda_fail(e, "prune wait"); break; }
            pc = ps.ring_hpc[i].as<int64_t>();
        }
        auto off = [&](int64_t col) { return prune ? pc[col - b.c0] : hc[col] - hc[b.c0]; };
        char *src_col = (char *)(prune ? ps.ring_pcol[i].p : dcol[i].p);
        char *src_row = (char *)(prune ? ps.ring_prow[i].p : drow[i].p);
        char *src_val = (char *)(prune ? ps.ring_pval[i].p : dval[i].p);
        int64_t c = b.c0;
        while (c < b.c1 && status == SPGEMM_OK) {
            // largest column range from c that fits one slot
            int64_t c1 = c + 1;
            auto bytes_of = [&](int64_t a, int64_t z) {
                const int64_t nnz = off(z) - off(a);
                return (size_t)((z - a + 1) * 8 + 15) / 16 * 16 + (size_t)(nnz * si + 15) / 16 * 16 +
                       (size_t)(nnz * sv);
            };
            int64_t lo = c + 1, hi = b.c1;
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo + 1) / 2;
                if (bytes_of(c, mid) <= slot_bytes) lo = mid; else hi = mid - 1;
            }
            c1 = lo;
            // a slot is free once its previous piece was delivered
            if ((int64_t)inflight.size() >= H) {
                status = deliver(inflight.front());
                inflight.pop_front();
                if (status != SPGEMM_OK) break;
            }
            const int slot = (int)(piece_no % H);
            const int64_t nnz = off(c1) - off(c);
            const int64_t o0 = off(c);
            char *hb = (char *)hslot[slot].p;
            const size_t cp_bytes = (size_t)((c1 - c + 1) * 8 + 15) / 16 * 16;
            const size_t ri_bytes = (size_t)(nnz * si + 15) / 16 * 16;
            e = cudaMemcpyAsync(hb, (int64_t *)src_col + (c - b.c0), (size_t)(c1 - c + 1) * 8,
                                cudaMemcpyDeviceToHost, copy);
            if (e == cudaSuccess && nnz)
                e = cudaMemcpyAsync(hb + cp_bytes, src_row + o0 * si, (size_t)(nnz * si),
                                    cudaMemcpyDeviceToHost, copy);
            if (e == cudaSuccess && nnz)
                e = cudaMemcpyAsync(hb + cp_bytes + ri_bytes, src_val + o0 * sv,
                                    (size_t)(nnz * sv), cudaMemcpyDeviceToHost, copy);
            if (e == cudaSuccess) e = cudaEventRecord(slot_evt[slot], copy);
            if (e != cudaSuccess) { status = cuda_fail(e, "D2H copy"); break; }
            inflight.push_back(Piece{t, c, c1, slot, slot_evt[slot], nnz});
            ++piece_no;
            c = c1;
        }
        if (status != SPGEMM_OK) break;
        if ((e = cudaEventRecord(freed[i], copy)) != cudaSuccess) { status = cuda_fail(e, "record"); break; }
    }
    while (!inflight.empty() && status == SPGEMM_OK) {
        status = deliver(inflight.front());
        inflight.pop_front();
    }
    // drain whatever is still in flight before the buffers go away
    cudaStreamSynchronize(compute);
    cudaStreamSynchronize(copy);
    int errw = 0;
    if (status == SPGEMM_OK) {
        e = cudaMemcpy(&errw, ps.err.p, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) status = cuda_fail(e, "error flag");
        else if (errw) {
            set_error("numeric: device error flags " + std::to_string(errw));
            status = SPGEMM_ERR_OVERFLOW;
        }
    }
    for (auto ev : slot_evt) if (ev) cudaEventDestroy(ev);
    cleanup();
    return status;
}
