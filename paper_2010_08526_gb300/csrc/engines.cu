// Dispatch on (index, value) type: one engine instantiation per pair.
#include "plan.h"

namespace spg {

#define SPG_DECL(I, V)                                                                      \
    EngineBase *make_engine_##I##_##V();                                                    \
    spgemm_status merge_##I##_##V(const spgemm_csc *, int, spgemm_csc *, cudaStream_t);     \
    spgemm_status multi_create_##I##_##V(MultiState &, const spgemm_csc *, const spgemm_csc *, \
                                         cudaStream_t);
#define SPG_DECL2(I, V)                                                                     \
    spgemm_status merge_noalloc_##I##_##V(const spgemm_csc *, int, spgemm_csc *, cudaStream_t,   \
                                          unsigned char *, size_t, int32_t *, int);             \
    spgemm_status prune_##I##_##V(const spgemm_csc *, double, int64_t, spgemm_csc *, cudaStream_t);
SPG_DECL2(i32, f64) SPG_DECL2(i32, f32) SPG_DECL2(i32, i64v)
SPG_DECL2(i64, f64) SPG_DECL2(i64, f32) SPG_DECL2(i64, i64v)
SPG_DECL(i32, f64) SPG_DECL(i32, f32) SPG_DECL(i32, i64v)
SPG_DECL(i64, f64) SPG_DECL(i64, f32) SPG_DECL(i64, i64v)

#define SPG_SWITCH(idx64, vtype, CALL)                                 \
    if (!(idx64)) {                                                    \
        if ((vtype) == SPGEMM_F64) return CALL(i32, f64);              \
        if ((vtype) == SPGEMM_F32) return CALL(i32, f32);              \
        if ((vtype) == SPGEMM_INT64) return CALL(i32, i64v);           \
    } else {                                                           \
        if ((vtype) == SPGEMM_F64) return CALL(i64, f64);              \
        if ((vtype) == SPGEMM_F32) return CALL(i64, f32);              \
        if ((vtype) == SPGEMM_INT64) return CALL(i64, i64v);           \
    }

EngineBase *make_engine_i32_mpf32();
EngineBase *make_engine_i32_mpf64();
EngineBase *make_engine_i64_mpf32();
EngineBase *make_engine_i64_mpf64();
EngineBase *make_engine_i32_oaf32();
EngineBase *make_engine_i32_oaf64();
EngineBase *make_engine_i32_oai64();
EngineBase *make_engine_i64_oaf32();
EngineBase *make_engine_i64_oaf64();
EngineBase *make_engine_i64_oai64();

EngineBase *make_engine(int idx64, int vtype, int semiring) {
    if (semiring == SPGEMM_MIN_PLUS) {   // float values only (checked at plan time)
        if (vtype == SPGEMM_F32) return idx64 ? make_engine_i64_mpf32() : make_engine_i32_mpf32();
        if (vtype == SPGEMM_F64) return idx64 ? make_engine_i64_mpf64() : make_engine_i32_mpf64();
        return nullptr;
    }
    if (semiring == SPGEMM_OR_AND) {     // any value type
        if (vtype == SPGEMM_F32) return idx64 ? make_engine_i64_oaf32() : make_engine_i32_oaf32();
        if (vtype == SPGEMM_F64) return idx64 ? make_engine_i64_oaf64() : make_engine_i32_oaf64();
        if (vtype == SPGEMM_INT64) return idx64 ? make_engine_i64_oai64() : make_engine_i32_oai64();
        return nullptr;
    }
#define MK(I, V) make_engine_##I##_##V()
    SPG_SWITCH(idx64, vtype, MK)
#undef MK
    return nullptr;
}

spgemm_status merge_dispatch(const spgemm_csc *parts, int nparts, spgemm_csc *out, cudaStream_t st) {
    const int idx64 = parts[0].idx_type == SPGEMM_I64;
    const int vtype = parts[0].val_type;
#define MG(I, V) merge_##I##_##V(parts, nparts, out, st)
    SPG_SWITCH(idx64, vtype, MG)
#undef MG
    set_error("unsupported type combination");
    return SPGEMM_ERR_INVALID;
}

spgemm_status prune_dispatch(const spgemm_csc *in, double thr, int64_t topk, spgemm_csc *out,
                             cudaStream_t st) {
    const int idx64 = in->idx_type == SPGEMM_I64;
    const int vtype = in->val_type;
#define PR(I, V) prune_##I##_##V(in, thr, topk, out, st)
    SPG_SWITCH(idx64, vtype, PR)
#undef PR
    set_error("unsupported type combination");
    return SPGEMM_ERR_INVALID;
}

spgemm_status merge_noalloc_dispatch(const spgemm_csc *parts, int nparts, spgemm_csc *out,
                                     cudaStream_t st, unsigned char *scratch, size_t cap,
                                     int32_t *stage, int nsm) {
    const int idx64 = parts[0].idx_type == SPGEMM_I64;
    const int vtype = parts[0].val_type;
#define MN(I, V) merge_noalloc_##I##_##V(parts, nparts, out, st, scratch, cap, stage, nsm)
    SPG_SWITCH(idx64, vtype, MN)
#undef MN
    set_error("unsupported type combination");
    return SPGEMM_ERR_INVALID;
}

spgemm_status multi_create_typed(MultiState &ms, const spgemm_csc *As, const spgemm_csc *Bs,
                                 cudaStream_t st) {
#define MC(I, V) multi_create_##I##_##V(ms, As, Bs, st)
    SPG_SWITCH(ms.idx64, ms.vtype, MC)
#undef MC
    set_error("unsupported type combination");
    return SPGEMM_ERR_INVALID;
}

}  // namespace spg
