// Engine instantiation for int32_t indices and int64_t values.
#include "engine.cuh"

namespace spg {
EngineBase *make_engine_i32_i64v() { return new Engine<int32_t, int64_t>(); }
spgemm_status merge_i32_i64v(const spgemm_csc *p, int np, spgemm_csc *o, cudaStream_t st) {
    return Engine<int32_t, int64_t>::merge(p, np, o, st);
}
spgemm_status multi_create_i32_i64v(MultiState &ms, const spgemm_csc *A, const spgemm_csc *B,
                                     cudaStream_t st) {
    return Engine<int32_t, int64_t>::multi_create(ms, A, B, st);
}
spgemm_status merge_noalloc_i32_i64v(const spgemm_csc *p, int np, spgemm_csc *o, cudaStream_t st,
                                     unsigned char *scratch, size_t cap, int32_t *stage, int nsm) {
    return Engine<int32_t, int64_t>::merge_noalloc(p, np, o, st, scratch, cap, stage, nsm);
}
spgemm_status prune_i32_i64v(const spgemm_csc *in, double thr, int64_t k, spgemm_csc *out, cudaStream_t st) {
    return Engine<int32_t, int64_t>::prune(in, thr, k, out, st);
}
}  // namespace spg
