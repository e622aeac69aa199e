// Engine instantiation for int64_t indices and double values.
#include "engine.cuh"

namespace spg {
EngineBase *make_engine_i64_f64() { return new Engine<int64_t, double>(); }
spgemm_status merge_i64_f64(const spgemm_csc *p, int np, spgemm_csc *o, cudaStream_t st) {
    return Engine<int64_t, double>::merge(p, np, o, st);
}
spgemm_status multi_create_i64_f64(MultiState &ms, const spgemm_csc *A, const spgemm_csc *B,
                                     cudaStream_t st) {
    return Engine<int64_t, double>::multi_create(ms, A, B, st);
}
spgemm_status merge_noalloc_i64_f64(const spgemm_csc *p, int np, spgemm_csc *o, cudaStream_t st,
                                     unsigned char *scratch, size_t cap, int32_t *stage, int nsm) {
    return Engine<int64_t, double>::merge_noalloc(p, np, o, st, scratch, cap, stage, nsm);
}
spgemm_status prune_i64_f64(const spgemm_csc *in, double thr, int64_t k, spgemm_csc *out, cudaStream_t st) {
    return Engine<int64_t, double>::prune(in, thr, k, out, st);
}
}  // namespace spg
