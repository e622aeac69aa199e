// Engine instantiation for int64_t indices and OrAnd<float> values (Boolean or-and semiring).
#include "engine.cuh"

namespace spg {
EngineBase *make_engine_i64_oaf32() { return new Engine<int64_t, OrAnd<float>>(); }
}  // namespace spg
