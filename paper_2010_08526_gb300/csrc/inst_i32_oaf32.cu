// Engine instantiation for int32_t indices and OrAnd<float> values (Boolean or-and semiring).
#include "engine.cuh"

namespace spg {
EngineBase *make_engine_i32_oaf32() { return new Engine<int32_t, OrAnd<float>>(); }
}  // namespace spg
