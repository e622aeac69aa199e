// Engine instantiation for int32_t indices and OrAnd<double> values (Boolean or-and semiring).
#include "engine.cuh"

namespace spg {
EngineBase *make_engine_i32_oaf64() { return new Engine<int32_t, OrAnd<double>>(); }
}  // namespace spg
