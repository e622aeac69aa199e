// Engine instantiation for int64_t indices and OrAnd<double> values (Boolean or-and semiring).
#include "engine.cuh"

namespace spg {
EngineBase *make_engine_i64_oaf64() { return new Engine<int64_t, OrAnd<double>>(); }
}  // namespace spg
