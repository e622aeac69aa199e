// Engine instantiation for int32_t indices and OrAnd<int64_t> values (Boolean or-and semiring).
#include "engine.cuh"

namespace spg {
EngineBase *make_engine_i32_oai64() { return new Engine<int32_t, OrAnd<int64_t>>(); }
}  // namespace spg
