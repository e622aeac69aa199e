// Engine instantiation for int64_t indices and OrAnd<int64_t> values (Boolean or-and semiring).
#include "engine.cuh"

namespace spg {
EngineBase *make_engine_i64_oai64() { return new Engine<int64_t, OrAnd<int64_t>>(); }
}  // namespace spg
