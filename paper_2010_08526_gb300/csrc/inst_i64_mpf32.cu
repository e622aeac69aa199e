// Engine instantiation for int64_t indices and MinPlus<float> values (min-plus semiring).
#include "engine.cuh"

namespace spg {
EngineBase *make_engine_i64_mpf32() { return new Engine<int64_t, MinPlus<float>>(); }
}  // namespace spg
