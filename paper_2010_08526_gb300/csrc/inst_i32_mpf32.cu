// Engine instantiation for int32_t indices and MinPlus<float> values (min-plus semiring).
#include "engine.cuh"

namespace spg {
EngineBase *make_engine_i32_mpf32() { return new Engine<int32_t, MinPlus<float>>(); }
}  // namespace spg
