// Engine instantiation for int32_t indices and MinPlus<double> values (min-plus semiring).
#include "engine.cuh"

namespace spg {
EngineBase *make_engine_i32_mpf64() { return new Engine<int32_t, MinPlus<double>>(); }
}  // namespace spg
