// Engine instantiation for int64_t indices and MinPlus<double> values (min-plus semiring).
#include "engine.cuh"

namespace spg {
EngineBase *make_engine_i64_mpf64() { return new Engine<int64_t, MinPlus<double>>(); }
}  // namespace spg
