// FP64 instantiation of the engine.
#include "sphst_engine_impl.cuh"

namespace sphst {
Engine *new_engine_f64() { return new EngineT<double>(); }
}  // namespace sphst
