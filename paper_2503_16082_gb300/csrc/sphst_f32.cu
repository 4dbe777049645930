// FP32 instantiation of the engine: pair arithmetic in FP32, positions as
// FP32 offsets from their cell origin, time-step control in FP64.
#include "sphst_engine_impl.cuh"

namespace sphst {
Engine *new_engine_f32() { return new EngineT<float>(); }
}  // namespace sphst
