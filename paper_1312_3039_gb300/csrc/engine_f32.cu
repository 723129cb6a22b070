// Mixed-precision instantiation: A, the CG vectors and the sparse products in
// FP32; iterates u, v, the cached M^-1 h, the scaling, the termination tests
// (with an FP64 copy of A) and all reductions in FP64.
#include "engine.cuh"

namespace scs {
EngineBase *make_engine_f32(const HostProblem &P, const scs_settings &st) { return new Engine<float>(P, st); }
}  // namespace scs
