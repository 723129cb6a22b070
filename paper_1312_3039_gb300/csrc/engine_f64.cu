// FP64 instantiation of the device solver (every vector and A in double).
#include "engine.cuh"

namespace scs {
EngineBase *make_engine_f64(const HostProblem &P, const scs_settings &st) { return new Engine<double>(P, st); }
}  // namespace scs
