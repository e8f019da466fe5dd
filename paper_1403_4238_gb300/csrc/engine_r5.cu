// Persistent engine, fast update and priority-init kernels for patch radius 5
// (one translation unit per radius so that the instantiations build in parallel).
#include "engine_impl.cuh"

namespace inp {
const EngineFns* engine_fns_r5() { return engine_fns_for<5>(); }
}  // namespace inp
