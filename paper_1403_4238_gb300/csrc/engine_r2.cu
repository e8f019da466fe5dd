// Persistent engine body, fast update and priority-init kernels for patch
// radius 2 (one translation unit per radius so that they build in parallel).
#include "engine_impl.cuh"

namespace inp {
__device__ void run_image_r2_s1(const EngineArgs& ea, int j, EngCtx& x) { run_image<2, 1>(ea, j, x); }
__device__ void run_image_r2_s2(const EngineArgs& ea, int j, EngCtx& x) { run_image<2, 2>(ea, j, x); }
const EngineFns* engine_fns_r2() { return engine_fns_for<2>(); }
}  // namespace inp
