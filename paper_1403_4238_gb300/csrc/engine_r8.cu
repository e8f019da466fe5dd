// Persistent engine body, fast update and priority-init kernels for patch
// radius 8 (one translation unit per radius so that they build in parallel).
#include "engine_impl.cuh"

namespace inp {
__device__ void run_image_r8_s1(const EngineArgs& ea, int j, EngCtx& x) { run_image<8, 1>(ea, j, x); }
__device__ void run_image_r8_s2(const EngineArgs& ea, int j, EngCtx& x) { run_image<8, 2>(ea, j, x); }
const EngineFns* engine_fns_r8() { return engine_fns_for<8>(); }
}  // namespace inp
