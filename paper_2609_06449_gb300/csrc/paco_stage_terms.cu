// Stage kernels for complex64 with the weighted-loss terms compiled in
// (paco_execute_weighted_power / paco_execute_weighted_input).
#include "paco_stage_launch.cuh"

namespace paco {
const void *stage_kernel_fn_terms_f32(int lgL, int minb) { return stage_kernel_fn<float, true>(lgL, minb); }
} // namespace paco
