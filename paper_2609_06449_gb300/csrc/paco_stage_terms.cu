// Stage kernels for complex64 with the weighted-loss terms compiled in
// (paco_execute_weighted_power / paco_execute_weighted_input): all terms, or
// the scalar factor on Phase I's loads alone.
#include "paco_stage_launch.cuh"

namespace paco {
const void *stage_kernel_fn_terms_f32(int lgL, int minb) { return stage_kernel_fn<float, 1>(lgL, minb); }
const void *stage_kernel_fn_scale_f32(int lgL, int minb) { return stage_kernel_fn<float, 2>(lgL, minb); }
} // namespace paco
