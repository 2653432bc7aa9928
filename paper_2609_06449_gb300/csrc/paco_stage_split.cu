// Stage kernels for the passes of a split stage (complex64, lengths 2^5..2^8).
#include "paco_stage_launch.cuh"

namespace paco {
const void *stage_kernel_fn_split_f32(int lgL, int minb) { return stage_kernel_fn_split<float>(lgL, minb); }
} // namespace paco
