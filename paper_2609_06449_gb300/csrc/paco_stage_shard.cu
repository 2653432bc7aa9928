// Stage kernels of the sharded form (paco_plan_create_sharded), complex64.
#include "paco_stage_launch.cuh"

namespace paco {
const void *stage_kernel_fn_shard_f32(int lgL, int minb) { return stage_kernel_fn_shard<float>(lgL, minb); }
} // namespace paco
