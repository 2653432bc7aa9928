// Stage kernels for complex64 (FP32 arithmetic).
#include "paco_stage_launch.cuh"

namespace paco {
const void *stage_kernel_fn_f32(int lgL, int minb) { return stage_kernel_fn<float>(lgL, minb); }
const void *stage_kernel_fn_special_f32(int lgL, int lgW, int lgK, int mode)
{
    return stage_kernel_fn_special<float>(lgL, lgW, lgK, mode);
}
} // namespace paco
