// Stage kernels for complex128 (FP64 arithmetic).
#include "paco_stage_launch.cuh"

namespace paco {
const void *stage_kernel_fn_f64(int lgL, int minb) { return stage_kernel_fn<double>(lgL, minb); }
const void *stage_kernel_fn_special_f64(int lgL, int lgW, int lgK, int mode)
{
    return stage_kernel_fn_special<double>(lgL, lgW, lgK, mode);
}
} // namespace paco
