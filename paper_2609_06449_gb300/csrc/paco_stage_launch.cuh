// paco_stage_launch.cuh -- instantiation and launch of the stage kernels for
// one real type (included once per type by paco_stage_f32.cu / _f64.cu).
#pragma once

#include "paco_stage.cuh"

namespace paco {

// lgL -> (A, B) = (2^ceil(lgL/2), 2^floor(lgL/2)), the balanced split.
template <typename R, int LGL>
struct StageKernel {
    static constexpr int A = 1 << ((LGL + 1) / 2);
    static constexpr int B = 1 << (LGL / 2);
    static const void *fn()
    {
        if constexpr (B == 1) return reinterpret_cast<const void *>(&paco_stage_kernel_b1<R, A>);
        else return reinterpret_cast<const void *>(&paco_stage_kernel<R, A, B>);
    }
};

template <typename R>
const void *stage_kernel_fn(int lgL)
{
    switch (lgL) {
    case 1: return StageKernel<R, 1>::fn();
    case 2: return StageKernel<R, 2>::fn();
    case 3: return StageKernel<R, 3>::fn();
    case 4: return StageKernel<R, 4>::fn();
    case 5: return StageKernel<R, 5>::fn();
    case 6: return StageKernel<R, 6>::fn();
    case 7: return StageKernel<R, 7>::fn();
    case 8: return StageKernel<R, 8>::fn();
    case 9: return StageKernel<R, 9>::fn();
    case 10: return StageKernel<R, 10>::fn();
    case 11: return StageKernel<R, 11>::fn();
    case 12: return StageKernel<R, 12>::fn();
    case 13: return StageKernel<R, 13>::fn();
    case 14: return StageKernel<R, 14>::fn();
    default: return nullptr;
    }
}

// Specialised kernels for the hot configurations: (A, B, log2 W, log2 K,
// mode).  Returns nullptr when there is none.
template <typename R>
const void *stage_kernel_fn_special(int lgL, int lgW, int lgK, int mode)
{
    if constexpr (sizeof(R) == 4) {
        if (lgL == 14 && lgW == 2 && lgK == 3) {
            if (mode == 1) return reinterpret_cast<const void *>(&paco_stage_kernel<R, 128, 128, 2, 3, 1, 2>);
            if (mode == 2) return reinterpret_cast<const void *>(&paco_stage_kernel<R, 128, 128, 2, 3, 2, 2>);
        }
    }
    return nullptr;
}

} // namespace paco
