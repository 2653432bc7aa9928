// paco_stage_launch.cuh -- instantiation and launch of the stage kernels for
// one real type (included once per type by paco_stage_f32.cu / _f64.cu).
#pragma once

#include "paco_stage.cuh"

namespace paco {

// lgL -> (A, B) = (2^ceil(lgL/2), 2^floor(lgL/2)), the balanced split.
template <typename R, int LGL, int TERMS>
struct StageKernel {
    static constexpr int A = 1 << ((LGL + 1) / 2);
    static constexpr int B = 1 << (LGL / 2);
    // minb: resident CTAs per SM the kernel is compiled for (2 caps the
    // registers at 64 per thread; complex64 only)
    static const void *fn(int minb)
    {
        if constexpr (B == 1) return TERMS ? nullptr : reinterpret_cast<const void *>(&paco_stage_kernel_b1<R, A>);
        else if constexpr (TERMS != 0) {
            if (minb == 2) return reinterpret_cast<const void *>(&paco_stage_kernel_terms<R, A, B, 2, TERMS>);
            return reinterpret_cast<const void *>(&paco_stage_kernel_terms<R, A, B, 1, TERMS>);
        } else if constexpr (sizeof(R) == 4) {
            if (minb == 2) return reinterpret_cast<const void *>(&paco_stage_kernel<R, A, B, -1, -1, 0, 2>);
            return reinterpret_cast<const void *>(&paco_stage_kernel<R, A, B>);
        } else return reinterpret_cast<const void *>(&paco_stage_kernel<R, A, B>);
    }
};

// The sharded-form stage kernel for length 2^lgL.
template <typename R>
const void *stage_kernel_fn_shard(int lgL, int minb)
{
#define PACO_SHARD_CASE(LG)                                                                          \
    case LG: {                                                                                       \
        constexpr int A_ = 1 << (((LG) + 1) / 2), B_ = 1 << ((LG) / 2);                              \
        if (minb == 2 && sizeof(R) == 4)                                                             \
            return reinterpret_cast<const void *>(&paco_stage_kernel_shard<R, A_, B_, 2>);           \
        return reinterpret_cast<const void *>(&paco_stage_kernel_shard<R, A_, B_, 1>);               \
    }
    switch (lgL) {
        PACO_SHARD_CASE(2) PACO_SHARD_CASE(3) PACO_SHARD_CASE(4) PACO_SHARD_CASE(5) PACO_SHARD_CASE(6)
        PACO_SHARD_CASE(7) PACO_SHARD_CASE(8) PACO_SHARD_CASE(9) PACO_SHARD_CASE(10) PACO_SHARD_CASE(11)
        PACO_SHARD_CASE(12) PACO_SHARD_CASE(13) PACO_SHARD_CASE(14)
    default: return nullptr;
    }
#undef PACO_SHARD_CASE
}

// One pass of a split stage, length 2^lgL (complex64, 2^5..2^8).
template <typename R>
const void *stage_kernel_fn_split(int lgL, int minb)
{
#define PACO_SPLIT_CASE(LG)                                                                          \
    case LG: {                                                                                       \
        constexpr int A_ = 1 << (((LG) + 1) / 2), B_ = 1 << ((LG) / 2);                              \
        if (minb == 2) return reinterpret_cast<const void *>(&paco_stage_kernel_split<R, A_, B_, 2>); \
        return reinterpret_cast<const void *>(&paco_stage_kernel_split<R, A_, B_, 1>);               \
    }
    switch (lgL) {
        PACO_SPLIT_CASE(5) PACO_SPLIT_CASE(6) PACO_SPLIT_CASE(7) PACO_SPLIT_CASE(8)
    default: return nullptr;
    }
#undef PACO_SPLIT_CASE
}

// The generic stage kernel for length 2^lgL; TERMS = 1: the variant with the
// weighted-loss terms (StageTerms) compiled in, 2: with the scalar factor on
// Phase I's loads alone.
template <typename R, int TERMS = 0>
const void *stage_kernel_fn(int lgL, int minb)
{
    switch (lgL) {
    case 1: return StageKernel<R, 1, TERMS>::fn(minb);
    case 2: return StageKernel<R, 2, TERMS>::fn(minb);
    case 3: return StageKernel<R, 3, TERMS>::fn(minb);
    case 4: return StageKernel<R, 4, TERMS>::fn(minb);
    case 5: return StageKernel<R, 5, TERMS>::fn(minb);
    case 6: return StageKernel<R, 6, TERMS>::fn(minb);
    case 7: return StageKernel<R, 7, TERMS>::fn(minb);
    case 8: return StageKernel<R, 8, TERMS>::fn(minb);
    case 9: return StageKernel<R, 9, TERMS>::fn(minb);
    case 10: return StageKernel<R, 10, TERMS>::fn(minb);
    case 11: return StageKernel<R, 11, TERMS>::fn(minb);
    case 12: return StageKernel<R, 12, TERMS>::fn(minb);
    case 13: return StageKernel<R, 13, TERMS>::fn(minb);
    case 14: return StageKernel<R, 14, TERMS>::fn(minb);
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
