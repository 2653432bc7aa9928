// Stage kernels of the tensor-core precision forms (complex64 data, radix-16
// sub-DFTs as mma.sync contractions; see paco_tc.cuh).  Lengths 2^8..2^14,
// where both factors of the in-tile split have a radix-16 pass.
#include "paco_plan.h"
#include "paco_stage.cuh"

namespace paco {

// Element (m, kk) of the real 32 x 32 matrix M, from FP64 sincospi.
static __device__ double tc_matrix_entry(int m, int kk)
{
    const int k = m & 15, j = kk & 15;
    double s, c;
    sincospi(2.0 * (double)((k * j) & 15) / 16.0, &s, &c);     // w_16^{-kj} = c - i s
    const bool re_out = m < 16, re_in = kk < 16;
    if (re_out && re_in) return c;          // Fr
    if (re_out && !re_in) return s;         // -Fi = s
    if (!re_out && re_in) return -s;        // Fi = -s
    return c;                               // Fr
}

// Fragment table: for term ta, m-tile mt, K half ks and lane, the four
// 32-bit registers a0..a3 of the m16n8k16 A operand (row-major 16 x 16):
// reg r holds rows g + 8*(r & 1), columns 2*q + 8*(r >> 1) + {0, 1}, with
// g = lane / 4, q = lane % 4 (lower column in the low half).
static __global__ void tc_table_kernel(int form, uint4 *out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int TA = (form == TC_BF16X3) ? 3 : 2;
    if (idx >= TA * 2 * 2 * 32) return;
    const int lane = idx & 31, ks = (idx >> 5) & 1, mt = (idx >> 6) & 1, ta = idx >> 7;
    const int g = lane >> 2, q = lane & 3;
    uint32_t reg[4];
    for (int r = 0; r < 4; ++r) {
        uint32_t packed = 0;
        for (int h = 0; h < 2; ++h) {
            const int m = 16 * mt + g + 8 * (r & 1);
            const int kk = 16 * ks + 2 * q + 8 * (r >> 1) + h;
            const float v = (float)tc_matrix_entry(m, kk);
            uint16_t bits;
            if (form == TC_BF16X3) {
                float rem = v;
                __nv_bfloat16 t = __float2bfloat16_rn(rem);
                for (int i = 0; i < ta; ++i) {
                    rem -= __bfloat162float(t);
                    t = __float2bfloat16_rn(rem);
                }
                bits = __bfloat16_as_ushort(t);
            } else {
                __half t = __float2half_rn(v);
                if (ta == 1) t = __float2half_rn(v - __half2float(t));
                bits = __half_as_ushort(t);
            }
            packed |= (uint32_t)bits << (16 * h);
        }
        reg[r] = packed;
    }
    out[idx] = make_uint4(reg[0], reg[1], reg[2], reg[3]);
}


template <int LGL, int FORM>
static const void *tc_fn()
{
    constexpr int A = 1 << ((LGL + 1) / 2), B = 1 << (LGL / 2);
    return reinterpret_cast<const void *>(&paco_stage_kernel<float, A, B, -1, -1, 0, 1, FORM>);
}

template <int FORM>
static const void *tc_fn_len(int lgL)
{
    switch (lgL) {
    case 8: return tc_fn<8, FORM>();
    case 9: return tc_fn<9, FORM>();
    case 10: return tc_fn<10, FORM>();
    case 11: return tc_fn<11, FORM>();
    case 12: return tc_fn<12, FORM>();
    case 13: return tc_fn<13, FORM>();
    case 14: return tc_fn<14, FORM>();
    default: return nullptr;
    }
}

const void *stage_kernel_fn_tc(int lgL, int form)
{
    if (form == TC_BF16X3) return tc_fn_len<TC_BF16X3>(lgL);
    if (form == TC_FP16) return tc_fn_len<TC_FP16>(lgL);
    return nullptr;
}

paco_status_t tc_table_create(int form, void **out)
{
    const int n = (form == TC_BF16X3) ? TcForm<TC_BF16X3>::TABLE_U4 : TcForm<TC_FP16>::TABLE_U4;
    PACO_CUDA_TRY(cudaMalloc(out, (size_t)n * sizeof(uint4)));
    tc_table_kernel<<<(n + 127) / 128, 128>>>(form, reinterpret_cast<uint4 *>(*out));
    PACO_CUDA_TRY(cudaGetLastError());
    return PACO_OK;
}

} // namespace paco
