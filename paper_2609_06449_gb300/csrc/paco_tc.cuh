// paco_tc.cuh -- radix-16 sub-DFTs as tensor-core contractions.
//
// The paper's leaves are exact constant-size DFTs (App. B, base case of the
// scheduler); here the 16-point leaf of a local FFT pass can instead be a
// dense contraction on the tensor cores.  A warp transforms the 32
// sequences its lanes hold (one 16-point sequence per lane) at once:
//
//     [Re y; Im y] (32 x 32) = M (32 x 32) * [Re x; Im x] (32 x 32),
//     M = [[Fr, -Fi], [Fi, Fr]],  F[k][j] = w_16^{-kj},
//
// column n being lane n's sequence.  mma.sync m16n8k16 with FP32
// accumulation computes it as 2 (rows of M) x 2 (K halves: Re, Im) x 4
// (groups of 8 sequences) tiles.  The contraction is register-to-register:
// its operands come from the FFT's registers through a small per-warp
// staging area, and the result goes back into the same registers, so the
// local-FFT pass around it is unchanged.
//
// Precision forms:
//   TC_BF16X3  x and M are each split into three bfloat16 terms
//              (v = v0 + v1 + v2, each the bf16 rounding of what remains);
//              the six products Mi*xj with i + j <= 2 recover ~24 bits,
//              i.e. FP32-level accuracy.
//   TC_FP16    one FP16 product; each sequence is scaled by a power of two
//              so that its largest component lies in [1, 2) before the
//              conversion and unscaled after (per-block scaling); M is
//              split into two FP16 terms (M0 + M1), so the error is that of
//              rounding x to 11 bits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "paco_common.cuh"

namespace paco {

enum { TC_NONE = 0, TC_BF16X3 = 1, TC_FP16 = 2 };

template <int FORM>
struct TcForm {
    static constexpr int TA = (FORM == TC_BF16X3) ? 3 : 2;   // terms of M
    static constexpr int TB = (FORM == TC_BF16X3) ? 3 : 1;   // terms of x
    // per-warp staging: operand terms [TB][plane][32 lanes][8 words], reused
    // for the FP32 result [32 lanes][33]
    static constexpr int IN_WORDS = TB * 2 * 32 * 8;
    static constexpr int OUT_WORDS = 32 * 33;
    static constexpr int WARP_WORDS = IN_WORDS > OUT_WORDS ? IN_WORDS : OUT_WORDS;
    static constexpr int TABLE_U4 = TA * 2 * 2 * 32;         // A fragments per term/m-tile/k-half/lane
};

// Extra dynamic shared memory of a TC stage CTA with `warps` warps (bytes).
__host__ __device__ inline int tc_smem_bytes(int form, int warps)
{
    if (form == TC_BF16X3)
        return TcForm<TC_BF16X3>::TABLE_U4 * 16 + warps * TcForm<TC_BF16X3>::WARP_WORDS * 4;
    if (form == TC_FP16)
        return TcForm<TC_FP16>::TABLE_U4 * 16 + warps * TcForm<TC_FP16>::WARP_WORDS * 4;
    return 0;
}

__device__ __forceinline__ void mma_bf16(float *d, const uint4 &a, uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_f16(float *d, const uint4 &a, uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&p);
}

__device__ __forceinline__ uint32_t pack_f16(float lo, float hi)
{
    __half2 p = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&p);
}

// Warp-collective contraction: v[0..16) of every lane (its 16-point
// sequence) -> the accumulator fragments of [Re y; Im y] for the warp's 32
// sequences: acc[nt][mt][i] is row m = 16 mt + g + 8 (i >> 1) (m < 16: Re of
// frequency m, else Im of m - 16) and column n = 8 nt + 2 q + (i & 1) (lane n's
// sequence), g = lane / 4, q = lane % 4.  scale_back: this lane's sequence
// scale (FP16 form; 1 otherwise).  All 32 lanes must call it together; ws is
// free again when it returns.
template <int FORM>
__device__ __forceinline__ void tc_contract(const cx<float> *v, const uint4 *tab, uint32_t *ws,
                                            float (&acc)[4][2][4], float &scale_back)
{
    using T = TcForm<FORM>;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, q = lane & 3;
    // ---- operand terms of this lane's sequence, row `lane` of each plane;
    //      words 0..3 and 4..7 swap on rows with bit 2 set (conflict-free reads)
    scale_back = 1.f;
    {
        const int sw = ((lane >> 2) & 1) << 2;
        if constexpr (FORM == TC_BF16X3) {
            float rem[32];
#pragma unroll
            for (int k = 0; k < 16; ++k) { rem[k] = v[k].x; rem[16 + k] = v[k].y; }
#pragma unroll
            for (int t = 0; t < 3; ++t) {
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    uint32_t w[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float a = rem[16 * p + 2 * i], b = rem[16 * p + 2 * i + 1];
                        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                        w[i] = *reinterpret_cast<const uint32_t *>(&h);
                        const float2 hf = __bfloat1622float2(h);
                        rem[16 * p + 2 * i] = a - hf.x;
                        rem[16 * p + 2 * i + 1] = b - hf.y;
                    }
                    uint4 *row = reinterpret_cast<uint4 *>(ws + ((t * 2 + p) * 32 + lane) * 8);
                    row[sw >> 2] = make_uint4(w[0], w[1], w[2], w[3]);
                    row[(sw >> 2) ^ 1] = make_uint4(w[4], w[5], w[6], w[7]);
                }
            }
        } else {
            float mx = 0.f;
#pragma unroll
            for (int k = 0; k < 16; ++k) mx = fmaxf(mx, fmaxf(fabsf(v[k].x), fabsf(v[k].y)));
            int e = (int)((__float_as_uint(mx) >> 23) & 0xff) - 127;   // mx in [2^e, 2^(e+1))
            if (e < -100) e = -100;
            if (e > 100) e = 100;
            const float s = __uint_as_float((uint32_t)(127 - e) << 23);
            scale_back = __uint_as_float((uint32_t)(127 + e) << 23);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                uint32_t w[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float a = p ? v[2 * i].y : v[2 * i].x;
                    const float b = p ? v[2 * i + 1].y : v[2 * i + 1].x;
                    w[i] = pack_f16(a * s, b * s);
                }
                uint4 *row = reinterpret_cast<uint4 *>(ws + (p * 32 + lane) * 8);
                row[sw >> 2] = make_uint4(w[0], w[1], w[2], w[3]);
                row[(sw >> 2) ^ 1] = make_uint4(w[4], w[5], w[6], w[7]);
            }
        }
    }
    __syncwarp();
    // ---- contraction: tile (mt, nt) of [Re y; Im y].  The matrix fragments
    //      of one (mt, K half) are loaded once and used for all four groups of
    //      eight sequences (the operand fragments, 4-byte reads, are re-read).
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) acc[nt][mt][0] = acc[nt][mt][1] = acc[nt][mt][2] = acc[nt][mt][3] = 0.f;
    const int rsw = ((g >> 2) & 1) << 2;        // swap of the source row n = 8 nt + g
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            uint4 af[T::TA];
#pragma unroll
            for (int ta = 0; ta < T::TA; ++ta) af[ta] = tab[((ta * 2 + mt) * 2 + ks) * 32 + lane];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                uint32_t bq[T::TB][2];
#pragma unroll
                for (int tb = 0; tb < T::TB; ++tb) {
                    const uint32_t *row = ws + ((tb * 2 + ks) * 32 + 8 * nt + g) * 8;
                    bq[tb][0] = row[q ^ rsw];           // k = 2q, 2q+1
                    bq[tb][1] = row[(q + 4) ^ rsw];     // k = 2q+8, 2q+9
                }
                float *d = acc[nt][mt];
                if constexpr (FORM == TC_BF16X3) {
                    // smallest products first
                    mma_bf16(d, af[2], bq[0][0], bq[0][1]);
                    mma_bf16(d, af[1], bq[1][0], bq[1][1]);
                    mma_bf16(d, af[0], bq[2][0], bq[2][1]);
                    mma_bf16(d, af[1], bq[0][0], bq[0][1]);
                    mma_bf16(d, af[0], bq[1][0], bq[1][1]);
                    mma_bf16(d, af[0], bq[0][0], bq[0][1]);
                } else {
                    mma_f16(d, af[1], bq[0][0], bq[0][1]);
                    mma_f16(d, af[0], bq[0][0], bq[0][1]);
                }
            }
        }
    }
    __syncwarp();                               // every operand read: ws is free
}

// Warp-collective: v[0..16) of every lane -> its natural-order 16-point DFT
// (the contraction, then the result transposed back through ws).
template <int FORM>
__device__ __forceinline__ void tc_dft16(cx<float> *v, const uint4 *tab, uint32_t *ws)
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, q = lane & 3;
    float acc[4][2][4];
    float scale_back;
    tc_contract<FORM>(v, tab, ws, acc, scale_back);
    // ---- result [n][m] (row stride 33), then each lane takes its row
    float *o = reinterpret_cast<float *>(ws);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int n = 8 * nt + 2 * q, m = 16 * mt + g;
            o[n * 33 + m] = acc[nt][mt][0];
            o[(n + 1) * 33 + m] = acc[nt][mt][1];
            o[n * 33 + m + 8] = acc[nt][mt][2];
            o[(n + 1) * 33 + m + 8] = acc[nt][mt][3];
        }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        v[k].x = o[lane * 33 + k] * scale_back;
        v[k].y = o[lane * 33 + 16 + k] * scale_back;
    }
    __syncwarp();                               // staging free for the next call
}

// Output (frequency s = g + 8 si, sequence n = 8 nt + 2 q + h) of the
// fragments of tc_contract, unscaled by that sequence's factor.
__device__ __forceinline__ cx<float> tc_frag_out(const float (&acc)[4][2][4], int nt, int h, int si, float sb)
{
    return make_cx<float>(acc[nt][0][h + 2 * si] * sb, acc[nt][1][h + 2 * si] * sb);
}

} // namespace paco
