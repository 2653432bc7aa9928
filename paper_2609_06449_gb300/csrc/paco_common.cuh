// paco_common.cuh -- device building blocks of the PACO stage kernels.
//
// Complex arithmetic on interleaved (re, im) pairs, the constant-size
// natural-order DFT leaves (radix 2, 4, 8, 16) that the paper's scheduler
// invokes at its base case ("constant-size natural-order DFT kernels",
// Fig. "cofft" in App. B), and the base-b digit reversal pi_ell of Sect. 3.2.
//
// Every DFT here is the forward one, y_s = sum_r v_r w_R^{-s r}; the inverse
// direction is obtained by conjugating on load and store.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace paco {

template <typename R>
struct cx {
    R x, y;
};

template <typename R>
__device__ __forceinline__ cx<R> make_cx(R a, R b) { cx<R> c; c.x = a; c.y = b; return c; }
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return make_cx<R>(a.x + b.x, a.y + b.y); }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return make_cx<R>(a.x - b.x, a.y - b.y); }
// complex product a*b
template <typename R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b)
{
    return make_cx<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// multiply by -i
template <typename R>
__device__ __forceinline__ cx<R> mul_mi(cx<R> a) { return make_cx<R>(a.y, -a.x); }

// Constants cos(pi/8), sin(pi/8), sqrt(1/2) to full double precision.
#define PACO_C8 0.92387953251128675612818318939678829
#define PACO_S8 0.38268343236508977172845998403039887
#define PACO_RH 0.70710678118654752440084436210484904

// multiply by w_8^{-1} = (1 - i)/sqrt(2)
template <typename R>
__device__ __forceinline__ cx<R> mul_w8_1(cx<R> a)
{
    const R h = R(PACO_RH);
    return make_cx<R>((a.x + a.y) * h, (a.y - a.x) * h);
}
// multiply by w_8^{-3} = (-1 - i)/sqrt(2)
template <typename R>
__device__ __forceinline__ cx<R> mul_w8_3(cx<R> a)
{
    const R h = R(PACO_RH);
    return make_cx<R>((a.y - a.x) * h, -(a.x + a.y) * h);
}
// multiply by the constant (c, s)
template <typename R>
__device__ __forceinline__ cx<R> mul_const(cx<R> a, R c, R s)
{
    return make_cx<R>(a.x * c - a.y * s, a.x * s + a.y * c);
}

// ---- natural-order DFT leaves, in place on v[0..R) ------------------------

template <typename R>
__device__ __forceinline__ void dft2(cx<R> *v)
{
    cx<R> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
}

template <typename R>
__device__ __forceinline__ void dft4_s(cx<R> &v0, cx<R> &v1, cx<R> &v2, cx<R> &v3)
{
    cx<R> t0 = v0 + v2, t1 = v0 - v2;
    cx<R> t2 = v1 + v3, t3 = mul_mi(v1 - v3);
    v0 = t0 + t2;
    v2 = t0 - t2;
    v1 = t1 + t3;
    v3 = t1 - t3;
}

template <typename R>
__device__ __forceinline__ void dft4(cx<R> *v) { dft4_s(v[0], v[1], v[2], v[3]); }

template <typename R>
__device__ __forceinline__ void dft8(cx<R> *v)
{
    // even / odd halves, then the w_8 combine
    cx<R> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    cx<R> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4_s(e0, e1, e2, e3);
    dft4_s(o0, o1, o2, o3);
    o1 = mul_w8_1(o1);
    o2 = mul_mi(o2);
    o3 = mul_w8_3(o3);
    v[0] = e0 + o0; v[4] = e0 - o0;
    v[1] = e1 + o1; v[5] = e1 - o1;
    v[2] = e2 + o2; v[6] = e2 - o2;
    v[3] = e3 + o3; v[7] = e3 - o3;
}

template <typename R>
__device__ __forceinline__ void dft16(cx<R> *v)
{
    // 4 x 4: column DFTs over j1 (stride 4), twiddle w_16^{-s0 j0}, row DFTs.
    dft4_s(v[0], v[4], v[8], v[12]);
    dft4_s(v[1], v[5], v[9], v[13]);
    dft4_s(v[2], v[6], v[10], v[14]);
    dft4_s(v[3], v[7], v[11], v[15]);
    const R c = R(PACO_C8), s = R(PACO_S8);
    // j0 = 1: s0 = 1, 2, 3 -> w^{-1}, w^{-2}, w^{-3}
    v[5] = mul_const(v[5], c, -s);
    v[9] = mul_w8_1(v[9]);
    v[13] = mul_const(v[13], s, -c);
    // j0 = 2: w^{-2}, w^{-4}, w^{-6}
    v[6] = mul_w8_1(v[6]);
    v[10] = mul_mi(v[10]);
    v[14] = mul_w8_3(v[14]);
    // j0 = 3: w^{-3}, w^{-6}, w^{-9}
    v[7] = mul_const(v[7], s, -c);
    v[11] = mul_w8_3(v[11]);
    v[15] = mul_const(v[15], -c, s);
    // row DFTs over j0 for each s0; output index s0 + 4*s1 sits at v[4*s0 + s1]
    dft4_s(v[0], v[1], v[2], v[3]);
    dft4_s(v[4], v[5], v[6], v[7]);
    dft4_s(v[8], v[9], v[10], v[11]);
    dft4_s(v[12], v[13], v[14], v[15]);
    // transpose the 4 x 4 index (s0, s1) -> natural order y[s0 + 4*s1]
    cx<R> t;
    t = v[1]; v[1] = v[4]; v[4] = t;
    t = v[2]; v[2] = v[8]; v[8] = t;
    t = v[3]; v[3] = v[12]; v[12] = t;
    t = v[6]; v[6] = v[9]; v[9] = t;
    t = v[7]; v[7] = v[13]; v[13] = t;
    t = v[11]; v[11] = v[14]; v[14] = t;
}

template <int RADIX, typename R>
__device__ __forceinline__ void dft(cx<R> *v)
{
    if constexpr (RADIX == 2) dft2(v);
    else if constexpr (RADIX == 4) dft4(v);
    else if constexpr (RADIX == 8) dft8(v);
    else if constexpr (RADIX == 16) dft16(v);
}

// ---- base-b digit reversal pi_ell (Sect. 3.2; App. A.1) -------------------
// u has ell digits of t bits (b = 2^t); bits = ell * t in [1, 31].  A full
// bit reversal reverses the digit order and the bits inside every digit; the
// per-digit fix-up restores the bit order inside each digit.
__device__ __forceinline__ uint32_t digit_reverse(uint32_t u, int bits, int t)
{
    uint32_t x = __brev(u) >> (32 - bits);
    switch (t) {
    case 2:
        x = ((x & 0x55555555u) << 1) | ((x >> 1) & 0x55555555u);
        break;
    case 3:
        x = (x & 0x12492492u) | ((x & 0x09249249u) << 2) | ((x >> 2) & 0x09249249u);
        break;
    case 4:
        x = ((x & 0x11111111u) << 3) | ((x & 0x22222222u) << 1) |
            ((x >> 1) & 0x22222222u) | ((x >> 3) & 0x11111111u);
        break;
    default:
        break;
    }
    return x;
}

// Arguments of one stage launch (see paco_stage.cuh).
struct StageArgs {
    const void *in;
    void *out;
    long long batch_stride; // N elements per transform
    int C;                  // row length (columns) of the input matrix view
    int out_ld;             // row length of the output matrix view
    int lgW, lgK;           // log2 tile width, log2 cluster size
    int mode;               // 1 fused stage 1, 2 stage 2, 3 Phase I alone
    int rev_bits, rev_t;    // digit reversal: ell*t bits, t bits per digit
    const void *twL;        // w_L^{-r}, r in [L]
    const void *twN_lo;     // w_N^{-r}, r in [2^twN_lo_bits]
    const void *twN_hi;     // w_N^{-(r << twN_lo_bits)}
    int twN_lo_bits;
    unsigned N_mask;        // N - 1
    int conj;               // 1: conjugate on load and store (dir = +1)
    int pad;                // shared-memory row padding (elements)
    const void *tc;         // tensor-core forms: fragment table (paco_tc.cuh)
};

} // namespace paco
