// paco_stage_args.cuh -- launch arguments of the stage kernels' variants
// (sharded form, split passes, weighted-loss terms), beside StageArgs.
#pragma once

namespace paco {

// The sharded form (paco_plan_create_sharded): rank `rank` of G holds input
// columns [rank Cl, (rank+1) Cl) of X (Cl = N2/G) and output columns
// [rank K1, (rank+1) K1) of Y (K1 = N1/G); blocks of N/G^2 items travel
// between ranks, buffers laid out [G][batch][Cl][K1] (block for / from rank g).
struct ShardArgs {
    long long c_base;       // rank * Cl: global column of local column 0 (Phase I twiddle)
    int lgCl, lgK1;         // log2 Cl, log2 K1
    long long bat_blk;      // batch * Cl * K1: stride between the blocks of two ranks
    long long bat_Cl;       // batch * Cl: the same in rows of K1 items
};

// A stage of length L = La Lb split into two passes through global memory
// (the local FFT's top split taken out of the CTA: pass A = La-point DFTs
// with the twiddle w_L^{-k_a j_b}, pass B = Lb-point DFTs with the stage's
// epilogue), scratch S holding the intermediate.  sub: 1 Phase I pass A
// (x -> S[j_b][c][k_a]), 2 Phase I pass B (S -> W[pi_m2(c)][k_a + La k_b]
// with w_N^{-k1 c}), 3 Phase III pass A (W rows pi_m2(j) -> S[j_b][k_a][v]),
// 4 Phase III pass B (S -> y[k_a + La k_b][v]).
struct SplitArgs {
    int sub;
    int lgC;                // log2 of the stage's column count
    int lgLa, lgLb;
    int rev_bits_c;         // sub 2: pi_m2 over log2 N2 bits
    const void *twS;        // w_L^{-r}, r < L (sub 1, 3)
};

// Element-wise terms of a weighted power loss, taken by the stage kernels
// built with them (paco_stage_kernel_terms); nullptr switches a term off.
struct StageTerms {
    const float *ld_w;      // mode 1: element n of the input is read as
    const double *ld_scale; //   ld_mult * (*ld_scale or 1) * (ld_w[n] or 1) * in[n]
    float ld_mult;
    int ld_on;              //   (1: that factor is applied)
    const float *st_w;      // mode 2: *st_loss += sum over n of st_w[n] |out[n]|^2,
    double *st_loss;
    int st_weighted;        //   and (1) out[n] = st_w[n] * y[n] is stored in place of y[n]
};

} // namespace paco
