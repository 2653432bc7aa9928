// paco_stage.cuh -- one PACO local-FFT stage as a CUDA kernel template.
//
// A stage computes a length-L DFT down every column of a row-major matrix
// (L rows, C columns), tile by tile:
//
//   mode 1  Phase I fused with the middle stage (Sect. 4.2): column DFTs of
//           the input view X[j1, j2] = x[j1*N2 + j2] (L = N1, C = N2), then
//           the top-level twiddle w_N^{-k1 c} (Eq. two-factor-ct; applied from
//           the logical coordinates, App. C.2 "application to twiddle
//           multiplication"), stored to W[pi_m2(c)][k1]: the full digit
//           reversal pi_m(a ++ c) = pi_m2(c) ++ pi_m1(a)
//           (Eq. full-middle-digit-reversal) resolved in the store address.
//   mode 2  Phase III (input-layout operator B_m2 = Omega P_pi, Lemma 1):
//           column v of W is read through the digit-reversed row map
//           j -> pi_m2(j) and its DFT is stored in natural order to
//           out[k2][v] (L = N2, C = N1).
//   mode 3  Phase I alone (A_m1 = P_pi Omega, Lemma 1): stored to
//           A-tilde[pi_m1(k1)][c], no twiddle (for the unfused pipeline).
//
// Inside a tile the length-L transform is split once, Cooley-Tukey style,
// as L = A*B with the balanced digit split of the paper's scheduler
// (A = 2^ceil(l/2), B = 2^floor(l/2); Sect. 4.1): j = j_hi*B + j_lo,
// k = k_lo + A*k_hi.
//
//   F1  A-point DFTs over j_hi for every (j_lo, column)  -> k_lo
//   tw  w_L^{-k_lo j_lo}  (the layout-aware twiddle, Eq. twop)
//   F2  B-point DFTs over j_lo for every (k_lo, column)  -> k_hi
//
// F1 and F2 each take one or two in-register radix passes (radix <= 16)
// with a shared-memory exchange between them.  A tile of W columns spans a
// thread-block cluster of K CTAs: CTA `rank` loads the j_lo range
// [rank*B/K, (rank+1)*B/K) and, after F1, sends each k_lo to the CTA that
// owns it (k_lo / (A/K)) through distributed shared memory -- the batch
// split of the paper's scheduler mapped onto the cluster.  Each thread holds
// EPT = min(16, L) elements.  Nothing is written to global memory except the
// stage output; no scratch.
#pragma once

#include <cooperative_groups.h>

#include "paco_common.cuh"
#include "paco_stage_args.cuh"
#include "paco_tc.cuh"

namespace paco {

namespace cg = cooperative_groups;

template <int X>
struct ilog2c { static constexpr int value = 1 + ilog2c<X / 2>::value; };
template <>
struct ilog2c<1> { static constexpr int value = 0; };

template <typename R>
__device__ __forceinline__ cx<R> ldg_cx(const cx<R> *p);
template <>
__device__ __forceinline__ cx<float> ldg_cx<float>(const cx<float> *p)
{
    float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return make_cx<float>(v.x, v.y);
}
template <>
__device__ __forceinline__ cx<double> ldg_cx<double>(const cx<double> *p)
{
    double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    return make_cx<double>(v.x, v.y);
}

template <typename R>
__device__ __forceinline__ cx<R> ldcg_cx(const cx<R> *p);
template <>
__device__ __forceinline__ cx<float> ldcg_cx<float>(const cx<float> *p)
{
    float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return make_cx<float>(v.x, v.y);
}
template <>
__device__ __forceinline__ cx<double> ldcg_cx<double>(const cx<double> *p)
{
    double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    return make_cx<double>(v.x, v.y);
}

template <typename R>
__device__ __forceinline__ void st_cx(cx<R> *p, cx<R> v) { *p = v; }

// Dynamic shared memory needed by a stage CTA (elements of cx<R>).
__host__ __device__ inline int stage_smem_elems(int A, int B, int K, int W, int pad)
{
    const int L = A * B;
    int lg = 0;
    while ((1 << lg) < L) ++lg;
    const int SL = 1 << ((lg + 1) / 2), SH = L / SL;
    const int Ak = A / K, Bk = B / K;
    const int P2 = B * W + pad;
    const int P1 = (K == 1) ? P2 : Bk * W;
    const int data = (A * P1 > Ak * P2) ? A * P1 : Ak * P2;
    return data + A + B + SL + SH + Ak * W + B * W;
}

// LGWC, LGKC, MC > 0 fix log2 W, log2 K and the mode at compile time (the
// hot configurations); 0 takes them from args at run time.  MINB is the
// minimum number of resident CTAs per SM requested from the compiler.
//
// stage_tile is the body: one tile (`tile`, transform base offset `boff`,
// cluster rank `rank`) computed by the calling CTA's NT = NE / EPT threads.
// LDCG loads the tile input through L2 only (ld.global.cg): for inputs that
// other CTAs of the same launch wrote (the batched persistent kernel).
// FORM != TC_NONE computes the radix-16 passes (F1 and F2 pass 1 when the
// radix is 16) as tensor-core contractions (paco_tc.cuh); its fragment table
// and per-warp staging follow the stage's shared memory.
// TERMS: the weighted-loss terms (StageTerms) are compiled in (1: all of
// them; 2: only the scalar factor on Phase I's loads).  SPLIT = 1: one pass of
// a split stage (SplitArgs).  SHARD: the
// sharded form's addresses (ShardArgs): Phase I on a local input slab with
// global twiddle columns, stored into the G send blocks; Phase III reading
// the received blocks; the output offset of the transform is boff_out.
template <typename R, int A, int B, int LGWC, int LGKC, int MC, bool LDCG, int FORM = TC_NONE, int TERMS = 0,
          bool SHARD = false, int SPLIT = 0>
__device__ __forceinline__ void stage_tile(const StageArgs &args, int tile, long long boff, int rank,
                                           unsigned char *smem_raw, const StageTerms *terms = nullptr,
                                           const ShardArgs *sh = nullptr, long long boff_out = 0,
                                           const SplitArgs *sp = nullptr)
{
    using C = cx<R>;
    constexpr int L = A * B;
    constexpr int EPT = L < 16 ? L : 16;          // elements per thread
    constexpr int RA1 = A >= 16 ? 16 : A;         // F1 radices
    constexpr int RA2 = A / RA1;
    constexpr int RB1 = B >= 16 ? 16 : B;         // F2 radices
    constexpr int RB2 = B / RB1;
    constexpr int LGL = ilog2c<L>::value;
    constexpr int LG_SL = (LGL + 1) / 2;
    constexpr int SL = 1 << LG_SL, SH = L / SL;
    static_assert(B >= 2, "B == 1 takes paco_stage_kernel_b1");
    static_assert(EPT % RA1 == 0 && EPT % RB1 == 0, "radix must divide EPT");
    static_assert(RA2 == 1 || EPT % RA2 == 0, "radix must divide EPT");
    static_assert(RB2 == 1 || EPT % RB2 == 0, "radix must divide EPT");

    const int lgW = (LGWC >= 0) ? LGWC : args.lgW;
    const int lgK = (LGKC >= 0) ? LGKC : args.lgK;
    const int W = 1 << lgW, K = 1 << lgK;
    const int Bk = B >> lgK, Ak = A >> lgK;
    const int S1 = Bk << lgW;                     // F1 sequences per CTA
    const int P2 = (B << lgW) + args.pad;         // F2 row stride
    const int P1 = (K == 1) ? P2 : S1;            // F1 row stride
    const int NT = blockDim.x;
    const int mode = MC ? MC : args.mode;

    C *sm = reinterpret_cast<C *>(smem_raw);
    const int data_elems = (A * P1 > Ak * P2) ? A * P1 : Ak * P2;
    C *twA = sm + data_elems;     // w_A^{-r}, r < A
    C *twB = twA + A;             // w_B^{-r}, r < B
    C *tlo = twB + B;             // w_L^{-r}, r < SL
    C *thi = tlo + SL;            // w_L^{-r*SL}, r < SH
    C *E1 = thi + SH;             // mode 1: w_N^{-k_lo c}     [W][Ak]
    C *E2 = E1 + Ak * W;          // mode 1: w_N^{-A k_hi c}   [B][W]
    const uint4 *tc_tab = nullptr;
    uint32_t *tc_ws = nullptr;
    if constexpr (FORM != TC_NONE) {
        static_assert(sizeof(R) == 4, "tensor-core forms are complex64");
        const int elems = data_elems + A + B + SL + SH + Ak * W + B * W;
        unsigned char *base = smem_raw + (((size_t)elems * sizeof(C) + 15) & ~(size_t)15);
        tc_tab = reinterpret_cast<const uint4 *>(base);
        tc_ws = reinterpret_cast<uint32_t *>(base + TcForm<FORM>::TABLE_U4 * 16) +
                (threadIdx.x >> 5) * TcForm<FORM>::WARP_WORDS;
        const uint4 *src = reinterpret_cast<const uint4 *>(args.tc);
        uint4 *dst = reinterpret_cast<uint4 *>(base);
        for (int r = threadIdx.x; r < TcForm<FORM>::TABLE_U4; r += blockDim.x) dst[r] = src[r];
    }

    const int tid = threadIdx.x;
    const int c0 = tile << lgW;
    const R csign = args.conj ? R(-1) : R(1);

    // ---- per-CTA twiddle tables (all forward, from FP64-generated tables)
    {
        const C *twL = reinterpret_cast<const C *>(args.twL);
        for (int r = tid; r < A; r += NT) twA[r] = ldg_cx(twL + r * B);
        for (int r = tid; r < B; r += NT) twB[r] = ldg_cx(twL + r * A);
        for (int r = tid; r < SL; r += NT) tlo[r] = ldg_cx(twL + r);
        for (int r = tid; r < SH; r += NT) thi[r] = ldg_cx(twL + r * SL);
        if constexpr (TERMS == 2) {
            // the scalar factor of Phase I's input, folded into the twiddle
            // every element takes after F1 (the DFT is linear): no per-element work
            if (mode == 1 && terms->ld_on) {
                const R f = R(terms->ld_mult) * (terms->ld_scale ? R(__ldg(terms->ld_scale)) : R(1));
                for (int r = tid; r < SH; r += NT) {
                    thi[r].x *= f;
                    thi[r].y *= f;
                }
            }
        }
        if constexpr (SPLIT != 0) {
            // one pass of a split stage: the tile's twiddles (its columns share j_b, or c)
            if (sp->sub == 1 || sp->sub == 3) {
                const C *twS = reinterpret_cast<const C *>(sp->twS);
                const int jb = c0 >> sp->lgC;
                for (int r = tid; r < (1 << sp->lgLa); r += NT) E1[r] = ldg_cx(twS + r * jb);   // w_L^{-k_a j_b}
            } else if (sp->sub == 2) {
                const C *nlo = reinterpret_cast<const C *>(args.twN_lo);
                const C *nhi = reinterpret_cast<const C *>(args.twN_hi);
                const unsigned lomask = (1u << args.twN_lo_bits) - 1u;
                const unsigned cw = (unsigned)(c0 >> sp->lgLa), ka0 = (unsigned)(c0 & ((1 << sp->lgLa) - 1));
                for (int e = tid; e < W; e += NT) {                                          // w_N^{-k_a c}
                    const unsigned r = ((ka0 + (unsigned)e) * cw) & args.N_mask;
                    E1[e] = cmul(ldg_cx(nlo + (r & lomask)), ldg_cx(nhi + (r >> args.twN_lo_bits)));
                }
                for (int e = tid; e < (1 << sp->lgLb); e += NT) {                             // w_N^{-La k_b c}
                    const unsigned r = (((unsigned)e << sp->lgLa) * cw) & args.N_mask;
                    E2[e] = cmul(ldg_cx(nlo + (r & lomask)), ldg_cx(nhi + (r >> args.twN_lo_bits)));
                }
            }
        }
        if (!SPLIT && mode == 1) {
            const C *nlo = reinterpret_cast<const C *>(args.twN_lo);
            const C *nhi = reinterpret_cast<const C *>(args.twN_hi);
            const unsigned lomask = (1u << args.twN_lo_bits) - 1u;
            const int nE1 = Ak << lgW, nE = nE1 + (B << lgW);
            for (int e = tid; e < nE; e += NT) {
                unsigned r;
                if (e < nE1) {
                    // E1 is [col][k_lo]: the epilogue reads it with k_lo fastest
                    const int lgAk = ilog2c<A>::value - lgK;
                    const unsigned klo = (unsigned)(rank * Ak + (e & (Ak - 1)));
                    unsigned c = (unsigned)(c0 + (e >> lgAk));
                    if constexpr (SHARD) c += (unsigned)sh->c_base;
                    r = (klo * c) & args.N_mask;
                } else {
                    const int e2 = e - nE1;
                    const unsigned khi = (unsigned)(e2 >> lgW);
                    unsigned c = (unsigned)(c0 + (e2 & (W - 1)));
                    if constexpr (SHARD) c += (unsigned)sh->c_base;
                    r = ((unsigned)A * khi * c) & args.N_mask;
                }
                E1[e] = cmul(ldg_cx(nlo + (r & lomask)), ldg_cx(nhi + (r >> args.twN_lo_bits)));
            }
        }
    }
    __syncthreads();

    C v[EPT];
    const C *gin = reinterpret_cast<const C *>(args.in) + boff;
    // weighted input (mode 1): one real factor per element
    bool ldw = false;
    R lds = R(1);
    if constexpr (TERMS == 1) {
        ldw = (mode == 1) && terms->ld_on;
        if (ldw) lds = R(terms->ld_mult) * (terms->ld_scale ? R(__ldg(terms->ld_scale)) : R(1));
    }

    // split pass A of Phase III: the tile's column block j_b lies in W's row block pi(j_b)
    [[maybe_unused]] long long cbase = 0;
    if constexpr (SPLIT != 0) {
        cbase = c0;
        if (sp->sub == 3)
            cbase = ((long long)digit_reverse((unsigned)(c0 >> sp->lgC), sp->lgLb, args.rev_t) << (sp->lgLa + sp->lgC)) +
                    (c0 & ((1 << sp->lgC) - 1));
    }

    // ---- F1 pass 1: radix RA1 over j_hi, span RA2; operands straight from HBM
    {
        constexpr int NB = EPT / RA1;
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int bfi = tid + NT * u;
            const int seq = bfi & (S1 - 1), jj = bfi / S1;
            const int jl = seq >> lgW, col = seq & (W - 1);
            const int jlo = rank * Bk + jl;
#pragma unroll
            for (int r = 0; r < RA1; ++r) {
                const int j = (jj + RA2 * r) * B + jlo;       // logical row in [L]
                unsigned row = (mode == 2) ? digit_reverse((unsigned)j, args.rev_bits, args.rev_t)
                                           : (unsigned)j;
                if constexpr (SHARD) {
                    // W row pi_m2(j), j = jh Cl + jl, is row pi(jl) of the block from rank jh
                    if (mode == 2)
                        row = (unsigned)((long long)(j >> sh->lgCl) * sh->bat_Cl) +
                              digit_reverse((unsigned)j & ((1u << sh->lgCl) - 1u), args.rev_bits, args.rev_t);
                }
                C x;
                if constexpr (SPLIT != 0) {
                    if (sp->sub != 3) row = (unsigned)j;               // natural rows (sub 3: pi over La's digits)
                    x = ldg_cx(gin + (long long)row * args.C + cbase + col);
                } else {
                    x = LDCG ? ldcg_cx(gin + (long long)row * args.C + c0 + col)
                             : ldg_cx(gin + (long long)row * args.C + c0 + col);
                }
                if constexpr (TERMS == 1) if (ldw) {
                    R f = lds;
                    if (terms->ld_w) f *= R(__ldg(terms->ld_w + boff + (long long)row * args.C + c0 + col));
                    x.x *= f;
                    x.y *= f;
                }
                x.y *= csign;
                v[u * RA1 + r] = x;
            }
            if constexpr (FORM != TC_NONE && RA1 == 16 && RA2 > 1) {
                // tensor-core contraction, twiddled and stored straight from the
                // accumulator fragments: lane n's sequence is bfi of lane n
                float acc[4][2][4];
                float sb;
                tc_contract<FORM>(v + u * RA1, tc_tab, tc_ws, acc, sb);
                const int lane = tid & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int n = 8 * nt + 2 * q + h;
                        const float sbn = (FORM == TC_FP16) ? __shfl_sync(0xffffffffu, sb, n) : 1.f;
                        const int bfn = (tid - lane) + n + NT * u;
                        const int seqn = bfn & (S1 - 1), jjn = bfn / S1;
#pragma unroll
                        for (int si = 0; si < 2; ++si) {
                            const int s = g + 8 * si;
                            C y = tc_frag_out(acc, nt, h, si, sbn);
                            if (s > 0) y = cmul(y, twA[s * jjn]);
                            sm[(jjn + RA2 * s) * P1 + seqn] = y;
                        }
                    }
                continue;
            }
            if constexpr (FORM != TC_NONE && RA1 == 16) tc_dft16<FORM>(v + u * RA1, tc_tab, tc_ws);
            else dft<RA1>(v + u * RA1);
            if constexpr (RA2 > 1) {
#pragma unroll
                for (int s = 1; s < RA1; ++s)
                    v[u * RA1 + s] = cmul(v[u * RA1 + s], twA[s * jj]);   // w_A^{-s jj}
#pragma unroll
                for (int s = 0; s < RA1; ++s)
                    sm[(jj + RA2 * s) * P1 + seq] = v[u * RA1 + s];
            }
        }
    }

    // ---- F1 pass 2 (if A > 16): radix RA2 over the span, groups g < 16.
    // After F1 the thread's element (u, k) has k_lo = kl_of(u, k).
    constexpr int RF = (RA2 > 1) ? RA2 : RA1;     // radix of F1's last pass
    constexpr int NBF = EPT / RF;
    if constexpr (RA2 > 1) {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NBF; ++u) {
            const int bfi = tid + NT * u;
            const int seq = bfi & (S1 - 1), g = bfi / S1;
#pragma unroll
            for (int r = 0; r < RA2; ++r) v[u * RA2 + r] = sm[(g * RA2 + r) * P1 + seq];
            dft<RA2>(v + u * RA2);
        }
    }

    // ---- twiddle w_L^{-k_lo j_lo}, then hand each k_lo to its owner
    if (K == 1) __syncthreads();                  // all F1 reads done before reuse
#pragma unroll
    for (int u = 0; u < NBF; ++u) {
        const int bfi = tid + NT * u;
        const int seq = bfi & (S1 - 1), hi = bfi / S1;   // hi = g (2 passes) or 0
        const int jl = seq >> lgW;
        const int jlo = rank * Bk + jl;
#pragma unroll
        for (int k = 0; k < RF; ++k) {
            const int klo = (RA2 > 1) ? (hi + RA1 * k) : k;
            const unsigned r = (unsigned)(klo * jlo);     // < L
            C t = cmul(tlo[r & (SL - 1)], thi[r >> LG_SL]);
            v[u * RF + k] = cmul(v[u * RF + k], t);
        }
    }
    if (K == 1) {
        // natural k_lo order in place of the F1 layout: sm[k_lo][j_lo][col]
#pragma unroll
        for (int u = 0; u < NBF; ++u) {
            const int bfi = tid + NT * u;
            const int seq = bfi & (S1 - 1), hi = bfi / S1;
#pragma unroll
            for (int k = 0; k < RF; ++k) {
                const int klo = (RA2 > 1) ? (hi + RA1 * k) : k;
                sm[klo * P2 + seq] = v[u * RF + k];
            }
        }
        __syncthreads();
    } else {
        cg::cluster_group cluster = cg::this_cluster();
        cluster.sync();                           // every CTA finished reading its F1 data
        const int lgAk = ilog2c<A>::value - lgK;
#pragma unroll
        for (int u = 0; u < NBF; ++u) {
            const int bfi = tid + NT * u;
            const int seq = bfi & (S1 - 1), hi = bfi / S1;
            const int jl = seq >> lgW, col = seq & (W - 1);
            const int jlo = rank * Bk + jl;
#pragma unroll
            for (int k = 0; k < RF; ++k) {
                const int klo = (RA2 > 1) ? (hi + RA1 * k) : k;
                const int dst = klo >> lgAk, al = klo & (Ak - 1);
                C *p = cluster.map_shared_rank(sm + al * P2 + (jlo << lgW) + col, dst);
                *p = v[u * RF + k];
            }
        }
        cluster.sync();                           // all of this CTA's F2 input has landed
    }

    // ---- F2 pass 1: radix RB1 over j_lo, span RB2
    constexpr int NB1 = EPT / RB1;
    C *gout = reinterpret_cast<C *>(args.out) + (SHARD ? boff_out : boff);
#pragma unroll
    for (int u = 0; u < NB1; ++u) {
        const int bfi = tid + NT * u;
        int col, jj, al;
        if (RB2 == 1 && mode == 1) {
            // single F2 pass in Phase I: k_lo fastest across threads, so the
            // stores below write runs of consecutive k1 of one W row (the row
            // pitch P2 is odd in mode 1: conflict-free shared-memory reads)
            al = bfi & (Ak - 1);
            col = (bfi >> (ilog2c<A>::value - lgK)) & (W - 1);
            jj = 0;
        } else {
            col = bfi & (W - 1);
            jj = (bfi >> lgW) % RB2;
            al = (bfi >> lgW) / RB2;
        }
#pragma unroll
        for (int r = 0; r < RB1; ++r) v[u * RB1 + r] = sm[al * P2 + ((jj + RB2 * r) << lgW) + col];
        if constexpr (FORM != TC_NONE && RB1 == 16 && RB2 > 1) {
            // as in F1: straight from the accumulator fragments (this pass uses
            // the col-fastest thread mapping whenever RB2 > 1)
            float acc[4][2][4];
            float sb;
            tc_contract<FORM>(v + u * RB1, tc_tab, tc_ws, acc, sb);
            const int lane = tid & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int n = 8 * nt + 2 * q + h;
                    const float sbn = (FORM == TC_FP16) ? __shfl_sync(0xffffffffu, sb, n) : 1.f;
                    const int bfn = (tid - lane) + n + NT * u;
                    const int coln = bfn & (W - 1);
                    const int jjn = (bfn >> lgW) % RB2;
                    const int aln = (bfn >> lgW) / RB2;
#pragma unroll
                    for (int si = 0; si < 2; ++si) {
                        const int s = g + 8 * si;
                        C y = tc_frag_out(acc, nt, h, si, sbn);
                        if (s > 0) y = cmul(y, twB[s * jjn]);
                        sm[aln * P2 + ((jjn + RB2 * s) << lgW) + coln] = y;
                    }
                }
            continue;
        }
        if constexpr (FORM != TC_NONE && RB1 == 16) tc_dft16<FORM>(v + u * RB1, tc_tab, tc_ws);
        else dft<RB1>(v + u * RB1);
        if constexpr (RB2 > 1) {
#pragma unroll
            for (int s = 1; s < RB1; ++s) v[u * RB1 + s] = cmul(v[u * RB1 + s], twB[s * jj]);
#pragma unroll
            for (int s = 0; s < RB1; ++s) sm[al * P2 + ((jj + RB2 * s) << lgW) + col] = v[u * RB1 + s];
        }
    }

    // ---- F2 pass 2 (if B > 16) and the store
    constexpr int RL = (RB2 > 1) ? RB2 : RB1;    // radix of the last pass
    constexpr int NBL = EPT / RL;
    bool stw = false;                             // weighted power of the output
    if constexpr (TERMS == 1) stw = (mode == 2) && terms->st_w != nullptr;
    R wpow = R(0);
    if constexpr (RB2 > 1) __syncthreads();
#pragma unroll
    for (int u = 0; u < NBL; ++u) {
        const int bfi = tid + NT * u;
        int al, col, hi;
        if constexpr (RB2 > 1) {
            if (mode == 1) {
                al = bfi & (Ak - 1);
                col = (bfi / Ak) & (W - 1);
                hi = bfi / (Ak << lgW);
            } else {
                col = bfi & (W - 1);
                al = (bfi >> lgW) & (Ak - 1);
                hi = (bfi >> lgW) / Ak;
            }
#pragma unroll
            for (int r = 0; r < RB2; ++r) v[u * RB2 + r] = sm[al * P2 + ((hi * RB2 + r) << lgW) + col];
            dft<RB2>(v + u * RB2);
        } else {
            // single F2 pass: the registers already hold the outputs of
            // butterfly (col, jj = 0, al), mapped as in F2 pass 1
            if (mode == 1) {
                al = bfi & (Ak - 1);
                col = (bfi >> (ilog2c<A>::value - lgK)) & (W - 1);
            } else {
                col = bfi & (W - 1);
                al = bfi >> lgW;
            }
            hi = 0;
        }
        const int klo = rank * Ak + al;
        const int c = c0 + col;
        float wv[TERMS == 1 ? RL : 1];                // the loss weights of this thread's outputs, loaded first
        if constexpr (TERMS == 1) if (stw) {
#pragma unroll
            for (int k = 0; k < RL; ++k) {
                const int khi = (RB2 > 1) ? (hi + RB1 * k) : k;
                wv[k] = __ldg(terms->st_w + boff + (long long)(klo + A * khi) * args.out_ld + c);
            }
        }
#pragma unroll
        for (int k = 0; k < RL; ++k) {
            const int khi = (RB2 > 1) ? (hi + RB1 * k) : k;
            const int kk = klo + A * khi;             // natural frequency in [L]
            C y = v[u * RL + k];
            long long idx;
            if constexpr (SPLIT != 0) {
                const int cc = c0 + col;                      // the pass's view column
                const int mC = (1 << sp->lgC) - 1;
                if (sp->sub == 1) {                           // S[j_b][c][k_a], view column j_b C + c
                    y = cmul(y, E1[kk]);
                    idx = ((long long)cc << sp->lgLa) + kk;
                } else if (sp->sub == 2) {                    // W[pi_m2(c)][k_a + La k_b], view column c La + k_a
                    y = cmul(y, cmul(E1[col], E2[kk]));
                    const unsigned cw = (unsigned)(cc >> sp->lgLa);
                    idx = (long long)digit_reverse(cw, sp->rev_bits_c, args.rev_t) * args.out_ld +
                          (cc & ((1 << sp->lgLa) - 1)) + ((long long)kk << sp->lgLa);
                } else if (sp->sub == 3) {                    // S[j_b][k_a][v], view column j_b C + v
                    y = cmul(y, E1[kk]);
                    idx = ((((long long)(c0 >> sp->lgC) << sp->lgLa) + kk) << sp->lgC) + (cc & mC);
                } else {                                      // y[k_a + La k_b][v], view column k_a C + v
                    idx = (long long)((cc >> sp->lgC) + (kk << sp->lgLa)) * args.out_ld + (cc & mC);
                }
            } else if (mode == 1) {
                y = cmul(y, cmul(E1[(col << (ilog2c<A>::value - lgK)) + al], E2[(khi << lgW) + col]));
                const unsigned urow = digit_reverse((unsigned)c, args.rev_bits, args.rev_t);
                if constexpr (SHARD) {
                    // block for the rank that owns k1 = kk, row pi(c) of the local columns
                    idx = (long long)(kk >> sh->lgK1) * sh->bat_blk + ((long long)urow << sh->lgK1) +
                          (kk & ((1 << sh->lgK1) - 1));
                } else {
                    idx = (long long)urow * args.out_ld + kk;
                }
            } else if (mode == 2) {
                idx = (long long)kk * args.out_ld + c;
                if constexpr (TERMS == 1) if (stw) {
                    wpow += R(wv[k]) * (y.x * y.x + y.y * y.y);
                    if (terms->st_weighted) {
                        y.x *= R(wv[k]);
                        y.y *= R(wv[k]);
                    }
                }
            } else {
                const unsigned arow = digit_reverse((unsigned)kk, args.rev_bits, args.rev_t);
                idx = (long long)arow * args.out_ld + c;
            }
            y.y *= csign;
            st_cx(gout + idx, y);
        }
    }
    if constexpr (TERMS == 1) if (stw) {
        if (NT & 31) {
            atomicAdd(terms->st_loss, (double)wpow);         // tiny tiles: one atomic per thread
        } else {
            // warp sums in the (now unused) tile buffer, then one FP64 atomic per CTA
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wpow += __shfl_xor_sync(0xffffffffu, wpow, o);
            double *wsum = reinterpret_cast<double *>(smem_raw);
            __syncthreads();                                  // every read of the tile is done
            if ((tid & 31) == 0) wsum[tid >> 5] = (double)wpow;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int i = 0; i < NT / 32; ++i) t += wsum[i];
                atomicAdd(terms->st_loss, t);
            }
        }
    }
}

template <typename R, int A, int B, int LGWC = -1, int LGKC = -1, int MC = 0, int MINB = 1, int FORM = TC_NONE>
__global__ void __launch_bounds__(512, MINB) paco_stage_kernel(const StageArgs args)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lgK = (LGKC >= 0) ? LGKC : args.lgK;
    int rank = 0;
    if ((1 << lgK) > 1) rank = (int)cg::this_cluster().block_rank();
    stage_tile<R, A, B, LGWC, LGKC, MC, false, FORM>(args, (int)(blockIdx.x >> lgK),
                                                     (long long)blockIdx.y * args.batch_stride, rank, smem_raw);
}

// The generic stage in the sharded form's addresses (ShardArgs): blockIdx.y =
// transform b; its input is at b * in_stride, its output at b * out_stride.
template <typename R, int A, int B, int MINB>
__global__ void __launch_bounds__(512, MINB) paco_stage_kernel_shard(const StageArgs args, const ShardArgs sh,
                                                                    long long in_stride, long long out_stride)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int rank = 0;
    if ((1 << args.lgK) > 1) rank = (int)cg::this_cluster().block_rank();
    stage_tile<R, A, B, -1, -1, 0, false, TC_NONE, 0, true>(
        args, (int)(blockIdx.x >> args.lgK), (long long)blockIdx.y * in_stride, rank, smem_raw, nullptr, &sh,
        (long long)blockIdx.y * out_stride);
}

// One pass of a split stage (SplitArgs); tiles of one CTA (no cluster).
template <typename R, int A, int B, int MINB>
__global__ void __launch_bounds__(512, MINB) paco_stage_kernel_split(const StageArgs args, const SplitArgs sp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    stage_tile<R, A, B, -1, 0, 0, false, TC_NONE, 0, false, 1>(
        args, (int)blockIdx.x, (long long)blockIdx.y * args.batch_stride, 0, smem_raw, nullptr, nullptr, 0, &sp);
}

// The generic stage with the element-wise terms of a weighted power loss
// (StageTerms) compiled in -- TM = 1 all of them, TM = 2 the scalar factor on
// Phase I's loads alone; paco_stage_kernel carries none of their code.
template <typename R, int A, int B, int MINB, int TM = 1>
__global__ void __launch_bounds__(512, MINB) paco_stage_kernel_terms(const StageArgs args, const StageTerms terms)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int rank = 0;
    if ((1 << args.lgK) > 1) rank = (int)cg::this_cluster().block_rank();
    stage_tile<R, A, B, -1, -1, 0, false, TC_NONE, TM>(args, (int)(blockIdx.x >> args.lgK),
                                                         (long long)blockIdx.y * args.batch_stride, rank, smem_raw,
                                                         &terms);
}

// L = A (B == 1): the whole transform is F1; store straight from F1's layout.
// Only tiny sizes take this path (L = 2).
template <typename R, int A>
__global__ void __launch_bounds__(512) paco_stage_kernel_b1(const StageArgs args)
{
    using C = cx<R>;
    static_assert(A <= 16, "single-factor path is for tiny transforms");
    constexpr int EPT = A;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    (void)smem_raw;
    const int lgW = args.lgW;
    const int W = 1 << lgW;
    const int NT = blockDim.x;
    const int tile = blockIdx.x;
    const long long boff = (long long)blockIdx.y * args.batch_stride;
    const int c0 = tile << lgW;
    const R csign = args.conj ? R(-1) : R(1);
    const C *gin = reinterpret_cast<const C *>(args.in) + boff;
    C *gout = reinterpret_cast<C *>(args.out) + boff;
    const int tid = threadIdx.x;
    if (tid >= W) return;
    (void)NT;
    const int col = tid, c = c0 + col;
    C v[EPT];
#pragma unroll
    for (int r = 0; r < A; ++r) {
        const unsigned row = (args.mode == 2) ? digit_reverse((unsigned)r, args.rev_bits, args.rev_t)
                                              : (unsigned)r;
        C x = ldg_cx(gin + (long long)row * args.C + c);
        x.y *= csign;
        v[r] = x;
    }
    dft<A>(v);
    const C *nlo = reinterpret_cast<const C *>(args.twN_lo);
    const C *nhi = reinterpret_cast<const C *>(args.twN_hi);
#pragma unroll
    for (int k = 0; k < A; ++k) {
        C y = v[k];
        long long idx;
        if (args.mode == 1) {
            const unsigned r = ((unsigned)k * (unsigned)c) & args.N_mask;
            y = cmul(y, cmul(ldg_cx(nlo + (r & ((1u << args.twN_lo_bits) - 1u))),
                             ldg_cx(nhi + (r >> args.twN_lo_bits))));
            const unsigned urow = digit_reverse((unsigned)c, args.rev_bits, args.rev_t);
            idx = (long long)urow * args.out_ld + k;
        } else if (args.mode == 2) {
            idx = (long long)k * args.out_ld + c;
        } else {
            const unsigned arow = digit_reverse((unsigned)k, args.rev_bits, args.rev_t);
            idx = (long long)arow * args.out_ld + c;
        }
        y.y *= csign;
        st_cx(gout + idx, y);
    }
}

} // namespace paco
