// paco_batched.cu -- many complex64 transforms of uneven power-of-two
// lengths in one persistent launch (paco_plan_create_batched).
//
// Every transform of length N = N1 * N2 follows the same three steps as the
// single-length plan: Phase I local FFTs down the N2 columns, the top-level
// twiddle w_N^{-k1 c} with the fused digit reversal (a, c) -> (pi_m2(c), k1)
// into W (Eq. 17), and Phase III local FFTs down W's columns read through
// pi_m2, stored as natural-order y (Lemma 1, Theorem 3).  The uneven batch is
// the batch-field recursion of the paper's scheduler taken to the machine:
// one queue of equal-sized work items (8192 elements each), claimed in order
// by a persistent grid.
//
//   small item  (N <= 2^13): G = 8192 / N whole transforms in one CTA.  Both
//               local FFTs run in shared memory; the redistribution is an
//               index map inside the CTA (self pairs only), so the transform
//               costs one HBM read and one HBM write per element.
//   stage item  (N >= 2^14): one tile of Phase I (mode 1) or Phase III
//               (mode 2) of one transform, the stage_tile body of the
//               single-length kernels with a tile of L x (8192 / L).  A
//               Phase III tile waits (bounded) on the transform's counter of
//               finished Phase I tiles.  Items are ordered so that a
//               transform's Phase III comes a fixed lag after its Phase I,
//               long enough to avoid waiting and short enough for W to stay
//               in L2 between the two (at best 16 B of HBM traffic per
//               element instead of 32).
//
// The plan's autotuner picks, per length, the N1 x N2 split and the radix b,
// and for the whole batch the kernel variant (one or two CTAs per SM) and the
// lag, by timing candidates at plan creation; it optimises time, so part of
// the L2 residency can be traded for faster tiles.
//
// Deadlock freedom: only Phase III items wait, and only on Phase I items of
// a lower queue index; those were claimed by running CTAs and never wait, so
// every wait ends without any assumption on how many CTAs are co-resident.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "paco_common.cuh"
#include "paco_plan.h"
#include "paco_stage.cuh"

namespace paco {

namespace batched {
constexpr int NT = 512;            // threads per CTA
constexpr int ITEM = 8192;         // elements per work item
constexpr int SMALL_MAX_LG = 13;   // whole-transform items up to 2^13
constexpr int STAGE_MIN_LG = 6;    // stage lengths built: 2^6 .. 2^10
constexpr int STAGE_MAX_LG = 10;
} // namespace batched

// One length class.
struct BLen {
    int lgN, lg1, lg2, t;          // N = 2^lgN = N1 * N2, N1 = 2^lg1, b = 2^t
    int small;                     // 1: whole-transform items
    int G;                         // small: transforms per item
    int ntiles1, ntiles2;          // stage items per transform
    const void *twN;               // small: w_N^{-r}, r < N
    StageArgs s1, s2;              // stage: mode 1 and mode 2 (in/out/conj set per item)
};

struct __align__(16) BItem {
    int kind;                      // 0 small group, 1 Phase I tile, 2 Phase III tile
    int len;                       // index into the length table
    int a;                         // kind 0: first entry of group_tx; else transform index
    int b;                         // kind 0: transforms in the group; else tile index
    long long off;                 // stage tiles: element offset of the transform
    long long pad;
};

struct BatchedArgs {
    const BItem *items;
    int nitems;
    const long long *off;          // element offset of every transform
    const BLen *lens;
    const int *group_tx;           // transforms of the small groups, grouped by length
    const void *in;
    void *out;
    unsigned *ctr;                 // [0] queue head, [1 + i] Phase I tiles done of transform i
    int *status;
    unsigned spin_limit;
    unsigned wait_bias;            // added to the Phase III wait target (0; tests of the bounded waits)
    int conj;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ---- whole transforms in shared memory ------------------------------------
// S holds G transforms (natural order) of N elements.  W of transform g is
// stored at S + g*N as rows of N1 with the columns XOR-swizzled by
// h(row) = pi_m2(row) mod min(N1, 32) (conflict-free Phase I stores and
// Phase III loads; any per-row bijection of the columns is a valid layout).
template <int LG1, int LG2>
__device__ __forceinline__ void small_group(const BatchedArgs &a, const BLen &ld, int gstart, int gcount,
                                            cx<float> *S, long long *s_off)
{
    using C = cx<float>;
    constexpr int N1 = 1 << LG1, N2 = 1 << LG2, LGN = LG1 + LG2, N = 1 << LGN;
    constexpr int G = batched::ITEM / N;
    constexpr int R1 = N1 < 16 ? N1 : 16, R2 = N1 / R1;        // Phase I radices
    constexpr int Q1 = N2 < 16 ? N2 : 16, Q2 = N2 / Q1;        // Phase III radices
    constexpr int LR1 = ilog2c<R1>::value, LR2 = ilog2c<R2>::value;
    constexpr int LQ1 = ilog2c<Q1>::value, LQ2 = ilog2c<Q2>::value;
    constexpr int HM = (N1 < 32 ? N1 : 32) - 1;                 // swizzle mask
    const int tid = threadIdx.x;
    const int t = ld.t;
    const bool cj = a.conj != 0;
    // w_N^{-r} = lo[r mod 2^LH] * hi[r >> LH], both halves in shared memory
    constexpr int LH = (LGN + 1) / 2;
    C *tw_lo = reinterpret_cast<C *>(s_off + G);
    C *tw_hi = tw_lo + (1 << LH);
    {
        const C *tw = reinterpret_cast<const C *>(ld.twN);
        for (int r = tid; r < (1 << LH); r += batched::NT) tw_lo[r] = tw[r];
        for (int r = tid; r < (N >> LH); r += batched::NT) tw_hi[r] = tw[r << LH];
    }
    auto twid = [&](int r) { return cmul(tw_lo[r & ((1 << LH) - 1)], tw_hi[r >> LH]); };
    // z^s, s < 16, for z = w_N^{-e}: from z, z^4, z^8 (three table reads)
    // and at most two products, zh[s >> 2] * zl[s & 3]
    auto powers = [&](C (&zl)[4], C (&zh)[4], int e) {
        const C z1 = twid(e & (N - 1)), z4 = twid((4 * e) & (N - 1)), z8 = twid((8 * e) & (N - 1));
        zl[0] = make_cx<float>(1.f, 0.f); zl[1] = z1; zl[2] = cmul(z1, z1); zl[3] = cmul(zl[2], z1);
        zh[0] = make_cx<float>(1.f, 0.f); zh[1] = z4; zh[2] = z8; zh[3] = cmul(z8, z4);
    };
    auto zpow = [&](const C (&zl)[4], const C (&zh)[4], int s_) {
        return ((s_ & 3) == 0) ? zh[s_ >> 2] : ((s_ >> 2) == 0) ? zl[s_ & 3] : cmul(zh[s_ >> 2], zl[s_ & 3]);
    };

    for (int g = tid; g < gcount; g += batched::NT) s_off[g] = a.off[a.group_tx[gstart + g]];
    __syncthreads();
    // load: 16-byte vectors, all issued before any use, conjugated for dir = +1
    {
        constexpr int NV = batched::ITEM / 2 / batched::NT;
        const float4 *src = reinterpret_cast<const float4 *>(a.in);
        float4 r4[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int e = tid + batched::NT * i;
            const int g = (2 * e) >> LGN, r = (2 * e) & (N - 1);
            r4[i] = (g < gcount) ? __ldg(src + ((s_off[g] + r) >> 1)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int e = tid + batched::NT * i;
            float4 v4 = r4[i];
            if (cj) { v4.y = -v4.y; v4.w = -v4.w; }
            S[2 * e] = make_cx<float>(v4.x, v4.y);
            S[2 * e + 1] = make_cx<float>(v4.z, v4.w);
        }
    }
    __syncthreads();

    C v[16];
    // ---- Phase I pass a: radix R1 over j_hi (j = j_hi*R2 + j_lo), twiddle
    //      w_N1^{-k_lo j_lo}, back in place (k_lo*R2 + j_lo)
    constexpr int NUa = 16 / R1;
#pragma unroll
    for (int q = 0; q < NUa; ++q) {
        const int u = tid + batched::NT * q;
        const int c = u & (N2 - 1);
        const int jl = (u >> LG2) & (R2 - 1);
        const int g = u >> (LG2 + LR2);
        C *base = S + g * N + jl * N2 + c;
#pragma unroll
        for (int r = 0; r < R1; ++r) v[q * R1 + r] = base[r * R2 * N2];
        dft<R1>(v + q * R1);
        if constexpr (R2 > 1) {
            C zl[4], zh[4];
            powers(zl, zh, jl * N2);                           // w_N1^{-jl} = w_N^{-jl N2}
#pragma unroll
            for (int s = 1; s < R1; ++s) v[q * R1 + s] = cmul(v[q * R1 + s], zpow(zl, zh, s));
#pragma unroll
            for (int s = 0; s < R1; ++s) base[s * R2 * N2] = v[q * R1 + s];
        }
    }
    // ---- Phase I pass b: radix R2 over j_lo; k1 = k_lo + R1 * k_hi
    constexpr int NUb = 16 / R2;
    if constexpr (R2 > 1) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NUb; ++q) {
            const int u = tid + batched::NT * q;
            const int c = u & (N2 - 1);
            const int kl = (u >> LG2) & (R1 - 1);
            const int g = u >> (LG2 + LR1);
            const C *base = S + g * N + kl * R2 * N2 + c;
#pragma unroll
            for (int r = 0; r < R2; ++r) v[q * R2 + r] = base[r * N2];
            dft<R2>(v + q * R2);
        }
    }
    __syncthreads();        // every Phase I read done before W overwrites S
    // ---- top-level twiddle w_N^{-k1 c} and the fused digit reversal:
    //      Z[k1][c] -> W[pi_m2(c)][k1]
    {
        constexpr int NUf = (R2 > 1) ? NUb : NUa;
        constexpr int RF = (R2 > 1) ? R2 : R1;
#pragma unroll
        for (int q = 0; q < NUf; ++q) {
            const int u = tid + batched::NT * q;
            const int c = u & (N2 - 1);
            const int kl = (R2 > 1) ? ((u >> LG2) & (R1 - 1)) : 0;
            const int g = (R2 > 1) ? (u >> (LG2 + LR1)) : (u >> LG2);
            const int urow = (int)digit_reverse((unsigned)c, LG2, t);
            C *row = S + g * N + urow * N1;
            const int h = c & HM;                              // pi_m2(urow) = c
#pragma unroll
            for (int k = 0; k < RF; ++k) {
                const int k1 = (R2 > 1) ? (kl + R1 * k) : k;
                row[k1 ^ h] = cmul(v[q * RF + k], twid(k1 * c));
            }
        }
    }
    __syncthreads();
    // ---- Phase III pass a: column v of W through the row map j -> pi_m2(j);
    //      radix Q1 over j_hi (j = j_hi*Q2 + j_lo), twiddle w_N2^{-k_lo j_lo}
    constexpr int NUc = 16 / Q1;
    constexpr int NUd = 16 / Q2;
    C *gout = reinterpret_cast<C *>(a.out);
#pragma unroll
    for (int q = 0; q < NUc; ++q) {
        const int u = tid + batched::NT * q;
        const int col = u & (N1 - 1);
        const int jl = (u >> LG1) & (Q2 - 1);
        const int g = u >> (LG1 + LQ2);
        C *base = S + g * N;
#pragma unroll
        for (int r = 0; r < Q1; ++r) {
            const int j = r * Q2 + jl;
            const int row = (int)digit_reverse((unsigned)j, LG2, t);
            v[q * Q1 + r] = base[row * N1 + (col ^ (j & HM))];
        }
        dft<Q1>(v + q * Q1);
        if constexpr (Q2 > 1) {
            C zl[4], zh[4];
            powers(zl, zh, jl * N1);                           // w_N2^{-jl} = w_N^{-jl N1}
#pragma unroll
            for (int s = 0; s < Q1; ++s) {
                C y = (s > 0) ? cmul(v[q * Q1 + s], zpow(zl, zh, s)) : v[q * Q1 + s];
                const int j = s * Q2 + jl;
                const int row = (int)digit_reverse((unsigned)j, LG2, t);
                base[row * N1 + (col ^ (j & HM))] = y;
            }
        } else if (g < gcount) {
            // single pass: k2 = s, natural-order y[k2 * N1 + col]
            C *dst = gout + s_off[g];
#pragma unroll
            for (int s = 0; s < Q1; ++s) {
                C y = v[q * Q1 + s];
                if (cj) y.y = -y.y;
                dst[s * N1 + col] = y;
            }
        }
    }
    if constexpr (Q2 > 1) {
        __syncthreads();
        // ---- Phase III pass b: radix Q2 over j_lo; k2 = k_lo + Q1 * k_hi
#pragma unroll
        for (int q = 0; q < NUd; ++q) {
            const int u = tid + batched::NT * q;
            const int col = u & (N1 - 1);
            const int kl = (u >> LG1) & (Q1 - 1);
            const int g = u >> (LG1 + LQ1);
            const C *base = S + g * N;
#pragma unroll
            for (int r = 0; r < Q2; ++r) {
                const int j = kl * Q2 + r;
                const int row = (int)digit_reverse((unsigned)j, LG2, t);
                v[q * Q2 + r] = base[row * N1 + (col ^ (j & HM))];
            }
            dft<Q2>(v + q * Q2);
            if (g < gcount) {
                C *dst = gout + s_off[g];
#pragma unroll
                for (int k = 0; k < Q2; ++k) {
                    C y = v[q * Q2 + k];
                    if (cj) y.y = -y.y;
                    dst[(kl + Q1 * k) * N1 + col] = y;
                }
            }
        }
    }
}

template <int LG1, int LG2>
__device__ __noinline__ void small_item(const BatchedArgs &a, const BLen &ld, int gs, int gc, cx<float> *S,
                                       long long *so)
{
    small_group<LG1, LG2>(a, ld, gs, gc, S, so);
}

// LDCG: Phase III reads W, written by other CTAs of this launch, through L2
// only; Phase I reads the launch's read-only input through the read-only path.
// One CTA per SM (128 registers): the body is inlined with the descriptor
// taken by value, so its fields live in registers instead of being re-read
// from shared memory after every barrier of the tile (measured ~20% faster
// per tile).  Two CTAs per SM (64 registers): inlining spills, so the body is
// a call.
template <int A, int B, bool LDCG>
__device__ __forceinline__ void stage_item_inline(const StageArgs sa, int tile, long long boff,
                                                  unsigned char *smem)
{
    stage_tile<float, A, B, -1, 0, 0, LDCG>(sa, tile, boff, 0, smem);
}
template <int A, int B, bool LDCG>
__device__ __noinline__ void stage_item_call(const StageArgs &sa, int tile, long long boff, unsigned char *smem)
{
    stage_tile<float, A, B, -1, 0, 0, LDCG>(sa, tile, boff, 0, smem);
}
template <int MINB, int A, int B, bool LDCG>
__device__ __forceinline__ void stage_item(const StageArgs &sa, int tile, long long boff, unsigned char *smem)
{
    if constexpr (MINB == 1) stage_item_inline<A, B, LDCG>(sa, tile, boff, smem);
    else stage_item_call<A, B, LDCG>(sa, tile, boff, smem);
}

__device__ __forceinline__ void small_dispatch(const BatchedArgs &a, const BLen &ld, int gs, int gc,
                                               cx<float> *S, long long *so)
{
    switch (ld.lgN) {
    case 4: small_item<2, 2>(a, ld, gs, gc, S, so); break;
    case 5: small_item<3, 2>(a, ld, gs, gc, S, so); break;
    case 6: small_item<3, 3>(a, ld, gs, gc, S, so); break;
    case 7: small_item<4, 3>(a, ld, gs, gc, S, so); break;
    case 8: small_item<4, 4>(a, ld, gs, gc, S, so); break;
    case 9: small_item<5, 4>(a, ld, gs, gc, S, so); break;
    case 10: small_item<5, 5>(a, ld, gs, gc, S, so); break;
    case 11: small_item<6, 5>(a, ld, gs, gc, S, so); break;
    case 12: small_item<6, 6>(a, ld, gs, gc, S, so); break;
    case 13: small_item<7, 6>(a, ld, gs, gc, S, so); break;
    default: break;
    }
}

template <int MINB, bool LDCG>
__device__ __forceinline__ void stage_dispatch(const StageArgs &sa, int lgL, int tile, long long boff,
                                               unsigned char *smem)
{
    switch (lgL) {
    case 6: stage_item<MINB, 8, 8, LDCG>(sa, tile, boff, smem); break;
    case 7: stage_item<MINB, 16, 8, LDCG>(sa, tile, boff, smem); break;
    case 8: stage_item<MINB, 16, 16, LDCG>(sa, tile, boff, smem); break;
    case 9: stage_item<MINB, 32, 16, LDCG>(sa, tile, boff, smem); break;
    case 10: stage_item<MINB, 32, 32, LDCG>(sa, tile, boff, smem); break;
    default: break;
    }
}

template <int MINB>
__global__ void __launch_bounds__(batched::NT, MINB) paco_batched_kernel(const __grid_constant__ BatchedArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BItem s_it;
    __shared__ int s_ok;
    __shared__ int s_key;                         // (length, kind) whose descriptor s_sa holds
    __shared__ StageArgs s_sa;
    const int tid = threadIdx.x;
    // Thread 0 keeps the next item (claimed and loaded) and the index of the
    // one after it (claimed) in registers: both round trips overlap the
    // current item.  Claiming ahead cannot deadlock: the lowest-indexed
    // claimed, unfinished item is always some CTA's current item, and it only
    // waits on lower-indexed items, which are all finished.
    BItem nit;
    int nidx = 0, nidx2 = 0;
    if (tid == 0) {
        s_key = -1;
        nidx = (int)atomicAdd(&a.ctr[0], 1u);
        nidx2 = (int)atomicAdd(&a.ctr[0], 1u);
        if (nidx < a.nitems) nit = a.items[nidx];
        else nit.kind = -1;
    }
    for (;;) {
        __syncthreads();                          // the previous item is done with shared memory
        if (tid == 0) {
            s_it = nit;
            nidx = nidx2;
            if (nidx < a.nitems) {
                nit = a.items[nidx];
                nidx2 = (int)atomicAdd(&a.ctr[0], 1u);
            } else {
                nit.kind = -1;
            }
        }
        __syncthreads();
        const BItem item = s_it;
        if (item.kind < 0) break;
        const BLen &ld = a.lens[item.len];
        if (item.kind == 0) {
            cx<float> *S = reinterpret_cast<cx<float> *>(smem_raw);
            long long *so = reinterpret_cast<long long *>(smem_raw + batched::ITEM * sizeof(cx<float>));
            small_dispatch(a, ld, item.a, item.b, S, so);
            continue;
        }
        const int key = item.len * 4 + item.kind;
        if (tid == 0 && s_key != key) {
            s_sa = (item.kind == 1) ? ld.s1 : ld.s2;
            s_sa.in = (item.kind == 1) ? a.in : a.out;
            s_sa.out = a.out;
            s_sa.conj = a.conj;
            s_key = key;
        }
        const StageArgs &sa = s_sa;
        const long long boff = item.off;
        if (item.kind == 2) {
            if (tid == 0) {
                const unsigned need = (unsigned)ld.ntiles1 + a.wait_bias;
                const unsigned *c = a.ctr + 1 + item.a;
                unsigned n = 0;
                int ok = 1;
                while (ld_acquire_u32(c) < need) {
                    if (++n > a.spin_limit) { ok = 0; break; }
                    __nanosleep(64);
                }
                if (!ok) atomicExch(a.status, (int)PACO_ERR_TIMEOUT);
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) continue;                  // reported through the status word
            stage_dispatch<MINB, true>(sa, ld.lg2, item.b, boff, smem_raw);
        } else {
            __syncthreads();                      // s_sa written
            stage_dispatch<MINB, false>(sa, ld.lg1, item.b, boff, smem_raw);
            __syncthreads();                      // every store of the tile issued
            if (tid == 0) {
                __threadfence();
                atomicAdd(a.ctr + 1 + item.a, 1u);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct LenCfg {
    int lg1 = 0, lg2 = 0, t = 1;
};

struct BatchedState {
    int64_t count = 0, total = 0;
    std::vector<int64_t> lengths;
    std::vector<long long> off;
    std::vector<int> lgs;                        // distinct log2 lengths, descending
    std::map<int, LenCfg> cfg;                   // per log2 length
    int minb = 1;                                // CTAs per SM (kernel variant)
    int lag_mult = 2;                            // Phase III lag, in grids
    // device
    BItem *d_items = nullptr;
    int nitems = 0;
    long long *d_off = nullptr;
    BLen *d_lens = nullptr;
    int *d_group = nullptr;
    unsigned *d_ctr = nullptr;
    size_t ctr_words = 0;
    std::vector<void *> tables;
    int smem = 0;
    int grid = 0;
    int tuned = 0;
};

static const void *batched_fn(int minb)
{
    return minb >= 2 ? (const void *)paco_batched_kernel<2> : (const void *)paco_batched_kernel<1>;
}

static int stage_smem_bytes(int lgL, int lgW, int mode)
{
    const int A = 1 << ((lgL + 1) / 2), B = 1 << (lgL / 2), W = 1 << lgW;
    return stage_smem_elems(A, B, 1, W, mode == 1 ? 1 : W) * 8;
}

void batched_destroy(BatchedState *bs)
{
    if (!bs) return;
    cudaFree(bs->d_items);
    cudaFree(bs->d_off);
    cudaFree(bs->d_lens);
    cudaFree(bs->d_group);
    cudaFree(bs->d_ctr);
    for (void *p : bs->tables) cudaFree(p);
    delete bs;
}

static void free_device(BatchedState *bs)
{
    cudaFree(bs->d_items); bs->d_items = nullptr;
    cudaFree(bs->d_lens); bs->d_lens = nullptr;
    cudaFree(bs->d_group); bs->d_group = nullptr;
    for (void *p : bs->tables) cudaFree(p);
    bs->tables.clear();
}

// Valid (lg1, lg2, t) for a length: both factors powers of b = 2^t.
static bool len_cfg_ok(int lgN, const LenCfg &c)
{
    if (c.lg1 + c.lg2 != lgN || c.t < 1 || c.t > 4) return false;
    if (c.lg1 % c.t || c.lg2 % c.t || c.lg1 < c.t || c.lg2 < c.t) return false;
    if (lgN <= batched::SMALL_MAX_LG) return c.lg1 == (lgN + 1) / 2;
    return c.lg1 >= batched::STAGE_MIN_LG && c.lg1 <= batched::STAGE_MAX_LG &&
           c.lg2 >= batched::STAGE_MIN_LG && c.lg2 <= batched::STAGE_MAX_LG;
}

static LenCfg default_cfg(int lgN)
{
    LenCfg c;
    c.lg1 = (lgN + 1) / 2;
    c.lg2 = lgN / 2;
    c.t = 1;
    for (int t = 4; t >= 1; --t) {
        LenCfg d = c;
        d.t = t;
        if (len_cfg_ok(lgN, d)) { c.t = t; break; }
    }
    return c;
}

// The work queue, in claim order (host only, no device state): transforms in
// decreasing length (stable); small ones (N <= 2^13) in groups of up to
// ITEM / N transforms of one length; every large transform's Phase I tiles
// (N / ITEM of them), then its Phase III tiles once `lag` more items have
// been queued after its last Phase I tile; small groups fill in at the end.
// Every Phase III tile thus follows all Phase I tiles of its transform, which
// is what makes the persistent launch deadlock-free.  len_index maps log2
// length to the descriptor index stored in the items.
static void schedule_items(const std::vector<int64_t> &lengths, const std::vector<long long> &off,
                           const std::map<int, int> &len_index, long long lag, std::vector<BItem> &items,
                           std::vector<int> &group)
{
    items.clear();
    group.clear();
    std::vector<int> order(lengths.size());
    for (size_t i = 0; i < lengths.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return lengths[(size_t)x] > lengths[(size_t)y]; });
    std::vector<BItem> small_items;
    std::vector<int> big;
    for (size_t k = 0; k < order.size();) {
        const int i = order[k];
        const int lg = ilog2_exact(lengths[(size_t)i]);
        if (lg > batched::SMALL_MAX_LG) { big.push_back(i); ++k; continue; }
        const int G = batched::ITEM >> lg;
        BItem it;
        memset(&it, 0, sizeof(it));
        it.kind = 0;
        it.len = len_index.at(lg);
        it.a = (int)group.size();
        int n = 0;
        while (k < order.size() && n < G && ilog2_exact(lengths[(size_t)order[k]]) == lg) {
            group.push_back(order[k]);
            ++k; ++n;
        }
        it.b = n;
        small_items.push_back(it);
    }
    auto ntiles = [&](int tr) { return (int)(lengths[(size_t)tr] / batched::ITEM); };
    std::deque<std::pair<int, long long>> pending;  // (transform, earliest position)
    auto emit_s2 = [&](int tr) {
        const int li = len_index.at(ilog2_exact(lengths[(size_t)tr]));
        for (int tl = 0; tl < ntiles(tr); ++tl) items.push_back(BItem{2, li, tr, tl, off[(size_t)tr], 0});
    };
    for (int tr : big) {
        const int li = len_index.at(ilog2_exact(lengths[(size_t)tr]));
        for (int tl = 0; tl < ntiles(tr); ++tl) items.push_back(BItem{1, li, tr, tl, off[(size_t)tr], 0});
        pending.emplace_back(tr, (long long)items.size() + lag);
        while (!pending.empty() && pending.front().second <= (long long)items.size()) {
            emit_s2(pending.front().first);
            pending.pop_front();
        }
    }
    size_t si = 0;
    while (!pending.empty() || si < small_items.size()) {
        if (!pending.empty() && (pending.front().second <= (long long)items.size() || si == small_items.size())) {
            emit_s2(pending.front().first);
            pending.pop_front();
        } else {
            items.push_back(small_items[si++]);
        }
    }
}

// Builds the device tables, the length descriptors and the item order for
// the current configuration.
static paco_status_t build_device(paco_plan *pl, BatchedState *bs)
{
    free_device(bs);
    int nsm = pl->num_sms;
    const void *fn = batched_fn(bs->minb);
    // shared memory: the largest stage tile or a small group
    int smem = batched::ITEM * 8 + (batched::ITEM / 16) * 8 + (128 + 64) * 8;
    for (int lg : bs->lgs) {
        const LenCfg &c = bs->cfg[lg];
        if (lg <= batched::SMALL_MAX_LG) continue;
        smem = std::max(smem, stage_smem_bytes(c.lg1, 13 - c.lg1, 1));
        smem = std::max(smem, stage_smem_bytes(c.lg2, 13 - c.lg2, 2));
    }
    bs->smem = smem;
    PACO_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int occ = 0;
    PACO_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, batched::NT, smem));
    if (occ < 1) return fail(PACO_ERR_UNSUPPORTED, "batched kernel does not fit on an SM");
    if (occ > bs->minb) occ = bs->minb;
    bs->grid = nsm * occ;

    // length descriptors and twiddle tables (FP64-generated)
    std::vector<BLen> lens;
    std::map<int, int> len_index;
    for (int lg : bs->lgs) {
        const LenCfg &c = bs->cfg[lg];
        BLen L;
        memset(&L, 0, sizeof(L));
        L.lgN = lg; L.lg1 = c.lg1; L.lg2 = c.lg2; L.t = c.t;
        const long long N = 1LL << lg, N1 = 1LL << c.lg1, N2 = 1LL << c.lg2;
        paco_status_t st;
        if (lg <= batched::SMALL_MAX_LG) {
            L.small = 1;
            L.G = batched::ITEM >> lg;
            void *tw = nullptr;
            if ((st = gen_table(8, &tw, N, N, 1, 0)) != PACO_OK) return st;
            bs->tables.push_back(tw);
            L.twN = tw;
        } else {
            void *t1 = nullptr, *t2 = nullptr, *lo = nullptr, *hi = nullptr;
            const int lob = (lg + 1) / 2;
            const long long nlo = 1LL << lob, nhi = N / nlo;
            if ((st = gen_table(8, &t1, N1, N1, 1, 0)) != PACO_OK) return st;
            bs->tables.push_back(t1);
            if ((st = gen_table(8, &t2, N2, N2, 1, 0)) != PACO_OK) return st;
            bs->tables.push_back(t2);
            if ((st = gen_table(8, &lo, N, nlo, 1, 0)) != PACO_OK) return st;
            bs->tables.push_back(lo);
            if ((st = gen_table(8, &hi, N, nhi, nlo, 0)) != PACO_OK) return st;
            bs->tables.push_back(hi);
            for (int s = 0; s < 2; ++s) {
                StageArgs &a = s ? L.s2 : L.s1;
                memset(&a, 0, sizeof(a));
                const int lgL = s ? c.lg2 : c.lg1;
                const long long Cc = s ? N1 : N2;
                int lgW = 13 - lgL;
                if ((1LL << lgW) > Cc) lgW = s ? c.lg1 : c.lg2;
                a.batch_stride = N;
                a.C = (int)Cc;
                a.out_ld = (int)N1;
                a.lgW = lgW;
                a.lgK = 0;
                a.mode = s ? 2 : 1;
                a.rev_bits = c.lg2;
                a.rev_t = c.t;
                a.twL = s ? t2 : t1;
                a.twN_lo = lo;
                a.twN_hi = hi;
                a.twN_lo_bits = lob;
                a.N_mask = (unsigned)(N - 1);
                a.pad = s ? (1 << lgW) : 1;
                if (s) L.ntiles2 = (int)(Cc >> lgW);
                else L.ntiles1 = (int)(Cc >> lgW);
                if ((1LL << lgL) * (1LL << lgW) != batched::ITEM)
                    return fail(PACO_ERR_UNSUPPORTED, "length 2^%d: stage tile is not %d elements", lg,
                                batched::ITEM);
            }
        }
        len_index[lg] = (int)lens.size();
        lens.push_back(L);
    }

    std::vector<BItem> items;
    std::vector<int> group;
    schedule_items(bs->lengths, bs->off, len_index, (long long)bs->lag_mult * bs->grid, items, group);
    bs->nitems = (int)items.size();

    PACO_CUDA_TRY(cudaMalloc(&bs->d_items, std::max<size_t>(1, items.size()) * sizeof(BItem)));
    PACO_CUDA_TRY(cudaMalloc(&bs->d_lens, std::max<size_t>(1, lens.size()) * sizeof(BLen)));
    PACO_CUDA_TRY(cudaMalloc(&bs->d_group, std::max<size_t>(1, group.size()) * sizeof(int)));
    if (!items.empty())
        PACO_CUDA_TRY(cudaMemcpy(bs->d_items, items.data(), items.size() * sizeof(BItem), cudaMemcpyHostToDevice));
    if (!lens.empty())
        PACO_CUDA_TRY(cudaMemcpy(bs->d_lens, lens.data(), lens.size() * sizeof(BLen), cudaMemcpyHostToDevice));
    if (!group.empty())
        PACO_CUDA_TRY(cudaMemcpy(bs->d_group, group.data(), group.size() * sizeof(int), cudaMemcpyHostToDevice));
    PACO_CUDA_TRY(cudaDeviceSynchronize());
    return PACO_OK;
}

static paco_status_t launch(const paco_plan *pl, const BatchedState *bs, const void *in, void *out, int dir,
                            cudaStream_t stream)
{
    BatchedArgs a;
    a.items = bs->d_items;
    a.nitems = bs->nitems;
    a.off = bs->d_off;
    a.lens = bs->d_lens;
    a.group_tx = bs->d_group;
    a.in = in;
    a.out = out;
    a.ctr = bs->d_ctr;
    a.status = pl->d_status;
    a.spin_limit = pl->dbg_spin_limit ? pl->dbg_spin_limit : 1u << 24;
    a.wait_bias = pl->dbg_wait_bias;
    a.conj = (dir == 1);
    PACO_CUDA_TRY(cudaMemsetAsync(bs->d_ctr, 0, bs->ctr_words * sizeof(unsigned), stream));
    const int grid = std::min<long long>(bs->grid, std::max(1, bs->nitems));
    void *params[] = {&a};
    PACO_CUDA_TRY(cudaLaunchKernel(batched_fn(bs->minb), dim3((unsigned)grid), dim3(batched::NT), params,
                                   (size_t)bs->smem, stream));
    return PACO_OK;
}

paco_status_t batched_execute(paco_plan *pl, const void *in, void *out, int dir, cudaStream_t stream)
{
    return launch(pl, pl->bs, in, out, dir, stream);
}

void batched_info(const paco_plan *pl, paco_plan_info_t *info)
{
    const BatchedState *bs = pl->bs;
    info->N = bs->total;
    info->batch = bs->count;
    info->dtype = pl->dtype;
    info->stage_threads[0] = info->stage_threads[1] = batched::NT;
    info->stage_smem[0] = info->stage_smem[1] = bs->smem;
    info->stage_cluster[0] = info->stage_cluster[1] = 1;
}

// ---- autotuner ----------------------------------------------------------------
// Times candidate configurations with CUDA events on plan-owned scratch
// buffers and keeps the fastest: per length class (b and the N1 x N2 split,
// on a sub-batch of that class alone), then the CTAs per SM and the Phase III
// lag on a sub-batch of the whole mix.
static float time_config(paco_plan *pl, BatchedState *bs, const void *in, void *out, int reps)
{
    if (build_device(pl, bs) != PACO_OK) return -1.f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r < reps + 1; ++r) {
        cudaEventRecord(e0, 0);
        if (launch(pl, bs, in, out, -1, 0) != PACO_OK) { best = -1.f; break; }
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess) { best = -1.f; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) best = std::min(best, ms);          // first run warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int h = 0;
    cudaMemcpy(&h, pl->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (h != 0) {
        cudaMemset(pl->d_status, 0, sizeof(int));
        return -1.f;
    }
    return best;
}

// A sub-batch: the first transforms of `src` (in order) up to `budget` elements.
static void sub_batch(const BatchedState &src, const std::vector<int> &pick, int64_t budget,
                      BatchedState *dst)
{
    dst->lengths.clear();
    dst->off.clear();
    int64_t tot = 0;
    for (int i : pick) {
        const int64_t n = src.lengths[(size_t)i];
        if (!dst->lengths.empty() && tot + n > budget) break;
        dst->lengths.push_back(n);
        dst->off.push_back(tot);
        tot += n;
    }
    dst->count = (int64_t)dst->lengths.size();
    dst->total = tot;
    std::vector<int> lgs;
    for (int64_t n : dst->lengths) lgs.push_back(ilog2_exact(n));
    std::sort(lgs.begin(), lgs.end(), std::greater<int>());
    lgs.erase(std::unique(lgs.begin(), lgs.end()), lgs.end());
    dst->lgs = lgs;
    dst->cfg = src.cfg;
    dst->minb = src.minb;
    dst->lag_mult = src.lag_mult;
}

static paco_status_t upload_offsets(BatchedState *bs)
{
    cudaFree(bs->d_off);
    cudaFree(bs->d_ctr);
    bs->d_off = nullptr;
    bs->d_ctr = nullptr;
    PACO_CUDA_TRY(cudaMalloc(&bs->d_off, std::max<size_t>(1, bs->off.size()) * sizeof(long long)));
    if (!bs->off.empty())
        PACO_CUDA_TRY(cudaMemcpy(bs->d_off, bs->off.data(), bs->off.size() * sizeof(long long),
                                 cudaMemcpyHostToDevice));
    bs->ctr_words = (size_t)bs->count + 1;
    PACO_CUDA_TRY(cudaMalloc(&bs->d_ctr, bs->ctr_words * sizeof(unsigned)));
    return PACO_OK;
}

static paco_status_t autotune(paco_plan *pl, BatchedState *bs)
{
    // sub-batches of at most 2^26 elements; scratch allocated here, freed below
    const int64_t budget = std::min<int64_t>(bs->total, int64_t(1) << 26);
    void *in = nullptr, *out = nullptr;
    PACO_CUDA_TRY(cudaMalloc(&in, (size_t)budget * 8));
    if (cudaMalloc(&out, (size_t)budget * 8) != cudaSuccess) {
        cudaFree(in);
        return fail(PACO_ERR_NOMEM, "autotune scratch");
    }
    cudaMemset(in, 0, (size_t)budget * 8);
    paco_status_t result = PACO_OK;
    // 1. per length class and per kernel variant (CTAs per SM): the split and
    //    the radix, each length timed alone
    std::map<int, LenCfg> best_cfg[3];
    for (int minb = 1; minb <= 2 && result == PACO_OK; ++minb) {
        for (int lg : bs->lgs) {
            std::vector<int> pick;
            for (int64_t i = 0; i < bs->count; ++i)
                if (ilog2_exact(bs->lengths[(size_t)i]) == lg) pick.push_back((int)i);
            BatchedState sub;
            sub_batch(*bs, pick, budget, &sub);
            sub.minb = minb;
            sub.lag_mult = 2;
            if (upload_offsets(&sub) != PACO_OK) { result = PACO_ERR_CUDA; break; }
            float best = -1.f;
            LenCfg bestc = bs->cfg[lg];
            for (int lg1 = 1; lg1 < lg; ++lg1) {
                for (int t = 1; t <= 4; ++t) {
                    LenCfg c;
                    c.lg1 = lg1; c.lg2 = lg - lg1; c.t = t;
                    if (!len_cfg_ok(lg, c)) continue;
                    sub.cfg[lg] = c;
                    const float ms = time_config(pl, &sub, in, out, 3);
                    if (ms > 0.f && (best < 0.f || ms < best)) { best = ms; bestc = c; }
                }
            }
            best_cfg[minb][lg] = bestc;
            free_device(&sub);
            cudaFree(sub.d_off);
            cudaFree(sub.d_ctr);
        }
    }
    // 2. CTAs per SM (with that variant's per-length choices) and the Phase III
    //    lag, on a sample of the whole mix that keeps its length distribution
    //    (every k-th transform)
    if (result == PACO_OK) {
        const int64_t k = std::max<int64_t>(1, (bs->total + budget - 1) / budget);
        std::vector<int> sample;
        for (int64_t i = 0; i < bs->count; i += k) sample.push_back((int)i);
        BatchedState sub;
        sub_batch(*bs, sample, budget, &sub);
        if (upload_offsets(&sub) == PACO_OK) {
            float best = -1.f;
            int bm = bs->minb, bl = bs->lag_mult;
            for (int minb = 1; minb <= 2; ++minb) {
                for (auto &kv : best_cfg[minb]) sub.cfg[kv.first] = kv.second;
                for (int lagm : {1, 2, 4}) {
                    sub.minb = minb;
                    sub.lag_mult = lagm;
                    const float ms = time_config(pl, &sub, in, out, 3);
                    if (ms > 0.f && (best < 0.f || ms < best)) { best = ms; bm = minb; bl = lagm; }
                }
            }
            bs->minb = bm;
            bs->lag_mult = bl;
            for (auto &kv : best_cfg[bm]) bs->cfg[kv.first] = kv.second;
        }
        free_device(&sub);
        cudaFree(sub.d_off);
        cudaFree(sub.d_ctr);
    }
    cudaFree(in);
    cudaFree(out);
    bs->tuned = 1;
    return result;
}

} // namespace paco

using namespace paco;

extern "C" paco_status_t paco_plan_create_batched_ex(paco_plan_t **out, const int64_t *lengths, int64_t count,
                                                     paco_dtype_t dtype, const paco_batched_opts_t *opts)
{
    if (!out) return fail(PACO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (count < 0 || (count > 0 && !lengths)) return fail(PACO_ERR_INVALID_ARG, "bad length list");
    if (count > (int64_t(1) << 24)) return fail(PACO_ERR_UNSUPPORTED, "more than 2^24 transforms");
    if (dtype != PACO_C64) return fail(PACO_ERR_UNSUPPORTED, "uneven batches are built for complex64 only");
    paco_batched_opts_t o;
    memset(&o, 0, sizeof(o));
    o.autotune = 1;
    if (opts) o = *opts;
    BatchedState *bs = new (std::nothrow) BatchedState();
    if (!bs) return fail(PACO_ERR_NOMEM, "out of host memory");
    bs->count = count;
    int64_t tot = 0;
    std::vector<int> lgs;
    for (int64_t i = 0; i < count; ++i) {
        const int64_t n = lengths[i];
        const int lg = ilog2_exact(n);
        if (lg < 4 || lg > 2 * batched::STAGE_MAX_LG) {
            delete bs;
            return fail(PACO_ERR_UNSUPPORTED, "length %lld: uneven batches take powers of two 2^4..2^20",
                        (long long)n);
        }
        bs->lengths.push_back(n);
        bs->off.push_back(tot);
        tot += n;
        lgs.push_back(lg);
    }
    if (tot > (int64_t(1) << 34)) {
        delete bs;
        return fail(PACO_ERR_UNSUPPORTED, "total length above 2^34");
    }
    bs->total = tot;
    std::sort(lgs.begin(), lgs.end(), std::greater<int>());
    lgs.erase(std::unique(lgs.begin(), lgs.end()), lgs.end());
    bs->lgs = lgs;
    for (int lg : lgs) {
        LenCfg c = default_cfg(lg);
        if (o.b) {
            LenCfg d = c;
            d.t = ilog2_exact(o.b);
            if (d.t < 1 || d.t > 4) {
                delete bs;
                return fail(PACO_ERR_INVALID_ARG, "radix b=%d must be 2, 4, 8 or 16", o.b);
            }
            if (len_cfg_ok(lg, d)) c = d;
        }
        bs->cfg[lg] = c;
    }
    bs->minb = (o.ctas_per_sm == 2) ? 2 : 1;
    bs->lag_mult = o.lag > 0 ? o.lag : 2;

    paco_plan *pl = new (std::nothrow) paco_plan();
    if (!pl) {
        delete bs;
        return fail(PACO_ERR_NOMEM, "out of host memory");
    }
    pl->dtype = dtype;
    pl->esize = 8;
    pl->N = tot > 0 ? tot : 1;
    pl->batch = count > 0 ? 1 : 0;
    pl->b = 2; pl->t = 1; pl->p = 1;
    pl->bs = bs;
    cudaGetDevice(&pl->device);
    cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, pl->device);
    paco_status_t st = PACO_OK;
    cudaError_t e = cudaMalloc(&pl->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(pl->d_status, 0, sizeof(int));
    if (e != cudaSuccess) st = fail(PACO_ERR_CUDA, "plan setup: %s", cudaGetErrorString(e));
    if (st == PACO_OK && count > 0) {
        if (o.autotune) st = autotune(pl, bs);
        if (st == PACO_OK) st = upload_offsets(bs);
        if (st == PACO_OK) st = build_device(pl, bs);
    }
    if (st != PACO_OK) {
        paco_plan_destroy(pl);
        return st;
    }
    *out = pl;
    return PACO_OK;
}

extern "C" paco_status_t paco_plan_create_batched(paco_plan_t **out, const int64_t *lengths, int64_t count,
                                                  paco_dtype_t dtype)
{
    return paco_plan_create_batched_ex(out, lengths, count, dtype, nullptr);
}

extern "C" paco_status_t paco_plan_batched_config(const paco_plan_t *pl, int64_t length, int *b, int *N1,
                                                  int *ctas_per_sm, int *lag)
{
    if (!pl || !pl->bs) return fail(PACO_ERR_INVALID_ARG, "not an uneven-batch plan");
    const int lg = ilog2_exact(length);
    auto it = pl->bs->cfg.find(lg);
    if (it == pl->bs->cfg.end()) return fail(PACO_ERR_INVALID_ARG, "length %lld is not in the plan", (long long)length);
    if (b) *b = 1 << it->second.t;
    if (N1) *N1 = 1 << it->second.lg1;
    if (ctas_per_sm) *ctas_per_sm = pl->bs->minb;
    if (lag) *lag = pl->bs->lag_mult;
    return PACO_OK;
}

extern "C" int64_t paco_debug_batched_schedule(const int64_t *lengths, int64_t count, int64_t lag_items,
                                               int32_t *kind, int32_t *index, int32_t *tile, int64_t cap,
                                               int32_t *group, int64_t group_cap)
{
    if (count < 0 || (count > 0 && !lengths) || lag_items < 0) return -1;
    std::vector<int64_t> len((size_t)count);
    std::vector<long long> off((size_t)count);
    std::map<int, int> li;
    long long tot = 0;
    for (int64_t i = 0; i < count; ++i) {
        const int lg = ilog2_exact(lengths[i]);
        if (lg < 4 || lg > 2 * batched::STAGE_MAX_LG) return -1;
        len[(size_t)i] = lengths[i];
        off[(size_t)i] = tot;
        tot += lengths[i];
        li[lg] = lg;
    }
    std::vector<BItem> items;
    std::vector<int> grp;
    schedule_items(len, off, li, lag_items, items, grp);
    if ((int64_t)items.size() > cap || (int64_t)grp.size() > group_cap) return -1;
    for (size_t k = 0; k < items.size(); ++k) {
        kind[k] = items[k].kind;
        index[k] = items[k].a;
        tile[k] = items[k].b;
    }
    for (size_t k = 0; k < grp.size(); ++k) group[k] = grp[k];
    return (int64_t)items.size();
}
