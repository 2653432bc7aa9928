// paco_panel.cuh -- L2-resident panel pipeline for a length-2^14 stage.
//
// The paper's local FFT on one slab is CO-Batched-FFT with n = L and
// s = slab width: a balanced transform split n = n1*n2 (here 128 x 128) into
// a first child group (s*n2 DFTs of length n1 over j_hi) and a second child
// group (s*n1 DFTs of length n2 over j_lo) with the layout-aware twiddle
// w_L^{-k_lo j_lo} between them (Sect. 4.1, Fig. "cofft", Eq. twop).  The
// analysis places the recursion frontier where a view fits in cache; on
// GB300 the cache that holds a slab is the 129 MB L2.  So each stage runs the
// two child groups of one panel (a group of columns) as two sub-passes:
//
//   sub-pass A: 128-point DFTs over j_hi of tiles read from HBM; twiddle;
//               written to an L2-resident panel buffer;
//   sub-pass B: 128-point DFTs over j_lo of that buffer; stage epilogue
//               (mode 1: top-level twiddle w_N^{-k1 c} and the digit-reversed
//               row pi_m2(c) of W, Eq. (17); mode 2: natural-order output).
//
// HBM is touched once per element per direction (the paper's two passes); the
// intermediate lives in a ring of NBUF panel buffers sized to stay in L2.
// One persistent kernel walks the tiles in the order A0, A1, B0, A2, B1, ...;
// a B tile waits for its panel's A tiles, an A tile waits until the panel
// that last used its buffer has been consumed.  Waits are bounded spins that
// record PACO_ERR_TIMEOUT and give up.  Every tile is 8192 elements: 512
// threads hold 16 each; a 128-point DFT is radix 16 (in registers) then radix
// 8 (after one shared-memory exchange).
#pragma once

#include "paco_common.cuh"

namespace paco {

struct PanelArgs {
    const void *in;        // stage input (batch of N elements)
    void *out;             // stage output
    void *scratch;         // NBUF panel buffers of L*P elements
    unsigned *ctr;         // [0] work counter, [1..np] A done, [np+1..2np] B done
    int *status;           // device status word (PACO_ERR_TIMEOUT on a wait that gave up)
    long long batch_stride;
    int C;                 // columns of the stage input matrix
    int out_ld;            // row length of the output matrix
    int P;                 // panel width (columns), a power of two >= 64
    int panels_per_batch;  // C / P
    int npanels;           // batch * C / P
    int mode;              // 1: stage 1 fused with the middle stage; 2: stage 2
    int rev_bits, rev_t;   // digit reversal pi_m2
    const void *twL;       // w_L^{-r}, r < L
    const void *twN_lo, *twN_hi;
    int twN_lo_bits;
    unsigned N_mask;
    int conj;
    unsigned spin_limit;
};

namespace panel {

constexpr int A = 128, B = 128, L = A * B;
constexpr int SP = 66;              // shared row stride (elements): conflict-free passes
constexpr int NT = 512;             // threads per CTA
constexpr int TILE = 8192;          // elements per tile
constexpr int NBUF = 3;             // panel buffers in the ring

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// L2 eviction policies (createpolicy) for the streams that pass through HBM
// once (evict first) and for the panel buffers that must stay (evict last).
__device__ __forceinline__ unsigned long long policy_evict_first()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long policy_evict_last()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float2 ld_stream(const float2 *p, unsigned long long pol)
{
    float2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
                 : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float2 ld_l2(const float2 *p)
{
    float2 v;
    asm volatile("ld.global.cg.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_hint(float2 *p, float2 v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;"
                 :: "l"(p), "f"(v.x), "f"(v.y), "l"(pol) : "memory");
}

__device__ __forceinline__ float2 f2mul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// shared slot of sequence (jl, c) in the stage-1 A tile: conflict-free both
// when lanes run over c (pass 1) and over jl then c (pass 2)
__device__ __forceinline__ int slot_s1a(int jl, int c) { return c * 4 + (jl ^ ((c >> 2) & 3)); }

// Pass 1 of a 128-point DFT: v[r] = x[t8 + 8 r]; radix 16 over r, twiddle
// w_128^{-s t8}, store output s of this thread at shared row t8 + 8 s.
__device__ __forceinline__ void pass1(cx<float> *v, float2 *sm, int t8, int slot, const float2 *w128)
{
    dft16(v);
#pragma unroll
    for (int s = 1; s < 16; ++s) {
        float2 w = w128[s * t8];
        float2 a = make_float2(v[s].x, v[s].y);
        float2 p = f2mul(a, w);
        v[s].x = p.x; v[s].y = p.y;
    }
#pragma unroll
    for (int s = 0; s < 16; ++s) sm[(t8 + 8 * s) * SP + slot] = make_float2(v[s].x, v[s].y);
}

// Pass 2: groups g = 2 gp + h (h < 2): radix 8 over t of rows g*8 + t; the
// output k' of group g is DFT index k = g + 16 k', left in v[8 h + k'].
__device__ __forceinline__ void pass2(cx<float> *v, const float2 *sm, int gp, int slot)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int g = 2 * gp + h;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            float2 a = sm[(g * 8 + t) * SP + slot];
            v[8 * h + t] = make_cx<float>(a.x, a.y);
        }
        dft8(v + 8 * h);
    }
}

} // namespace panel

#ifdef PACO_PANEL_KERNEL_TU
// Launch: grid = persistent CTAs (co-residency is not required for
// progress: a tile only ever waits for tiles dequeued before it).
__global__ void __launch_bounds__(panel::NT, 2) paco_panel_kernel(const PanelArgs args)
{
    using namespace panel;
    extern __shared__ __align__(16) float2 sm[];          // A rows x SP
    __shared__ float2 w128[A];                           // w_128^{-r} = w_L^{-128 r}
    __shared__ float2 tlo[128];                          // w_L^{-r}, r < 128
    __shared__ float2 E1[64], E2[B];                     // mode 1 epilogue factors
    __shared__ unsigned rtab[16];                        // pi(1024 r)
    __shared__ int s_tile[2], s_abort;                  // tile index by iteration parity

    const int tid = threadIdx.x;
    const float2 *twL = reinterpret_cast<const float2 *>(args.twL);
    for (int r = tid; r < A; r += NT) {
        w128[r] = __ldg(twL + r * B);
        tlo[r] = __ldg(twL + r);
    }
    if (tid < 16 && args.mode == 2)
        rtab[tid] = digit_reverse((unsigned)tid << 10, args.rev_bits, args.rev_t);
    if (tid == 0) {
        s_tile[0] = (int)atomicAdd(args.ctr, 1u);
        s_abort = 0;
    }
    const float csign = args.conj ? -1.f : 1.f;
    const unsigned long long pol_first = policy_evict_first();
    const unsigned long long pol_last = policy_evict_last();
    const int T = (L / TILE) * args.P;                    // tiles per phase per panel
    const int np = args.npanels;
    const long long total = 2LL * np * T;
    const float2 *gin = reinterpret_cast<const float2 *>(args.in);
    float2 *gout = reinterpret_cast<float2 *>(args.out);
    float2 *scr = reinterpret_cast<float2 *>(args.scratch);
    unsigned *doneA = args.ctr + 1, *doneB = args.ctr + 1 + np;
    __syncthreads();

    for (int iter = 0;; ++iter) {
        const long long g = s_tile[iter & 1];
        if (g >= total) break;
        // decode the tile: blocks A0 | A1 B0 | A2 B1 | ... | B(np-1)
        const int bi = (int)(g / T), t = (int)(g % T);
        bool isB;
        int q;
        if (bi == 0) { isB = false; q = 0; }
        else if (bi == 2 * np - 1) { isB = true; q = np - 1; }
        else { q = (bi + 1) / 2; isB = !(bi & 1); if (isB) q -= 1; }
        // wait for the dependency
        if (tid == 0) {
            const unsigned *dep = nullptr;
            if (isB) dep = doneA + q;
            else if (q >= NBUF) dep = doneB + (q - NBUF);
            if (dep) {
                unsigned it = 0;
                while (ld_acquire(dep) < (unsigned)T) {
                    if (++it > args.spin_limit) {
                        atomicExch(args.status, 5 /* PACO_ERR_TIMEOUT */);
                        s_abort = 1;
                        break;
                    }
                    __nanosleep(200);
                }
            }
            s_tile[(iter + 1) & 1] = (int)atomicAdd(args.ctr, 1u);   // prefetch the next tile index
        }
        __syncthreads();
        if (s_abort) break;
        __threadfence();

        const int bidx = q / args.panels_per_batch, pcol = q % args.panels_per_batch;
        const long long boff = (long long)bidx * args.batch_stride;
        const int colbase = pcol * args.P;                     // first column of the panel
        float2 *buf = scr + (size_t)(q % NBUF) * ((size_t)L * args.P);
        cx<float> v[16];

        if (args.mode == 1 && !isB) {
            // A tile of stage 1: 4 j_lo x 16 columns; X[j_hi*128 + j_lo][c]
            const int ncg = args.P >> 4;
            const int j0 = (t / ncg) * 4, c0 = (t % ncg) * 16;
            {
                const int c = tid & 15, jl = (tid >> 4) & 3, t8 = tid >> 6;
                const float2 *src = gin + boff + (long long)(j0 + jl) * args.C + colbase + c0 + c;
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    float2 x = ld_stream(src + (long long)((t8 + 8 * r) * B) * args.C, pol_first);
                    v[r] = make_cx<float>(x.x, x.y * csign);
                }
                pass1(v, sm, t8, slot_s1a(jl, c), w128);
            }
            __syncthreads();
            {
                const int jl = tid & 3, c = (tid >> 2) & 15, gp = tid >> 6;
                pass2(v, sm, gp, slot_s1a(jl, c));
                const int jlo = j0 + jl;
                float2 *dst = buf + ((size_t)(c0 + c) * A) * B + jlo;
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int klo = 2 * gp + h + 16 * k;
                        const unsigned rr = (unsigned)(klo * jlo);                 // < L
                        const float2 w = f2mul(tlo[rr & 127], w128[rr >> 7]);       // w_L^{-rr}
                        const float2 y = f2mul(make_float2(v[8 * h + k].x, v[8 * h + k].y), w);
                        st_hint(dst + (size_t)klo * B, y, pol_last);
                    }
            }
        } else if (args.mode == 1) {
            // B tile of stage 1: 64 k_lo x 1 column; reads buf[c][k_lo][j_lo]
            const int cl = t >> 1, k0 = (t & 1) * 64;
            const unsigned cglob = (unsigned)(colbase + cl);
            if (tid < 64 + B) {
                unsigned r;
                if (tid < 64) r = ((unsigned)(k0 + tid) * cglob) & args.N_mask;
                else r = ((unsigned)A * (unsigned)(tid - 64) * cglob) & args.N_mask;
                const float2 *nlo = reinterpret_cast<const float2 *>(args.twN_lo);
                const float2 *nhi = reinterpret_cast<const float2 *>(args.twN_hi);
                const float2 w = f2mul(__ldg(nlo + (r & ((1u << args.twN_lo_bits) - 1u))),
                                       __ldg(nhi + (r >> args.twN_lo_bits)));
                if (tid < 64) E1[tid] = w; else E2[tid - 64] = w;
            }
            {
                const int t8 = tid & 7, k = tid >> 3;
                const float2 *src = buf + ((size_t)cl * A + k0 + k) * B + t8;
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    float2 x = ld_l2(src + 8 * r);
                    v[r] = make_cx<float>(x.x, x.y);
                }
                pass1(v, sm, t8, k, w128);
            }
            __syncthreads();
            {
                const int k = tid & 63, gp = tid >> 6;
                pass2(v, sm, gp, k);
                const unsigned urow = digit_reverse(cglob, args.rev_bits, args.rev_t);
                float2 *dst = gout + boff + (long long)urow * args.out_ld + k0 + k;
                const float2 e1 = E1[k];
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const int khi = 2 * gp + h + 16 * kk;
                        float2 y = f2mul(make_float2(v[8 * h + kk].x, v[8 * h + kk].y), f2mul(e1, E2[khi]));
                        y.y *= csign;
                        st_hint(dst + A * khi, y, pol_first);
                    }
            }
        } else if (!isB) {
            // A tile of stage 2: 1 j_lo x 64 columns; W[pi(j_hi*128 + j_lo)][v]
            const int nvg = args.P >> 6;
            const int jlo = t / nvg, v0 = (t % nvg) * 64;
            {
                const int vv = tid & 63, t8 = tid >> 6;
                const unsigned base = digit_reverse((unsigned)(jlo + (t8 << 7)), args.rev_bits, args.rev_t);
                const float2 *src = gin + boff + colbase + v0 + vv;
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    float2 x = ld_stream(src + (long long)(base | rtab[r]) * args.C, pol_first);
                    v[r] = make_cx<float>(x.x, x.y * csign);
                }
                pass1(v, sm, t8, vv, w128);
            }
            __syncthreads();
            {
                const int vv = tid & 63, gp = tid >> 6;
                pass2(v, sm, gp, vv);
                float2 *dst = buf + (size_t)jlo * args.P + v0 + vv;
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int klo = 2 * gp + h + 16 * k;
                        const unsigned rr = (unsigned)(klo * jlo);
                        const float2 w = f2mul(tlo[rr & 127], w128[rr >> 7]);
                        const float2 y = f2mul(make_float2(v[8 * h + k].x, v[8 * h + k].y), w);
                        st_hint(dst + (size_t)klo * B * args.P, y, pol_last);
                    }
            }
        } else {
            // B tile of stage 2: 1 k_lo x 64 columns; reads buf[k_lo][j_lo][v]
            const int nvg = args.P >> 6;
            const int klo = t / nvg, v0 = (t % nvg) * 64;
            {
                const int vv = tid & 63, t8 = tid >> 6;
                const float2 *src = buf + ((size_t)klo * B + t8) * args.P + v0 + vv;
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    float2 x = ld_l2(src + (size_t)(8 * r) * args.P);
                    v[r] = make_cx<float>(x.x, x.y);
                }
                pass1(v, sm, t8, vv, w128);
            }
            __syncthreads();
            {
                const int vv = tid & 63, gp = tid >> 6;
                pass2(v, sm, gp, vv);
                float2 *dst = gout + boff + colbase + v0 + vv;
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const int khi = 2 * gp + h + 16 * kk;
                        float2 y = make_float2(v[8 * h + kk].x, v[8 * h + kk].y * csign);
                        st_hint(dst + (long long)(klo + A * khi) * args.out_ld, y, pol_first);
                    }
            }
        }
        // publish the tile
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd(isB ? doneB + q : doneA + q, 1u);
    }
}

#endif // PACO_PANEL_KERNEL_TU

} // namespace paco
