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

#include <cuda.h>                 // CUtensorMap (type only)

#include "paco_common.cuh"

namespace paco {

struct PanelArgs {
    // Tensor maps for the TMA-fed kernel (__grid_constant__, 64-byte aligned):
    //   map_in:  stage 1: X as (c, j_lo, j_hi, batch), box (16, 4, 128, 1);
    //            stage 2: W rows split into runs of digit-reversal bits (see
    //            map_rows_* below), box (64, ..) = the 128 rows of one j_lo.
    //   map_scr: the scratch ring as (v, rows), box (64, 128) (stage 2).
    CUtensorMap map_in;
    CUtensorMap map_scr;
    int map_rank;                  // rank of map_in (stage 2)
    int map_run_start[4];          // stage 2: bit position of each row dimension
    int map_run_fixed[4];          // 1: the run is fixed by j_lo (box 1), 0: spanned
    unsigned vmask;                // stage 2: row bits spanned by j_hi
    const void *in;        // stage input (batch of N elements)
    void *out;             // stage output
    void *scratch;         // NBUF panel buffers of L*P elements
    unsigned *ctr;         // [0] work counter, [1..np] A done, [np+1..2np] B done
    int *status;           // device status word (PACO_ERR_TIMEOUT on a wait that gave up)
    long long batch_stride;
    int C;                 // columns of the stage input matrix
    int out_ld;            // row length of the output matrix
    int P;                 // panel width (columns), a power of two >= 64
    int lgP;               // log2 P
    int panels_per_batch;  // C / P (a power of two)
    int lgPpb;             // log2 panels_per_batch
    int npanels;           // batch * C / P
    int mode;              // 1: stage 1 fused with the middle stage; 2: stage 2
    int rev_bits, rev_t;   // digit reversal pi_m2
    const void *twL;       // w_L^{-r}, r < L
    const void *twN_lo, *twN_hi;
    int twN_lo_bits;
    unsigned N_mask;
    int conj;
    unsigned spin_limit;
    int use_tensor;                // 1: tiles arrive by tensor TMA
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

__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
// drop a consumed 128-byte scratch line from L2 without writing it back
__device__ __forceinline__ void discard_l2(const void *p)
{
    asm volatile("discard.global.L2 [%0], 128;" :: "l"(p) : "memory");
}

__device__ __forceinline__ float2 f2mul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// shared slot of sequence (jl, c) in the stage-1 A tile: conflict-free both
// when lanes run over c (pass 1) and over jl then c (pass 2)
__device__ __forceinline__ int slot_s1a(int jl, int c) { return c * 4 + (jl ^ ((c >> 2) & 3)); }

// Pass 1 of a 128-point DFT: v[r] = x[t8 + 8 r]; radix 16 over r, twiddle
// w_128^{-s t8} from w16[s*8 + t8] (lanes that differ in t8 read consecutive
// entries), store output s of this thread at shared row t8 + 8 s.
__device__ __forceinline__ void pass1(cx<float> *v, float2 *sm, int t8, int slot, const float2 *w16)
{
    dft16(v);
#pragma unroll
    for (int s = 1; s < 16; ++s) {
        float2 w = w16[s * 8 + t8];
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

// One decoded tile of the pipeline order A0 | A1 B0 | A2 B1 | ... | B(np-1).
struct Tile {
    int g;         // position in the order (>= total: none)
    int isB, q, t;
};

__device__ __forceinline__ Tile decode_tile(int g, int lgT, int np)
{
    Tile d;
    d.g = g;
    const unsigned gu = (unsigned)g;                  // total < 2^31 tiles
    const int bi = (int)(gu >> lgT);
    d.t = (int)(gu & ((1u << lgT) - 1u));
    if (bi == 0) { d.isB = 0; d.q = 0; }
    else if (bi == 2 * np - 1) { d.isB = 1; d.q = np - 1; }
    else { d.q = (bi + 1) / 2; d.isB = !(bi & 1); if (d.isB) d.q -= 1; }
    return d;
}

// tiles per phase per panel: T = L * P / TILE = 2 P
__device__ __forceinline__ int tiles_per_phase(const PanelArgs &a) { return 2 << a.lgP; }

// the counter a tile waits on, or nullptr
__device__ __forceinline__ const unsigned *tile_dep(const PanelArgs &a, const Tile &d)
{
    if (d.isB) return a.ctr + 1 + d.q;
    if (d.q >= panel::NBUF) return a.ctr + 1 + a.npanels + (d.q - panel::NBUF);
    return nullptr;
}

// Per warp: 1 if the tile's dependency is met (acquired); with `block`, spin
// (bounded) until it is.  Returns -1 when a bounded wait gave up.
__device__ __forceinline__ int warp_acquire(const PanelArgs &a, const Tile &d, bool block)
{
    const unsigned *dep = tile_dep(a, d);
    if (!dep) return 1;
    int ok = 0;
    if ((threadIdx.x & 31) == 0) {
        unsigned it = 0;
        for (;;) {
            if (panel::ld_acquire(dep) >= (unsigned)tiles_per_phase(a)) { ok = 1; break; }
            if (!block) break;
            if (++it > a.spin_limit) {
                atomicExch(a.status, 5 /* PACO_ERR_TIMEOUT */);
                ok = -1;
                break;
            }
            __nanosleep(100);
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok;
}

__device__ __forceinline__ float2 *panel_buf(const PanelArgs &a, int q)
{
    return reinterpret_cast<float2 *>(a.scratch) + ((size_t)(q % panel::NBUF) << (14 + a.lgP));
}

// Issue the 16 loads of this thread's pass-1 operands for tile d.
__device__ __forceinline__ void load_tile(const PanelArgs &a, const Tile &d, cx<float> *v,
                                          const unsigned *rtab)
{
    using namespace panel;
    const float2 *gin = reinterpret_cast<const float2 *>(a.in);
    const int tid = threadIdx.x;
    const int bidx = d.q >> a.lgPpb, pcol = d.q & (a.panels_per_batch - 1);
    const long long boff = (long long)bidx * a.batch_stride;
    const int colbase = pcol << a.lgP;
    const float2 *buf = panel_buf(a, d.q);
    if (a.mode == 1 && !d.isB) {
        const unsigned long long pol = policy_evict_first();
        const int j0 = (d.t >> (a.lgP - 4)) * 4, c0 = (d.t & ((a.P >> 4) - 1)) * 16;
        const int cc = tid & 15, jl = (tid >> 4) & 3, t8 = tid >> 6;
        const float2 *src = gin + boff + (long long)(j0 + jl) * a.C + colbase + c0 + cc +
                            (long long)(t8 * B) * a.C;
        const long long step = (long long)(8 * B) * a.C;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            float2 x = ld_stream(src + r * step, pol);
            v[r] = make_cx<float>(x.x, x.y);
        }
    } else if (a.mode == 1) {
        const int cl = d.t >> 1, k0 = (d.t & 1) * 64;
        const int t8 = tid & 7, k = tid >> 3;
        const float2 *src = buf + ((size_t)cl * A + k0 + k) * B + t8;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            float2 x = ld_l2(src + 8 * r);
            v[r] = make_cx<float>(x.x, x.y);
        }
    } else if (!d.isB) {
        const int jlo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
        const int vv = tid & 63, t8 = tid >> 6;
        const unsigned base = digit_reverse((unsigned)(jlo + (t8 << 7)), a.rev_bits, a.rev_t);
        const float2 *src = gin + boff + colbase + v0 + vv;
        const unsigned long long pol = policy_evict_first();
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            float2 x = ld_stream(src + (long long)(base | rtab[r]) * a.C, pol);
            v[r] = make_cx<float>(x.x, x.y);
        }
    } else {
        const int klo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
        const int vv = tid & 63, t8 = tid >> 6;
        const float2 *src = buf + ((size_t)klo * B + t8) * a.P + v0 + vv;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            float2 x = ld_l2(src + (size_t)(8 * r) * a.P);
            v[r] = make_cx<float>(x.x, x.y);
        }
    }
}

// Per-tile twiddle tables, built before pass 1 and read in pass 2:
//  A tiles: TW[jl][k_lo] = w_L^{-k_lo j_lo}    (stage 1: 4 x 128; stage 2: 1 x 128)
//  stage-1 B tiles: E1[k] = w_N^{-(k0+k) c}, E2[k_hi] = w_N^{-128 k_hi c}
__device__ __forceinline__ void tile_tables(const PanelArgs &a, const Tile &d, float2 *TW,
                                            float2 *E1, float2 *E2, const float2 *w128,
                                            const float2 *tlo)
{
    using namespace panel;
    const int tid = threadIdx.x;
    if (!d.isB) {
        int jlo, klo;
        int jl = 0;
        if (a.mode == 1) {
            jl = tid >> 7;
            jlo = (d.t >> (a.lgP - 4)) * 4 + jl;
            klo = tid & 127;
        } else {
            if (tid >= 128) return;
            jlo = d.t >> (a.lgP - 6);
            klo = tid;
        }
        const unsigned rr = (unsigned)(klo * jlo);
        TW[klo * 4 + jl] = f2mul(tlo[rr & 127], w128[rr >> 7]);     // [k_lo][jl]: conflict-free reads
    } else if (a.mode == 1) {
        if (tid >= 64 + B) return;
        const int pcol = d.q & (a.panels_per_batch - 1);
        const unsigned cglob = (unsigned)((pcol << a.lgP) + (d.t >> 1));
        const int k0 = (d.t & 1) * 64;
        unsigned r;
        if (tid < 64) r = ((unsigned)(k0 + tid) * cglob) & a.N_mask;
        else r = ((unsigned)A * (unsigned)(tid - 64) * cglob) & a.N_mask;
        const float2 *nlo = reinterpret_cast<const float2 *>(a.twN_lo);
        const float2 *nhi = reinterpret_cast<const float2 *>(a.twN_hi);
        const float2 w = f2mul(__ldg(nlo + (r & ((1u << a.twN_lo_bits) - 1u))),
                               __ldg(nhi + (r >> a.twN_lo_bits)));
        if (tid < 64) E1[tid] = w; else E2[tid - 64] = w;
    }
}

// Pass 1 (operands in v), block barrier, pass 2 and the stores of tile d.
// `abort_out` receives the block's abort flag, read right after the mid-tile
// barrier: every write to it happens before that barrier in the same step, so
// all warps see the same value.
__device__ __forceinline__ void compute_tile(const PanelArgs &a, const Tile &d, cx<float> *v,
                                             float2 *sm, const float2 *w16, const float2 *TW,
                                             const float2 *E1, const float2 *E2,
                                             const volatile int *s_abort, int &abort_out)
{
    using namespace panel;
    const int tid = threadIdx.x;
    const int bidx = d.q >> a.lgPpb, pcol = d.q & (a.panels_per_batch - 1);
    const long long boff = (long long)bidx * a.batch_stride;
    const int colbase = pcol << a.lgP;
    float2 *buf = panel_buf(a, d.q);
    float2 *gout = reinterpret_cast<float2 *>(a.out);
    const float cs = a.conj ? -1.f : 1.f;

    if (a.mode == 1 && !d.isB) {
        const int j0 = (d.t >> (a.lgP - 4)) * 4, c0 = (d.t & ((a.P >> 4) - 1)) * 16;
        {
            const int cc = tid & 15, jl = (tid >> 4) & 3, t8 = tid >> 6;
            if (cs < 0.f) {
#pragma unroll
                for (int r = 0; r < 16; ++r) v[r].y = -v[r].y;
            }
            pass1(v, sm, t8, slot_s1a(jl, cc), w16);
        }
        __syncthreads();
        abort_out = *s_abort;
        const int jl = tid & 3, cc = (tid >> 2) & 15, gp = tid >> 6;
        pass2(v, sm, gp, slot_s1a(jl, cc));
        float2 *dst = buf + ((size_t)(c0 + cc) * A) * B + j0 + jl;
        const float2 *tw = TW + jl;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int klo = 2 * gp + h + 16 * k;
                const float2 y = f2mul(make_float2(v[8 * h + k].x, v[8 * h + k].y), tw[klo * 4]);
                st_hint(dst + (size_t)klo * B, y, policy_evict_last());
            }
    } else if (a.mode == 1) {
        const int cl = d.t >> 1, k0 = (d.t & 1) * 64;
        const unsigned cglob = (unsigned)(colbase + cl);
        {
            const int t8 = tid & 7, k = tid >> 3;
            pass1(v, sm, t8, k, w16);
        }
        __syncthreads();
        abort_out = *s_abort;
        discard_l2(buf + ((size_t)cl * A + k0) * B + 16 * tid);        // consumed lines
        const int k = tid & 63, gp = tid >> 6;
        pass2(v, sm, gp, k);
        const unsigned urow = digit_reverse(cglob, a.rev_bits, a.rev_t);
        float2 *dst = gout + boff + (long long)urow * a.out_ld + k0 + k;
        const float2 e1 = E1[k];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const int khi = 2 * gp + h + 16 * kk;
                float2 y = f2mul(f2mul(make_float2(v[8 * h + kk].x, v[8 * h + kk].y), e1), E2[khi]);
                if (cs < 0.f) y.y = -y.y;
                st_hint(dst + A * khi, y, policy_evict_first());
            }
    } else if (!d.isB) {
        const int jlo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
        {
            const int vv = tid & 63, t8 = tid >> 6;
            if (cs < 0.f) {
#pragma unroll
                for (int r = 0; r < 16; ++r) v[r].y = -v[r].y;
            }
            pass1(v, sm, t8, vv, w16);
        }
        __syncthreads();
        abort_out = *s_abort;
        const int vv = tid & 63, gp = tid >> 6;
        pass2(v, sm, gp, vv);
        float2 *dst = buf + (size_t)jlo * a.P + v0 + vv;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int klo = 2 * gp + h + 16 * k;
                const float2 y = f2mul(make_float2(v[8 * h + k].x, v[8 * h + k].y), TW[klo * 4]);
                st_hint(dst + (size_t)klo * B * a.P, y, policy_evict_last());
            }
    } else {
        const int klo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
        {
            const int vv = tid & 63, t8 = tid >> 6;
            pass1(v, sm, t8, vv, w16);
        }
        __syncthreads();
        abort_out = *s_abort;
        discard_l2(buf + ((size_t)klo * B + (tid >> 2)) * a.P + v0 + 16 * (tid & 3));
        const int vv = tid & 63, gp = tid >> 6;
        pass2(v, sm, gp, vv);
        float2 *dst = gout + boff + colbase + v0 + vv;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const int khi = 2 * gp + h + 16 * kk;
                float2 y = make_float2(v[8 * h + kk].x, cs < 0.f ? -v[8 * h + kk].y : v[8 * h + kk].y);
                st_hint(dst + (long long)(klo + A * khi) * a.out_ld, y, policy_evict_first());
            }
    }
}

// Persistent kernel.  With PREFETCH (one CTA per SM) each thread keeps two
// register sets: while tile i is computed from one, the loads of tile i+1 are
// already in flight into the other (issued only when tile i+1's dependency is
// met, so a CTA never blocks while it holds an unfinished tile).  Without it
// (two CTAs per SM) the other CTA covers a CTA's load latency.
template <bool PREFETCH>
__global__ void __launch_bounds__(panel::NT, PREFETCH ? 1 : 2)
    paco_panel_kernel(const __grid_constant__ PanelArgs args)
{
    using namespace panel;
    extern __shared__ __align__(16) float2 sm[];          // A rows x SP
    __shared__ float2 w128[A];                           // w_128^{-r} = w_L^{-128 r}
    __shared__ float2 w16[128];                          // w_128^{-s t8} at [s*8 + t8]
    __shared__ float2 tlo[128];                          // w_L^{-r}, r < 128
    __shared__ float2 TW[512];                           // per-tile w_L table (A tiles)
    __shared__ float2 E1[64], E2[B];                     // stage-1 B tiles: w_N factors
    __shared__ unsigned rtab[16];                        // pi(1024 r)
    __shared__ int s_tile[3];                            // tile indices i, i+1, i+2
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x;
    const float2 *twL = reinterpret_cast<const float2 *>(args.twL);
    for (int r = tid; r < A; r += NT) {
        w128[r] = __ldg(twL + r * B);
        tlo[r] = __ldg(twL + r);
        w16[r] = __ldg(twL + ((r >> 3) * (r & 7)) * B);
    }
    if (tid < 16 && args.mode == 2)
        rtab[tid] = digit_reverse((unsigned)tid << 10, args.rev_bits, args.rev_t);
    if (tid == 0) {
        s_tile[0] = (int)atomicAdd(args.ctr, 1u);
        s_tile[1] = (int)atomicAdd(args.ctr, 1u);
        s_abort = 0;
    }
    const int lgT = args.lgP + 1;                        // T = 2 P tiles per phase
    const int total = (2 * args.npanels) << lgT;
    __syncthreads();

    cx<float> va[16];
    cx<float> vb[PREFETCH ? 16 : 1];
    Tile cur = decode_tile(s_tile[0], lgT, args.npanels);
    if (cur.g < total) {
        if (warp_acquire(args, cur, true) < 0) s_abort = 1;
        load_tile(args, cur, va, rtab);
    }

    // one iteration computes `cur` from X (and, with PREFETCH, loads the next
    // tile into Y ahead of time)
    auto step = [&](cx<float> *X, cx<float> *Y, int iter) -> bool {
        if (cur.g >= total) return false;
        bool have_next = false;
        if constexpr (PREFETCH) {
            const Tile nx = decode_tile(s_tile[(iter + 1) % 3], lgT, args.npanels);
            if (nx.g < total && warp_acquire(args, nx, false) == 1) {
                load_tile(args, nx, Y, rtab);
                have_next = true;
            }
        }
        unsigned nn = 0;
        if (tid == 0) nn = atomicAdd(args.ctr, 1u);           // index of tile i+2
        tile_tables(args, cur, TW, E1, E2, w128, tlo);
        int ab = 0;
        compute_tile(args, cur, X, sm, w16, TW, E1, E2, &s_abort, ab);
        if (tid == 0) s_tile[(iter + 2) % 3] = (int)nn;
        __syncthreads();
        if (ab) return false;
        if (tid == 0)
            red_release_add(args.ctr + 1 + (cur.isB ? args.npanels : 0) + cur.q, 1u);
        cur = decode_tile(s_tile[(iter + 1) % 3], lgT, args.npanels);
        if (cur.g < total && !have_next) {
            if (warp_acquire(args, cur, true) < 0) s_abort = 1;
            load_tile(args, cur, Y, rtab);
        }
        return true;
    };
    if constexpr (PREFETCH) {
        for (int iter = 0;; iter += 2) {
            if (!step(va, vb, iter)) break;
            if (!step(vb, va, iter + 1)) break;
        }
    } else {
        for (int iter = 0;; ++iter)
            if (!step(va, va, iter)) break;
    }
}


// ---------------------------------------------------------------------------
// TMA-fed variant: one CTA per SM, a ring of NSTAGE shared-memory stage
// buffers filled by bulk asynchronous copies (cp.async.bulk, completion on an
// mbarrier).  A stage buffer is first the landing zone of a tile's operands,
// then the exchange buffer between its two radix passes.  The copies of tile
// i+NSTAGE are issued as soon as tile i has released its buffer, so about
// NSTAGE-1 tiles of HBM reads are in flight per SM without holding registers.
// ---------------------------------------------------------------------------
namespace tma {

constexpr int NSTAGE = 3;
constexpr int STAGE_ELEMS = panel::A * panel::SP;       // 8448 (>= 8192 landing)
constexpr unsigned TILE_BYTES = panel::TILE * 8;        // 65536

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ unsigned mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok;
}
// global -> shared bulk copy; `bytes` and both addresses multiples of 16
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes,
                                          unsigned long long *bar, unsigned long long pol)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
                 " [%0], [%1], %2, [%3], %4;"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *map, int c0, int c1,
                                       unsigned long long *bar, unsigned long long pol)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
                 " [%0], [%1, {%2, %3}], [%4], %5;"
                 :: "r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar)), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void tma_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                       unsigned long long *bar, unsigned long long pol)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
                 " [%0], [%1, {%2, %3, %4}], [%5], %6;"
                 :: "r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void tma_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                       unsigned long long *bar, unsigned long long pol)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6], %7;"
                 :: "r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar)),
                    "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void tma_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                       int c4, unsigned long long *bar, unsigned long long pol)
{
    asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
                 " [%0], [%1, {%2, %3, %4, %5, %6}], [%7], %8;"
                 :: "r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
                    "r"(smem_u32(bar)), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Bounded wait for a stage buffer; returns 0 when it gave up.
__device__ __forceinline__ int wait_stage(unsigned long long *bar, unsigned parity, unsigned limit)
{
    unsigned it = 0;
    while (!mbar_try_wait(bar, parity))
        if (++it > limit) return 0;
    return 1;
}

// Warp 0 issues the bulk copies of tile d into stage buffer sbuf.  Landing
// layouts (elements of the 8192-element tile):
//   stage-1 A: (j_hi, jl, c) at (j_hi*4 + jl)*16 + c     512 copies of 128 B
//   stage-1 B: (k, j)        at k*128 + j                 1 copy of 64 KiB
//   stage-2 A: (j_hi, v)     at j_hi*64 + v               128 copies of 512 B
//   stage-2 B: (j, v)        at j*64 + v                  128 copies of 512 B
__device__ __forceinline__ void issue_tile(const PanelArgs &a, const Tile &d, float2 *sbuf,
                                           unsigned long long *bar)
{
    using namespace panel;
    const int lane = threadIdx.x & 31;
    if (lane == 0) mbar_expect_tx(bar, TILE_BYTES);
    __syncwarp();
    const int bidx = d.q >> a.lgPpb, pcol = d.q & (a.panels_per_batch - 1);
    const long long boff = (long long)bidx * a.batch_stride;
    const int colbase = pcol << a.lgP;
    const float2 *gin = reinterpret_cast<const float2 *>(a.in);
    const float2 *buf = panel_buf(a, d.q);
    if (a.use_tensor) {
        if (lane == 0) {
            const unsigned long long pol = policy_evict_first();
            if (a.mode == 1 && !d.isB) {
                const int j0 = (d.t >> (a.lgP - 4)) * 4, c0 = (d.t & ((a.P >> 4) - 1)) * 16;
                tma_4d(sbuf, &a.map_in, colbase + c0, j0, 0, bidx, bar, pol);
            } else if (a.mode == 1) {
                const int cl = d.t >> 1, k0 = (d.t & 1) * 64;
                bulk_load(sbuf, buf + ((size_t)cl * A + k0) * B, TILE_BYTES, bar, pol);
            } else if (!d.isB) {
                const int jlo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
                const unsigned uf = digit_reverse((unsigned)jlo, a.rev_bits, a.rev_t);  // row bits set by j_lo
                int c[5];
                c[0] = colbase + v0;
                const int R = a.map_rank;
                for (int k = 1; k < R; ++k) {
                    const int st = a.map_run_start[k - 1];
                    const int en = (k < R - 1) ? a.map_run_start[k] : a.rev_bits;
                    c[k] = a.map_run_fixed[k - 1] ? (int)((uf >> st) & ((1u << (en - st)) - 1u)) : 0;
                }
                c[R - 1] += bidx << (a.rev_bits - a.map_run_start[R - 2]);      // batch folded on top
                if (R == 3) tma_3d(sbuf, &a.map_in, c[0], c[1], c[2], bar, pol);
                else if (R == 4) tma_4d(sbuf, &a.map_in, c[0], c[1], c[2], c[3], bar, pol);
                else tma_5d(sbuf, &a.map_in, c[0], c[1], c[2], c[3], c[4], bar, pol);
            } else {
                const int klo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
                tma_2d(sbuf, &a.map_scr, v0, ((d.q % NBUF) << 14) + klo * B, bar, pol);
            }
        }
        return;
    }
    if (a.mode == 1 && !d.isB) {
        const unsigned long long pol = policy_evict_first();
        const int j0 = (d.t >> (a.lgP - 4)) * 4, c0 = (d.t & ((a.P >> 4) - 1)) * 16;
        const float2 *src0 = gin + boff + colbase + c0;
#pragma unroll 4
        for (int m = 0; m < 16; ++m) {
            const int idx = lane + 32 * m, jh = idx >> 2, jl = idx & 3;
            bulk_load(sbuf + idx * 16, src0 + (long long)(jh * B + j0 + jl) * a.C, 128, bar, pol);
        }
    } else if (a.mode == 1) {
        if (lane == 0) {
            const int cl = d.t >> 1, k0 = (d.t & 1) * 64;
            bulk_load(sbuf, buf + ((size_t)cl * A + k0) * B, TILE_BYTES, bar, policy_evict_first());
        }
    } else if (!d.isB) {
        const unsigned long long pol = policy_evict_first();
        const int jlo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
        const float2 *src0 = gin + boff + colbase + v0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int jh = lane + 32 * m;
            const unsigned row = digit_reverse((unsigned)(jlo + (jh << 7)), a.rev_bits, a.rev_t);
            bulk_load(sbuf + jh * 64, src0 + (long long)row * a.C, 512, bar, pol);
        }
    } else {
        const unsigned long long pol = policy_evict_first();
        const int klo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = lane + 32 * m;
            bulk_load(sbuf + j * 64, buf + ((size_t)klo * B + j) * a.P + v0, 512, bar, pol);
        }
    }
}

} // namespace tma

// Pass-1 operands of tile d from its landing layout.  `lrow[j_hi]` is the
// landing row of logical j_hi for stage-2 A tiles loaded by tensor TMA (the
// box keeps the physical row order of W).
__device__ __forceinline__ void read_landing(const PanelArgs &a, const Tile &d, cx<float> *v,
                                             const float2 *sbuf, const unsigned char *lrow)
{
    const int tid = threadIdx.x;
    if (a.mode == 1 && !d.isB) {
        const int cc = tid & 15, jl = (tid >> 4) & 3, t8 = tid >> 6;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const float2 x = sbuf[((t8 + 8 * r) * 4 + jl) * 16 + cc];
            v[r] = make_cx<float>(x.x, x.y);
        }
    } else if (a.mode == 1) {
        const int t8 = tid & 7, k = tid >> 3;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const float2 x = sbuf[k * 128 + t8 + 8 * r];
            v[r] = make_cx<float>(x.x, x.y);
        }
    } else if (!d.isB && a.use_tensor) {
        const int vv = tid & 63, t8 = tid >> 6;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const float2 x = sbuf[lrow[t8 + 8 * r] * 64 + vv];
            v[r] = make_cx<float>(x.x, x.y);
        }
    } else {
        const int vv = tid & 63, t8 = tid >> 6;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const float2 x = sbuf[(t8 + 8 * r) * 64 + vv];
            v[r] = make_cx<float>(x.x, x.y);
        }
    }
}

// Radix-16 pass of tile d in registers (conjugation of the stage input, DFT,
// w_128 twiddles); returns the thread's t8 and exchange slot.
__device__ __forceinline__ void pass1_regs(const PanelArgs &a, const Tile &d, cx<float> *v,
                                           const float2 *w16, int &t8, int &slot)
{
    using namespace panel;
    const int tid = threadIdx.x;
    if (a.mode == 1 && !d.isB) {
        const int cc = tid & 15, jl = (tid >> 4) & 3;
        t8 = tid >> 6;
        slot = slot_s1a(jl, cc);
    } else if (a.mode == 1) {
        t8 = tid & 7;
        slot = tid >> 3;
    } else {
        t8 = tid >> 6;
        slot = tid & 63;
    }
    if (!d.isB && a.conj) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r].y = -v[r].y;
    }
    dft16(v);
#pragma unroll
    for (int s = 1; s < 16; ++s) {
        const float2 w = w16[s * 8 + t8];
        const float2 p = f2mul(make_float2(v[s].x, v[s].y), w);
        v[s].x = p.x; v[s].y = p.y;
    }
}

// Radix-8 pass from the exchange layout and the stores of tile d.
__device__ __forceinline__ void pass2_store(const PanelArgs &a, const Tile &d, cx<float> *v,
                                            const float2 *sm, const float2 *TW, const float2 *E1,
                                            const float2 *E2)
{
    using namespace panel;
    const int tid = threadIdx.x;
    const int bidx = d.q >> a.lgPpb, pcol = d.q & (a.panels_per_batch - 1);
    const long long boff = (long long)bidx * a.batch_stride;
    const int colbase = pcol << a.lgP;
    float2 *buf = panel_buf(a, d.q);
    float2 *gout = reinterpret_cast<float2 *>(a.out);
    if (a.mode == 1 && !d.isB) {
        const int j0 = (d.t >> (a.lgP - 4)) * 4, c0 = (d.t & ((a.P >> 4) - 1)) * 16;
        const int jl = tid & 3, cc = (tid >> 2) & 15, gp = tid >> 6;
        pass2(v, sm, gp, slot_s1a(jl, cc));
        float2 *dst = buf + ((size_t)(c0 + cc) * A) * B + j0 + jl;
        const unsigned long long pol = policy_evict_last();
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int klo = 2 * gp + h + 16 * k;
                st_hint(dst + (size_t)klo * B, f2mul(make_float2(v[8 * h + k].x, v[8 * h + k].y), TW[klo * 4 + jl]), pol);
            }
    } else if (a.mode == 1) {
        const int cl = d.t >> 1, k0 = (d.t & 1) * 64;
        const unsigned cglob = (unsigned)(colbase + cl);
        const int k = tid & 63, gp = tid >> 6;
        pass2(v, sm, gp, k);
        const unsigned urow = digit_reverse(cglob, a.rev_bits, a.rev_t);
        float2 *dst = gout + boff + (long long)urow * a.out_ld + k0 + k;
        const float2 e1 = E1[k];
        const unsigned long long pol = policy_evict_first();
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const int khi = 2 * gp + h + 16 * kk;
                float2 y = f2mul(f2mul(make_float2(v[8 * h + kk].x, v[8 * h + kk].y), e1), E2[khi]);
                if (a.conj) y.y = -y.y;
                st_hint(dst + A * khi, y, pol);
            }
    } else if (!d.isB) {
        const int jlo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
        const int vv = tid & 63, gp = tid >> 6;
        pass2(v, sm, gp, vv);
        float2 *dst = buf + (size_t)jlo * a.P + v0 + vv;
        const unsigned long long pol = policy_evict_last();
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int klo = 2 * gp + h + 16 * k;
                st_hint(dst + (size_t)klo * B * a.P, f2mul(make_float2(v[8 * h + k].x, v[8 * h + k].y), TW[klo * 4]), pol);
            }
    } else {
        const int klo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
        const int vv = tid & 63, gp = tid >> 6;
        pass2(v, sm, gp, vv);
        float2 *dst = gout + boff + colbase + v0 + vv;
        const unsigned long long pol = policy_evict_first();
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const int khi = 2 * gp + h + 16 * kk;
                float2 y = make_float2(v[8 * h + kk].x, a.conj ? -v[8 * h + kk].y : v[8 * h + kk].y);
                st_hint(dst + (long long)(klo + A * khi) * a.out_ld, y, pol);
            }
    }
}

// Drop the consumed scratch lines of a B tile (one 128-byte line per thread).
__device__ __forceinline__ void discard_consumed(const PanelArgs &a, const Tile &d)
{
    using namespace panel;
    const int tid = threadIdx.x;
    const float2 *buf = panel_buf(a, d.q);
    if (a.mode == 1) {
        const int cl = d.t >> 1, k0 = (d.t & 1) * 64;
        discard_l2(buf + ((size_t)cl * A + k0) * B + 16 * tid);
    } else {
        const int klo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
        discard_l2(buf + ((size_t)klo * B + (tid >> 2)) * a.P + v0 + 16 * (tid & 3));
    }
}

// Lane 0 of the calling warp acquires `dep`; blocking (bounded) or one probe.
// Returns 1 when met, 0 when not (probe), -1 when a bounded wait gave up.
__device__ __forceinline__ int acquire_dep(const PanelArgs &a, const unsigned *dep, bool block)
{
    if (!dep) return 1;
    int ok = 0;
    if ((threadIdx.x & 31) == 0) {
        unsigned it = 0;
        for (;;) {
            if (panel::ld_acquire(dep) >= (unsigned)tiles_per_phase(a)) { ok = 1; break; }
            if (!block) break;
            if (++it > a.spin_limit) {
                atomicExch(a.status, 5 /* PACO_ERR_TIMEOUT */);
                ok = -1;
                break;
            }
            __nanosleep(100);
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok;
}

__device__ __forceinline__ void named_barrier_consumers()
{
    asm volatile("bar.sync 1, %0;" :: "n"(panel::NT) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tma::smem_u32(bar)) : "memory");
}

// Warp-specialised persistent kernel: warps 0..15 compute (consumers), warp
// 16 produces.  The producer takes tile indices from the queue in order,
// resolves each tile's dependency (bounded blocking waits are safe there: a
// tile only depends on tiles dequeued before it), and fills stage buffer
// i % NSTAGE with bulk copies once the consumers have released it; `full`
// carries the data, `empty` returns the buffer.  Tile info travels with the
// full barrier (written before the producer's release-arrive).
__global__ void __launch_bounds__(panel::NT + 32, 1) paco_panel_tma_kernel(const __grid_constant__ PanelArgs args)
{
    using namespace panel;
    using namespace tma;
    extern __shared__ __align__(1024) float2 stage[];     // NSTAGE x STAGE_ELEMS
    __shared__ __align__(8) unsigned long long full[NSTAGE], empty[NSTAGE];
    __shared__ float2 w128[A];
    __shared__ float2 w16[128];
    __shared__ float2 tlo[128];
    __shared__ float2 TW[512];
    __shared__ float2 E1[64], E2[B];
    __shared__ int s_info[NSTAGE];                       // tile index held by each stage
    __shared__ unsigned char lrow[A];                    // stage 2 (tensor): landing row of j_hi
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x;
    const float2 *twL = reinterpret_cast<const float2 *>(args.twL);
    for (int r = tid; r < A; r += blockDim.x) {
        w128[r] = __ldg(twL + r * B);
        tlo[r] = __ldg(twL + r);
        w16[r] = __ldg(twL + ((r >> 3) * (r & 7)) * B);
    }
    if (tid < A && args.mode == 2) {
        // landing row of j_hi: the spanned row bits of pi(j_hi * 128), packed
        const unsigned u = digit_reverse((unsigned)tid << 7, args.rev_bits, args.rev_t);
        unsigned r = 0;
        int o = 0;
        for (int bit = 0; bit < args.rev_bits; ++bit)
            if ((args.vmask >> bit) & 1u) r |= ((u >> bit) & 1u) << o++;
        lrow[tid] = (unsigned char)r;
    }
    if (tid == 0) {
        for (int k = 0; k < NSTAGE; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], 1);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int lgT = args.lgP + 1;
    const int total = (2 * args.npanels) << lgT;
    __syncthreads();

    if (tid >= NT) {
        // ---------------- producer warp ----------------
        const int lane = tid & 31;
        unsigned eparity = 0;
        for (int i = 0;; ++i) {
            const int b = i % NSTAGE;
            if (i >= NSTAGE) {
                int ok = 1;
                if (lane == 0) ok = wait_stage(&empty[b], (eparity >> b) & 1u, 1u << 22);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                eparity ^= 1u << b;
                if (!ok) s_abort = 1;
            }
            int g = 0;
            if (lane == 0) {
                g = (int)atomicAdd(args.ctr, 1u);
                if (s_abort) g = total;                      // stop: hand the consumers a terminator
            }
            g = __shfl_sync(0xffffffffu, g, 0);
            const Tile d = decode_tile(g, lgT, args.npanels);
            if (g < total) {
                if (acquire_dep(args, tile_dep(args, d), true) < 0) {
                    s_abort = 1;
                    g = total;
                }
            }
            if (lane == 0) s_info[b] = g;
            if (g >= total) {
                if (lane == 0) mbar_arrive(&full[b]);        // no data: consumers see the end
                break;
            }
            fence_async_global();                            // scratch written by other CTAs, then read by TMA
            fence_async_shared();                            // consumers' reads of stage b, then TMA writes
            issue_tile(args, d, stage + b * STAGE_ELEMS, &full[b]);
        }
        return;
    }

    // ---------------- consumer warps ----------------
    unsigned fparity = 0;
    cx<float> v[16];
    for (int i = 0;; ++i) {
        const int b = i % NSTAGE;
        float2 *sbuf = stage + b * STAGE_ELEMS;
        if (!wait_stage(&full[b], (fparity >> b) & 1u, 1u << 22)) s_abort = 1;
        fparity ^= 1u << b;
        const int g = s_info[b];                             // same for every consumer
        if (g >= total) break;
        const Tile d = decode_tile(g, lgT, args.npanels);
        if (d.isB) discard_consumed(args, d);
        tile_tables(args, d, TW, E1, E2, w128, tlo);
        read_landing(args, d, v, sbuf, lrow);
        int t8, slot;
        pass1_regs(args, d, v, w16, t8, slot);
        named_barrier_consumers();                           // landing reads done
#pragma unroll
        for (int s = 0; s < 16; ++s) sbuf[(t8 + 8 * s) * SP + slot] = make_float2(v[s].x, v[s].y);
        named_barrier_consumers();                           // exchange and tables written
        pass2_store(args, d, v, sbuf, TW, E1, E2);
        named_barrier_consumers();                           // stage b and tables free; stores issued
        if (tid == 0) {
            red_release_add(args.ctr + 1 + (d.isB ? args.npanels : 0) + d.q, 1u);
            mbar_arrive(&empty[b]);
        }
    }
}

#endif // PACO_PANEL_KERNEL_TU

} // namespace paco
