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
// intermediate lives in a ring of NBUF panel buffers sized to stay in L2 and
// its lines are discarded from L2 once consumed, so they are never written
// back.  The tiles run in the order A0 | A1 B0 | A2 B1 | ... | B(np-1): a B
// tile needs all A tiles of its panel; an A tile needs the panel that last
// used its buffer to be consumed.
//
// One persistent CTA per SM: a producer warp takes tiles from a global queue
// in order, resolves their dependencies (bounded waits that record
// PACO_ERR_TIMEOUT), builds the tile's twiddle tables and fills a ring of
// NSTAGE shared-memory stage buffers with one tiled tensor TMA per tile
// (cp.async.bulk.tensor, completion on an mbarrier).  Sixteen consumer warps
// compute: every tile is 8192 elements, 16 per thread; a 128-point DFT is
// radix 16 in registers, an exchange through the stage buffer (which first
// was the tile's landing zone), then radix 8.
#pragma once

#include <cuda.h>                 // CUtensorMap (type only)

#include "paco_common.cuh"

namespace paco {

struct PanelArgs {
    // Tensor maps (__grid_constant__ parameter, 64-byte aligned):
    //   map_in:  stage 1: X as (c, j_lo, j_hi, batch), box (16, 4, 128, 1);
    //            stage 2: the rows of W split into runs of the bits that
    //            pi_m2(j_lo + 128 j_hi) spans over j_hi (box: the run) or
    //            fixes by j_lo (box 1), plus the columns, box 64 wide.
    //   map_scr: stage 1: the scratch ring as (j_lo & 7, k_lo, j_lo >> 3, c),
    //            box (8, 64, 16, 1); stage 2: as (v, rows), box (64, 128).
    CUtensorMap map_in;
    CUtensorMap map_scr;
    int map_rank;                  // rank of map_in (stage 2)
    int map_run_start[4];          // stage 2: first row bit of each row dimension
    int map_run_fixed[4];          // 1: the run is fixed by j_lo (box 1), 0: spanned
    unsigned vmask;                // stage 2: row bits spanned by j_hi
    const void *in;                // stage input (batch of N elements)
    void *out;                     // stage output
    void *scratch;                 // NBUF panel buffers of L*P elements
    unsigned *ctr;                 // [0] tile queue, [1..np] A done, [np+1..2np] B done
    int *status;                   // device status word (PACO_ERR_TIMEOUT)
    long long batch_stride;
    int C;                         // columns of the stage input matrix
    int out_ld;                    // row length of the output matrix
    int P;                         // panel width (columns), a power of two >= 64
    int lgP;                       // log2 P
    int panels_per_batch;          // C / P (a power of two)
    int lgPpb;                     // log2 panels_per_batch
    int npanels;                   // batch * C / P
    int mode;                      // 1: stage 1 fused with the middle stage; 2: stage 2
    int rev_bits, rev_t;           // digit reversal pi_m2
    const void *twL;               // w_L^{-r}, r < L
    const void *twN_lo, *twN_hi;
    int twN_lo_bits;
    unsigned N_mask;
    int conj;
    unsigned spin_limit;
    int use_tensor;                // 1: tiles arrive by tensor TMA, 0: by bulk copies
    unsigned dep_bias;             // added to every dependency target (0; tests of the bounded waits)
};

namespace panel {

constexpr int A = 128, B = 128, L = A * B;
constexpr int SP = 66;              // exchange row stride (elements): conflict-free passes
constexpr int NT = 512;             // consumer threads per CTA
constexpr int TILE = 8192;          // elements per tile
constexpr int NBUF = 3;             // panel buffers in the L2 ring
constexpr int NSTAGE = 3;           // shared-memory stage buffers
constexpr int STAGE_ELEMS = A * SP; // 8448 (>= 8192 landing)
constexpr unsigned TILE_BYTES = TILE * 8;

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

// Twiddles of a thread computed in registers from a few table entries (a
// shared-memory read costs more than the products here: the consumers are
// bound by shared-memory traffic).  seq8: out[k] = b * s^k, k < 8, from b,
// s and s^4; at most four roundings on top of the tables'.
__device__ __forceinline__ void seq8(float2 *out, float2 b, float2 s1, float2 s4)
{
    const float2 s2 = f2mul(s1, s1), s3 = f2mul(s2, s1);
    out[0] = b;
    out[1] = f2mul(b, s1);
    out[2] = f2mul(b, s2);
    out[3] = f2mul(b, s3);
    const float2 b4 = f2mul(b, s4);
    out[4] = b4;
    out[5] = f2mul(b4, s1);
    out[6] = f2mul(b4, s2);
    out[7] = f2mul(b4, s3);
}

// exchange slot of sequence (jl, c) in the stage-1 A tile: conflict-free both
// when lanes run over c (pass 1) and over jl then c (pass 2)
__device__ __forceinline__ int slot_s1a(int jl, int c) { return c * 4 + (jl ^ ((c >> 2) & 3)); }

// Pass 2: groups g = 2 gp + h (h < 2): radix 8 over t of exchange rows g*8 + t;
// the output k' of group g is DFT index k = g + 16 k', left in v[8 h + k'].
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

// ---- mbarrier / TMA ------------------------------------------------------
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
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ unsigned mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok;
}
// Bounded wait for an mbarrier phase; returns 0 when it gave up.
__device__ __forceinline__ int mbar_wait(unsigned long long *bar, unsigned parity, unsigned limit)
{
    unsigned it = 0;
    while (!mbar_try_wait(bar, parity))
        if (++it > limit) return 0;
    return 1;
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
__device__ __forceinline__ void named_barrier_consumers()
{
    asm volatile("bar.sync 1, %0;" :: "n"(NT) : "memory");
}

} // namespace panel

#ifdef PACO_PANEL_KERNEL_TU

// One decoded tile of the order A0 | A1 B0 | A2 B1 | ... | B(np-1).
struct Tile {
    int g;         // position in the order (>= total: none)
    int isB, q, t;
};

__device__ __forceinline__ Tile decode_tile(int g, int lgT, int np)
{
    Tile d;
    d.g = g;
    const unsigned gu = (unsigned)g;
    const int bi = (int)(gu >> lgT);
    d.t = (int)(gu & ((1u << lgT) - 1u));
    if (bi == 0) { d.isB = 0; d.q = 0; }
    else if (bi == 2 * np - 1) { d.isB = 1; d.q = np - 1; }
    else { d.q = (bi + 1) / 2; d.isB = !(bi & 1); if (d.isB) d.q -= 1; }
    return d;
}

// tiles per phase per panel: L * P / TILE = 2 P
__device__ __forceinline__ int tiles_per_phase(const PanelArgs &a) { return 2 << a.lgP; }

// the counter a tile waits on, or nullptr
__device__ __forceinline__ const unsigned *tile_dep(const PanelArgs &a, const Tile &d)
{
    if (d.isB) return a.ctr + 1 + d.q;
    if (d.q >= panel::NBUF) return a.ctr + 1 + a.npanels + (d.q - panel::NBUF);
    return nullptr;
}

__device__ __forceinline__ float2 *panel_buf(const PanelArgs &a, int q)
{
    return reinterpret_cast<float2 *>(a.scratch) + ((size_t)(q % panel::NBUF) << (14 + a.lgP));
}

// Lane 0 of the calling warp acquires `dep` (bounded blocking wait).
// Returns 1 when met, -1 when the wait gave up.
__device__ __forceinline__ int acquire_dep(const PanelArgs &a, const unsigned *dep)
{
    if (!dep) return 1;
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
        unsigned it = 0;
        while (panel::ld_acquire(dep) < (unsigned)tiles_per_phase(a) + a.dep_bias) {
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

// ---- producer -------------------------------------------------------------

// The copies of tile d into stage buffer sbuf (warp-wide call).  Landing
// layouts (elements of the 8192-element tile):
//   stage-1 A: (j_hi, jl, c)        at (j_hi*4 + jl)*16 + c
//   stage-1 B: (j_lo>>3, k, j_lo&7) at ((j_lo>>3)*64 + k)*8 + (j_lo&7)
//   stage-2 A: (landing row of j_hi, v) at lrow(j_hi)*64 + v  (tensor form);
//              (j_hi, v) at j_hi*64 + v (bulk form)
//   stage-2 B: (j, v)               at j*64 + v
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
    const unsigned long long pol = policy_evict_first();
    if (a.use_tensor) {
        if (lane != 0) return;
        if (a.mode == 1 && !d.isB) {
            const int j0 = (d.t >> (a.lgP - 4)) * 4, c0 = (d.t & ((a.P >> 4) - 1)) * 16;
            tma_4d(sbuf, &a.map_in, colbase + c0, j0, 0, bidx, bar, pol);
        } else if (a.mode == 1) {
            const int cl = d.t >> 1, k0 = (d.t & 1) * 64;
            tma_4d(sbuf, &a.map_scr, 0, k0, 0, ((d.q % NBUF) << a.lgP) + cl, bar, pol);
        } else if (!d.isB) {
            const int jlo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
            const unsigned uf = digit_reverse((unsigned)jlo, a.rev_bits, a.rev_t);   // row bits fixed by j_lo
            int c[5];
            c[0] = colbase + v0;
            const int R = a.map_rank;
            for (int k = 1; k < R; ++k) {
                const int st = a.map_run_start[k - 1];
                const int en = (k < R - 1) ? a.map_run_start[k] : a.rev_bits;
                c[k] = a.map_run_fixed[k - 1] ? (int)((uf >> st) & ((1u << (en - st)) - 1u)) : 0;
            }
            c[R - 1] += bidx << (a.rev_bits - a.map_run_start[R - 2]);         // batch on the top run
            if (R == 3) tma_3d(sbuf, &a.map_in, c[0], c[1], c[2], bar, pol);
            else if (R == 4) tma_4d(sbuf, &a.map_in, c[0], c[1], c[2], c[3], bar, pol);
            else tma_5d(sbuf, &a.map_in, c[0], c[1], c[2], c[3], c[4], bar, pol);
        } else {
            const int klo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
            tma_2d(sbuf, &a.map_scr, v0, ((d.q % NBUF) << 14) + klo * B, bar, pol);
        }
        return;
    }
    // bulk-copy form (no tensor maps): one copy per contiguous run
    if (a.mode == 1 && !d.isB) {
        const int j0 = (d.t >> (a.lgP - 4)) * 4, c0 = (d.t & ((a.P >> 4) - 1)) * 16;
        const float2 *src0 = gin + boff + colbase + c0;
        for (int m = 0; m < 16; ++m) {
            const int idx = lane + 32 * m, jh = idx >> 2, jl = idx & 3;
            bulk_load(sbuf + idx * 16, src0 + (long long)(jh * B + j0 + jl) * a.C, 128, bar, pol);
        }
    } else if (a.mode == 1) {
        const int cl = d.t >> 1, k0 = (d.t & 1) * 64;
        if (lane < 16)
            bulk_load(sbuf + lane * 512, buf + (((size_t)cl * 16 + lane) * A + k0) * 8, 4096, bar, pol);
    } else if (!d.isB) {
        const int jlo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
        const float2 *src0 = gin + boff + colbase + v0;
        for (int m = 0; m < 4; ++m) {
            const int jh = lane + 32 * m;
            const unsigned row = digit_reverse((unsigned)(jlo + (jh << 7)), a.rev_bits, a.rev_t);
            bulk_load(sbuf + jh * 64, src0 + (long long)row * a.C, 512, bar, pol);
        }
    } else {
        const int klo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
        for (int m = 0; m < 4; ++m) {
            const int j = lane + 32 * m;
            bulk_load(sbuf + j * 64, buf + ((size_t)klo * B + j) * a.P + v0, 512, bar, pol);
        }
    }
}

// Twiddle tables of tile d for its stage (warp-wide call by the producer):
//   A tiles: TW[k_lo*4 + jl] = w_L^{-k_lo j_lo}   (stage 2: jl = 0 only)
//   stage-1 B: E1[k] = w_N^{-(k0+k) c},  E2[k_hi] = w_N^{-128 k_hi c}
__device__ __forceinline__ void build_tables(const PanelArgs &a, const Tile &d, float2 *TW,
                                             float2 *E1, float2 *E2, const float2 *w128,
                                             const float2 *tlo)
{
    using namespace panel;
    const int lane = threadIdx.x & 31;
    if (!d.isB) {
        if (a.mode == 1) {
            const int j0 = (d.t >> (a.lgP - 4)) * 4;
            for (int e = lane; e < 512; e += 32) {
                const int klo = e >> 2, jl = e & 3;
                const unsigned rr = (unsigned)(klo * (j0 + jl));                 // < L
                TW[e] = f2mul(tlo[rr & 127], w128[rr >> 7]);
            }
        } else {
            const int jlo = d.t >> (a.lgP - 6);
            for (int klo = lane; klo < A; klo += 32) {
                const unsigned rr = (unsigned)(klo * jlo);
                TW[klo * 4] = f2mul(tlo[rr & 127], w128[rr >> 7]);
            }
        }
    } else if (a.mode == 1) {
        const int pcol = d.q & (a.panels_per_batch - 1);
        const unsigned cglob = (unsigned)((pcol << a.lgP) + (d.t >> 1));
        const int k0 = (d.t & 1) * 64;
        const float2 *nlo = reinterpret_cast<const float2 *>(a.twN_lo);
        const float2 *nhi = reinterpret_cast<const float2 *>(a.twN_hi);
        const unsigned lomask = (1u << a.twN_lo_bits) - 1u;
        constexpr int PER = (64 + B) / 32;                   // 6 entries per lane
        float2 lo[PER], hi[PER];
#pragma unroll
        for (int m = 0; m < PER; ++m) {                      // all loads in flight first
            const int e = lane + 32 * m;
            const unsigned r = (e < 64) ? (((unsigned)(k0 + e) * cglob) & a.N_mask)
                                        : (((unsigned)A * (unsigned)(e - 64) * cglob) & a.N_mask);
            lo[m] = __ldg(nlo + (r & lomask));
            hi[m] = __ldg(nhi + (r >> a.twN_lo_bits));
        }
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int e = lane + 32 * m;
            const float2 w = f2mul(lo[m], hi[m]);
            if (e < 64) E1[e] = w; else E2[e - 64] = w;
        }
    }
}

// ---- consumers ------------------------------------------------------------

// Pass-1 operands of tile d from its landing layout; lrow[j_hi] is the landing
// row of logical j_hi for stage-2 A tiles that arrive by tensor TMA (the box
// keeps the physical row order of W).
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
        const int t8 = tid & 7, k = tid >> 3;                 // lanes over (t8, k): consecutive words
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const float2 x = sbuf[(r * 64 + k) * 8 + t8];
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
// w_128^{-s t8} twiddles from w16[s*8 + t8]); returns the thread's t8 and its
// exchange slot.
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
    // w_128^{-s t8} = z^s, z = w_128^{-t8}: z^(4a + c) = z4^a * z^c from the
    // table entries z, z^4, z^8 (s = 1, 4, 8 of w16[s * 8 + t8])
    const float2 z1 = w16[8 + t8], z4 = w16[32 + t8], z8 = w16[64 + t8];
    const float2 z2 = f2mul(z1, z1), z3 = f2mul(z2, z1), z12 = f2mul(z8, z4);
    const float2 zl[4] = {make_float2(1.f, 0.f), z1, z2, z3};
    const float2 zh[4] = {make_float2(1.f, 0.f), z4, z8, z12};
#pragma unroll
    for (int s = 1; s < 16; ++s) {
        float2 w;
        if ((s & 3) == 0) w = zh[s >> 2];
        else if ((s >> 2) == 0) w = zl[s & 3];
        else w = f2mul(zh[s >> 2], zl[s & 3]);
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
        // scratch layout [c][j_lo >> 3][k_lo][j_lo & 7]
        const int j0 = (d.t >> (a.lgP - 4)) * 4, c0 = (d.t & ((a.P >> 4) - 1)) * 16;
        const int jl = tid & 3, cc = (tid >> 2) & 15, gp = tid >> 6;
        pass2(v, sm, gp, slot_s1a(jl, cc));
        const int jlo = j0 + jl;
        float2 *dst = buf + ((size_t)(c0 + cc) * 16 + (jlo >> 3)) * (A * 8) + (jlo & 7);
        const unsigned long long pol = policy_evict_last();
        // TW[klo][jl] = w_L^{-klo jlo}, klo = 2 gp + h + 16 k: b_h * s^k
        const float2 s1 = TW[16 * 4 + jl], s4 = TW[64 * 4 + jl];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 tw[8];
            seq8(tw, TW[(2 * gp + h) * 4 + jl], s1, s4);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int klo = 2 * gp + h + 16 * k;
                st_hint(dst + klo * 8, f2mul(make_float2(v[8 * h + k].x, v[8 * h + k].y), tw[k]), pol);
            }
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
        // E2[khi] = w_N^{-128 khi c}, khi = 2 gp + h + 16 kk: (e1 E2[2 gp + h]) * s^kk
        const float2 s1 = E2[16], s4 = E2[64];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 tw[8];
            seq8(tw, f2mul(e1, E2[2 * gp + h]), s1, s4);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const int khi = 2 * gp + h + 16 * kk;
                float2 y = f2mul(make_float2(v[8 * h + kk].x, v[8 * h + kk].y), tw[kk]);
                if (a.conj) y.y = -y.y;
                st_hint(dst + A * khi, y, pol);
            }
        }
    } else if (!d.isB) {
        // scratch layout [k_lo][j_lo][v]
        const int jlo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
        const int vv = tid & 63, gp = tid >> 6;
        pass2(v, sm, gp, vv);
        float2 *dst = buf + (size_t)jlo * a.P + v0 + vv;
        const unsigned long long pol = policy_evict_last();
        // TW[klo] = w_L^{-klo jlo}, klo = 2 gp + h + 16 k: b_h * s^k
        const float2 s1 = TW[16 * 4], s4 = TW[64 * 4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 tw[8];
            seq8(tw, TW[(2 * gp + h) * 4], s1, s4);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int klo = 2 * gp + h + 16 * k;
                st_hint(dst + (size_t)klo * B * a.P, f2mul(make_float2(v[8 * h + k].x, v[8 * h + k].y), tw[k]), pol);
            }
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
        discard_l2(buf + (((size_t)cl * 16 + (tid >> 5)) * A + k0) * 8 + 16 * (tid & 31));
    } else {
        const int klo = d.t >> (a.lgP - 6), v0 = (d.t & ((a.P >> 6) - 1)) * 64;
        discard_l2(buf + ((size_t)klo * B + (tid >> 2)) * a.P + v0 + 16 * (tid & 3));
    }
}

// Warps 0..15 consume, warp 16 produces.  The producer takes tile indices in
// queue order, resolves each tile's dependency (a bounded blocking wait is
// safe there: a tile depends only on tiles dequeued before it), builds its
// twiddle tables and fills stage buffer i % NSTAGE once the consumers have
// released it; `full` carries data and tables, `empty` returns the buffer.
__global__ void __launch_bounds__(panel::NT + 32, 1)
    paco_panel_kernel(const __grid_constant__ PanelArgs args)
{
    using namespace panel;
    extern __shared__ __align__(1024) float2 stage[];     // NSTAGE x STAGE_ELEMS
    __shared__ __align__(8) unsigned long long full[NSTAGE], empty[NSTAGE];
    __shared__ float2 w128[A];                           // w_128^{-r} = w_L^{-128 r}
    __shared__ float2 w16[128];                          // w_128^{-s t8} at [s*8 + t8]
    __shared__ float2 tlo[128];                          // w_L^{-r}, r < 128
    __shared__ float2 TWs[NSTAGE][512];                  // per-stage w_L table (A tiles)
    __shared__ float2 E1s[NSTAGE][64], E2s[NSTAGE][B];   // per-stage w_N factors (stage-1 B)
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
    const int lgT = args.lgP + 1;                        // T = 2 P tiles per phase
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
                if (lane == 0) ok = mbar_wait(&empty[b], (eparity >> b) & 1u, 1u << 22);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                eparity ^= 1u << b;
                if (!ok && lane == 0) s_abort = 1;
            }
            int g = 0;
            if (lane == 0) {
                g = (int)atomicAdd(args.ctr, 1u);
                if (s_abort) g = total;                      // stop: hand the consumers a terminator
            }
            g = __shfl_sync(0xffffffffu, g, 0);
            const Tile d = decode_tile(g, lgT, args.npanels);
            if (g < total && acquire_dep(args, tile_dep(args, d)) < 0) {
                if (lane == 0) s_abort = 1;
                g = total;
            }
            if (lane == 0) s_info[b] = g;
            if (g >= total) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[b]);        // no data: consumers see the end
                break;
            }
            build_tables(args, d, TWs[b], E1s[b], E2s[b], w128, tlo);
            __syncwarp();                                    // tables written before the arrive
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
        if (!mbar_wait(&full[b], (fparity >> b) & 1u, 1u << 22)) s_abort = 1;
        fparity ^= 1u << b;
        const int g = s_info[b];                             // the same for every consumer
        if (g >= total) break;
        const Tile d = decode_tile(g, lgT, args.npanels);
        if (d.isB) discard_consumed(args, d);
        read_landing(args, d, v, sbuf, lrow);
        int t8, slot;
        pass1_regs(args, d, v, w16, t8, slot);
        named_barrier_consumers();                           // landing reads done
#pragma unroll
        for (int s = 0; s < 16; ++s) sbuf[(t8 + 8 * s) * SP + slot] = make_float2(v[s].x, v[s].y);
        named_barrier_consumers();                           // exchange written
        pass2_store(args, d, v, sbuf, TWs[b], E1s[b], E2s[b]);
        named_barrier_consumers();                           // stage b free; stores issued
        if (tid == 0) {
            red_release_add(args.ctr + 1 + (d.isB ? args.npanels : 0) + d.q, 1u);
            mbar_arrive(&empty[b]);
        }
    }
}

#endif // PACO_PANEL_KERNEL_TU

} // namespace paco
