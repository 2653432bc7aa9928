// paco_panel.cuh -- L2-resident panel pipeline for a length-2^14 stage.
//
// The paper's local FFT on one slab is CO-Batched-FFT with n = L and
// s = slab width: a balanced transform split n = n1*n2 (here 128 x 128) into
// a first child group (s*n2 DFTs of length n1 over j_hi) and a second child
// group (s*n1 DFTs of length n2 over j_lo) with the layout-aware twiddle
// w_L^{-k_lo j_lo} between them (Sect. 4.1, Fig. "cofft", Eq. twop).  The
// analysis places the recursion frontier where a view fits in cache; on
// GB300 the cache that holds a slab is the 129 MB L2.  So each stage runs the
// two child groups of one panel (a group of P columns) as two sub-passes:
//
//   sub-pass A: 128-point DFTs over j_hi of tiles read from HBM; twiddle
//               w_L^{-k_lo j_lo}; written to an L2-resident panel buffer;
//   sub-pass B: 128-point DFTs over j_lo of that buffer; stage epilogue
//               (mode 1: top-level twiddle w_N^{-k1 c} and the digit-reversed
//               row pi_m2(c) of W, Eq. (17); mode 2: natural-order output).
//
// HBM is touched once per element per direction (the paper's two passes); the
// intermediate lives in a ring of NBUF panel buffers sized to stay in L2 and
// its lines are discarded from L2 once consumed, so they are never written
// back.  Tiles run in the order A0 | A1 B0 | A2 B1 | ... | B(np-1): a B tile
// needs all A tiles of its panel; an A tile needs the panel that last used
// its buffer to be consumed.
//
// One persistent CTA per SM, three roles and no CTA-wide barrier:
//   * a producer warp claims tiles from a global queue in order (one claim
//     ahead), resolves their dependencies (bounded waits that record
//     PACO_ERR_TIMEOUT) and lands each tile in one of NSTAGE shared-memory
//     stage buffers with two tiled tensor TMA loads (boxes of 16 sequences x
//     128 points, 128-byte swizzle); a table warp builds the tile's twiddle
//     tables while the loads fly;
//   * sixteen consumer warps in two groups of eight take alternate tiles; each
//     warp owns four whole sequences of its tile: radix 16 in registers, the
//     radix-16 -> radix-8 exchange inside the warp's own part of the stage
//     buffer (warp synchronisation only), radix 8, the output twiddle;
//     results are written back in place (or, for stage-1 A tiles, stored to
//     the panel buffer with 16-byte stores);
//   * a storer warp writes each finished tile out with two TMA tensor stores
//     (one store group in flight) and returns stage buffers to the producer
//     once the stores have read them;
//   * a publisher warp makes the completed tiles count: the storer hands it
//     each completion through a shared-memory ring, and it publishes them to
//     the panel counters other CTAs wait on, one GPU-scope fence per batch
//     (the fence is the costly part, so it stays off the storer's path).
// The 128-byte swizzle makes every shared-memory access of a warp (landing
// reads, both sides of the exchange, the output staging) conflict-free.
#pragma once

#include <cuda.h>                 // CUtensorMap (type only)

#include "paco_common.cuh"

namespace paco {

struct PanelArgs {
    // Tensor maps (__grid_constant__ parameter, 64-byte aligned), all with
    // 8-byte elements, 128-byte swizzle and 16-element inner boxes:
    //   map_ld:     A-tile loads.  Stage 1: X as (c, j_lo, j_hi + 128 batch),
    //               box (16, 1, 128).  Stage 2: the rows pi_m2(j_lo + 128 j_hi)
    //               of W split into runs of row bits (see panel_prepare).
    //   map_ld_alt: stage 2 with b = 4: map_ld moved by 64 rows (row bit 6,
    //               fixed by j_lo, selects the map).
    //   map_scr_ld: B-tile loads from the panel ring, box (16, 128, 1).
    //   map_scr_st: stage 2: A-tile stores into the panel ring, box (16, 1, 128).
    //   map_out:    B-tile stores.  Stage 1: W as (k_lo, k_hi, u + N2 batch),
    //               box (16, 128, 1); stage 2: Y as (v, k_lo, k_hi + 128 batch),
    //               box (16, 1, 128).
    CUtensorMap map_ld;
    CUtensorMap map_ld_alt;
    CUtensorMap map_scr_ld;
    CUtensorMap map_scr_st;
    CUtensorMap map_out;
    void *scratch;                 // NBUF panel buffers of L*P elements
    unsigned *ctr;                 // [0] tile queue, [1..np] A done, [np+1..2np] B done
    int *status;                   // device status word (PACO_ERR_TIMEOUT)
    int P;                         // panel width (columns), a power of two >= 64
    int lgP;
    int panels_per_batch;          // C / P (a power of two)
    int lgPpb;
    int npanels;                   // batch * C / P
    int N2rows;                    // stage 1: rows of W per transform (N2)
    int rev_bits, rev_t;           // digit reversal pi_m2
    const void *twL;               // w_L^{-r}, r < L
    const void *twN_lo, *twN_hi;   // w_N^{-r} in two levels (stage 1)
    int twN_lo_bits;
    unsigned N_mask;
    int conj;                      // 1: conjugate on load and store (dir = +1)
    unsigned spin_limit;           // poll limit of the dependency waits
    unsigned dep_bias;             // added to every dependency target (0; tests of the bounded waits)
};

namespace panel {

constexpr int A = 128, B = 128, L = A * B;
constexpr int NCW = 16;                  // consumer warps
constexpr int WPG = 8;                   // consumer warps per group (one tile)
constexpr int NT = (NCW + 4) * 32;       // + producer, storer, table and publisher warps
constexpr int PQ = 64;                   // completions the storer may hand the publisher at once
constexpr int TILE = 4096;               // elements per tile (32 sequences x 128)
constexpr int NBOX = 2;                  // TMA boxes per tile
constexpr int NBUF = 3;                  // panel buffers in the L2 ring
constexpr int NSTAGE = 6;                // shared-memory stage buffers
constexpr unsigned BOX_BYTES = 16384;    // 16 sequences x 128 points x 8 B
constexpr unsigned TILE_BYTES = NBOX * BOX_BYTES;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // give up an mbarrier wait after 2 s

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
__device__ __forceinline__ void st_v4_hint(void *p, float4 v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;"
                 :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol) : "memory");
}
__device__ __forceinline__ void red_relaxed_add(unsigned *p, unsigned v)
{
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// drop a consumed 128-byte scratch line from L2 without writing it back
__device__ __forceinline__ void discard_l2(const void *p)
{
    asm volatile("discard.global.L2 [%0], 128;" :: "l"(p) : "memory");
}

__device__ __forceinline__ float2 f2mul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
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
// non-blocking test of the completion of the phase of the given parity
__device__ __forceinline__ unsigned mbar_test(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok;
}
// try_wait with a suspend-time hint: the thread sleeps until the phase
// completes or about 0.5 ms pass, instead of spinning on the issue slots.
__device__ __forceinline__ unsigned mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity), "r"(500000u) : "memory");
    return ok;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the completion of the mbarrier phase of the given parity;
// returns 0 when it gave up after `limit_ns` nanoseconds.
__device__ __forceinline__ int mbar_wait(unsigned long long *bar, unsigned parity, unsigned long long limit_ns)
{
    if (mbar_try_wait(bar, parity)) return 1;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return 0;
    return 1;
}
__device__ __forceinline__ void tma_ld_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                          unsigned long long *bar, unsigned long long pol)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
                 " [%0], [%1, {%2, %3, %4}], [%5], %6;"
                 :: "r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void tma_ld_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                          unsigned long long *bar, unsigned long long pol)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6], %7;"
                 :: "r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar)),
                    "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void tma_ld_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                          int c4, unsigned long long *bar, unsigned long long pol)
{
    asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
                 " [%0], [%1, {%2, %3, %4, %5, %6}], [%7], %8;"
                 :: "r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
                    "r"(smem_u32(bar)), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void tma_st_3d(const CUtensorMap *map, int c0, int c1, int c2, const void *src,
                                          unsigned long long pol)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group.L2::cache_hint"
                 " [%0, {%1, %2, %3}], [%4], %5;"
                 :: "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src)), "l"(pol) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait1() { asm volatile("cp.async.bulk.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

__device__ __forceinline__ float2 lds2(unsigned addr)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void sts2(unsigned addr, float2 v)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" :: "r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// Stage-2 A tiles (rows of W read through the digit reversal): the landing
// row of logical j_hi = t8 + 8 s is lo(t8) + 8 hi(s), fixed by the order of
// the row dimensions of map_ld (see panel_prepare).  b = 2: the row
// dimensions are (pi bits 4-6, pi bits 0-3): lo = 3-bit reversal, hi = 4-bit
// reversal.  b = 4: (pi bit 7, pi bits 4-5, pi bits 0-3): lo = identity,
// hi swaps the two bit pairs of s.
template <int B2>
__host__ __device__ constexpr int land_lo(int t8)
{
    return B2 == 2 ? (((t8 & 1) << 2) | (t8 & 2) | ((t8 >> 2) & 1)) : t8;
}
template <int B2>
__host__ __device__ constexpr int land_hi(int s)
{
    return B2 == 2 ? (((s & 1) << 3) | ((s & 2) << 1) | ((s >> 1) & 2) | ((s >> 3) & 1))
         : B2 == 4 ? (((s & 3) << 2) | ((s >> 2) & 3))
                   : s;
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

// tiles per phase per panel: L * P / TILE = 4 P; a panel's counters complete there
__device__ __forceinline__ unsigned tiles_per_phase(const PanelArgs &a) { return 4u << a.lgP; }

// the counter a tile waits on, or nullptr
__device__ __forceinline__ const unsigned *tile_dep(const PanelArgs &a, const Tile &d)
{
    if (d.isB) return a.ctr + 1 + d.q;
    if (d.q >= panel::NBUF) return a.ctr + 1 + a.npanels + (d.q - panel::NBUF);
    return nullptr;
}
// the counter a tile's completion counts towards
__device__ __forceinline__ unsigned *tile_ctr(const PanelArgs &a, const Tile &d)
{
    return a.ctr + 1 + (d.isB ? a.npanels : 0) + d.q;
}

// Tile coordinates inside its panel (32 sequences).  Consecutive tiles cover
// neighbouring column blocks of the same rows, so the CTAs working at one
// time read and write whole 1 KiB panel rows:
//   A tiles:     j_lo = t >> (lgP - 5), 32 columns from c0 = 32 (t & (P/32 - 1))
//   stage-1 B:   column cl = t >> 2, 32 k_lo from k0 = 32 (t & 3)
//   stage-2 B:   k_lo = t >> (lgP - 5), 32 columns from v0 = 32 (t & (P/32 - 1))
__device__ __forceinline__ int tile_hi(const PanelArgs &a, const Tile &d, int mode)
{
    return (mode == 1 && d.isB) ? (d.t >> 2) : (d.t >> (a.lgP - 5));
}
__device__ __forceinline__ int tile_lo32(const PanelArgs &a, const Tile &d, int mode)
{
    return (mode == 1 && d.isB) ? ((d.t & 3) << 5) : ((d.t & ((a.P >> 5) - 1)) << 5);
}

// Lane 0 of the calling warp acquires `dep` (bounded blocking wait).
// Returns 1 when met, -1 when the wait gave up.
__device__ __forceinline__ int acquire_dep(const PanelArgs &a, const unsigned *dep)
{
    if (!dep) return 1;
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
        unsigned it = 0;
        while (panel::ld_acquire(dep) < tiles_per_phase(a) + a.dep_bias) {
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

// The two TMA loads of tile d into stage buffer sbuf (lane 0 of the producer).
template <int MODE, int B2>
__device__ __forceinline__ void issue_loads(const PanelArgs &a, const Tile &d, unsigned char *sbuf,
                                            unsigned long long *bar)
{
    using namespace panel;
    mbar_expect_tx(bar, TILE_BYTES);
    const int bidx = d.q >> a.lgPpb, pcol = d.q & (a.panels_per_batch - 1);
    const int colbase = pcol << a.lgP;
    const int slot = d.q % NBUF;
    const int hi = tile_hi(a, d, MODE), lo = tile_lo32(a, d, MODE);
    const unsigned long long pol = policy_evict_first();
#pragma unroll
    for (int x = 0; x < NBOX; ++x) {
        void *bx = sbuf + x * BOX_BYTES;
        if (!d.isB) {
            if (MODE == 1) {
                tma_ld_3d(bx, &a.map_ld, colbase + lo + 16 * x, hi, bidx * 128, bar, pol);
            } else {
                const unsigned u = digit_reverse((unsigned)hi, a.rev_bits, a.rev_t);   // pi(j_lo): fixed row bits
                if (B2 == 2) {
                    tma_ld_4d(bx, &a.map_ld, colbase + lo + 16 * x, 0, 0, (int)(u >> 7) + (bidx << 7), bar, pol);
                } else {
                    const CUtensorMap *m = ((u >> 6) & 1u) ? &a.map_ld_alt : &a.map_ld;
                    tma_ld_5d(bx, m, colbase + lo + 16 * x, 0, 0, 0, (int)(u >> 8) + (bidx << 6), bar, pol);
                }
            }
        } else if (MODE == 1) {
            tma_ld_3d(bx, &a.map_scr_ld, lo + 16 * x, 0, slot * a.P + hi, bar, pol);
        } else {
            tma_ld_3d(bx, &a.map_scr_ld, lo + 16 * x, 0, slot * 128 + hi, bar, pol);
        }
    }
}

// Twiddle tables of tile d (warp-wide call by the producer):
//   A tiles:    TW[k] = w_L^{-k j_lo}, k < 128, from the block's tables
//               tlo[r] = w_L^{-r} and w128[r] = w_L^{-128 r} (r < 128)
//   stage-1 B:  E1[e] = w_N^{-(k0+e) c} (e < 32), E2[k_hi] = w_N^{-128 k_hi c}
template <int MODE>
__device__ __forceinline__ void build_tables(const PanelArgs &a, const Tile &d, float2 *TW, float2 *E1,
                                             float2 *E2, const float2 *tlo, const float2 *w128)
{
    using namespace panel;
    const int lane = threadIdx.x & 31;
    if (!d.isB) {
        const unsigned jlo = (unsigned)tile_hi(a, d, MODE);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const unsigned r = (unsigned)(lane + 32 * m) * jlo;                 // < L
            TW[lane + 32 * m] = f2mul(tlo[r & 127u], w128[r >> 7]);
        }
    } else if (MODE == 1) {
        const int pcol = d.q & (a.panels_per_batch - 1);
        const unsigned cglob = (unsigned)((pcol << a.lgP) + tile_hi(a, d, MODE));
        const int k0 = tile_lo32(a, d, MODE);
        const float2 *nlo = reinterpret_cast<const float2 *>(a.twN_lo);
        const float2 *nhi = reinterpret_cast<const float2 *>(a.twN_hi);
        const unsigned lomask = (1u << a.twN_lo_bits) - 1u;
        constexpr int PER = (32 + B) / 32;                   // 5 entries per lane
        float2 lo[PER], hi[PER];
#pragma unroll
        for (int m = 0; m < PER; ++m) {                      // all loads in flight first
            const int e = lane + 32 * m;
            const unsigned r = (e < 32) ? (((unsigned)(k0 + e) * cglob) & a.N_mask)
                                        : (((unsigned)A * (unsigned)(e - 32) * cglob) & a.N_mask);
            lo[m] = __ldg(nlo + (r & lomask));
            hi[m] = __ldg(nhi + (r >> a.twN_lo_bits));
        }
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int e = lane + 32 * m;
            const float2 w = f2mul(lo[m], hi[m]);
            if (e < 32) E1[e] = w; else E2[e - 32] = w;
        }
    }
}

// ---- consumer ---------------------------------------------------------------

__device__ __forceinline__ void cmul_into(cx<float> &v, float2 w)
{
    const float2 p = panel::f2mul(make_float2(v.x, v.y), w);
    v.x = p.x;
    v.y = p.y;
}

// One consumer warp's part of tile d in stage buffer sb (shared address):
// warp wl (0..7 within its group) owns columns 4 (wl & 3) .. 4 (wl & 3) + 3
// of box wl >> 2.  Lane l has q = l & 7 (t8 in pass 1, gp in pass 2) and
// column c = 4 (wl & 3) + (l >> 3), so each half-warp (the unit an 8-byte
// shared access is served in) holds all eight values of q for two columns
// sharing a 16-byte chunk.
// Shared address of (row r, column c) of a box: r*128 + ((c>>1) ^ (r&7))*16
// + (c&1)*8 (the TMA 128-byte swizzle).
// Pass 2 gives lane gp the sequence outputs k = k16 + 16 k8 for two k16:
//   paired (stage-1 A, stored from registers as 16-byte pairs): k16 = 2gp + h;
//   staged (all other tiles, written back as the store image): k16 = gp + 8h,
//   so that the image rows k of the eight gp differ in k & 7.
template <int MODE, int B2>
__device__ __forceinline__ void consume_tile(const PanelArgs &a, const Tile &d, unsigned sb,
                                             const float2 *TW, const float2 *E1, const float2 *E2,
                                             const float2 *w16)
{
    using namespace panel;
    const int wl = (threadIdx.x >> 5) & (WPG - 1), lane = threadIdx.x & 31;
    const int q = lane & 7;
    const int col = 4 * (wl & 3) + (lane >> 3);              // column in the box
    const int cc = col >> 1, half = col & 1;
    const unsigned box = sb + (unsigned)(wl >> 2) * BOX_BYTES + (unsigned)half * 8u;
    const bool paired = (MODE == 1 && !d.isB);

    cx<float> v[16];
    // ---- landing -> registers: v[s] = logical point t8 + 8 s, t8 = q
    {
        const int lo = (MODE == 2 && !d.isB) ? land_lo<B2>(q) : q;
        const unsigned base = box + (unsigned)(lo << 7) + (unsigned)((cc ^ lo) << 4);
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            const int hs = (MODE == 2 && !d.isB) ? land_hi<B2>(s) : s;
            const float2 x = lds2(base + (unsigned)hs * 1024u);
            v[s] = make_cx<float>(x.x, x.y);
        }
    }
    if (!d.isB && a.conj) {
#pragma unroll
        for (int s = 0; s < 16; ++s) v[s].y = -v[s].y;
    }
    dft16(v);
#pragma unroll
    for (int s = 1; s < 16; ++s) cmul_into(v[s], w16[s * 8 + q]);     // w_128^{-k16 t8}
    // ---- exchange inside the warp's columns: X1[t8][k16] at row
    // R = 8 k16 + (t8 ^ m(k16)), m = k16 >> 1 (paired) or k16 & 7 (staged);
    // its row & 7 is a bijection of t8 (the writes) and of gp (the reads), so
    // every access is conflict-free.
    const unsigned e0 = box + (unsigned)(q << 7) + (unsigned)((cc ^ q) << 4);
    __syncwarp();                                             // landing reads of the other lanes done
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const unsigned m = paired ? (unsigned)(k >> 1) : (unsigned)(k & 7);
        sts2((e0 ^ (m * 0x90u)) + (unsigned)k * 1024u, make_float2(v[k].x, v[k].y));
    }
    __syncwarp();
    {
        // paired: row 8 (2gp + h) + (t ^ gp); staged: row 8 (gp + 8h) + (t ^ gp)
        const unsigned rb = e0 + (paired ? (unsigned)q * 2048u : (unsigned)q * 1024u);
        const unsigned hs = paired ? 1024u : 8192u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const float2 x = lds2((rb ^ (unsigned)(t * 0x90)) + (unsigned)h * hs);
                v[8 * h + t] = make_cx<float>(x.x, x.y);
            }
            dft8(v + 8 * h);
        }
    }
    // v[8 h + k8] = output k = k16(h) + 16 k8 of the lane's sequence
    const int kb0 = paired ? 2 * q : q, kbs = paired ? 1 : 8;   // k16(h) = kb0 + kbs h
    if (!d.isB) {
        // A tiles: w_L^{-k j_lo} = TW[k]
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < 8; ++k) cmul_into(v[8 * h + k], TW[kb0 + kbs * h + 16 * k]);
    } else if (MODE == 1) {
        // stage-1 B: w_N^{-(k_lo + 128 k_hi) c} = E1[column] E2[k_hi]
        const float2 e1 = E1[16 * (wl >> 2) + col];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < 8; ++k) cmul_into(v[8 * h + k], f2mul(e1, E2[kb0 + kbs * h + 16 * k]));
    }
    if (d.isB && a.conj) {
#pragma unroll
        for (int s = 0; s < 16; ++s) v[s].y = -v[s].y;
    }
    if (paired) {
        // panel buffer [c][j_lo][k_lo]: 16-byte stores of (k, k + 1), k = 2q + 16 k8
        const int jlo = tile_hi(a, d, MODE);
        const int cl = tile_lo32(a, d, MODE) + 16 * (wl >> 2) + col;     // column in the panel
        float2 *dst = reinterpret_cast<float2 *>(a.scratch) +
                      ((((size_t)(d.q % NBUF) << a.lgP) + (size_t)cl) * 128 + (size_t)jlo) * 128 + 2 * q;
        const unsigned long long pol = policy_evict_last();
#pragma unroll
        for (int k = 0; k < 8; ++k)
            st_v4_hint(dst + 16 * k, make_float4(v[k].x, v[k].y, v[8 + k].x, v[8 + k].y), pol);
    } else {
        // in place, row = output index k = q + 8h + 16 k8: the tile's store image
        __syncwarp();                                         // exchange reads of the other lanes done
        const unsigned ob = box + (unsigned)(q << 7) + (unsigned)((cc ^ q) << 4);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < 8; ++k)
                sts2(ob + (unsigned)h * 1024u + (unsigned)k * 2048u, make_float2(v[8 * h + k].x, v[8 * h + k].y));
        fence_async_shared();                                 // visible to the TMA stores
    }
}

// ---- storer -> publisher ring -------------------------------------------------

// Completed tiles travel from the storer to the publisher as pointers to the
// counter they count towards; bit 0 set: the tile was written by TMA stores
// (the publisher orders those writes before its release with a proxy fence).
struct PubRing {
    unsigned long long slot[panel::PQ];
    int tail;                      // entries appended (storer)
    int head;                      // entries published (publisher)
    int fin;                       // the storer appends no more
};

__device__ __forceinline__ int ld_acquire_cta(const int *p)
{
    int v;
    asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(panel::smem_u32(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta(int *p, int v)
{
    asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" :: "r"(panel::smem_u32(p)), "r"(v) : "memory");
}

// Storer side: append one completion (bounded wait while the ring is full).
__device__ __forceinline__ void pub_push(PubRing &r, int &tail, unsigned *ctr, int async, int *status)
{
    if (tail - ld_acquire_cta(&r.head) >= panel::PQ) {
        const unsigned long long t0 = panel::global_ns();
        while (tail - ld_acquire_cta(&r.head) >= panel::PQ) {
            if (panel::global_ns() - t0 > panel::WAIT_NS) { atomicExch(status, 5); return; }
            __nanosleep(200);
        }
    }
    r.slot[tail % panel::PQ] = (unsigned long long)ctr | (unsigned long long)async;
    st_release_cta(&r.tail, ++tail);
}

// Warps 0..15 consume (groups 0 and 1 take even and odd tiles), warp 16
// produces, warp 17 stores, warp 18 builds the twiddle tables, warp 19
// publishes the completions.
template <int MODE, int B2>
__global__ void __launch_bounds__(panel::NT, 1)
    paco_panel_kernel(const __grid_constant__ PanelArgs args)
{
    using namespace panel;
    extern __shared__ __align__(1024) unsigned char stage_raw[];
    __shared__ __align__(8) unsigned long long full[NSTAGE], done[NSTAGE], empty[NSTAGE], posted[NSTAGE];
    __shared__ float2 w16[128];                           // w_128^{-s t8} at [s*8 + t8]
    __shared__ float2 tlo[128], w128[128];                // w_L^{-r}, w_L^{-128 r}, r < 128
    __shared__ float2 TWs[NSTAGE][128];                   // per-stage w_L table (A tiles)
    __shared__ float2 E1s[NSTAGE][32], E2s[NSTAGE][B];    // per-stage w_N factors (stage-1 B)
    __shared__ int s_info[NSTAGE];                        // tile index held by each stage
    __shared__ PubRing ring;
    __shared__ volatile int s_abort;

    // the dynamic buffer starts 1024-aligned (the 128-byte swizzle needs it)
    unsigned char *stage = stage_raw + ((1024u - (smem_u32(stage_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float2 *twL = reinterpret_cast<const float2 *>(args.twL);
    for (int r = tid; r < 128; r += blockDim.x) {
        w16[r] = __ldg(twL + ((r >> 3) * (r & 7)) * B);
        tlo[r] = __ldg(twL + r);
        w128[r] = __ldg(twL + r * B);
    }
    if (tid == 0) {
        for (int k = 0; k < NSTAGE; ++k) {
            mbar_init(&full[k], 2);                       // the load arrival (with bytes) + the tables
            mbar_init(&done[k], WPG);
            mbar_init(&empty[k], 1);
            mbar_init(&posted[k], 1);                     // the tile index is in s_info

        }
        s_abort = 0;
        ring.tail = ring.head = ring.fin = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int lgT = args.lgP + 2;                        // T = 4 P tiles per phase
    const int total = (2 * args.npanels) << lgT;
    __syncthreads();

    if (warp == NCW) {
        // ---------------- producer ----------------
        const unsigned *depA = nullptr, *depB = nullptr;  // the counters last found complete
        int gnext = 0;
        if (lane == 0) gnext = (int)atomicAdd(args.ctr, 1u);
        int i = 0, ends = 0;
        for (;; ++i) {
            const int b = i % NSTAGE;
            if (i >= NSTAGE && lane == 0 &&
                !mbar_wait(&empty[b], (unsigned)((i / NSTAGE - 1) & 1), WAIT_NS)) {
                s_abort = 1;
                atomicExch(args.status, 5);
                // the stage was not returned: let its load land before reusing it
                mbar_wait(&full[b], (unsigned)(((i - NSTAGE) / NSTAGE) & 1), WAIT_NS);
            }
            __syncwarp();
            int g = 0;
            if (lane == 0) {
                g = s_abort ? total : gnext;
                if (g < total && !ends) gnext = (int)atomicAdd(args.ctr, 1u);   // claim one ahead
            }
            g = __shfl_sync(0xffffffffu, g, 0);
            if (ends) g = total;
            const Tile d = decode_tile(g, lgT, args.npanels);
            bool fresh = false;                               // a dependency newly acquired
            if (g < total) {
                const unsigned *dep = tile_dep(args, d);
                const unsigned *&cache = d.isB ? depB : depA;
                if (dep && dep != cache) {
                    if (acquire_dep(args, dep) < 0) {
                        if (lane == 0) s_abort = 1;
                        g = total;
                    } else {
                        cache = dep;
                        fresh = true;
                    }
                }
            }
            if (g >= total) {
                // end marker for this group; then one for the other group
                if (lane == 0) {
                    s_info[b] = total;
                    mbar_arrive(&posted[b]);
                    mbar_arrive(&full[b]);
                    mbar_arrive(&full[b]);
                }
                if (++ends == 2) break;
                continue;
            }
            if (lane == 0) {
                s_info[b] = g;
                mbar_arrive(&posted[b]);                      // the table warp may start
                if (fresh) fence_async_global();              // panel data of other CTAs, then TMA reads
                fence_async_shared();                         // consumers' accesses of stage b, then TMA writes
                issue_loads<MODE, B2>(args, d, stage + b * TILE_BYTES, &full[b]);
            }
        }
        // Iterations i-1 and i posted the end markers on stages whose earlier
        // loads had been consumed.  The loads of iterations i-NSTAGE+1 .. i-2
        // may still be in flight: wait (bounded) for them before exiting.  No
        // later phase was posted on their stages, so each parity names the
        // current or the just-completed phase.
        if (lane == 0)
            for (int j = (i - NSTAGE + 1 < 0 ? 0 : i - NSTAGE + 1); j < i - 1; ++j)
                mbar_wait(&full[j % NSTAGE], (unsigned)((j / NSTAGE) & 1), WAIT_NS);
        return;
    }
    if (warp == NCW + 2) {
        // ---------------- twiddle tables ----------------
        for (int i = 0;; ++i) {
            const int b = i % NSTAGE;
            const int ok = mbar_wait(&posted[b], (unsigned)((i / NSTAGE) & 1), WAIT_NS);   // every lane
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) { s_abort = 1; atomicExch(args.status, 5); }
                break;
            }
            const int g = s_info[b];
            if (g >= total) break;
            build_tables<MODE>(args, decode_tile(g, lgT, args.npanels), TWs[b], E1s[b], E2s[b], tlo, w128);
            __syncwarp();                                     // tables written before the arrive
            if (lane == 0) mbar_arrive(&full[b]);
        }
        return;
    }
    if (warp == NCW + 1) {
        // ---------------- storer ----------------
        if (lane == 0) {
            int tail = 0;
            int last_b = -1;                                  // stage of the newest store group
            unsigned *last_a = nullptr;                       // its A-tile counter (stage 2), if any
            for (int i = 0;; ++i) {
                const int b = i % NSTAGE;
                const unsigned par = (unsigned)((i / NSTAGE) & 1);
                if (!mbar_test(&done[b], par)) {
                    // about to wait: nothing stays held back meanwhile (the stage
                    // returns once the stores have read it; an A tile counts once written)
                    if (last_b >= 0) {
                        bulk_wait_read0();
                        mbar_arrive(&empty[last_b]);
                        if (last_a) {
                            bulk_wait0();
                            pub_push(ring, tail, last_a, 1, args.status);
                        }
                        last_b = -1;
                        last_a = nullptr;
                    }
                    if (!mbar_wait(&done[b], par, WAIT_NS)) {
                        s_abort = 1;
                        atomicExch(args.status, 5);
                        break;
                    }
                }
                const int g = s_info[b];
                if (g >= total) break;
                const Tile d = decode_tile(g, lgT, args.npanels);
                unsigned *ctr = tile_ctr(args, d);
                if (!d.isB && MODE == 1) {
                    // the consumers stored this tile to the panel buffer themselves
                    pub_push(ring, tail, ctr, 0, args.status);
                    mbar_arrive(&empty[b]);
                    continue;
                }
                if (d.isB) pub_push(ring, tail, ctr, 0, args.status);   // its panel lines were read
                const int bidx = d.q >> args.lgPpb, pcol = d.q & (args.panels_per_batch - 1);
                const int colbase = pcol << args.lgP;
                const int hi = tile_hi(args, d, MODE), lo = tile_lo32(args, d, MODE);
                const unsigned char *src = stage + b * TILE_BYTES;
                if (!d.isB) {
                    const unsigned long long pol = policy_evict_last();
#pragma unroll
                    for (int x = 0; x < NBOX; ++x)
                        tma_st_3d(&args.map_scr_st, lo + 16 * x, hi, (d.q % NBUF) * 128, src + x * BOX_BYTES, pol);
                } else if (MODE == 1) {
                    const unsigned long long pol = policy_evict_first();
                    const unsigned u = digit_reverse((unsigned)(colbase + hi), args.rev_bits, args.rev_t);
                    const int row = (int)u + bidx * args.N2rows;
#pragma unroll
                    for (int x = 0; x < NBOX; ++x)
                        tma_st_3d(&args.map_out, lo + 16 * x, 0, row, src + x * BOX_BYTES, pol);
                } else {
                    const unsigned long long pol = policy_evict_first();
#pragma unroll
                    for (int x = 0; x < NBOX; ++x)
                        tma_st_3d(&args.map_out, colbase + lo + 16 * x, hi, bidx * 128, src + x * BOX_BYTES, pol);
                }
                bulk_commit();
                if (last_b >= 0) {
                    // the previous group has read its stage; an A tile's completion
                    // is published once its stores are written
                    bulk_wait_read1();
                    mbar_arrive(&empty[last_b]);
                    if (last_a) {
                        bulk_wait1();
                        pub_push(ring, tail, last_a, 1, args.status);
                    }
                }
                last_b = b;
                last_a = d.isB ? nullptr : ctr;
            }
            bulk_wait0();
            if (last_b >= 0) {
                mbar_arrive(&empty[last_b]);
                if (last_a) pub_push(ring, tail, last_a, 1, args.status);
            }
            st_release_cta(&ring.fin, 1);
        }
        return;
    }
    if (warp == NCW + 3) {
        // ---------------- publisher ----------------
        if (lane == 0) {
            int head = 0;
            unsigned long long idle_since = 0;
            for (;;) {
                const int fin = ld_acquire_cta(&ring.fin);
                const int tail = ld_acquire_cta(&ring.tail);
                if (tail == head) {
                    if (fin) break;
                    const unsigned long long now = global_ns();
                    if (!idle_since) idle_since = now;
                    else if (now - idle_since > 2 * WAIT_NS) break;   // the storer gave up
                    __nanosleep(256);
                    continue;
                }
                idle_since = 0;
                int async = 0;
                for (int k = head; k < tail; ++k) async |= (int)(ring.slot[k % PQ] & 1ull);
                if (async) fence_async_global();              // TMA-stored panel data, then the release
                fence_acq_rel_gpu();                          // one fence publishes the batch
                unsigned *run = nullptr;
                unsigned n = 0;
                for (int k = head; k < tail; ++k) {
                    unsigned *c = reinterpret_cast<unsigned *>(ring.slot[k % PQ] & ~1ull);
                    if (c != run) {
                        if (run) red_relaxed_add(run, n);
                        run = c;
                        n = 0;
                    }
                    ++n;
                }
                if (run) red_relaxed_add(run, n);
                head = tail;
                st_release_cta(&ring.head, head);
            }
        }
        return;
    }

    // ---------------- consumer warps ----------------
    const unsigned stage_base = smem_u32(stage);
    for (int i = warp / WPG;; i += 2) {
        const int b = i % NSTAGE;
        const int ok = mbar_wait(&full[b], (unsigned)((i / NSTAGE) & 1), WAIT_NS);   // every lane
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) { s_abort = 1; atomicExch(args.status, 5); }
            break;
        }
        const int g = s_info[b];
        if (g >= total) {
            if (lane == 0) mbar_arrive(&done[b]);
            break;
        }
        const Tile d = decode_tile(g, lgT, args.npanels);
        if (d.isB) {
            // drop the consumed panel lines (now in shared memory): one 128-byte
            // box row per lane, rows 32 (wl & 3) + lane of box wl >> 2
            const int hi = tile_hi(args, d, MODE), lo = tile_lo32(args, d, MODE);
            const int wl = warp & (WPG - 1);
            const int bx = wl >> 2, row = 32 * (wl & 3) + lane;
            const float2 *sc = reinterpret_cast<const float2 *>(args.scratch);
            const size_t slot = (size_t)(d.q % NBUF);
            const float2 *line = (MODE == 1)
                ? sc + (((slot << args.lgP) + (size_t)hi) * 128 + (size_t)row) * 128 + lo + 16 * bx
                : sc + ((slot * 128 + (size_t)hi) * 128 + (size_t)row) * (size_t)args.P + lo + 16 * bx;
            discard_l2(line);
        }
        consume_tile<MODE, B2>(args, d, stage_base + (unsigned)b * TILE_BYTES, TWs[b], E1s[b], E2s[b], w16);
        __syncwarp();
        if (lane == 0) mbar_arrive(&done[b]);
    }
}

#endif // PACO_PANEL_KERNEL_TU

} // namespace paco
