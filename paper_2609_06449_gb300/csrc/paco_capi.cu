// paco_capi.cu -- host side of the C ABI declared in include/paco.h.
//
// Plan construction (legality per Sect. 2, Eq. exact-divisibility; tile and
// cluster choice; FP64 twiddle tables generated on the device), execution
// (two stage launches per Theorem 3's composition, Eq. (10)), the unfused
// three-pass form, the host-buffer form, and error reporting.
#include <cuda.h>            // CUtensorMap types (no libcuda link: the encoder comes
#include <cudaTypedefs.h>    // from cudaGetDriverEntryPointByVersion)
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <string>

#include "../../include/paco.h"
#include "paco_plan.h"
#include "paco_common.cuh"
#include "paco_stage_args.cuh"
#include "paco_panel_host.h"
#include "paco_stage.cuh"

namespace paco {
const void *stage_kernel_fn_f32(int lgL, int minb);
const void *stage_kernel_fn_f64(int lgL, int minb);
const void *stage_kernel_fn_special_f32(int lgL, int lgW, int lgK, int mode);
const void *stage_kernel_fn_special_f64(int lgL, int lgW, int lgK, int mode);
const void *stage_kernel_fn_terms_f32(int lgL, int minb);
const void *stage_kernel_fn_scale_f32(int lgL, int minb);
const void *stage_kernel_fn_shard_f32(int lgL, int minb);
const void *stage_kernel_fn_split_f32(int lgL, int minb);
} // namespace paco

using namespace paco;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

paco_status_t paco::fail(paco_status_t st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

extern "C" const char *paco_last_error(void) { return g_last_error.c_str(); }

namespace paco {
void set_last_error(const char *msg) { g_last_error = msg; }
} // namespace paco
extern "C" const char *paco_version(void) { return "paco-gb300 0.1"; }

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
int paco::ilog2_exact(int64_t v)
{
    if (v <= 0 || (v & (v - 1))) return -1;
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

// w_M^{-(r*mult)} for r in [count], generated in FP64 with sincospi.
template <typename R>
__global__ void twiddle_gen_kernel(cx<R> *out, long long M, long long count, long long mult)
{
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= count) return;
    long long e = (r * mult) % M;
    double s, c;
    sincospi(2.0 * (double)e / (double)M, &s, &c);
    out[r] = make_cx<R>((R)c, (R)(-s));
}

paco_status_t paco::gen_table(int esize, void **dst, long long M, long long count, long long mult,
                              cudaStream_t stream)
{
    size_t bytes = (size_t)count * (size_t)esize;
    PACO_CUDA_TRY(cudaMalloc(dst, bytes));
    int threads = 256;
    long long blocks = (count + threads - 1) / threads;
    if (esize == 8)
        twiddle_gen_kernel<float><<<(unsigned)blocks, threads, 0, stream>>>((cx<float> *)*dst, M, count, mult);
    else
        twiddle_gen_kernel<double><<<(unsigned)blocks, threads, 0, stream>>>((cx<double> *)*dst, M, count, mult);
    PACO_CUDA_TRY(cudaGetLastError());
    return PACO_OK;
}

// Tile width W and cluster size K for a stage of length 2^lgL over C columns:
// about 64 KiB of tile per CTA, at least 32 B per row segment, and at most
// 16 columns for L >= 128, 64 for L = 32, 64, none for L <= 16 (measured on
// GB300, one 2^28-point complex64 pass: L = 16 4.04 -> 1.02 ms with 512
// columns instead of 16; L = 32 1.76 -> 0.79 ms and L = 64 0.97 -> 0.76 ms
// with 64; L = 128 and 256 are fastest with 16).
static void choose_tile(const paco_plan *pl, int lgL, int64_t C, int req_w, int req_k, int mode,
                        int *lgW_out, int *lgK_out)
{
    const int lgE = pl->esize == 8 ? 3 : 4;
    const int lgBudget = 16 - lgE;                   // elements per CTA: 8192 (c64) / 4096 (c128)
    int lgC = ilog2_exact(C);
    int lgW;
    if (req_w > 0) lgW = ilog2_exact(req_w);
    else {
        int lgWmin = 5 - lgE;                        // 32-byte rows: 4 (c64) / 2 (c128)
        lgW = lgBudget - lgL;
        if (lgW < lgWmin) lgW = lgWmin;
        const int lgWmax = (lgL <= 4) ? lgBudget : (lgL <= 6) ? 6 : 4;
        if (lgW > lgWmax) lgW = lgWmax;
    }
    if (lgW > lgC) lgW = lgC;
    if (lgW < 0) lgW = 0;
    int lgK;
    if (req_k > 0) lgK = ilog2_exact(req_k);
    else {
        lgK = lgL + lgW - lgBudget;
        if (lgK < 0) lgK = 0;
    }
    // the cluster splits both factors of L
    int lgB = lgL / 2;
    if (lgK > lgB) lgK = lgB;
    // Phase I (complex64): a tile that needs a cluster is replaced by a
    // single-CTA tile of at least two columns (measured at L = 2^12: 1.84 vs
    // 2.30 ms for 16 x 2^24; Phase III keeps the cluster, its reads and
    // writes both being row segments of the tile width)
    if (mode == 1 && pl->esize == 8 && req_w == 0 && req_k == 0 && lgK > 0 && lgBudget - lgL >= 1 &&
        (int64_t(1) << (lgBudget - lgL)) <= C) {
        lgW = lgBudget - lgL;
        lgK = 0;
    }
    *lgW_out = lgW;
    *lgK_out = lgK;
}

static const int kPanelWidth = 128;
static const bool kDefaultTwoCtas = true;

// A complex64 stage of length 2^12 or 2^13 runs as two passes through the
// plan's scratch: the single-tile kernel at those lengths needs four radix
// passes and three exchanges per tile, while passes of length 2^6 / 2^7 run
// near the memory bound (measured on GB300, one 2^28-point pass: L = 64
// 0.76 ms, L = 128 0.71 ms, against 1.8-2.4 ms for L = 4096 and 3.2 ms for
// L = 8192 in one pass).
static paco_status_t setup_split(paco_plan *pl, StageCfg *sc, int lgL, int64_t C, int mode, int lgLa_req = 0)
{
    // pass lengths: powers of b (so that pi_m2(j_a Lb + j_b) = pi(j_b) La + pi(j_a)),
    // both between 2^5 and 2^8; La the larger unless given (the 3-D DFT's middle axis)
    int lgLa = lgLa_req;
    if (!lgLa) {
        lgLa = (lgL + 1) / 2;
        while (lgLa % pl->t) ++lgLa;
    }
    const int lgLb = lgL - lgLa;
    if (lgLa % pl->t || lgLb % pl->t || lgLa < 5 || lgLb < 5 || lgLa > 8 || lgLb > 8) return PACO_OK;
    const int lgC = ilog2_exact(C);
    for (int p = 0; p < 2; ++p) {
        const int lgLs = p == 0 ? lgLa : lgLb;
        const int64_t Cv = ((int64_t)1 << (p == 0 ? lgLb : lgLa)) * C;   // the pass's view columns
        int lgW = 0, lgK = 0;
        choose_tile(pl, lgLs, Cv, 0, 0, 2, &lgW, &lgK);
        if (lgW > lgC) lgW = lgC;                        // a tile stays inside one column block
        if (mode == 1 && p == 1 && lgW > lgLa) lgW = lgLa;
        const int As = 1 << ((lgLs + 1) / 2), Bs = 1 << (lgLs / 2), W = 1 << lgW;
        const bool fits = lgK == 0 && ((p == 0 && (1 << lgLa) <= (As + Bs) * W) ||
                                       (p == 1 && (mode == 2 || (1 << lgLb) <= Bs * W)));
        if (!fits) return PACO_OK;                       // not split: the single-pass kernel runs
        const int pad = (mode == 1 && p == 0) ? 1 : W;
        sc->sp_lgW[p] = lgW;
        sc->sp_threads[p] = (int)(((int64_t)1 << lgLs) * W / 16);
        sc->sp_smem[p] = stage_smem_elems(As, Bs, 1, W, pad) * pl->esize;
        sc->sp_ntiles[p] = (int)(Cv / W);
        const int minb = (pl->req_ctas == 1 || sc->sp_smem[p] > 113 * 1024) ? 1 : 2;
        sc->sp_fn[p] = stage_kernel_fn_split_f32(lgLs, minb);
        if (!sc->sp_fn[p] || sc->sp_threads[p] > 512) return PACO_OK;
        PACO_CUDA_TRY(cudaFuncSetAttribute(sc->sp_fn[p], cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    }
    paco_status_t st;
    if ((st = gen_table(8, &sc->sp_tw[0], (long long)1 << lgLa, (long long)1 << lgLa, 1, 0)) != PACO_OK ||
        (st = gen_table(8, &sc->sp_tw[1], (long long)1 << lgLb, (long long)1 << lgLb, 1, 0)) != PACO_OK)
        return st;
    sc->lgLa = lgLa;
    sc->lgLb = lgLb;
    sc->split = 1;
    return PACO_OK;
}

static paco_status_t setup_stage(paco_plan *pl, StageCfg *sc, int lgL, int64_t C, int mode,
                                 int req_w, int req_k)
{
    sc->lgL = lgL;
    if (!pl->form && !pl->shard_G && pl->esize == 8 && lgL == 14 && (mode == 1 || mode == 2) &&
        C >= kPanelWidth && req_w == 0 && req_k == 0 && pl->req_split != 1 && !(pl->dims == 3 && mode == 2)) {
        sc->panel = 1;
        sc->P = kPanelWidth;
        sc->fn = panel_kernel_fn(mode, pl->b);
        if (!sc->fn) return fail(PACO_ERR_UNSUPPORTED, "panel stage: radix %d", pl->b);
        sc->smem = panel_smem_bytes();
        sc->threads = panel::NT;                             // 16 consumer warps + producer + storer
        PACO_CUDA_TRY(cudaFuncSetAttribute(sc->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, sc->smem));
        return PACO_OK;
    }
    choose_tile(pl, lgL, C, req_w, req_k, mode, &sc->lgW, &sc->lgK);
    if (sc->lgW < 0 || sc->lgK < 0 || sc->lgK > 3)
        return fail(PACO_ERR_INVALID_ARG, "tile width / cluster size must be powers of two, cluster <= 8");
    const int A = 1 << ((lgL + 1) / 2), B = 1 << (lgL / 2);
    const int W = 1 << sc->lgW, K = 1 << sc->lgK;
    if ((int64_t)W > C) return fail(PACO_ERR_INVALID_ARG, "tile width %d exceeds %lld columns", W, (long long)C);
    if (K > 1 && (A % K || B % K)) return fail(PACO_ERR_INVALID_ARG, "cluster %d does not divide the split %dx%d", K, A, B);
    const int L = 1 << lgL;
    const int EPT = L < 16 ? L : 16;
    const int64_t NE = (int64_t)A * (B / K) * W;     // elements per CTA
    sc->ntiles = (int)(C / W);
    if (pl->form) {
        sc->fn = stage_kernel_fn_tc(lgL, pl->form);
        if (!sc->fn) return fail(PACO_ERR_UNSUPPORTED, "tensor-core forms need stage lengths 2^8..2^14");
    } else {
        sc->fn = (pl->esize == 8) ? stage_kernel_fn_special_f32(lgL, sc->lgW, sc->lgK, mode)
                                  : stage_kernel_fn_special_f64(lgL, sc->lgW, sc->lgK, mode);
        if (!sc->fn) sc->fn = (pl->esize == 8) ? stage_kernel_fn_f32(lgL, 1) : stage_kernel_fn_f64(lgL, 1);
    }
    if (!sc->fn) return fail(PACO_ERR_UNSUPPORTED, "stage length 2^%d is not built (max 2^14)", lgL);
    if (B == 1) {
        sc->threads = W;
        sc->smem = 0;
    } else {
        if (NE % EPT) return fail(PACO_ERR_INVALID_ARG, "tile too small");
        sc->threads = (int)(NE / EPT);
        const int pad = (mode == 1) ? 1 : W;
        sc->smem = stage_smem_elems(A, B, K, W, pad) * pl->esize;
    }
    if (pl->form) sc->smem = ((sc->smem + 15) & ~15) + tc_smem_bytes(pl->form, (sc->threads + 31) / 32);
    if (sc->threads > 512 || sc->threads < 1)
        return fail(PACO_ERR_INVALID_ARG, "tile of %lld elements needs %d threads (max 512)",
                    (long long)NE, sc->threads);
    if (sc->smem > 227 * 1024)
        return fail(PACO_ERR_INVALID_ARG, "tile needs %d bytes of shared memory (max 227 KiB)", sc->smem);
    // two resident CTAs per SM (registers capped at 64) for the generic
    // complex64 kernels, when asked for, or by default where two tiles fit
    const bool generic = !pl->form && pl->esize == 8 && B > 1 &&
                         !stage_kernel_fn_special_f32(lgL, sc->lgW, sc->lgK, mode);
    const bool two = generic && (pl->req_ctas == 2 ||
                                 (pl->req_ctas == 0 && kDefaultTwoCtas && sc->smem <= 113 * 1024));
    if (two) sc->fn = stage_kernel_fn_f32(lgL, 2);
    PACO_CUDA_TRY(cudaFuncSetAttribute(sc->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024));
    if (pl->shard_G && mode != 3) {
        // the sharded form's variant of the generic kernel (block addresses)
        sc->fn = stage_kernel_fn_shard_f32(lgL, (two || !generic) ? 2 : 1);
        if (!sc->fn || B == 1) return fail(PACO_ERR_UNSUPPORTED, "sharded form: stage length 2^%d is not built", lgL);
        PACO_CUDA_TRY(cudaFuncSetAttribute(sc->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        return PACO_OK;
    }
    if (pl->dims == 3 && mode == 2) {
        // the 3-D DFT: Phase III is the N2' x N3 plane's two passes (whatever its length)
        paco_status_t st = setup_split(pl, sc, lgL, C, mode, pl->lgLa3);
        if (st != PACO_OK) return st;
        if (!sc->split)
            return fail(PACO_ERR_UNSUPPORTED, "dims = 3: no pass configuration for the %lld x %lld plane over %lld columns",
                        1LL << pl->lgLa3, (long long)pl->N3, (long long)C);
    } else if (!pl->form && !pl->shard_G && pl->esize == 8 && pl->req_split >= 0 &&
        (lgL == 12 || lgL == 13 || (lgL == 14 && pl->req_split == 1)) && mode != 3 && req_w == 0 && req_k == 0) {
        paco_status_t st = setup_split(pl, sc, lgL, C, mode);
        if (st != PACO_OK) return st;
    }
    if (!pl->form && pl->esize == 8 && B > 1) {
        // the weighted-loss variant of the generic kernel (runtime tile width and
        // cluster size, so it also stands in for a specialised kernel)
        sc->fn_terms = stage_kernel_fn_terms_f32(lgL, (two || !generic) ? 2 : 1);
        sc->fn_scale = stage_kernel_fn_scale_f32(lgL, (two || !generic) ? 2 : 1);
        for (const void *f : {sc->fn_terms, sc->fn_scale})
            if (f) PACO_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    }
    return PACO_OK;
}

static paco_status_t plan_build(paco_plan **out, const paco_plan_opts_t *o, int shard_G = 0, int shard_rank = 0)
{
    *out = nullptr;
    if (!o) return fail(PACO_ERR_INVALID_ARG, "opts is NULL");
    // dims = 3: the N1 x N2' x N3 array is the pipeline's N1 x (N2' N3) view;
    // Phase III runs as the split stage La x Lb = N2' x N3 with ones for its
    // middle twiddle, i.e. the 2-D DFT of each N2' x N3 plane
    paco_plan_opts_t o3;
    int lgLa3 = 0;
    if (o->dims == 3) {
        if (shard_G) return fail(PACO_ERR_UNSUPPORTED, "dims = 3: not built for the sharded form");
        if (o->dtype != PACO_C64) return fail(PACO_ERR_UNSUPPORTED, "dims = 3: complex64 only");
        const int la = ilog2_exact(o->N2), lb = ilog2_exact(o->N3);
        const int tb = (o->b == 2 || o->b == 4 || o->b == 8 || o->b == 16) ? ilog2_exact(o->b) : 1;
        if (la < 5 || la > 8 || lb < 5 || lb > 8 || la % tb || lb % tb)
            return fail(PACO_ERR_UNSUPPORTED, "dims = 3: N2=%lld and N3=%lld must be powers of b in 2^5..2^8",
                        (long long)o->N2, (long long)o->N3);
        if (la + lb > 14) return fail(PACO_ERR_UNSUPPORTED, "dims = 3: N2 N3 = 2^%d exceeds 2^14", la + lb);
        o3 = *o;
        o3.N2 = o->N2 * o->N3;
        o = &o3;
        lgLa3 = la;
    } else if (o->N3 != 0 && o->N3 != 1) {
        return fail(PACO_ERR_INVALID_ARG, "N3=%lld is for dims = 3 only", (long long)o->N3);
    }
    if (o->b != 2 && o->b != 4 && o->b != 8 && o->b != 16)
        return fail(PACO_ERR_INVALID_ARG, "radix b=%d must be 2, 4, 8 or 16", o->b);
    if (o->dtype != PACO_C64 && o->dtype != PACO_C128 && o->dtype != PACO_C64_TC_BF16X3 &&
        o->dtype != PACO_C64_TC_FP16)
        return fail(PACO_ERR_UNSUPPORTED, "dtype %d is not built", (int)o->dtype);
    if (o->batch < 0) return fail(PACO_ERR_INVALID_ARG, "batch %lld < 0", (long long)o->batch);
    if (o->ctas_per_sm < 0 || o->ctas_per_sm > 2)
        return fail(PACO_ERR_INVALID_ARG, "ctas_per_sm=%d must be 0, 1 or 2", o->ctas_per_sm);
    const int t = ilog2_exact(o->b);
    const int l1 = ilog2_exact(o->N1), l2 = ilog2_exact(o->N2);
    if (l1 < 1 || l1 % t) return fail(PACO_ERR_INVALID_ARG, "N1=%lld is not a power of b=%d (>= b)", (long long)o->N1, o->b);
    if (l2 < 1 || l2 % t) return fail(PACO_ERR_INVALID_ARG, "N2=%lld is not a power of b=%d (>= b)", (long long)o->N2, o->b);
    if (l1 + l2 > 32) return fail(PACO_ERR_UNSUPPORTED, "N = 2^%d exceeds 2^32", l1 + l2);
    if (l1 > 14 || l2 > 14) return fail(PACO_ERR_UNSUPPORTED, "factors above 2^14 are not built");
    const bool tc = (o->dtype == PACO_C64_TC_BF16X3 || o->dtype == PACO_C64_TC_FP16);
    if (tc && (l1 < 8 || l2 < 8))
        return fail(PACO_ERR_UNSUPPORTED, "tensor-core forms need N1, N2 >= 2^8 (radix-16 passes in both stages)");
    const int m1 = l1 / t, m2 = l2 / t;
    int p = o->p;
    if (p == 0) {
        int e = (m1 < m2 ? m1 : m2) / 2;
        if (e < 1) e = 1;
        p = 1 << (t * e);
    }
    const int lp = ilog2_exact(p);
    if (p < 2 || lp < 0 || lp % t || p > o->N1 || p > o->N2 || o->N1 % p || o->N2 % p)
        return fail(PACO_ERR_INVALID_ARG, "p=%d must be a power of b=%d with 2 <= p, p | N1, p | N2", p, o->b);

    paco_plan *pl = new (std::nothrow) paco_plan();
    if (!pl) return fail(PACO_ERR_NOMEM, "out of host memory");
    pl->N1 = o->N1; pl->N2 = o->N2; pl->N = o->N1 * o->N2; pl->batch = o->batch;
    pl->b = o->b; pl->t = t; pl->p = p; pl->m1 = m1; pl->m2 = m2;
    pl->dtype = o->dtype;
    pl->esize = (o->dtype == PACO_C128) ? 16 : 8;
    pl->shard_G = shard_G;
    pl->shard_rank = shard_rank;
    pl->req_split = o->split;
    if (o->dims < 0 || o->dims > 3) {
        delete pl;
        return fail(PACO_ERR_INVALID_ARG, "dims=%d must be 1, 2 or 3", o->dims);
    }
    pl->dims = (o->dims == 0) ? 1 : o->dims;
    pl->lgLa3 = lgLa3;
    pl->N3 = (o->dims == 3) ? o->N2 >> lgLa3 : 1;
    pl->req_ctas = o->ctas_per_sm;
    pl->form = (o->dtype == PACO_C64_TC_BF16X3) ? TC_BF16X3 : (o->dtype == PACO_C64_TC_FP16) ? TC_FP16 : TC_NONE;
    if (pl->form) {
        paco_status_t ts = tc_table_create(pl->form, &pl->tc);
        if (ts != PACO_OK) {
            delete pl;
            return ts;
        }
    }
    cudaGetDevice(&pl->device);

    paco_status_t st;
    const int64_t C1 = shard_G ? pl->N2 / shard_G : pl->N2;   // columns of each stage's matrix
    const int64_t C2 = shard_G ? pl->N1 / shard_G : pl->N1;
    if ((st = setup_stage(pl, &pl->st[0], l1, C1, 1, o->tile_w, o->cluster)) != PACO_OK ||
        (st = setup_stage(pl, &pl->ph1, l1, pl->N2, 3, o->tile_w, o->cluster)) != PACO_OK ||
        (st = setup_stage(pl, &pl->st[1], l2, C2, 2, o->tile_w, o->cluster)) != PACO_OK) {
        paco_plan_destroy(pl);
        return st;
    }
    // FP64-generated twiddle tables: w_N1^{-r}, w_N2^{-r}, and w_N^{-r} in
    // two levels (r = hi * 2^h + lo).  The 2-D DFT has no top-level twiddle:
    // its w_N tables are w_1 = 1 (every kernel then multiplies by one).
    const int lgN = l1 + l2;
    pl->twN_lo_bits = (lgN + 1) / 2;
    const long long nlo = 1LL << pl->twN_lo_bits, nhi = (1LL << lgN) / nlo;
    const long long Mtw = (pl->dims >= 2) ? 1 : pl->N;
    if ((st = gen_table(pl->esize, &pl->twL1, pl->N1, pl->N1, 1, 0)) != PACO_OK ||
        (st = gen_table(pl->esize, &pl->twL2, pl->N2, pl->N2, 1, 0)) != PACO_OK ||
        (st = gen_table(pl->esize, &pl->twN_lo, Mtw, nlo, 1, 0)) != PACO_OK ||
        (st = gen_table(pl->esize, &pl->twN_hi, Mtw, nhi, nlo, 0)) != PACO_OK ||
        (pl->dims == 3 && (st = gen_table(pl->esize, &pl->tw_ones, 1, pl->N2, 1, 0)) != PACO_OK)) {
        paco_plan_destroy(pl);
        return st;
    }
    cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, pl->device);
    if (!shard_G && cluster_eligible(pl)) {
        if ((st = cluster_setup(pl)) != PACO_OK) {
            paco_plan_destroy(pl);
            return st;
        }
        pl->fused = 1;
    }
    size_t scratch_elems = 0, words = 0;
    for (int k = 0; k < 2; ++k) {
        const StageCfg &sc = pl->st[k];
        if (!sc.panel) continue;
        const int64_t C = (k == 0) ? pl->N2 : pl->N1;
        scratch_elems = std::max(scratch_elems, (size_t)panel::NBUF * ((size_t)1 << sc.lgL) * sc.P);
        words = std::max(words, (size_t)(2 * pl->batch * (C / sc.P) + 1));
    }
    if (scratch_elems) {
        cudaError_t ea = cudaMalloc(&pl->scratch, scratch_elems * pl->esize);
        if (ea == cudaSuccess) ea = cudaMalloc((void **)&pl->ctr, words * sizeof(unsigned));
        if (ea != cudaSuccess) {
            paco_plan_destroy(pl);
            return fail(PACO_ERR_NOMEM, "panel scratch: %s", cudaGetErrorString(ea));
        }
        pl->ctr_words = words;
    }
    if ((pl->st[0].split || pl->st[1].split) && pl->batch > 0) {
        cudaError_t ea = cudaMalloc(&pl->split_scratch, (size_t)(pl->N * pl->batch) * pl->esize);
        if (ea != cudaSuccess) {
            paco_plan_destroy(pl);
            return fail(PACO_ERR_NOMEM, "split-stage scratch: %s", cudaGetErrorString(ea));
        }
    }
    cudaError_t e = cudaMalloc(&pl->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(pl->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        paco_plan_destroy(pl);
        return fail(PACO_ERR_CUDA, "plan setup: %s", cudaGetErrorString(e));
    }
    *out = pl;
    return PACO_OK;
}

extern "C" paco_status_t paco_plan_create_ex(paco_plan_t **out, const paco_plan_opts_t *opts)
{
    if (!out) return fail(PACO_ERR_INVALID_ARG, "out is NULL");
    return plan_build(out, opts);
}

extern "C" paco_plan_t *paco_plan_create(int64_t N1, int64_t N2, int b, int64_t batch,
                                         paco_dtype_t dtype)
{
    paco_plan_opts_t o;
    memset(&o, 0, sizeof(o));
    o.N1 = N1; o.N2 = N2; o.b = b; o.batch = batch; o.dtype = dtype;
    paco_plan *pl = nullptr;
    plan_build(&pl, &o);
    return pl;
}

extern "C" void paco_plan_destroy(paco_plan_t *pl)
{
    if (!pl) return;
    batched_destroy(pl->bs);
    restore_destroy(pl);
    cudaFree(pl->tc);
    cudaFree(pl->twL1);
    cudaFree(pl->twL2);
    cudaFree(pl->twN_lo);
    cudaFree(pl->twN_hi);
    cudaFree(pl->twN_full);
    cudaFree(pl->tw_ones);
    cudaFree(pl->split_scratch);
    for (int k = 0; k < 2; ++k)
        for (int p = 0; p < 2; ++p) cudaFree(pl->st[k].sp_tw[p]);
    cudaFree(pl->d_status);
    cudaFree(pl->scratch);
    cudaFree(pl->ctr);
    delete pl;
}

extern "C" paco_status_t paco_plan_info(const paco_plan_t *pl, paco_plan_info_t *info)
{
    if (!pl || !info) return fail(PACO_ERR_INVALID_ARG, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->N3 = 1;
    if (pl->bs) {
        batched_info(pl, info);
        return PACO_OK;
    }
    info->N1 = pl->N1; info->N2 = pl->N2 / pl->N3; info->N3 = pl->N3; info->N = pl->N; info->batch = pl->batch;
    info->b = pl->b; info->p = pl->p; info->m1 = pl->m1; info->m2 = pl->m2;
    info->dtype = pl->dtype;
    const int64_t line = 128 / pl->esize;
    info->slab_width_ok = (pl->N1 / pl->p >= line) && (pl->N2 / pl->p >= line);
    const int64_t p = pl->p;
    info->items_per_pair = pl->N / (p * p);
    info->h = pl->N / p - pl->N / (p * p);
    info->mu = pl->N - pl->N / p;
    info->fused_cluster = pl->fused;
    info->shard_G = pl->shard_G;
    info->shard_rank = pl->shard_rank;
    info->stage_split[0] = pl->st[0].split;
    info->stage_split[1] = pl->st[1].split;
    info->dims = pl->dims;
    for (int s = 0; s < 2; ++s) {
        info->stage_tile_w[s] = 1 << pl->st[s].lgW;
        info->stage_cluster[s] = 1 << pl->st[s].lgK;
        info->stage_threads[s] = pl->st[s].threads;
        info->stage_smem[s] = pl->st[s].smem;
    }
    return PACO_OK;
}

// ---------------------------------------------------------------------------
// execution
// ---------------------------------------------------------------------------
static paco_status_t launch_panel(const paco_plan *pl, const StageCfg &sc, int mode,
                                  const void *in, void *out, int dir, cudaStream_t stream)
{
    PanelLaunch l;
    memset(&l, 0, sizeof(l));
    l.mode = mode;
    l.b = pl->b;
    l.C = (mode == 1) ? pl->N2 : pl->N1;
    l.batch = pl->batch;
    l.N = pl->N;
    l.P = sc.P;
    l.in = in;
    l.out = out;
    l.scratch = pl->scratch;
    l.ctr = pl->ctr;
    l.status = pl->d_status;
    l.twL = (mode == 1) ? pl->twL1 : pl->twL2;
    l.twN_lo = pl->twN_lo;
    l.twN_hi = pl->twN_hi;
    l.twN_lo_bits = pl->twN_lo_bits;
    l.conj = (dir == 1);
    l.spin_limit = pl->dbg_spin_limit;
    l.dep_bias = pl->dbg_wait_bias;
    PanelArgs a;
    paco_status_t st = panel_prepare(l, &a);
    if (st != PACO_OK) return st;
    const size_t words = (size_t)(2 * a.npanels + 1);
    PACO_CUDA_TRY(cudaMemsetAsync(pl->ctr, 0, words * sizeof(unsigned), stream));
    const long long total = 2LL * a.npanels * ((long long)panel::L / panel::TILE) * sc.P;
    long long grid = (long long)pl->num_sms;                 // one persistent CTA per SM
    if (grid > total) grid = total;
    void *params[] = {&a};
    PACO_CUDA_TRY(cudaLaunchKernel(sc.fn, dim3((unsigned)grid), dim3((unsigned)sc.threads), params,
                                   (size_t)sc.smem, stream));
    return PACO_OK;
}

// The two passes of a split stage: in -> scratch (pass A), scratch -> out (pass B).
static paco_status_t launch_split(const paco_plan *pl, const StageCfg &sc, int mode, const void *in, void *out,
                                  int dir, cudaStream_t stream)
{
    const int64_t C = (mode == 1) ? pl->N2 : pl->N1;
    const int lgC = ilog2_exact(C);
    for (int p = 0; p < 2; ++p) {
        const int sub = (mode == 1) ? 1 + p : 3 + p;
        StageArgs a;
        memset(&a, 0, sizeof(a));
        a.batch_stride = pl->N;
        a.lgW = sc.sp_lgW[p];
        a.lgK = 0;
        a.mode = (sub == 1) ? 1 : 2;
        a.rev_t = pl->t;
        a.rev_bits = (sub == 3) ? sc.lgLa : sc.lgLb;     // sub 3: rows pi over La's digits (others: natural rows)
        a.conj = (dir == 1);
        a.N_mask = (unsigned)(pl->N - 1);
        a.twN_lo = pl->twN_lo;
        a.twN_hi = pl->twN_hi;
        a.twN_lo_bits = pl->twN_lo_bits;
        a.pad = (sub == 1) ? 1 : (1 << sc.sp_lgW[p]);
        a.twL = sc.sp_tw[p];
        a.C = (int)((sub == 1) ? (C << sc.lgLb) : (sub == 2) ? (C << sc.lgLa) : (sub == 3) ? C : (C << sc.lgLa));
        a.out_ld = (int)((sub == 2) ? ((int64_t)1 << (sc.lgLa + sc.lgLb)) : C);
        SplitArgs sa;
        memset(&sa, 0, sizeof(sa));
        sa.sub = sub;
        sa.lgC = lgC;
        sa.lgLa = sc.lgLa;
        sa.lgLb = sc.lgLb;
        sa.rev_bits_c = (mode == 1) ? lgC : 0;
        sa.twS = (mode == 1) ? pl->twL1 : (pl->dims == 3) ? pl->tw_ones : pl->twL2;
        const void *src = (p == 0) ? in : pl->split_scratch;
        void *dst = (p == 0) ? pl->split_scratch : out;
        for (int64_t b0 = 0; b0 < pl->batch; b0 += 65535) {
            const int64_t nb = (pl->batch - b0 < 65535) ? pl->batch - b0 : 65535;
            StageArgs ab = a;
            ab.in = (const char *)src + (size_t)(b0 * pl->N) * pl->esize;
            ab.out = (char *)dst + (size_t)(b0 * pl->N) * pl->esize;
            void *params[] = {&ab, &sa};
            PACO_CUDA_TRY(cudaLaunchKernel(sc.sp_fn[p], dim3((unsigned)sc.sp_ntiles[p], (unsigned)nb, 1),
                                           dim3((unsigned)sc.sp_threads[p], 1, 1), params, (size_t)sc.sp_smem[p],
                                           stream));
        }
    }
    return PACO_OK;
}

static paco_status_t launch_stage(const paco_plan *pl, const StageCfg &sc, int mode,
                                  const void *in, void *out, int dir, cudaStream_t stream,
                                  const StageTerms *terms = nullptr)
{
    if (sc.panel) {
        if (terms) return fail(PACO_ERR_UNSUPPORTED, "weighted terms: not in the 2^14 panel stages");
        return launch_panel(pl, sc, mode, in, out, dir, stream);
    }
    if (terms && !sc.fn_terms)
        return fail(PACO_ERR_UNSUPPORTED, "weighted terms: complex64 plans with both factors >= 4 only");
    if (sc.split && !terms) return launch_split(pl, sc, mode, in, out, dir, stream);
    StageArgs a;
    memset(&a, 0, sizeof(a));
    a.in = in;
    a.out = out;
    a.batch_stride = pl->N;
    a.lgW = sc.lgW;
    a.lgK = sc.lgK;
    a.mode = mode;
    a.rev_t = pl->t;
    a.conj = (dir == 1);
    a.N_mask = (unsigned)(pl->N - 1);
    a.twN_lo = pl->twN_lo;
    a.twN_hi = pl->twN_hi;
    a.twN_lo_bits = pl->twN_lo_bits;
    a.pad = (mode == 1) ? 1 : (1 << sc.lgW);
    a.tc = pl->tc;
    if (mode == 1 || mode == 3) {         // over the input view: L = N1, C = N2
        a.C = (int)pl->N2;
        a.twL = pl->twL1;
        if (mode == 1) { a.out_ld = (int)pl->N1; a.rev_bits = pl->m2 * pl->t; }
        else { a.out_ld = (int)pl->N2; a.rev_bits = pl->m1 * pl->t; }
    } else {                              // over W: L = N2, C = N1
        a.C = (int)pl->N1;
        a.twL = pl->twL2;
        a.out_ld = (int)pl->N1;
        a.rev_bits = pl->m2 * pl->t;
    }
    const int K = 1 << sc.lgK;
    for (int64_t b0 = 0; b0 < pl->batch; b0 += 65535) {
        const int64_t nb = (pl->batch - b0 < 65535) ? pl->batch - b0 : 65535;
        StageArgs ab = a;
        ab.in = (const char *)in + (size_t)(b0 * pl->N) * pl->esize;
        ab.out = (char *)out + (size_t)(b0 * pl->N) * pl->esize;
        StageTerms tb;
        memset(&tb, 0, sizeof(tb));
        if (terms) {
            tb = *terms;
            if (tb.ld_w) tb.ld_w += b0 * pl->N;
            if (tb.st_w) tb.st_w += b0 * pl->N;
        }
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3((unsigned)(sc.ntiles * K), (unsigned)nb, 1);
        cfg.blockDim = dim3((unsigned)sc.threads, 1, 1);
        cfg.dynamicSmemBytes = (size_t)sc.smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)K;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void *params[] = {&ab, &tb};
        const void *fn = !terms ? sc.fn : (terms->ld_on && !terms->ld_w && !terms->st_w) ? sc.fn_scale : sc.fn_terms;
        PACO_CUDA_TRY(cudaLaunchKernelExC(&cfg, fn, params));
    }
    return PACO_OK;
}

static bool overlap(const void *a, const void *b, size_t bytes)
{
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + bytes && y < x + bytes;
}

static paco_status_t check_exec(const paco_plan *pl, const void *in, const void *out, int dir,
                                bool allow_inplace)
{
    if (!pl) return fail(PACO_ERR_INVALID_ARG, "plan is NULL");
    if (pl->shard_G) return fail(PACO_ERR_UNSUPPORTED, "a sharded plan runs through paco_shard_stage1 / stage2");
    if (dir != -1 && dir != 1) return fail(PACO_ERR_INVALID_ARG, "dir=%d must be -1 or +1", dir);
    if (pl->batch == 0) return PACO_OK;
    if (!in || !out) return fail(PACO_ERR_INVALID_ARG, "NULL buffer");
    if (((uintptr_t)in | (uintptr_t)out) & 15u)
        return fail(PACO_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    const size_t bytes = (size_t)(pl->N * pl->batch) * pl->esize;
    if (overlap(in, out, bytes) && !(allow_inplace && in == out))
        return fail(PACO_ERR_ALIASING, "input and output overlap");
    return PACO_OK;
}

static void set_device(const paco_plan *pl)
{
    int d = -1;
    cudaGetDevice(&d);
    if (d != pl->device) cudaSetDevice(pl->device);
}

extern "C" paco_status_t paco_execute(paco_plan_t *pl, const void *in, void *out, int dir,
                                      paco_stream_t stream)
{
    paco_status_t st = check_exec(pl, in, out, dir, false);
    if (st != PACO_OK || pl->batch == 0) return st;
    set_device(pl);
    cudaStream_t s = (cudaStream_t)stream;
    if (pl->bs) return batched_execute(pl, in, out, dir, s);
    if (pl->fused) return launch_cluster(pl, in, out, dir, nullptr, s);
    if ((st = launch_stage(pl, pl->st[0], 1, in, out, dir, s)) != PACO_OK) return st;
    return launch_stage(pl, pl->st[1], 2, out, out, dir, s);
}

// ---------------------------------------------------------------------------
// sharded form (Sect. 4.2, App. C.5 across G ranks)
// ---------------------------------------------------------------------------
extern "C" paco_status_t paco_plan_create_sharded(paco_plan_t **out, const paco_shard_opts_t *o)
{
    if (!out || !o) return fail(PACO_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (o->dtype != PACO_C64) return fail(PACO_ERR_UNSUPPORTED, "sharded form: complex64 only");
    const int t = (o->b == 2 || o->b == 4 || o->b == 8 || o->b == 16) ? ilog2_exact(o->b) : -1;
    if (t < 0) return fail(PACO_ERR_INVALID_ARG, "radix b=%d must be 2, 4, 8 or 16", o->b);
    const int lg = ilog2_exact(o->G);
    if (o->G < 2 || lg < 0 || lg % t || o->G > o->N1 || o->G > o->N2 || o->N1 % o->G || o->N2 % o->G)
        return fail(PACO_ERR_INVALID_ARG, "G=%d must be a power of b=%d with 2 <= G, G | N1, G | N2", o->G, o->b);
    if (o->N2 / o->G < o->b) return fail(PACO_ERR_INVALID_ARG, "G=%d leaves fewer than b=%d columns per rank", o->G, o->b);
    if (o->rank < 0 || o->rank >= o->G) return fail(PACO_ERR_INVALID_ARG, "rank %d not in [0, %d)", o->rank, o->G);
    if (o->batch < 0 || o->batch > 65535) return fail(PACO_ERR_INVALID_ARG, "batch %lld not in [0, 65535]", (long long)o->batch);
    paco_plan_opts_t po;
    memset(&po, 0, sizeof(po));
    po.N1 = o->N1; po.N2 = o->N2; po.b = o->b; po.p = o->G; po.batch = o->batch; po.dtype = o->dtype;
    po.dims = o->dims;
    paco_status_t st = plan_build(out, &po, o->G, o->rank);
    if (st != PACO_OK || !o->restore) return st;
    if ((o->N1 * o->N2) / o->G > INT32_MAX) {
        paco_plan_destroy(*out);
        *out = nullptr;
        return fail(PACO_ERR_UNSUPPORTED, "restore: N/G must stay below 2^31");
    }
    if ((st = restore_setup(*out)) != PACO_OK) {
        paco_plan_destroy(*out);
        *out = nullptr;
    }
    return st;
}

static paco_status_t launch_shard(const paco_plan *pl, int mode, const void *in, void *out, int dir,
                                  cudaStream_t stream)
{
    const StageCfg &sc = pl->st[mode == 1 ? 0 : 1];
    const int64_t G = pl->shard_G, Cl = pl->N2 / G, K1 = pl->N1 / G;
    StageArgs a;
    memset(&a, 0, sizeof(a));
    a.in = in;
    a.out = out;
    a.lgW = sc.lgW;
    a.lgK = sc.lgK;
    a.mode = mode;
    a.rev_t = pl->t;
    a.rev_bits = ilog2_exact(Cl);                  // the digit reversal of a rank's local columns / rows
    a.conj = (dir == 1);
    a.N_mask = (unsigned)(pl->N - 1);
    a.twN_lo = pl->twN_lo;
    a.twN_hi = pl->twN_hi;
    a.twN_lo_bits = pl->twN_lo_bits;
    a.pad = (mode == 1) ? 1 : (1 << sc.lgW);
    if (mode == 1) { a.C = (int)Cl; a.twL = pl->twL1; a.out_ld = (int)K1; }
    else { a.C = (int)K1; a.twL = pl->twL2; a.out_ld = (int)K1; }
    ShardArgs sh;
    memset(&sh, 0, sizeof(sh));
    sh.c_base = (long long)pl->shard_rank * Cl;
    sh.lgCl = ilog2_exact(Cl);
    sh.lgK1 = ilog2_exact(K1);
    sh.bat_blk = (long long)pl->batch * Cl * K1;
    sh.bat_Cl = (long long)pl->batch * Cl;
    long long in_stride = (mode == 1) ? pl->N / G : Cl * K1;
    long long out_stride = (mode == 1) ? Cl * K1 : pl->N / G;
    const int K = 1 << sc.lgK;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(sc.ntiles * K), (unsigned)pl->batch, 1);
    cfg.blockDim = dim3((unsigned)sc.threads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)sc.smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *params[] = {&a, &sh, &in_stride, &out_stride};
    PACO_CUDA_TRY(cudaLaunchKernelExC(&cfg, sc.fn, params));
    return PACO_OK;
}

static paco_status_t check_shard(const paco_plan *pl, const void *in, const void *out, int dir, const char *fn)
{
    if (!pl) return fail(PACO_ERR_INVALID_ARG, "plan is NULL");
    if (!pl->shard_G) return fail(PACO_ERR_UNSUPPORTED, "%s takes a sharded plan (paco_plan_create_sharded)", fn);
    if (dir != -1 && dir != 1) return fail(PACO_ERR_INVALID_ARG, "dir=%d must be -1 or +1", dir);
    if (pl->batch == 0) return PACO_OK;
    if (!in || !out) return fail(PACO_ERR_INVALID_ARG, "NULL buffer");
    if (((uintptr_t)in | (uintptr_t)out) & 15u) return fail(PACO_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    if (overlap(in, out, (size_t)(pl->N / pl->shard_G * pl->batch) * pl->esize))
        return fail(PACO_ERR_ALIASING, "input and output overlap");
    return PACO_OK;
}

extern "C" paco_status_t paco_shard_stage1(paco_plan_t *pl, const void *x_local, void *send, int dir,
                                           paco_stream_t stream)
{
    paco_status_t st = check_shard(pl, x_local, send, dir, "paco_shard_stage1");
    if (st != PACO_OK || pl->batch == 0) return st;
    set_device(pl);
    return launch_shard(pl, 1, x_local, send, dir, (cudaStream_t)stream);
}

extern "C" paco_status_t paco_shard_stage2(paco_plan_t *pl, const void *recv, void *y_local, int dir,
                                           paco_stream_t stream)
{
    paco_status_t st = check_shard(pl, recv, y_local, dir, "paco_shard_stage2");
    if (st != PACO_OK || pl->batch == 0) return st;
    set_device(pl);
    return launch_shard(pl, 2, recv, y_local, dir, (cudaStream_t)stream);
}

// Plans whose two stages are the generic stage kernels take the weighted terms.
static paco_status_t check_weighted(const paco_plan *pl, const char *fn)
{
    if (pl->bs) return fail(PACO_ERR_UNSUPPORTED, "%s takes a single-length plan", fn);
    if (pl->dims == 3) return fail(PACO_ERR_UNSUPPORTED, "%s: not built for dims = 3 plans", fn);
    if (pl->st[0].panel || pl->st[1].panel)
        return fail(PACO_ERR_UNSUPPORTED, "%s: plans with a 2^14 complex64 factor (panel stages) are not supported", fn);
    if (!pl->st[0].fn_terms || !pl->st[1].fn_terms)
        return fail(PACO_ERR_UNSUPPORTED, "%s: plain complex64 plans with both factors >= 4 only", fn);
    return PACO_OK;
}

extern "C" paco_status_t paco_execute_weighted_power(paco_plan_t *pl, const void *in, void *out, const float *w,
                                                     double *loss, int out_weighted, int dir, paco_stream_t stream)
{
    paco_status_t st = check_exec(pl, in, out, dir, false);
    if (st != PACO_OK) return st;
    if ((st = check_weighted(pl, "paco_execute_weighted_power")) != PACO_OK) return st;
    if (!w || !loss) return fail(PACO_ERR_INVALID_ARG, "paco_execute_weighted_power: w and loss required");
    if (((uintptr_t)w & 3u) || ((uintptr_t)loss & 7u))
        return fail(PACO_ERR_INVALID_ARG, "paco_execute_weighted_power: w must be 4-byte, loss 8-byte aligned");
    set_device(pl);
    cudaStream_t s = (cudaStream_t)stream;
    PACO_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(double), s));
    if (pl->batch == 0) return PACO_OK;
    StageTerms t;
    memset(&t, 0, sizeof(t));
    t.st_w = w;
    t.st_loss = loss;
    t.st_weighted = out_weighted ? 1 : 0;
    if ((st = launch_stage(pl, pl->st[0], 1, in, out, dir, s)) != PACO_OK) return st;
    return launch_stage(pl, pl->st[1], 2, out, out, dir, s, &t);
}

extern "C" paco_status_t paco_execute_weighted_input(paco_plan_t *pl, const void *in, void *out, const float *w,
                                                     const double *scale, float mult, int dir,
                                                     paco_stream_t stream)
{
    paco_status_t st = check_exec(pl, in, out, dir, false);
    if (st != PACO_OK) return st;
    if ((st = check_weighted(pl, "paco_execute_weighted_input")) != PACO_OK) return st;
    if (((uintptr_t)w & 3u) || ((uintptr_t)scale & 7u))
        return fail(PACO_ERR_INVALID_ARG, "paco_execute_weighted_input: w must be 4-byte, scale 8-byte aligned");
    if (pl->batch == 0) return PACO_OK;
    set_device(pl);
    cudaStream_t s = (cudaStream_t)stream;
    StageTerms t;
    memset(&t, 0, sizeof(t));
    t.ld_w = w;
    t.ld_scale = scale;
    t.ld_mult = mult;
    t.ld_on = 1;
    if ((st = launch_stage(pl, pl->st[0], 1, in, out, dir, s, &t)) != PACO_OK) return st;
    return launch_stage(pl, pl->st[1], 2, out, out, dir, s);
}

extern "C" paco_status_t paco_execute_stage1(paco_plan_t *pl, const void *in, void *W, int dir,
                                             paco_stream_t stream)
{
    paco_status_t st = check_exec(pl, in, W, dir, false);
    if (st != PACO_OK || pl->batch == 0) return st;
    if (pl->bs) return fail(PACO_ERR_UNSUPPORTED, "%s takes a single-length plan", "paco_execute_stage1");
    set_device(pl);
    return launch_stage(pl, pl->st[0], 1, in, W, dir, (cudaStream_t)stream);
}

extern "C" paco_status_t paco_execute_stage2(paco_plan_t *pl, const void *W, void *out, int dir,
                                             paco_stream_t stream)
{
    paco_status_t st = check_exec(pl, W, out, dir, true);
    if (st != PACO_OK || pl->batch == 0) return st;
    if (pl->bs) return fail(PACO_ERR_UNSUPPORTED, "%s takes a single-length plan", "paco_execute_stage2");
    set_device(pl);
    return launch_stage(pl, pl->st[1], 2, W, out, dir, (cudaStream_t)stream);
}

extern "C" paco_status_t paco_execute_phase1(paco_plan_t *pl, const void *in, void *out, int dir,
                                             paco_stream_t stream)
{
    paco_status_t st = check_exec(pl, in, out, dir, false);
    if (st != PACO_OK || pl->batch == 0) return st;
    if (pl->bs) return fail(PACO_ERR_UNSUPPORTED, "%s takes a single-length plan", "paco_execute_phase1");
    set_device(pl);
    return launch_stage(pl, pl->ph1, 3, in, out, dir, (cudaStream_t)stream);
}

extern "C" paco_status_t paco_permute(paco_plan_t *pl, const void *A_tilde, void *W, int dir,
                                      paco_stream_t stream)
{
    paco_status_t st = check_exec(pl, A_tilde, W, dir, false);
    if (st != PACO_OK || pl->batch == 0) return st;
    if (pl->bs) return fail(PACO_ERR_UNSUPPORTED, "paco_permute takes a single-length plan");
    set_device(pl);
    return launch_permute(pl, A_tilde, W, dir, (cudaStream_t)stream);
}

extern "C" paco_status_t paco_execute_host(paco_plan_t *pl, const void *h_in, void *h_out,
                                           void *d_in, void *d_out, int dir, paco_stream_t stream)
{
    paco_status_t st = check_exec(pl, d_in, d_out, dir, false);
    if (st != PACO_OK || pl->batch == 0) return st;
    if (!h_in || !h_out) return fail(PACO_ERR_INVALID_ARG, "NULL host buffer");
    set_device(pl);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)(pl->N * pl->batch) * pl->esize;
    PACO_CUDA_TRY(cudaMemcpyAsync(d_in, h_in, bytes, cudaMemcpyHostToDevice, s));
    if ((st = paco_execute(pl, d_in, d_out, dir, stream)) != PACO_OK) return st;
    PACO_CUDA_TRY(cudaMemcpyAsync(h_out, d_out, bytes, cudaMemcpyDeviceToHost, s));
    return PACO_OK;
}

extern "C" paco_status_t paco_plan_check(paco_plan_t *pl)
{
    if (!pl) return fail(PACO_ERR_INVALID_ARG, "plan is NULL");
    set_device(pl);
    PACO_CUDA_TRY(cudaDeviceSynchronize());
    int h = 0;
    PACO_CUDA_TRY(cudaMemcpy(&h, pl->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    PACO_CUDA_TRY(cudaMemset(pl->d_status, 0, sizeof(int)));
    if (h == PACO_ERR_TIMEOUT) return fail(PACO_ERR_TIMEOUT, "a bounded device wait gave up");
    if (h != 0) return fail(PACO_ERR_DEVICE, "device status word %d", h);
    return PACO_OK;
}

extern "C" paco_status_t paco_debug_exchange_counts(paco_plan_t *pl, const void *in, void *out, int dir,
                                                   int64_t *counts, paco_stream_t stream)
{
    paco_status_t st = check_exec(pl, in, out, dir, false);
    if (st != PACO_OK) return st;
    if (!pl->fused) return fail(PACO_ERR_UNSUPPORTED, "paco_debug_exchange_counts: the plan is not a one-launch cluster plan");
    if (!counts) return fail(PACO_ERR_INVALID_ARG, "counts is NULL");
    set_device(pl);
    const int p = pl->p;
    unsigned *d = nullptr;
    PACO_CUDA_TRY(cudaMalloc(&d, sizeof(unsigned) * p * p));
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned) * p * p, s);
    if (e == cudaSuccess && pl->batch > 0) st = launch_cluster(pl, in, out, dir, d, s);
    unsigned h[256] = {0};
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(unsigned) * p * p, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(PACO_ERR_CUDA, "paco_debug_exchange_counts: %s", cudaGetErrorString(e));
    if (st != PACO_OK) return st;
    for (int k = 0; k < p * p; ++k) counts[k] = (int64_t)h[k];
    return PACO_OK;
}

extern "C" paco_status_t paco_debug_set_waits(paco_plan_t *pl, unsigned spin_limit, unsigned wait_bias)
{
    if (!pl) return fail(PACO_ERR_INVALID_ARG, "plan is NULL");
    pl->dbg_spin_limit = spin_limit;
    pl->dbg_wait_bias = wait_bias;
    return PACO_OK;
}

extern "C" int64_t paco_digit_reverse(int64_t u, int b, int ell)
{
    int t = ilog2_exact(b);
    if (t < 1 || t > 4 || ell < 0 || (int64_t)ell * t > 31) return -1;
    const int bits = ell * t;
    if (u < 0 || u >= (int64_t(1) << bits)) return -1;
    if (bits == 0) return 0;
    // same construction as the device map: reverse all bits, then restore the
    // bit order inside every t-bit digit
    uint32_t x = 0, v = (uint32_t)u;
    for (int i = 0; i < bits; ++i) x |= ((v >> i) & 1u) << (bits - 1 - i);
    uint32_t y = 0;
    for (int d = 0; d < ell; ++d) {
        uint32_t dig = (x >> (d * t)) & ((1u << t) - 1u);
        uint32_t r = 0;
        for (int i = 0; i < t; ++i) r |= ((dig >> i) & 1u) << (t - 1 - i);
        y |= r << (d * t);
    }
    return (int64_t)y;
}
