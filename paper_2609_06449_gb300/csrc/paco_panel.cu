// paco_panel.cu -- the panel-pipeline stage kernel (length-2^14 stages,
// complex64) and the host code that prepares one launch of it: the tensor
// maps of its loads and stores and its arguments (used by plans and by
// paco_execute_noalloc).
#define PACO_PANEL_KERNEL_TU
#include "paco_panel.cuh"

#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "paco_panel_host.h"

namespace paco {

template __global__ void paco_panel_kernel<1, 0>(const __grid_constant__ PanelArgs);
template __global__ void paco_panel_kernel<2, 2>(const __grid_constant__ PanelArgs);
template __global__ void paco_panel_kernel<2, 4>(const __grid_constant__ PanelArgs);

const void *panel_kernel_fn(int mode, int b)
{
    if (mode == 1) return reinterpret_cast<const void *>(&paco_panel_kernel<1, 0>);
    if (mode == 2 && b == 2) return reinterpret_cast<const void *>(&paco_panel_kernel<2, 2>);
    if (mode == 2 && b == 4) return reinterpret_cast<const void *>(&paco_panel_kernel<2, 4>);
    return nullptr;
}

// stage buffers plus the slack that aligns them to 1024 bytes
int panel_smem_bytes() { return panel::NSTAGE * (int)panel::TILE_BYTES + 1024; }

namespace {

PFN_cuTensorMapEncodeTiled_v12000 tensor_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// 8-byte elements, 128-byte swizzle (16-element inner box).
bool encode(CUtensorMap *m, const void *base, int rank, const cuuint64_t *dims, const cuuint64_t *strides,
            const cuuint32_t *box, bool promote)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_encoder();
    if (!enc) return false;
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)rank, const_cast<void *>(base), dims, strides,
               box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               promote ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int lg2(int64_t v)
{
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return ((int64_t(1) << l) == v) ? l : -1;
}

} // namespace

// Stage 2 reads, for a fixed j_lo, the 128 rows u = pi_m2(j_lo + 128 j_hi) of
// W (14 row bits).  pi is a bit permutation, so these rows are the rows whose
// bits outside the image of j_hi's bits equal those of pi(j_lo): a tensor box
// whose row dimensions are the runs of spanned bits (box = the run) and fixed
// bits (box 1).  The spanned runs are ordered so that the landing row's low
// three bits are the images of j_hi's bits 0-2 (a bijection of t8), which
// keeps the consumers' swizzled reads conflict-free:
//   b = 2 (pi = 14-bit reversal; j_hi bit k -> row bit 6 - k): dimensions
//         (v, rows bits 4-6, bits 0-3, bits 7-13 + batch): rank 4;
//   b = 4 (base-4 digit reversal; j_hi bits 0,1,2 -> row bits 7,4,5): (v,
//         bit 7, bits 4-5, bits 0-3, bits 8-13 + batch) with row bit 6 fixed
//         by j_lo, folded into a second map based 64 rows further: rank 5.
// The landing order this gives is land_lo / land_hi in paco_panel.cuh.
paco_status_t panel_prepare(const PanelLaunch &l, PanelArgs *a)
{
    memset(a, 0, sizeof(*a));
    const int E = 8;
    const int lgC = lg2(l.C), lgP = lg2(l.P);
    if (lgC < 7 || lgP < 6 || l.P > l.C || l.batch < 1 || (l.b != 2 && l.b != 4) || (l.mode != 1 && l.mode != 2))
        return fail(PACO_ERR_UNSUPPORTED, "panel stage: unsupported geometry (C=%lld, P=%d, b=%d)",
                    (long long)l.C, l.P, l.b);
    a->scratch = l.scratch;
    a->ctr = l.ctr;
    a->status = l.status;
    a->P = l.P;
    a->lgP = lgP;
    a->panels_per_batch = (int)(l.C / l.P);
    a->lgPpb = lgC - lgP;
    a->npanels = (int)(l.batch * a->panels_per_batch);
    a->rev_t = (l.b == 2) ? 1 : 2;
    a->twL = l.twL;
    a->twN_lo = l.twN_lo;
    a->twN_hi = l.twN_hi;
    a->twN_lo_bits = l.twN_lo_bits;
    a->N_mask = (unsigned)(l.N - 1);
    a->conj = l.conj;
    a->spin_limit = l.spin_limit ? l.spin_limit : 1u << 22;
    a->dep_bias = l.dep_bias;
    const cuuint64_t P = (cuuint64_t)l.P, NB = (cuuint64_t)panel::NBUF;
    const cuuint64_t C = (cuuint64_t)l.C, batch = (cuuint64_t)l.batch;
    bool ok = true;
    if (l.mode == 1) {
        // stage 1: L = N1 = 2^14 rows of X, C = N2 columns; W is N2 x N1
        a->N2rows = (int)l.C;
        a->rev_bits = lgC;
        {   // X as (c, j_lo, j_hi + 128 batch)
            const cuuint64_t dims[3] = {C, 128, 128 * batch};
            const cuuint64_t str[2] = {C * E, 128 * C * E};
            const cuuint32_t box[3] = {16, 1, 128};
            ok = ok && encode(&a->map_ld, l.in, 3, dims, str, box, true);
        }
        {   // panel ring [c][j_lo][k_lo] as (k_lo, j_lo, c)
            const cuuint64_t dims[3] = {128, 128, NB * P};
            const cuuint64_t str[2] = {128 * E, 128 * 128 * E};
            const cuuint32_t box[3] = {16, 128, 1};
            ok = ok && encode(&a->map_scr_ld, l.scratch, 3, dims, str, box, false);
            ok = ok && encode(&a->map_scr_st, l.scratch, 3, dims, str, box, false);   // unused in stage 1
        }
        {   // W (row length N1 = 2^14) as (k_lo, k_hi, u + N2 batch)
            const cuuint64_t dims[3] = {128, 128, C * batch};
            const cuuint64_t str[2] = {128 * E, 16384 * E};
            const cuuint32_t box[3] = {16, 128, 1};
            ok = ok && encode(&a->map_out, l.out, 3, dims, str, box, false);
        }
        a->map_ld_alt = a->map_ld;
    } else {
        // stage 2: L = N2 = 2^14 rows of W, C = N1 columns; Y is N2 x N1
        a->N2rows = 16384;
        a->rev_bits = 14;
        const cuuint64_t R = C * E;                           // row stride of W
        if (l.b == 2) {
            const cuuint64_t dims[4] = {C, 8, 16, 128 * batch};
            const cuuint64_t str[3] = {16 * R, R, 128 * R};
            const cuuint32_t box[4] = {16, 8, 16, 1};
            ok = ok && encode(&a->map_ld, l.in, 4, dims, str, box, true);
            a->map_ld_alt = a->map_ld;
        } else {
            const cuuint64_t dims[5] = {C, 2, 4, 16, 64 * batch};
            const cuuint64_t str[4] = {128 * R, 16 * R, R, 256 * R};
            const cuuint32_t box[5] = {16, 2, 4, 16, 1};
            ok = ok && encode(&a->map_ld, l.in, 5, dims, str, box, true);
            ok = ok && encode(&a->map_ld_alt, static_cast<const char *>(l.in) + 64 * R, 5, dims, str, box, true);
        }
        {   // panel ring [k_lo][j_lo][v] as (v, j_lo, k_lo)
            const cuuint64_t dims[3] = {P, 128, 128 * NB};
            const cuuint64_t str[2] = {P * E, 128 * P * E};
            const cuuint32_t bld[3] = {16, 128, 1}, bst[3] = {16, 1, 128};
            ok = ok && encode(&a->map_scr_ld, l.scratch, 3, dims, str, bld, false);
            ok = ok && encode(&a->map_scr_st, l.scratch, 3, dims, str, bst, false);
        }
        {   // Y as (v, k_lo, k_hi + 128 batch)
            const cuuint64_t dims[3] = {C, 128, 128 * batch};
            const cuuint64_t str[2] = {C * E, 128 * C * E};
            const cuuint32_t box[3] = {16, 1, 128};
            ok = ok && encode(&a->map_out, l.out, 3, dims, str, box, false);
        }
    }
    if (!ok) return fail(PACO_ERR_CUDA, "panel stage: tensor map encoding failed");
    return PACO_OK;
}

} // namespace paco
