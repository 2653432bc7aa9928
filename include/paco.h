/*
 * paco.h -- C ABI of the PACO FFT library for one GB300 (sm_103a).
 *
 * PACO ("A Fully Cache-Oblivious Parallel FFT with One Global
 * Redistribution") computes the canonical length-N DFT
 *
 *     y = Omega_N x,  (Omega_N)_{k,j} = w_N^{-kj},  w_N = exp(2*pi*i/N)
 *
 * (Sect. 2, "Model and Main Result") for N = N1*N2, N1 = b^m1, N2 = b^m2,
 * as LocalFFT -> one fused base-b digit-reversal permutation -> LocalFFT
 * (Sect. 3, Eq. (10)).  On one GPU the paper's p processors are p virtual
 * slabs; its one global redistribution (PARA-CO-DRP_b, Sect. 4.2) is the HBM
 * pass between the two stage kernels.
 *
 * Data layout (all entry points):
 *   - Complex data are interleaved (re, im): PACO_C64 = two floats (8 B),
 *     PACO_C128 = two doubles (16 B).  Buffers are device pointers unless an
 *     entry point says "host", aligned to 16 bytes, holding `batch`
 *     transforms back to back (stride N elements).
 *   - Input of one transform: x in natural order, i.e. the row-major
 *     N1 x N2 view X[j1, j2] = x[j1*N2 + j2] (Sect. 2, input view).
 *   - Output of one transform: the row-major N2 x N1 view
 *     Y[k2, k1] = y[k1 + k2*N1] (Eq. factor-swapped-output-view), which is
 *     natural-order y when read flat.  Slab q' of the output (Eq. (3),
 *     owner1 = floor(k1*p/N1)) is the column range k1 in [q'N1/p,(q'+1)N1/p).
 *   - dir = -1 computes the paper's transform (w^{-kj}); dir = +1 computes the
 *     unnormalised conjugate transform (w^{+kj}).  The paper defines only
 *     the forward transform; +1 is this library's reading (the adjoint).
 *
 * Ownership: the caller owns every buffer passed in.  A plan owns its
 * twiddle tables and a device status word; it holds no N-sized scratch (a
 * plan with a 2^14 complex64 factor also owns a 48 MiB ring of L2-resident
 * panel buffers and its counters).
 * Execution entry points enqueue work on `stream` and return without
 * synchronising; they allocate nothing.
 *
 * Errors: every entry point returns a paco_status_t (plan constructors that
 * return a pointer return NULL instead).  On failure a message for the
 * calling thread is available from paco_last_error().  Errors detected while
 * kernels run are reported by paco_plan_check().
 */
#ifndef PACO_H
#define PACO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without including the CUDA headers; NULL = legacy stream. */
typedef struct CUstream_st *paco_stream_t;

typedef struct paco_plan paco_plan_t;

typedef enum {
    PACO_OK = 0,
    PACO_ERR_INVALID_ARG = 1, /* sizes, radix, p, pointers, dir out of contract */
    PACO_ERR_UNSUPPORTED = 2, /* legal for the paper, not built here */
    PACO_ERR_ALIASING = 3,    /* in == out where the entry point forbids it */
    PACO_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    PACO_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
    PACO_ERR_NOMEM = 6,       /* plan allocation failed */
    PACO_ERR_DEVICE = 7       /* a device-side check set the status word */
} paco_status_t;

typedef enum {
    PACO_C64 = 0,           /* complex float in/out, FP32 arithmetic */
    PACO_C128 = 1,          /* complex double in/out, FP64 arithmetic */
    PACO_C64_TC_BF16X3 = 2, /* complex float in/out; radix-16 sub-DFTs as
                               3-term-split BF16 tensor-core products (six per
                               contraction, FP32 accumulation): complex64
                               accuracy; factors N1, N2 in 2^8..2^14 */
    PACO_C64_TC_FP16 = 3    /* complex float in/out; radix-16 sub-DFTs as FP16
                               tensor-core products with per-block scaling
                               (relative L2 error about 4e-4); factors N1, N2
                               in 2^8..2^14 */
} paco_dtype_t;

/* Plan options for paco_plan_create_ex.  Zero fields take defaults. */
typedef struct {
    int64_t N1, N2;      /* the two factors, N = N1*N2 (Sect. 2) */
    int b;               /* digit-reversal radix: 2, 4, 8 or 16 (b = 2^t) */
    int p;               /* virtual slabs; 0 = default b^floor(min(m1,m2)/2),
                            raised to b if that is 1 */
    int64_t batch;       /* transforms per execute, >= 0 */
    paco_dtype_t dtype;
    int tile_w;          /* columns per tile; 0 = default */
    int cluster;         /* CTAs per cluster (1, 2, 4, 8); 0 = default */
    int ctas_per_sm;     /* resident CTAs per SM the stage kernels are compiled
                            for (1 or 2; complex64 stage kernels only); 0 = default */
    int split;           /* complex64 stages of 2^12..2^14 as two passes through an
                            N * batch scratch (paco_plan_info.stage_split): 0 =
                            default (2^12, 2^13; 2^14 keeps the L2 panel pipeline),
                            1 = 2^14 as well, -1 = never */
    int dims;            /* 0 or 1: the 1-D DFT of length N (the paper's transform);
                            2: the 2-D DFT of the N1 x N2 view, out[k2][k1] =
                            sum_{j1,j2} x[j1 N2 + j2] w_N1^{-k1 j1} w_N2^{-k2 j2},
                            i.e. returned transposed (N2 x N1 row-major) -- the
                            same pipeline without the top-level twiddle: a slab
                            decomposition of the 2-D FFT with one redistribution;
                            3: the 3-D DFT of the N1 x N2 x N3 array (row-major,
                            x[(j1 N2 + j2) N3 + j3]), returned with its axes
                            reversed: out[(k3 N2 + k2) N1 + k1] = sum x[..]
                            w_N1^{-k1 j1} w_N2^{-k2 j2} w_N3^{-k3 j3}.  The
                            pipeline runs on the N1 x (N2 N3) view without the
                            top-level twiddle, Phase III as two passes over the
                            N2 x N3 planes (Sect. 4.1's top split, with ones for
                            its twiddle).  complex64, not sharded; N2 and N3
                            powers of b in 2^5..2^8 with N2 N3 <= 2^14; p must
                            divide N1 and N2 N3; the weighted entry points
                            reject it (PACO_ERR_UNSUPPORTED) */
    int64_t N3;          /* dims = 3: the third axis; 0 (or 1) otherwise, else
                            PACO_ERR_INVALID_ARG */
} paco_plan_opts_t;

/* Read-only description of a plan (paco_plan_info). */
typedef struct {
    int64_t N1, N2, N, batch;
    int b, p, m1, m2;
    paco_dtype_t dtype;
    int slab_width_ok;           /* N1/p and N2/p span >= 128 B (Eq. (5)) */
    int64_t items_per_pair;      /* N/p^2 (Eq. fused-global-pairwise-volume) */
    int64_t h;                   /* (N/p)(1 - 1/p) (Eq. fused-global-h-volume) */
    int64_t mu;                  /* N(1 - 1/p) (Eq. fused-global-total-volume) */
    int stage_tile_w[2];         /* tile width used by stage 1 / stage 2 */
    int stage_cluster[2];        /* cluster size used by stage 1 / stage 2 */
    int stage_threads[2];        /* threads per CTA */
    int stage_smem[2];           /* dynamic shared memory per CTA, bytes */
    int fused_cluster;           /* 1: paco_execute runs the whole transform as one
                                    cluster launch (see paco_execute) */
    int shard_G;                 /* sharded plan: G ranks (0: not sharded) */
    int shard_rank;              /* sharded plan: this rank */
    int stage_split[2];          /* 1: the stage runs as two passes through the plan's
                                    N * batch scratch (complex64 stages of 2^12, 2^13) */
    int dims;                    /* 1: the 1-D DFT; 2: the 2-D DFT of the N1 x N2 view;
                                    3: the 3-D DFT of the N1 x N2 x N3 array (m2, p,
                                    items_per_pair, h and mu then refer to the
                                    pipeline's second factor N2 N3) */
    int64_t N3;                  /* dims = 3: the third axis; 1 otherwise */
} paco_plan_info_t;

/*
 * paco_plan_create -- plan `batch` PACO transforms of size N = N1*N2 with
 * digit-reversal radix b (Sect. 2: b = 2^t, N1 = b^m1, N2 = b^m2, p | N1,
 * p | N2, Eq. exact-divisibility) in precision `dtype`, on the current CUDA
 * device.  Builds the twiddle tables in FP64 on the device and waits for
 * them.  Returns NULL on error (paco_last_error() says why): N1 or N2 not a
 * power of b, b not in {2,4,8,16}, N > 2^32, batch < 0, or a dtype that is
 * not built.  The default p is described at paco_plan_opts_t.
 */
paco_plan_t *paco_plan_create(int64_t N1, int64_t N2, int b, int64_t batch,
                              paco_dtype_t dtype);

/* paco_plan_create_ex -- as paco_plan_create with explicit options (p, tile,
 * cluster, CTAs per SM).  p must be a power of b with p >= 2, p | N1 and p | N2
 * (Eq. exact-divisibility).  Writes the plan to *out (NULL on error). */
paco_status_t paco_plan_create_ex(paco_plan_t **out, const paco_plan_opts_t *opts);

/* paco_plan_destroy -- free the plan's tables.  NULL is accepted.  The
 * caller must ensure no work using the plan is still running. */
void paco_plan_destroy(paco_plan_t *plan);

/* paco_plan_info -- fill *info for the plan. */
paco_status_t paco_plan_info(const paco_plan_t *plan, paco_plan_info_t *info);

/*
 * paco_execute -- y = PACO(x) for every transform of the batch (Theorem 3):
 * Phase I (LocalFFT, output layout, Lemma 1) with the top-level twiddle and
 * the full digit reversal pi_m of Eq. (full-middle-digit-reversal) fused into
 * its stores (the PARA-CO-DRP_b middle stage, Sect. 4.2), then Phase III
 * (LocalFFT, input layout) reading that layout.  `in` and `out` are device
 * buffers of batch*N elements of the plan's dtype; `out` also holds the
 * intermediate W = Z-hat (Eq. (17)) between the two kernels, so no scratch
 * is used.  in == out, or overlapping buffers, return PACO_ERR_ALIASING.
 * batch = 0 is a no-op.  Asynchronous on `stream`.  A complex64 plan with
 * N1 = N2 = 256, p = 4 or 8 and batch <= 16 (where one launch is faster than
 * two) runs as ONE launch (paco_plan_info.fused_cluster): a thread-block
 * cluster of K = 16 CTAs per transform (8 where the GPU cannot host a
 * 16-CTA cluster), processor q of Sect. 2 being the K/p CTAs that hold its
 * slab -- Phase I on the input columns in shared memory, then PARA-CO-DRP_b
 * (Sect. 4.2, App. C.5) as one all-to-all of asynchronous stores into the
 * other CTAs' shared memory (N/p^2 items per ordered pair of processors, a
 * CTA's items for itself kept in the CTA), then Phase
 * III on its output columns; W never reaches global memory.  The launch
 * allows programmatic dependent launch (it waits for the preceding kernels
 * before it reads `in`).  A device-side wait of this form that gives up after
 * 2 s sets the status word that paco_plan_check reads (PACO_ERR_TIMEOUT).
 * Executions of one plan
 * must not overlap in time (a plan with a 2^14 complex64 factor, and an
 * uneven-batch plan, run pipelines whose ring buffers and counters the plan
 * owns): use one plan per concurrently used stream.
 */
paco_status_t paco_execute(paco_plan_t *plan, const void *in, void *out, int dir,
                           paco_stream_t stream);

/*
 * The sharded form -- PARA-CO-DRP across G ranks (Sect. 4.2, App. C.5; one
 * GPU per rank, G = p processors).  Rank g holds input slab g, the columns
 * c in [g Cl, (g+1) Cl) of X = x viewed N1 x N2 (Cl = N2/G), and gets output
 * slab g, the columns k1 in [g K1, (g+1) K1) of Y = y viewed N2 x N1
 * (K1 = N1/G).  Per rank:
 *   paco_shard_stage1  Phase I on the local slab (length-N1 column DFTs, the
 *                      top-level twiddle w_N^{-k1 c} at the global column c),
 *                      stored as G send blocks of N/G^2 items (Theorem 4):
 *                      block q' holds k1 in rank q''s slab, its rows in the
 *                      order pi(c - g Cl) -- the digit reversal over the
 *                      local column's digits, the part of pi_m2 that stays on
 *                      the rank (Eq. (17) with c = g Cl + c_l: pi_m2(c) =
 *                      pi(c_l) G + pi(g));
 *   (exchange)         block q' of every rank's send buffer goes to rank q',
 *                      into block g of its receive buffer (an all-to-all of
 *                      equal blocks, e.g. NCCL grouped send/recv or
 *                      torch.distributed.all_to_all_single; the caller runs
 *                      it -- this library holds no communicator);
 *   paco_shard_stage2  Phase III on the local output columns, reading W row
 *                      pi_m2(j), j = j_h Cl + j_l, as row pi(j_l) of the block
 *                      from rank j_h.
 * Layouts (complex64, device): x_local [batch][N1][Cl]; send and recv
 * [G][batch][Cl][K1] (block for / from rank g, N/G^2 items per transform);
 * y_local [batch][N2][K1].  G must be a power of b with 2 <= G, G | N1 and
 * G | N2, N2/G >= b; batch <= 65535.  dir = +1 is the conjugate transform, as in
 * paco_execute.  A sharded plan takes only these two calls (paco_execute and
 * the others return PACO_ERR_UNSUPPORTED).
 */
typedef struct {
    int64_t N1, N2;
    int b;
    int G;               /* ranks */
    int rank;            /* this rank, in [0, G) */
    int64_t batch;
    paco_dtype_t dtype;  /* PACO_C64 */
    int restore;         /* 1: also build the maps of paco_shard_restore_* */
    int dims;            /* 2: the 2-D DFT of the N1 x N2 view (as paco_plan_opts_t.dims):
                            the slab-decomposed 2-D FFT across the G ranks; 3 is
                            not built for the sharded form (PACO_ERR_UNSUPPORTED) */
} paco_shard_opts_t;

paco_status_t paco_plan_create_sharded(paco_plan_t **out, const paco_shard_opts_t *opts);
/* x_local -> send (Phase I of the rank's slab, packed for the exchange); in != out */
paco_status_t paco_shard_stage1(paco_plan_t *plan, const void *x_local, void *send, int dir,
                                paco_stream_t stream);
/* recv -> y_local (Phase III of the rank's output columns); in != out */
paco_status_t paco_shard_stage2(paco_plan_t *plan, const void *recv, void *y_local, int dir,
                                paco_stream_t stream);

/*
 * paco_probe_tc05_dft128 -- measurement probe (the paper has no
 * counterpart): the 128-point DFT sub-pass of a 2^14 stage on the tcgen05
 * tensor cores, y[b][k][c] = sum_j w_128^{-jk} x[b][j][c] for every b < batch,
 * k < 128, c < C (complex64, [batch][128][C], device, 16-byte aligned, C a
 * multiple of 64, in != out), as a BF16x3 complex GEMM with FP32 accumulators
 * in tensor memory (relative error about 1e-5: the operands are kept to
 * about 2^-17).  With ms != NULL the call waits and returns the kernel's
 * CUDA-event time; a wait for the tensor-core operations that gives up
 * returns PACO_ERR_TIMEOUT.  Builds its 128 KiB operand table on first use.
 */
paco_status_t paco_probe_tc05_dft128(const void *x, void *y, int64_t batch, int64_t C, float *ms,
                                     paco_stream_t stream);

/*
 * Restoring the input's ownership -- the second redistribution the paper
 * leaves out (Sect. 6, Limitations): after paco_shard_stage2 rank q holds
 * y_local = Y[:, q K1 .. (q+1) K1) (K1 = N1/G); afterwards rank r holds y in
 * the layout its input had, y viewed N1 x N2, columns j in [r Cl, (r+1) Cl)
 * (Cl = N2/G): [batch][N1][Cl].  Element k of y moves from rank
 * floor((k mod N1) / K1) to rank floor((k mod N2) / Cl); each block carries
 * its items in increasing k.  Block sizes differ between pairs unless
 * N1 = N2 (then every item stays on its rank).  Per rank:
 *   paco_shard_restore_pack    y_local -> send, [G][batch][send_counts[r]]
 *   (exchange)                 block r of every rank's send buffer to rank r,
 *                              into block q (the sender) of its receive buffer,
 *                              [G][batch][recv_counts[q]] (an all-to-all with
 *                              uneven splits: counts times batch);
 *   paco_shard_restore_unpack  recv -> x_layout, [batch][N1][Cl].
 * The plan must be created with paco_shard_opts_t.restore = 1 (it then owns
 * two int32 maps of N/G entries; N/G < 2^31); otherwise
 * PACO_ERR_UNSUPPORTED.  Buffers: device, complex64, 8-byte aligned, in != out.
 * paco_shard_restore_counts gives the block sizes per transform (G entries
 * each, either pointer may be NULL).  paco_shard_restore_maps is the host
 * computation of one rank's maps and counts (no device needed; arrays of
 * N/G and G entries, NULL to skip), for tests and for callers that move the
 * data themselves.
 */
paco_status_t paco_shard_restore_counts(const paco_plan_t *plan, int64_t *send_counts, int64_t *recv_counts);
paco_status_t paco_shard_restore_pack(paco_plan_t *plan, const void *y_local, void *send, paco_stream_t stream);
paco_status_t paco_shard_restore_unpack(paco_plan_t *plan, const void *recv, void *x_layout, paco_stream_t stream);
paco_status_t paco_shard_restore_maps(int64_t N1, int64_t N2, int G, int rank, int32_t *pack_map,
                                      int64_t *send_counts, int32_t *unpack_map, int64_t *recv_counts);

/*
 * paco_execute_weighted_power -- paco_execute plus the weighted power of the
 * result, for a spectral loss: y = F^dir x as paco_execute computes it, and
 * *loss = sum over the whole batch of w[n] |y[n]|^2, accumulated by the
 * Phase III kernel as it stores y (the sum is not a separate pass; *loss is
 * set to 0 on `stream` first, then added to atomically in FP64: its rounding
 * order varies between runs).  out_weighted = 0 stores y in `out`; 1 stores
 * w ⊙ y instead (what the loss's backward needs, at no extra cost: the
 * kernel already holds w[n]).  w: device, batch*N floats in the layout of y;
 * loss: device, one double, 8-byte aligned.  The paper's transform is
 * unchanged (Theorem 3); the loss is an epilogue of the last stage.  Plans
 * with a 2^14 complex64 factor (panel stages) and uneven-batch plans return
 * PACO_ERR_UNSUPPORTED; a one-launch cluster plan runs its two stage launches
 * here.  Asynchronous on `stream`.
 */
paco_status_t paco_execute_weighted_power(paco_plan_t *plan, const void *in, void *out, const float *w,
                                          double *loss, int out_weighted, int dir, paco_stream_t stream);

/*
 * paco_execute_weighted_input -- out = F^dir (s * w ⊙ in) with the
 * element-wise product applied as Phase I loads its input (no separate
 * pass): s = mult * (*scale), or mult when scale is NULL; w = NULL applies
 * the scalar s alone.  w: device, batch*N floats in the layout of `in`;
 * scale: device double or NULL.  With dir = +1, in = w ⊙ y (the output of
 * paco_execute_weighted_power with out_weighted = 1), w = NULL, mult = 2 and
 * scale the incoming gradient g of that loss, out is the loss's gradient
 * with respect to x, F^H (2 g w ⊙ F x) (the conjugate transform being F^H).
 * Same plans and errors as paco_execute_weighted_power.
 */
paco_status_t paco_execute_weighted_input(paco_plan_t *plan, const void *in, void *out, const float *w,
                                          const double *scale, float mult, int dir, paco_stream_t stream);

/*
 * paco_execute_stage1 -- Phase I and the fused middle stage only: writes
 * W[u][v] = Z-hat[u, v] = Z[v, pi_m2(u)] with Z[v, c] = A[v, c] w_N^{dir*vc}
 * and A the length-N1 column DFTs (Sect. 4.2, local pack and Eq. (17)),
 * as a row-major N2 x N1 array per transform.  in != W required.
 */
paco_status_t paco_execute_stage1(paco_plan_t *plan, const void *in, void *W, int dir,
                                  paco_stream_t stream);

/*
 * paco_execute_stage2 -- Phase III only: for every column v of W (N2 x N1,
 * Eq. (17) layout), the length-N2 DFT of the logical input W[pi_m2(j)][v]
 * (input-layout operator B_m2 = Omega P_pi, Lemma 1), written to
 * out[k2][v].  W == out is allowed (in place); partial overlap is not.
 */
paco_status_t paco_execute_stage2(paco_plan_t *plan, const void *W, void *out, int dir,
                                  paco_stream_t stream);

/*
 * paco_execute_phase1 -- Phase I alone, unfused: the output-layout local FFT
 * A-tilde[a, c] = A[pi_m1(a), c] (Lemma 1, Eq. output-layout-local-operator)
 * written as a row-major N1 x N2 array per transform, with no twiddle and no
 * redistribution.  Together with paco_permute and paco_execute_stage2 it
 * forms the unfused three-pass pipeline.  in != out required.
 */
paco_status_t paco_execute_phase1(paco_plan_t *plan, const void *in, void *out, int dir,
                                  paco_stream_t stream);

/*
 * paco_permute -- the middle stage PARA-CO-DRP_b as a standalone pass
 * (App. C.5): reads A-tilde (N1 x N2, layout of paco_execute_phase1) and
 * writes W[pi_m2(c)][pi_m1(a)] = A-tilde[a][c] * w_N^{dir*pi_m1(a)*c}
 * (N2 x N1), i.e. pack with the fused twiddle, the all-to-all of N/p^2-item
 * blocks, the per-block transpose and the unpack, in one gather.  in != W.
 */
paco_status_t paco_permute(paco_plan_t *plan, const void *A_tilde, void *W, int dir,
                           paco_stream_t stream);

/*
 * paco_execute_host -- paco_execute on HOST buffers: copies h_in (batch*N
 * elements, pinned or pageable host memory) to the device buffer d_in,
 * runs paco_execute(d_in -> d_out), and copies d_out back to h_out, all
 * enqueued on `stream`; returns once the work is enqueued (synchronise the
 * stream before reading h_out).  d_in and d_out are caller-owned device
 * buffers of batch*N elements and must not overlap.
 */
paco_status_t paco_execute_host(paco_plan_t *plan, const void *h_in, void *h_out,
                                void *d_in, void *d_out, int dir, paco_stream_t stream);

/*
 * paco_plan_check -- synchronise the device, then read and clear the plan's
 * device status word.  Returns PACO_OK, PACO_ERR_DEVICE or PACO_ERR_TIMEOUT
 * for errors raised by kernels since the last check, or PACO_ERR_CUDA.
 */
paco_status_t paco_plan_check(paco_plan_t *plan);

/* paco_last_error -- message for the last failure on the calling thread
 * ("" if none).  The string stays valid until the thread's next call. */
const char *paco_last_error(void);

/*
 * paco_digit_reverse -- pi_ell(u) in base b (Sect. 3.2, App. A.1): the
 * ell-digit base-b string of u written in reverse digit order; the same map
 * the kernels compute.  Returns -1 if b is not in {2,4,8,16}, ell*log2(b)
 * exceeds 31, or u >= b^ell.  Host-only, no GPU needed.
 */
int64_t paco_digit_reverse(int64_t u, int b, int ell);

/* paco_version -- library version string. */
const char *paco_version(void);

/*
 * Uneven batches.  The paper transforms one length at a time; its
 * scheduler splits the transform and the batch dimensions with the same
 * recursion (Sect. 4.1, batch field of the digit split), which is what a
 * batch of many lengths needs.  This library runs such a batch as one
 * persistent launch over a queue of equal-sized work items (the method per
 * transform is unchanged: Phase I, fused twiddle + digit reversal, Phase III).
 *
 * paco_plan_create_batched -- plan for `count` complex64 transforms whose
 * lengths are lengths[0..count) (each a power of two, 2^4 .. 2^20; the
 * factorisation N = N1*N2 and the radix b are chosen per length).  Buffers
 * passed to paco_execute / paco_execute_host hold the transforms back to
 * back in the given order (transform i starts at element
 * sum_{j<i} lengths[j]); each is computed as by a single-length plan (natural
 * order in and out).  The default constructor autotunes: it times candidate
 * configurations on plan-owned scratch buffers (allocated and freed inside
 * the call, up to 2 x 512 MiB) and keeps the fastest.  Returns
 * PACO_ERR_UNSUPPORTED for other dtypes or lengths, PACO_ERR_INVALID_ARG for
 * a NULL list with count > 0.  Execution of such a plan is one
 * cudaMemsetAsync of its counters and one kernel launch on `stream`, so it can
 * be captured in a CUDA graph.  paco_execute_stage1/2, _phase1 and
 * paco_permute return PACO_ERR_UNSUPPORTED for it; paco_plan_info reports
 * N = the total length and batch = count.
 */
typedef struct {
    int autotune;     /* 1: time candidates at plan creation (default constructor) */
    int b;            /* 0: per length; else the radix for every length it fits */
    int ctas_per_sm;  /* 1 or 2 resident CTAs per SM (autotuned when autotune=1) */
    int lag;          /* Phase III lag after Phase I, in grids of work items (0: 2) */
} paco_batched_opts_t;

paco_status_t paco_plan_create_batched(paco_plan_t **out, const int64_t *lengths, int64_t count,
                                       paco_dtype_t dtype);
paco_status_t paco_plan_create_batched_ex(paco_plan_t **out, const int64_t *lengths, int64_t count,
                                          paco_dtype_t dtype, const paco_batched_opts_t *opts);

/* paco_plan_batched_config -- the configuration an uneven-batch plan uses
 * for one of its lengths (radix b, first factor N1) and overall (CTAs per SM,
 * Phase III lag).  Any output pointer may be NULL.  PACO_ERR_INVALID_ARG if
 * the plan is not an uneven batch or does not hold that length. */
paco_status_t paco_plan_batched_config(const paco_plan_t *plan, int64_t length, int *b, int *N1,
                                       int *ctas_per_sm, int *lag);

/*
 * paco_debug_set_waits -- test hook for the kernels' bounded waits (the
 * paper has no counterpart).  The pipelined kernels (the 2^14 panel stages,
 * the uneven-batch kernel) wait on completion counters of other CTAs; each
 * wait gives up after a poll limit and records PACO_ERR_TIMEOUT in the plan's
 * status word (read by paco_plan_check) instead of hanging.  spin_limit
 * replaces the default poll limit (0 restores it); wait_bias is added to every
 * counter target, so with wait_bias > 0 no such wait can be met: the next
 * execution of the plan returns garbage and paco_plan_check reports
 * PACO_ERR_TIMEOUT, and the CUDA context stays usable.  In the one-launch
 * cluster form (fused_cluster = 1) wait_bias > 0 makes each CTA's transaction
 * barrier expect 8 * wait_bias bytes that never come, so its 2 s wait runs
 * out the same way.  Set both to 0 for normal use.  Returns
 * PACO_ERR_INVALID_ARG for a NULL plan.
 */
paco_status_t paco_debug_set_waits(paco_plan_t *plan, unsigned spin_limit, unsigned wait_bias);

/*
 * paco_debug_exchange_counts -- test hook (the paper has no counterpart):
 * runs paco_execute of a one-launch cluster plan (fused_cluster = 1) once,
 * counting the items each CTA writes to each destination CTA in the
 * all-to-all, added up per ordered pair of processors, and stores them in
 * counts[q * p + q'] (p x p, source processor q, destination q'), for every
 * transform of the batch added together; waits
 * for the result.  Theorem 4 fixes each count at batch * N/p^2.  Allocates a
 * small device buffer (a test hook, not an execution entry point).
 * PACO_ERR_UNSUPPORTED for other plans.
 */
paco_status_t paco_debug_exchange_counts(paco_plan_t *plan, const void *in, void *out, int dir,
                                         int64_t *counts, paco_stream_t stream);

/*
 * paco_debug_batched_schedule -- test hook (host only, no GPU): the work
 * queue an uneven-batch plan executes, in claim order, for `count` lengths
 * (powers of two 2^4..2^20) and a Phase III lag of `lag_items` items.  Item k
 * is kind[k] = 0 (a group of small transforms: group[index[k] ..
 * index[k] + tile[k]) lists them), 1 (Phase I tile tile[k] of transform
 * index[k]) or 2 (Phase III tile tile[k] of transform index[k]).  Returns the
 * number of items, or -1 for bad arguments or when `cap` / `group_cap` is too
 * small.
 */
int64_t paco_debug_batched_schedule(const int64_t *lengths, int64_t count, int64_t lag_items,
                                    int32_t *kind, int32_t *index, int32_t *tile, int64_t cap,
                                    int32_t *group, int64_t group_cap);

/*
 * paco_probe_fp64_peak -- measure the FP64 fused multiply-add rate of the
 * current device (the paper has no counterpart: it is the denominator of the
 * complex128 roofline, since those transforms are bound by FP64 arithmetic
 * on this GPU).  One launch of 8 blocks per SM x 256 threads, each running 8
 * independent chains of 16 * iters FMAs, timed with CUDA events on `stream`
 * after a short warm-up launch; synchronises the stream.  *gflops receives
 * the rate (an FMA counts as two flops) at whatever clock the GPU ran, *ms
 * (may be NULL) the kernel time.  PACO_ERR_INVALID_ARG for iters < 1 or a
 * NULL gflops.  Allocates nothing.
 */
paco_status_t paco_probe_fp64_peak(int64_t iters, double *gflops, float *ms, paco_stream_t stream);

/* Largest batch that paco_execute_noalloc accepts. */
#define PACO_NOALLOC_MAX_BATCH 16

/*
 * paco_execute_noalloc -- the complex64 transform of paco_execute for
 * N1 = N2 = 2^14 (N = 2^28, b = 2 or 4), for callers that cannot allocate
 * device memory: code running while a CUDA graph is captured, inside a
 * framework whose pool owns the device memory, or anywhere the allocator must
 * not be touched after start-up.  The paper has no counterpart; this is a
 * deployment form of the same kernels.  No plan: everything it needs (panel
 * buffers, pipeline counters, status word, twiddle tables; about 24.4 MiB)
 * lives in device arrays that the library reserves on every GPU that loads it,
 * until the process exits.  The call allocates and frees nothing.
 *   in, out  device buffers of batch * 2^28 complex64 values, 16-byte aligned,
 *            not overlapping (layout as paco_execute); 0 <= batch <=
 *            PACO_NOALLOC_MAX_BATCH, larger batches return
 *            PACO_ERR_INVALID_ARG; b other than 2 or 4 too.
 * The first call on a device takes the arrays' device addresses and fills the
 * twiddle tables (synchronously); make it before any stream capture.  Later
 * calls only enqueue work on `stream`.  All calls on one device share the
 * arrays and each leaves its intermediates there: calls whose work overlaps on
 * the GPU race and must be ordered by the caller.  Argument and launch errors
 * are returned by the call (message from paco_last_error()); errors raised
 * while its kernels run (a bounded wait that gave up) are recorded in the
 * library's status word on the device and returned by the next
 * paco_noalloc_check() on that device.
 */
paco_status_t paco_execute_noalloc(const void *in, void *out, int b, int64_t batch, int dir,
                                   paco_stream_t stream);

/*
 * paco_noalloc_check -- the device-side status of paco_execute_noalloc on
 * the current device: synchronises the device, reads and clears the status
 * word the kernels write, and returns PACO_OK, PACO_ERR_TIMEOUT (a bounded
 * wait gave up: the output of the call that raised it is not valid) or
 * PACO_ERR_DEVICE; PACO_ERR_CUDA if the device cannot be read.  Allocates
 * nothing.  PACO_OK when paco_execute_noalloc has not run on the device.
 */
paco_status_t paco_noalloc_check(void);

/*
 * paco_debug_noalloc_set_waits -- test hook for the bounded waits of
 * paco_execute_noalloc, as paco_debug_set_waits is for a plan (the paper has
 * no counterpart): spin_limit replaces the default poll limit (0 restores
 * it), wait_bias is added to every dependency target, so with wait_bias > 0
 * the next call's waits give up and paco_noalloc_check reports
 * PACO_ERR_TIMEOUT while the CUDA context stays usable.  Applies to calls
 * made after it, on every device.  Set both to 0 for normal use.
 */
void paco_debug_noalloc_set_waits(unsigned spin_limit, unsigned wait_bias);

#ifdef __cplusplus
}
#endif

#endif /* PACO_H */
