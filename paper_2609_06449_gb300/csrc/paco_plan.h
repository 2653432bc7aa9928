// paco_plan.h -- host-side plan state shared by the library's translation
// units (not part of the C ABI; include/paco.h is the public interface).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/paco.h"

namespace paco {

struct StageCfg {
    int lgL = 0;      // log2 of the transform length of this stage
    int lgW = 0;      // log2 tile width
    int lgK = 0;      // log2 cluster size
    int threads = 0;
    int smem = 0;     // dynamic shared memory, bytes
    int ntiles = 0;   // column tiles per transform
    const void *fn = nullptr;
    const void *fn_terms = nullptr;   // the same stage with the weighted-loss terms (complex64), or nullptr
    const void *fn_scale = nullptr;   // ... with the scalar factor on Phase I's loads alone
    int panel = 0;    // 1: L2-resident panel pipeline (paco_panel.cuh)
    int P = 0;        // panel width (columns)
    // split = 1: the stage runs as two passes through the plan's scratch (pass A
    // of length 2^lgLa, pass B of length 2^lgLb; SplitArgs in paco_stage_args.cuh)
    int split = 0;
    int lgLa = 0, lgLb = 0;
    int sp_lgW[2] = {0, 0}, sp_threads[2] = {0, 0}, sp_smem[2] = {0, 0}, sp_ntiles[2] = {0, 0};
    const void *sp_fn[2] = {nullptr, nullptr};
    void *sp_tw[2] = {nullptr, nullptr};   // w_{2^lgLa}^{-r} and w_{2^lgLb}^{-r}
};

struct BatchedState;  // paco_batched.cu

} // namespace paco

struct paco_plan {
    int64_t N1 = 0, N2 = 0, N = 0, batch = 0;
    int b = 0, t = 0, p = 0, m1 = 0, m2 = 0;
    paco_dtype_t dtype = PACO_C64;
    int esize = 8;                 // bytes per complex element
    int device = 0;
    paco::StageCfg st[2];          // stage 1 (L = N1, C = N2), stage 2 (L = N2, C = N1)
    paco::StageCfg ph1;            // Phase I alone (mode 3), same geometry as st[0]
    void *twL1 = nullptr, *twL2 = nullptr, *twN_lo = nullptr, *twN_hi = nullptr;
    int twN_lo_bits = 0;
    int *d_status = nullptr;
    void *scratch = nullptr;       // panel ring buffers (L2-sized, not N-sized)
    unsigned *ctr = nullptr;       // panel pipeline counters
    size_t ctr_words = 0;
    int num_sms = 0;
    int form = 0;                  // tensor-core precision form (paco_tc.cuh), 0 = plain
    int req_ctas = 0;              // requested CTAs per SM of the stage kernels (0 = default)
    int req_split = 0;             // paco_plan_opts_t.split
    int dims = 1;                  // 2: the 2-D DFT (the top-level twiddle tables hold ones)
    int64_t N3 = 1;                // dims = 3: the third axis; N2 (the pipeline's factor) is N2' N3
    int lgLa3 = 0;                 // dims = 3: log2 of the middle axis N2' (Phase III's first split pass)
    void *tw_ones = nullptr;       // dims = 3: ones in place of Phase III's split twiddle w_N2^{-k_a j_b}
    unsigned dbg_spin_limit = 0;   // paco_debug_set_waits: poll limit of the bounded waits (0 = default)
    unsigned dbg_wait_bias = 0;    // paco_debug_set_waits: added to the dependency targets
    void *tc = nullptr;            // its fragment table
    int fused = 0;                 // 1: paco_execute is one cluster launch (paco_cluster.cu)
    int fused_k = 8;               //   its CTAs per transform (16 where the device allows that cluster)
    void *twN_full = nullptr;      // one-launch form: w_N^{-r}, r < N
    void *split_scratch = nullptr; // split stages: the intermediate of their two passes (N * batch)
    int shard_G = 0;               // sharded form (paco_plan_create_sharded): ranks, 0 = not sharded
    int shard_rank = 0;
    void *rs_maps = nullptr;       // restoring the input's ownership (paco_restore.cu): pack and unpack maps
    void *rs_off = nullptr;        //   their block offsets (send, then receive; G + 1 each)
    int64_t *rs_send_counts = nullptr, *rs_recv_counts = nullptr;   // host copies of the block sizes
    // uneven batch (paco_plan_create_batched): N = total elements, batch = 1
    paco::BatchedState *bs = nullptr;
};

namespace paco {

paco_status_t fail(paco_status_t st, const char *fmt, ...);
int ilog2_exact(int64_t v);
// FP64-generated table of w_M^{-(r*mult)}, r in [count], complex of `esize` bytes
paco_status_t gen_table(int esize, void **dst, long long M, long long count, long long mult,
                        cudaStream_t stream);

// paco_stage_tc.cu
const void *stage_kernel_fn_tc(int lgL, int form);
paco_status_t tc_table_create(int form, void **out);

// paco_permute.cu
paco_status_t launch_permute(const paco_plan *pl, const void *A_tilde, void *W, int dir,
                             cudaStream_t stream);

// paco_cluster.cu
bool cluster_eligible(const paco_plan *pl);
paco_status_t cluster_setup(paco_plan *pl);
paco_status_t launch_cluster(const paco_plan *pl, const void *in, void *out, int dir, unsigned *pair_count,
                             cudaStream_t stream);

// paco_restore.cu
paco_status_t restore_setup(paco_plan *pl);
void restore_destroy(paco_plan *pl);

// paco_batched.cu
paco_status_t batched_execute(paco_plan *pl, const void *in, void *out, int dir, cudaStream_t stream);
void batched_destroy(BatchedState *bs);
void batched_info(const paco_plan *pl, paco_plan_info_t *info);

} // namespace paco

#define PACO_CUDA_TRY(call)                                                                    \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return ::paco::fail(PACO_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
