// paco_cluster.cu -- the whole PACO transform of a small size in one launch,
// with the paper's p processors as groups of CTAs of one thread-block cluster.
//
// N1 = N2 = 256, p in {4, 8}.  The transform runs on a cluster of K CTAs
// (K = 16 where the GPU allows that cluster size, else 8; K is a multiple of
// p): processor q of Sect. 2 is the group of K/p consecutive CTAs, and CTA r
// owns 256/K of its slab's columns on both sides, so that more SMs share the
// work of one transform.  CTA r:
//   Phase I    owns input columns c in [r 256/K, (r+1) 256/K) of X = x viewed
//              N1 x N2 (processor q = floor(r p / K) owns slab q, Eq.
//              input-slab-owner) and computes their length-256 DFTs in shared
//              memory (radix 16 x 16);
//   middle     each result A[v][c] takes the top-level twiddle w_N^{-vc} and
//              goes straight to the CTA that owns output column v (its
//              processor owns v by Eq. (3)), at row pi_m2(c) of that CTA's
//              part of W = Z-hat (Eq. (17)): the fused digit reversal of
//              PARA-CO-DRP (Sect. 4.2, App. C.5) as the addresses of one
//              all-to-all through distributed shared memory -- N/K^2 items per
//              ordered pair of CTAs, N/p^2 per ordered pair of processors; a
//              CTA's items for itself stay in its own shared memory;
//   Phase III  computes the length-256 DFTs of its output columns over the
//              digit-reversed rows (Lemma 1, input layout) and writes columns
//              k1 in [r 256/K, (r+1) 256/K) of Y = y viewed N2 x N1.
// Synchronisation: one split cluster barrier (arrive at entry, wait before the
// first remote store) makes sure every CTA of the cluster runs and has set up
// its transaction barrier; the all-to-all is asynchronous stores
// (st.async) that count their bytes on the destination CTA's barrier, so a
// CTA starts Phase III as soon as its own N/K items have landed, with no
// second cluster-wide barrier.  The wait is bounded (2 s): a CTA that gives up
// sets the plan's status word to PACO_ERR_TIMEOUT and finishes the launch with
// whatever landed.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>

#include "../../include/paco.h"
#include "paco_common.cuh"
#include "paco_plan.h"

namespace paco {

struct ClusterArgs {
    const float2 *in;
    float2 *out;
    long long N;                 // 65536
    int p;                       // processors (counts are kept per pair of processors)
    int rev_t;                   // digit reversal pi_m2 over 8 bits, t bits per digit
    int conj;                    // dir = +1: conjugate on load and store
    const float2 *tw256;         // w_256^{-r}, r < 256
    const float2 *twN;           // w_N^{-r}, r < N
    int *status;                 // device status word (PACO_ERR_TIMEOUT)
    unsigned *pair_count;        // p x p counts of items sent (test hook), or nullptr
    unsigned long long wait_ns;  // limit of the bounded wait
    unsigned extra_tx;           // test hook: bytes expected beyond the N/K items (0 in use)
};

namespace {

constexpr int L = 256;

__device__ __forceinline__ cx<float> ld_cx(const float2 *p)
{
    const float2 v = *p;
    return make_cx<float>(v.x, v.y);
}
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ unsigned map_rank(unsigned addr, int rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
// 8-byte store into another CTA's shared memory that counts its bytes on
// that CTA's transaction barrier
__device__ __forceinline__ void st_async_v2(unsigned addr, float x, float y, unsigned bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];"
                 :: "r"(addr), "f"(x), "f"(y), "r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ cx<float> cmul2(cx<float> a, float2 w)
{
    return make_cx<float>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
// Column swizzle of a row of a CTA's W part.  Row pi_m2(c) has the bits of
// c's low nibble in its high nibble (for every digit width t | 4), so the 16
// lanes of a half-warp, which hold 16 consecutive c, write 16 different
// banks in the exchange, and read one row's 16 columns in Phase III.
__device__ __forceinline__ int sw(int row) { return row >> 4; }

// Rotate v left by r (0 <= r < 16, uniform across the warp) without dynamic
// register indexing: out[k] = v[(k + r) & 15], four conditional shifts.
__device__ __forceinline__ void rotate16(cx<float> *v, int r)
{
#pragma unroll
    for (int b = 1; b < 16; b <<= 1) {
        const bool on = (r & b) != 0;
        cx<float> t[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) t[k] = on ? v[(k + b) & 15] : v[k];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = t[k];
    }
}

// One length-256 DFT per column of a W-column block, as radix 16 x 16 with
// one exchange through buf.  Pass 1: thread (col, t16) -- col = tid % W,
// t16 = tid / W -- brings its 16 inputs x[t16 + 16 s] in v (the caller loads
// them) and the 15 inner twiddles w_256^{-s t16}, s = 1..15, in tw.  Pass 2:
// thread (col2, u) -- (tid % W, tid / W) when T16_FAST is false, else
// (tid / 16, tid % 16) -- gets outputs u + 16 k', k' < 16, of column col2 in
// v.  buf holds the intermediate (k16, t16) of column col at row
// 16 k16 + t16, column col ^ k16: conflict-free for both pass-2 roles.
template <bool T16_FAST>
__device__ __forceinline__ void dft256_cols(cx<float> *v, float2 *buf, int W, int col, int t16,
                                            const float2 *tw)
{
    dft16(v);
#pragma unroll
    for (int s = 1; s < 16; ++s) v[s] = cmul2(v[s], tw[s - 1]);
    __syncthreads();                                          // the loads from buf are done
#pragma unroll
    for (int s = 0; s < 16; ++s) buf[(s * 16 + t16) * W + (col ^ s)] = make_float2(v[s].x, v[s].y);
    __syncthreads();
    const int tid = threadIdx.x;
    const int col2 = T16_FAST ? tid / 16 : tid % W, u = T16_FAST ? tid % 16 : tid / W;
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = ld_cx(&buf[(u * 16 + t) * W + (col2 ^ u)]);
    dft16(v);
}

} // namespace

// K CTAs per transform (a cluster), 4096 / K threads each.
template <int K>
__global__ void __launch_bounds__(4096 / K, K == 16 ? 2 : 1) paco_cluster_kernel(const ClusterArgs a)
{
    extern __shared__ __align__(16) float2 smem[];
    constexpr int NK = 65536 / K;                             // items per CTA
    float2 *bufA = smem;                                      // the in-CTA exchanges of the length-256 DFTs
    float2 *bufB = smem + NK;                                 // this CTA's part of W, filled by the all-to-all
    __shared__ __align__(8) unsigned long long full;          // counts the bytes that land in bufB
    __shared__ unsigned cnt[16];
    constexpr int W1 = L / K, W2 = L / K;                     // input and output columns of a CTA
    unsigned q;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(q));  // this CTA
    const long long tr = (long long)(blockIdx.x / K);         // the transform of this cluster
    const int tid = threadIdx.x;
    const int col = tid % W1, t16 = tid / W1;                 // Phase I pass 1; Phase III: (vl, u16) = (col, t16)
    const int colB = tid / 16, tB = tid % 16;                 // Phase I pass 2: column q W1 + colB, outputs tB + 16 k
    const int cglob = (int)q * W1 + col, cB = (int)q * W1 + colB;
    const unsigned fullA = smem_u32(&full);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(fullA) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(fullA), "r"((unsigned)(NK * sizeof(float2)) + a.extra_tx) : "memory");
    }
    if (a.pair_count && tid < 16) cnt[tid] = 0;
    // (the barrier's initialisation is ordered by the fence above)
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");

    // Twiddles first: the plan's tables are not written by the preceding
    // kernels, so their loads overlap the wait for those kernels.
    float2 tw[15];                                            // w_256^{-s t16}: the same in both phases
#pragma unroll
    for (int s = 1; s < 16; ++s) tw[s - 1] = __ldg(&a.tw256[(s * t16) & 255]);
    float2 wt[16];                                            // w_N^{-vc}, v = tB + 16 k, c = cB (vc < N)
#pragma unroll
    for (int k = 0; k < 16; ++k) wt[k] = __ldg(&a.twN[(tB + 16 * k) * cB]);
    // Programmatic dependent launch: wait for the kernels before this one
    // (they may write x or read y), then let the next kernel start its CTAs.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    const float2 *x = a.in + tr * a.N;
    float2 *y = a.out + tr * a.N;

    // ---- Phase I on input columns c = q W1 + col
    cx<float> v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        v[s] = ld_cx(x + (long long)(t16 + 16 * s) * L + cglob);   // row t16 + 16 s of X
        if (a.conj) v[s].y = -v[s].y;
    }
    dft256_cols<true>(v, bufA, W1, col, t16, tw);
    // v[k] = A[v][c] with c = cB, v = tB + 16 k (the natural frequency k1)
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = cmul2(v[k], wt[k]);  // Z[v][c] = A[v][c] w_N^{-vc}
    const int row = (int)digit_reverse((unsigned)cB, 8, a.rev_t);   // pi_m2(c): its row of W
    // Send order: warp w of CTA q starts at k = (q + w) mod 16, so that at
    // every step the CTAs' stores spread over all destinations; the 16 lanes
    // of a half-warp fill 16 consecutive columns of one destination row.
    const int rho = ((int)q + (tid >> 5)) & 15;
    rotate16(v, rho);
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");   // all CTAs run, barriers set up
    const unsigned bufB_a = smem_u32(bufB);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int vf = tB + 16 * ((j + rho) & 15);            // k1 = v
        const int qd = vf / W2, vl = vf % W2;                 // the CTA that owns output column v, local column
        const unsigned dst = map_rank(bufB_a + (unsigned)(row * W2 + (vl ^ sw(row))) * 8u, qd);
        st_async_v2(dst, v[j].x, v[j].y, map_rank(fullA, qd));
        if (a.pair_count) atomicAdd(&cnt[qd], 1u);
    }
    // every item of this CTA's part has landed (bounded wait)
    if (!mbar_try_wait(fullA, 0)) {
        const unsigned long long t0 = global_ns();
        while (!mbar_try_wait(fullA, 0)) {
            if (global_ns() - t0 > a.wait_ns) {                // give up: flag it, finish the launch
                atomicExch(a.status, (int)PACO_ERR_TIMEOUT);
                break;
            }
        }
    }
    if (a.pair_count) {                                       // per ordered pair of processors
        __syncthreads();
        if (tid < K) {
            const int g = K / a.p;
            atomicAdd(&a.pair_count[((int)q / g) * a.p + tid / g], cnt[tid]);
        }
    }

    // ---- Phase III on output columns v = q W2 + vl, logical rows j -> pi_m2(j)
    const int vl = col, u16 = t16;
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int rj = (int)digit_reverse((unsigned)(u16 + 16 * s), 8, a.rev_t);
        v[s] = ld_cx(&bufB[rj * W2 + (vl ^ sw(rj))]);
    }
    dft256_cols<false>(v, bufA, W2, vl, u16, tw);
    const int k1 = (int)q * W2 + vl;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int k2 = u16 + 16 * k;
        y[(long long)k2 * L + k1] = make_float2(v[k].x, a.conj ? -v[k].y : v[k].y);   // Y[k2][k1] = y[k1 + k2 N1]
    }
}

const void *cluster_kernel_fn(int K)
{
    return K == 16 ? reinterpret_cast<const void *>(&paco_cluster_kernel<16>)
                   : reinterpret_cast<const void *>(&paco_cluster_kernel<8>);
}

// The one-launch form applies to complex64 plans with N1 = N2 = 256 and p = 4
// or 8, up to 16 transforms: it keeps one transform on one cluster of K SMs,
// which is latency-bound, and from 32 transforms on the two stage launches,
// which stream the whole batch through all SMs, take less time (measured on
// GB300: 15.8 vs 16.5 us at 16 transforms, 24.8 vs 21.5 us at 32).
bool cluster_eligible(const paco_plan *pl)
{
    return pl->dtype == PACO_C64 && pl->N1 == 256 && pl->N2 == 256 && (pl->p == 4 || pl->p == 8) &&
           pl->batch <= 16;
}

// CTAs per transform on the current device: 16 when a 16-CTA cluster of this
// kernel can be resident, else 8 (queried once per device; concurrent first
// calls compute the same answer).
int cluster_size()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    const int known = cache[dev].load(std::memory_order_relaxed);
    if (known) return known;
    int k = 8;
    if (cudaFuncSetAttribute(cluster_kernel_fn(16), cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
        cudaSuccess) {
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3(16, 1, 1);
        cfg.blockDim = dim3(256, 1, 1);
        cfg.dynamicSmemBytes = 2 * 4096 * sizeof(float2);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 16;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, cluster_kernel_fn(16), &cfg) == cudaSuccess && n > 0) k = 16;
    }
    cudaGetLastError();                                       // a refused query leaves no error behind
    cache[dev].store(k, std::memory_order_relaxed);
    return k;
}

paco_status_t launch_cluster(const paco_plan *pl, const void *in, void *out, int dir, unsigned *pair_count,
                             cudaStream_t stream)
{
    ClusterArgs a;
    memset(&a, 0, sizeof(a));
    a.in = static_cast<const float2 *>(in);
    a.out = static_cast<float2 *>(out);
    a.N = pl->N;
    a.p = pl->p;
    a.rev_t = pl->t;
    a.conj = (dir == 1);
    a.tw256 = static_cast<const float2 *>(pl->twL2);
    a.twN = static_cast<const float2 *>(pl->twN_full);
    a.status = pl->d_status;
    a.pair_count = pair_count;
    a.wait_ns = 2000000000ull;
    a.extra_tx = 8u * pl->dbg_wait_bias;          // paco_debug_set_waits: a wait that runs out
    const int K = pl->fused_k;                    // chosen at plan creation on the plan's device
    const int threads = (int)(pl->N / K / 16);
    const size_t smem = 2 * (size_t)(pl->N / K) * sizeof(float2);
    for (int64_t b0 = 0; b0 < pl->batch; b0 += 8192) {
        const int64_t nb = (pl->batch - b0 < 8192) ? pl->batch - b0 : 8192;
        ClusterArgs ab = a;
        ab.in = a.in + b0 * pl->N;
        ab.out = a.out + b0 * pl->N;
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3((unsigned)(nb * K), 1, 1);
        cfg.blockDim = dim3((unsigned)threads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)K;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // the kernel waits (griddepcontrol)
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 2;
        void *params[] = {&ab};
        PACO_CUDA_TRY(cudaLaunchKernelExC(&cfg, cluster_kernel_fn(K), params));
    }
    return PACO_OK;
}

// Kernel attributes and the plan's full table of w_N^{-r}, r < N (512 KiB).
paco_status_t cluster_setup(paco_plan *pl)
{
    PACO_CUDA_TRY(cudaFuncSetAttribute(cluster_kernel_fn(8), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       2 * 8192 * (int)sizeof(float2)));
    PACO_CUDA_TRY(cudaFuncSetAttribute(cluster_kernel_fn(16), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       2 * 4096 * (int)sizeof(float2)));
    pl->fused_k = cluster_size();
    return gen_table(8, &pl->twN_full, (pl->dims >= 2) ? 1 : pl->N, pl->N, 1, 0);   // ones for the 2-D DFT
}

} // namespace paco
