// paco_tc05.cu -- the 128-point DFT sub-pass of a 2^14 stage on the 5th-generation
// tensor cores (tcgen05), as a measured alternative to the FP32 radix-16 x 8
// leaf of the panel kernel (the paper's leaves are exact DFTs, Sect. 4.1; this
// is an approximate contraction with a stated error).
//
//   y[b][k][c] = sum_j w_128^{-jk} x[b][j][c],   k, j < 128, c < C
//
// as the complex GEMM Y = F X with F[k][j] = w_128^{-jk}, in real arithmetic
//   Yr = Fr Xr - Fi Xi,   Yi = Fi Xr + Fr Xi,
// each real product in BF16x3 form: F = F0 + F1 and X = X0 + X1 split into
// bf16 terms, F0 X0 + F0 X1 + F1 X0 accumulated in FP32 (the F1 X1 term and
// the residuals beyond two terms, about 2^-17 relative, are dropped).
//
// One persistent CTA per SM (256 threads).  Shared memory holds the four F
// operands (Fr0, Fr1, Fi0, Fi1: 128 x 128 bf16 each, 128 KiB, loaded once)
// and the four X operands of a tile of 64 sequences (Xr0, Xr1, Xi0, Xi1:
// 64 x 128 bf16 each), all K-major in the 128-byte swizzle layout the MMA
// descriptors address.  Per tile one thread issues 96 tcgen05.mma
// (M = 128, N = 64, K = 16, kind::f16, bf16 in, FP32 accumulators in TMEM:
// Yr in columns 0..63, Yi in 64..127; -Fi by the instruction's negate-A bit)
// and commits them to an mbarrier; the eight warps read the accumulators back
// with tcgen05.ld (warp w: TMEM lanes 32 (w mod 4).., columns half w / 4) and
// store 256-byte runs of y.  The next tile's x is loaded into registers while
// the MMAs run.  (A double-buffered variant with 32-sequence tiles, MMAs of
// tile i+1 issued before tile i's epilogue, measured slower: 2.64 against
// 1.37 ms for 2^28 points -- the time per tile is set by the number of MMA
// instructions, about 64 ns each, not by their size.)  The wait for the MMAs
// is bounded (2 s; status PACO_ERR_TIMEOUT) and the TMEM columns are freed on
// every path.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/paco.h"
#include "paco_plan.h"

namespace paco {
namespace tc05 {

constexpr int L = 128;                   // DFT length
constexpr int NS = 64;                   // sequences per tile (MMA N)
constexpr int THREADS = 256;
constexpr int A_BYTES = L * L * 2;       // one 128 x 128 bf16 operand
constexpr int B_BYTES = NS * L * 2;      // one 64 x 128 bf16 operand
constexpr int SMEM_BYTES = 4 * A_BYTES + 4 * B_BYTES + 1024;   // + alignment slack
constexpr int TMEM_COLS = 128;           // Yr and Yi, NS columns each
constexpr unsigned long long WAIT_NS = 2000000000ull;

// Byte offset of element (row r, k) in a K-major operand of R rows and K = 128
// in the 128-byte swizzle layout: two atoms of 64 k (128 B per row), 8-row
// groups 1024 B apart, 16-byte chunk index XOR (r mod 8).
__host__ __device__ inline uint32_t sw128_off(int r, int k, int R)
{
    return (uint32_t)((k >> 6) * (R * 128) + r * 128 + ((((k & 63) >> 3) ^ (r & 7)) << 4) + ((k & 7) << 1));
}

// Shared-memory matrix descriptor: start address, leading byte offset (unused
// by swizzled K-major layouts), stride byte offset 1024 (8 rows x 128 B), the
// fixed 0b001 at bits 46-48, swizzle mode 2 (128 B) at bits 61-63.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), bf16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28; bit 13 negates A.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NS >> 3) << 17) |
                           ((uint32_t)(L >> 4) << 24);
constexpr uint32_t IDESC_NEG_A = IDESC | (1u << 13);

__device__ int g_status;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &h, __nv_bfloat16 &l)
{
    h = __float2bfloat16_rn(v);
    l = __float2bfloat16_rn(v - __bfloat162float(h));
}

// F operands in the operand layout: [Fr0 | Fr1 | Fi0 | Fi1], each 128 x 128,
// row k (output), column j (input), from FP64 sincospi.
__global__ void tc05_table_kernel(__nv_bfloat16 *out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= L * L) return;
    const int k = idx / L, j = idx % L;
    double s, c;
    sincospi((double)((j * k) & (L - 1)) / (L / 2), &s, &c);   // angle 2 pi jk / 128
    const float fr = (float)c, fi = (float)(-s);              // w_128^{-jk}
    __nv_bfloat16 h, l;
    const uint32_t o = sw128_off(k, j, L) / 2;
    split_bf16(fr, h, l);
    out[o] = h;
    out[A_BYTES / 2 + o] = l;
    split_bf16(fi, h, l);
    out[2 * A_BYTES / 2 + o] = h;
    out[3 * A_BYTES / 2 + o] = l;
}

// x and y: [batch][128][C] complex64; tiles of NS columns, tile t -> (b, c0).
__global__ void __launch_bounds__(THREADS, 1) tc05_dft128_kernel(const float2 *__restrict__ x, float2 *__restrict__ y,
                                                                 const uint4 *__restrict__ table, long long ntiles,
                                                                 int C)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);   // swizzle atoms need 1 KiB alignment
    unsigned char *sA = smem;                          // Fr0, Fr1, Fi0, Fi1
    unsigned char *sB = smem + 4 * A_BYTES;            // Xr0, Xr1, Xi0, Xi1
    __shared__ __align__(8) unsigned long long done;   // MMA completion
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_per_b = C / NS;

    // F operands, once per CTA
    for (int i = tid; i < 4 * A_BYTES / 16; i += THREADS)
        reinterpret_cast<uint4 *>(sA)[i] = table[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_slot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t bar = smem_u32(&done);
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);

    // loader role: unit u = tid + 256 i, i < 4: sequence n = u % 64, points j = 8 (u / 64) + e
    float2 xv[4][8];
    auto load_tile = [&](long long t) {
        const long long bb = t / tiles_per_b;
        const int c0 = (int)(t % tiles_per_b) * NS;
        const float2 *xb = x + bb * (long long)L * C + c0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int u = tid + THREADS * i, n = u & (NS - 1), jc = u >> 6;
#pragma unroll
            for (int e = 0; e < 8; ++e) xv[i][e] = __ldg(xb + (long long)(8 * jc + e) * C + n);
        }
    };

    uint32_t phase = 0;
    bool failed = false;
    long long t = blockIdx.x;
    if (t < ntiles) load_tile(t);
    for (; t < ntiles; t += gridDim.x) {
        // X operands of this tile: bf16 hi / lo of the real and imaginary parts
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int u = tid + THREADS * i, n = u & (NS - 1), jc = u >> 6;
            __align__(16) __nv_bfloat16 rh[8], rl[8], ih[8], il[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                split_bf16(xv[i][e].x, rh[e], rl[e]);
                split_bf16(xv[i][e].y, ih[e], il[e]);
            }
            const uint32_t o = sw128_off(n, 8 * jc, NS);
            *reinterpret_cast<uint4 *>(sB + 0 * B_BYTES + o) = *reinterpret_cast<const uint4 *>(rh);
            *reinterpret_cast<uint4 *>(sB + 1 * B_BYTES + o) = *reinterpret_cast<const uint4 *>(rl);
            *reinterpret_cast<uint4 *>(sB + 2 * B_BYTES + o) = *reinterpret_cast<const uint4 *>(ih);
            *reinterpret_cast<uint4 *>(sB + 3 * B_BYTES + o) = *reinterpret_cast<const uint4 *>(il);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> MMA reads
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // (A operand, B operand) per product, Yr then Yi; Yr's last three negate A (-Fi)
            const int ta[2][6] = {{0, 0, 1, 2, 2, 3}, {2, 2, 3, 0, 0, 1}};
            const int tb[2][6] = {{0, 1, 0, 2, 3, 2}, {0, 1, 0, 2, 3, 2}};
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const uint32_t d = tmem + (uint32_t)(part * NS);
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const uint32_t id = (part == 0 && q >= 3) ? IDESC_NEG_A : IDESC;
#pragma unroll
                    for (int kk = 0; kk < L / 16; ++kk) {
                        const uint32_t ka = (uint32_t)((kk >> 2) * (L * 128) + (kk & 3) * 32);
                        const uint32_t kb = (uint32_t)((kk >> 2) * (NS * 128) + (kk & 3) * 32);
                        mma(d, sdesc(a0 + ta[part][q] * A_BYTES + ka), sdesc(b0 + tb[part][q] * B_BYTES + kb), id,
                            (q > 0 || kk > 0) ? 1u : 0u);
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(bar) : "memory");
        }
        // the next tile's x while the MMAs run
        const long long tn = t + gridDim.x;
        if (tn < ntiles) load_tile(tn);
        // wait for the MMAs (bounded)
        if (!mbar_try(bar, phase)) {
            const unsigned long long t0 = gtime();
            while (!mbar_try(bar, phase)) {
                if (gtime() - t0 > WAIT_NS) {
                    failed = true;
                    break;
                }
            }
        }
        phase ^= 1u;
        if (__syncthreads_or(failed)) {                   // the same decision in every thread
            if (tid == 0) atomicExch(&g_status, (int)PACO_ERR_TIMEOUT);
            // the MMAs may still be in flight: one more bounded wait before TMEM is freed
            const unsigned long long t0 = gtime();
            while (!mbar_try(bar, phase ^ 1u) && gtime() - t0 < WAIT_NS) {
            }
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // accumulators -> y: warp w reads lanes 32 (w mod 4).., columns 32 (w / 4)..
        {
            const int m = 32 * (warp & 3) + lane;         // output point k
            const int h = warp >> 2;
            const uint32_t ta_r = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * h);
            uint32_t r[32], im[32];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                           "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                           "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                         : "r"(ta_r));
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                         : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]),
                           "=r"(im[6]), "=r"(im[7]), "=r"(im[8]), "=r"(im[9]), "=r"(im[10]), "=r"(im[11]),
                           "=r"(im[12]), "=r"(im[13]), "=r"(im[14]), "=r"(im[15]), "=r"(im[16]), "=r"(im[17]),
                           "=r"(im[18]), "=r"(im[19]), "=r"(im[20]), "=r"(im[21]), "=r"(im[22]), "=r"(im[23]),
                           "=r"(im[24]), "=r"(im[25]), "=r"(im[26]), "=r"(im[27]), "=r"(im[28]), "=r"(im[29]),
                           "=r"(im[30]), "=r"(im[31])
                         : "r"(ta_r + (uint32_t)NS));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const long long bb = t / tiles_per_b;
            const int c0 = (int)(t % tiles_per_b) * NS + 32 * h;
            float4 *yo = reinterpret_cast<float4 *>(y + bb * (long long)L * C + (long long)m * C + c0);
#pragma unroll
            for (int i = 0; i < 16; ++i)
                yo[i] = make_float4(__uint_as_float(r[2 * i]), __uint_as_float(im[2 * i]),
                                    __uint_as_float(r[2 * i + 1]), __uint_as_float(im[2 * i + 1]));
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();                                  // TMEM and the X operands free for the next tile
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

} // namespace tc05
} // namespace paco

extern "C" paco_status_t paco_probe_tc05_dft128(const void *x, void *y, int64_t batch, int64_t C, float *ms,
                                                paco_stream_t stream)
{
    using namespace paco;
    using namespace paco::tc05;
    if (!x || !y || batch < 0 || C < NS || C % NS || C > (1 << 24))
        return fail(PACO_ERR_INVALID_ARG, "paco_probe_tc05_dft128: C a multiple of %d, buffers required", NS);
    if (((uintptr_t)x | (uintptr_t)y) & 15u) return fail(PACO_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    const size_t bytes = (size_t)batch * L * C * sizeof(float2);
    if ((const char *)x < (const char *)y + bytes && (const char *)y < (const char *)x + bytes)
        return fail(PACO_ERR_ALIASING, "input and output overlap");
    static void *table = nullptr;                     // the F operands (128 KiB), built once per process
    static int table_dev = -1;
    int dev = 0, sms = 0;
    PACO_CUDA_TRY(cudaGetDevice(&dev));
    cudaStream_t s = (cudaStream_t)stream;
    if (!table || table_dev != dev) {
        PACO_CUDA_TRY(cudaMalloc(&table, 4 * A_BYTES));
        tc05_table_kernel<<<L * L / 256, 256, 0, s>>>(static_cast<__nv_bfloat16 *>(table));
        PACO_CUDA_TRY(cudaGetLastError());
        PACO_CUDA_TRY(cudaFuncSetAttribute(tc05_dft128_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        table_dev = dev;
    }
    if (batch == 0) return PACO_OK;
    PACO_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long ntiles = batch * (C / NS);
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms) {
        PACO_CUDA_TRY(cudaEventCreate(&e0));
        PACO_CUDA_TRY(cudaEventCreate(&e1));
        PACO_CUDA_TRY(cudaEventRecord(e0, s));
    }
    tc05_dft128_kernel<<<grid, THREADS, SMEM_BYTES, s>>>(static_cast<const float2 *>(x), static_cast<float2 *>(y),
                                                         static_cast<const uint4 *>(table), ntiles, (int)C);
    PACO_CUDA_TRY(cudaGetLastError());
    if (ms) {
        PACO_CUDA_TRY(cudaEventRecord(e1, s));
        PACO_CUDA_TRY(cudaEventSynchronize(e1));
        PACO_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        int st = 0;
        PACO_CUDA_TRY(cudaMemcpyFromSymbol(&st, g_status, sizeof(int)));
        if (st) {
            int zero = 0;
            cudaMemcpyToSymbol(g_status, &zero, sizeof(int));
            return fail(PACO_ERR_TIMEOUT, "paco_probe_tc05_dft128: the wait for the tensor-core MMAs gave up");
        }
    }
    return PACO_OK;
}
