// paco_permute.cu -- the middle stage PARA-CO-DRP_b as a standalone pass
// (App. C.5, the unfused form of the one global redistribution).
//
// Input: A-tilde[a][c] = A[pi_m1(a)][c], the Phase I output layout (Lemma 1),
// row-major N1 x N2 per transform.  Output: W[u][v] = Z[v][pi_m2(u)] with
// Z[v][c] = A[v][c] * w_N^{dir*v*c} (Eq. 17 and the top-level twiddle of the
// two-factor Cooley-Tukey identity), row-major N2 x N1.  Element (a, c) goes
// to (pi_m2(c), pi_m1(a)): the fused digit reversal pi_m(a ++ c).
//
// On one GPU the p^2 slab-pair blocks of the paper's all-to-all are not
// separate messages; the pass is a gather over 32 x 32 tiles chosen so that
// both sides are row segments: the tile covers the contiguous output columns
// v in [v0, v0 + 32) (input rows a = pi_m1(v), each read as a contiguous run
// of 32 columns c) and the contiguous input columns c in [c0, c0 + 32)
// (output rows u = pi_m2(c), each written as a run of 32 columns v).  Every
// element is read once and written once (16 B per c64 element).
#include <cuda_runtime.h>

#include "paco_common.cuh"
#include "paco_plan.h"

namespace paco {

struct PermuteArgs {
    const void *in;
    void *out;
    long long batch;
    long long N;           // elements per transform
    int N1, N2;
    int bits1, bits2, t;   // log2 N1, log2 N2, bits per base-b digit
    unsigned N_mask;
    const void *twN_lo, *twN_hi;
    int twN_lo_bits;
    int conj;              // dir = +1: w_N^{+v c}
};

template <typename R>
__global__ void __launch_bounds__(256) paco_permute_kernel(const PermuteArgs a)
{
    using C = cx<R>;
    __shared__ C tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;           // 32 x 8
    const int TV = a.N1 < 32 ? a.N1 : 32, TC = a.N2 < 32 ? a.N2 : 32;
    const int v0 = blockIdx.x * TV, c0 = blockIdx.y * TC;
    const C *lo = reinterpret_cast<const C *>(a.twN_lo);
    const C *hi = reinterpret_cast<const C *>(a.twN_hi);
    const unsigned lomask = (1u << a.twN_lo_bits) - 1u;
    for (long long bt = blockIdx.z; bt < a.batch; bt += gridDim.z) {
        const C *src = reinterpret_cast<const C *>(a.in) + bt * a.N;
        C *dst = reinterpret_cast<C *>(a.out) + bt * a.N;
        if (tx < TC) {
            // all loads of the thread first (4 rows of the tile), then the twiddles
            const unsigned c = (unsigned)(c0 + tx);
            C x[4], w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = ty + 8 * q;
                if (i < TV) {
                    const unsigned v = (unsigned)(v0 + i);
                    const unsigned arow = digit_reverse(v, a.bits1, a.t);     // a = pi_m1(v)
                    const unsigned r = (v * c) & a.N_mask;
                    x[q] = src[(long long)arow * a.N2 + c];
                    w[q] = cmul(lo[r & lomask], hi[r >> a.twN_lo_bits]);      // w_N^{-vc}
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = ty + 8 * q;
                if (i < TV) {
                    C wq = w[q];
                    if (a.conj) wq.y = -wq.y;
                    tile[i][tx] = cmul(x[q], wq);
                }
            }
        }
        __syncthreads();
        if (tx < TV) {
            for (int j = ty; j < TC; j += 8) {
                const unsigned u = digit_reverse((unsigned)(c0 + j), a.bits2, a.t);   // u = pi_m2(c)
                dst[(long long)u * a.N1 + v0 + tx] = tile[tx][j];
            }
        }
        __syncthreads();
    }
}

paco_status_t launch_permute(const paco_plan *pl, const void *A_tilde, void *W, int dir,
                             cudaStream_t stream)
{
    PermuteArgs a;
    a.in = A_tilde;
    a.out = W;
    a.batch = pl->batch;
    a.N = pl->N;
    a.N1 = (int)pl->N1;
    a.N2 = (int)pl->N2;
    a.bits1 = pl->m1 * pl->t;
    a.bits2 = pl->m2 * pl->t;
    a.t = pl->t;
    a.N_mask = (unsigned)(pl->N - 1);
    a.twN_lo = pl->twN_lo;
    a.twN_hi = pl->twN_hi;
    a.twN_lo_bits = pl->twN_lo_bits;
    a.conj = (dir == 1);
    const int TV = a.N1 < 32 ? a.N1 : 32, TC = a.N2 < 32 ? a.N2 : 32;
    const long long gz = pl->batch < 65535 ? pl->batch : 65535;
    dim3 grid((unsigned)(a.N1 / TV), (unsigned)(a.N2 / TC), (unsigned)gz);
    if (pl->esize == 8)
        paco_permute_kernel<float><<<grid, dim3(32, 8), 0, stream>>>(a);
    else
        paco_permute_kernel<double><<<grid, dim3(32, 8), 0, stream>>>(a);
    PACO_CUDA_TRY(cudaGetLastError());
    return PACO_OK;
}

} // namespace paco
