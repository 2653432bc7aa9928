// paco_restore.cu -- restoring the input's ownership after the sharded form:
// the second redistribution that the paper leaves out (Sect. 6, Limitations:
// after PACO processor q owns output columns k1 of Y, not slab q of the
// natural layout).  Rank q holds y_local = Y[:, q K1 .. (q+1) K1) (the
// output of paco_shard_stage2); afterwards rank r holds y viewed N1 x N2 in
// the input's layout, columns j in [r Cl, (r+1) Cl) (Cl = N2/G), i.e. the
// same slab of y that rank r held of x.
//
// Element k of y sits at (k2, k1) = (k / N1, k mod N1) before and at
// (i, j) = (k / N2, k mod N2) after: it moves from rank floor(k1 / K1) to
// rank floor(j / Cl).  Both sides enumerate the items of a block in
// increasing k, so a block needs no index of its own: the sender gathers in
// that order (pack map), the receiver scatters in that order (unpack map).
// The maps are built on the host once per plan (N/G entries each); the
// block sizes differ between pairs unless N1 = N2 (then every item stays on
// its rank: k1 = j).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/paco.h"
#include "paco_plan.h"

namespace {

// Pack (rank q): pos -> local index of y_local [N2][K1] (k2 K1 + k1l), block
// by block (r = 0..G-1).  Unpack (rank r): pos -> local index of the
// restored [N1][Cl] (i Cl + jl), block by block (q = 0..G-1).
void build_maps(int64_t N1, int64_t N2, int G, int rank, int32_t *pack, int64_t *send_counts, int32_t *unpack,
                int64_t *recv_counts)
{
    const int64_t K1 = N1 / G, Cl = N2 / G;
    if (pack || send_counts) {
        std::vector<std::vector<int32_t>> blk(G);
        for (int64_t k2 = 0; k2 < N2; ++k2)
            for (int64_t k1l = 0; k1l < K1; ++k1l) {         // increasing k = k1 + k2 N1
                const int64_t k = rank * K1 + k1l + k2 * N1;
                blk[(int)((k % N2) / Cl)].push_back((int32_t)(k2 * K1 + k1l));
            }
        int64_t pos = 0;
        for (int r = 0; r < G; ++r) {
            if (send_counts) send_counts[r] = (int64_t)blk[r].size();
            if (pack) std::memcpy(pack + pos, blk[r].data(), blk[r].size() * sizeof(int32_t));
            pos += (int64_t)blk[r].size();
        }
    }
    if (unpack || recv_counts) {
        std::vector<std::vector<int32_t>> blk(G);
        for (int64_t i = 0; i < N1; ++i)
            for (int64_t jl = 0; jl < Cl; ++jl) {           // increasing k = i N2 + j
                const int64_t k = i * N2 + rank * Cl + jl;
                blk[(int)((k % N1) / K1)].push_back((int32_t)(i * Cl + jl));
            }
        int64_t pos = 0;
        for (int q = 0; q < G; ++q) {
            if (recv_counts) recv_counts[q] = (int64_t)blk[q].size();
            if (unpack) std::memcpy(unpack + pos, blk[q].data(), blk[q].size() * sizeof(int32_t));
            pos += (int64_t)blk[q].size();
        }
    }
}

// the block of position pos: off[g] <= pos < off[g + 1] (off in shared memory)
__device__ __forceinline__ int block_of(const long long *off, int G, long long pos)
{
    int lo = 0, hi = G;                                       // off[lo] <= pos < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= pos) lo = mid;
        else hi = mid;
    }
    return lo;
}

// send [G][batch][count] <- y_local [batch][N/G] through the pack map
__global__ void restore_pack_kernel(const float2 *__restrict__ y, float2 *__restrict__ send,
                                    const int32_t *__restrict__ map, const long long *__restrict__ off_g, int G,
                                    long long n, long long batch)
{
    extern __shared__ long long off[];
    for (int i = threadIdx.x; i <= G; i += blockDim.x) off[i] = off_g[i];
    __syncthreads();
    const long long total = n * batch;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / n, pos = e - b * n;
        const int r = block_of(off, G, pos);
        const long long cnt = off[r + 1] - off[r];
        send[off[r] * batch + b * cnt + (pos - off[r])] = __ldg(&y[b * n + map[pos]]);
    }
}

// out [batch][N/G] <- recv [G][batch][count] through the unpack map
__global__ void restore_unpack_kernel(const float2 *__restrict__ recv, float2 *__restrict__ out,
                                      const int32_t *__restrict__ map, const long long *__restrict__ off_g, int G,
                                      long long n, long long batch)
{
    extern __shared__ long long off[];
    for (int i = threadIdx.x; i <= G; i += blockDim.x) off[i] = off_g[i];
    __syncthreads();
    const long long total = n * batch;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / n, pos = e - b * n;
        const int q = block_of(off, G, pos);
        const long long cnt = off[q + 1] - off[q];
        out[b * n + map[pos]] = __ldg(&recv[off[q] * batch + b * cnt + (pos - off[q])]);
    }
}

} // namespace

extern "C" paco_status_t paco_shard_restore_maps(int64_t N1, int64_t N2, int G, int rank, int32_t *pack_map,
                                                 int64_t *send_counts, int32_t *unpack_map, int64_t *recv_counts)
{
    using paco::fail;
    if (G < 1 || rank < 0 || rank >= G || N1 < G || N2 < G || N1 % G || N2 % G || N1 * N2 / G > INT32_MAX)
        return fail(PACO_ERR_INVALID_ARG, "paco_shard_restore_maps: G | N1, G | N2, 0 <= rank < G, N/G < 2^31");
    build_maps(N1, N2, G, rank, pack_map, send_counts, unpack_map, recv_counts);
    return PACO_OK;
}

namespace paco {

// Built at plan creation when paco_shard_opts_t.restore is set.
paco_status_t restore_setup(paco_plan *pl)
{
    const int G = pl->shard_G;
    const int64_t n = pl->N / G;
    std::vector<int32_t> pack(n), unpack(n);
    std::vector<int64_t> sc(G), rc(G);
    build_maps(pl->N1, pl->N2, G, pl->shard_rank, pack.data(), sc.data(), unpack.data(), rc.data());
    std::vector<long long> off(2 * (G + 1), 0);
    for (int g = 0; g < G; ++g) {
        off[g + 1] = off[g] + sc[g];
        off[G + 1 + g + 1] = off[G + 1 + g] + rc[g];
    }
    pl->rs_send_counts = new int64_t[G];
    pl->rs_recv_counts = new int64_t[G];
    std::memcpy(pl->rs_send_counts, sc.data(), G * sizeof(int64_t));
    std::memcpy(pl->rs_recv_counts, rc.data(), G * sizeof(int64_t));
    PACO_CUDA_TRY(cudaMalloc(&pl->rs_maps, 2 * (size_t)n * sizeof(int32_t)));
    PACO_CUDA_TRY(cudaMalloc(&pl->rs_off, off.size() * sizeof(long long)));
    PACO_CUDA_TRY(cudaMemcpy(pl->rs_maps, pack.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
    PACO_CUDA_TRY(cudaMemcpy(static_cast<int32_t *>(pl->rs_maps) + n, unpack.data(), n * sizeof(int32_t),
                             cudaMemcpyHostToDevice));
    PACO_CUDA_TRY(cudaMemcpy(pl->rs_off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice));
    return PACO_OK;
}

void restore_destroy(paco_plan *pl)
{
    cudaFree(pl->rs_maps);
    cudaFree(pl->rs_off);
    delete[] pl->rs_send_counts;
    delete[] pl->rs_recv_counts;
}

} // namespace paco

static paco_status_t restore_check(const paco_plan_t *pl, const void *a, const void *b, const char *fn)
{
    using paco::fail;
    if (!pl) return fail(PACO_ERR_INVALID_ARG, "%s: plan is NULL", fn);
    if (!pl->rs_maps) return fail(PACO_ERR_UNSUPPORTED, "%s: a sharded plan created with restore = 1", fn);
    if (pl->batch == 0) return PACO_OK;
    if (!a || !b) return fail(PACO_ERR_INVALID_ARG, "%s: NULL buffer", fn);
    if (((uintptr_t)a | (uintptr_t)b) & 7u) return fail(PACO_ERR_INVALID_ARG, "%s: buffers must be 8-byte aligned", fn);
    const size_t bytes = (size_t)(pl->N / pl->shard_G * pl->batch) * sizeof(float2);
    const char *x = (const char *)a, *y = (const char *)b;
    if (x < y + bytes && y < x + bytes) return fail(PACO_ERR_ALIASING, "%s: buffers overlap", fn);
    return PACO_OK;
}

static paco_status_t restore_launch(const paco_plan_t *pl, bool pack, const void *in, void *out, cudaStream_t s)
{
    const int G = pl->shard_G;
    const long long n = pl->N / G;
    int dev = 0, sms = 0;
    PACO_CUDA_TRY(cudaGetDevice(&dev));
    PACO_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long total = n * pl->batch;
    long long blocks = (total + 255) / 256;
    if (blocks > 8LL * sms) blocks = 8LL * sms;
    const int32_t *map = static_cast<const int32_t *>(pl->rs_maps) + (pack ? 0 : n);
    const long long *off = static_cast<const long long *>(pl->rs_off) + (pack ? 0 : G + 1);
    const size_t smem = (size_t)(G + 1) * sizeof(long long);
    if (pack)
        restore_pack_kernel<<<(unsigned)blocks, 256, smem, s>>>(static_cast<const float2 *>(in),
                                                                static_cast<float2 *>(out), map, off, G, n,
                                                                pl->batch);
    else
        restore_unpack_kernel<<<(unsigned)blocks, 256, smem, s>>>(static_cast<const float2 *>(in),
                                                                  static_cast<float2 *>(out), map, off, G, n,
                                                                  pl->batch);
    PACO_CUDA_TRY(cudaGetLastError());
    return PACO_OK;
}

extern "C" paco_status_t paco_shard_restore_counts(const paco_plan_t *pl, int64_t *send_counts, int64_t *recv_counts)
{
    using paco::fail;
    if (!pl) return fail(PACO_ERR_INVALID_ARG, "paco_shard_restore_counts: plan is NULL");
    if (!pl->rs_maps) return fail(PACO_ERR_UNSUPPORTED, "paco_shard_restore_counts: a sharded plan created with restore = 1");
    for (int g = 0; g < pl->shard_G; ++g) {
        if (send_counts) send_counts[g] = pl->rs_send_counts[g];
        if (recv_counts) recv_counts[g] = pl->rs_recv_counts[g];
    }
    return PACO_OK;
}

extern "C" paco_status_t paco_shard_restore_pack(paco_plan_t *pl, const void *y_local, void *send,
                                                 paco_stream_t stream)
{
    paco_status_t st = restore_check(pl, y_local, send, "paco_shard_restore_pack");
    if (st != PACO_OK || pl->batch == 0) return st;
    return restore_launch(pl, true, y_local, send, (cudaStream_t)stream);
}

extern "C" paco_status_t paco_shard_restore_unpack(paco_plan_t *pl, const void *recv, void *x_layout,
                                                   paco_stream_t stream)
{
    paco_status_t st = restore_check(pl, recv, x_layout, "paco_shard_restore_unpack");
    if (st != PACO_OK || pl->batch == 0) return st;
    return restore_launch(pl, false, recv, x_layout, (cudaStream_t)stream);
}
