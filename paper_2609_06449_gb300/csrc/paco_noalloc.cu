// paco_noalloc.cu -- paco_execute_noalloc: the complex64 transform of
// N1 = N2 = 2^14 run only from memory the library reserves when it is loaded.
//
// Some callers cannot allocate device memory: code that runs while a CUDA
// graph is being captured, inside a framework whose memory pool owns every
// byte of the device, or in a context that must not touch the allocator after
// start-up.  This entry point serves them: the panel buffers the length-2^14
// stages stream through, the pipeline counters, the status word and the
// twiddle tables are file-scope __device__ arrays, so a call allocates and
// frees nothing.  Every GPU that loads the library holds these arrays (about
// 24.4 MiB) until the process exits.
//
// In host code the names of these arrays are host-side stand-ins, not device
// addresses; the device addresses come from cudaGetSymbolAddress, taken once
// per device (with that device current) by the first call on the device, which
// also fills the twiddle tables.  That first call should therefore come before
// any stream capture.  All calls on a device share the arrays and each call
// leaves them holding its own intermediates: the counters are cleared on the
// stream at the start of every stage; calls whose work overlaps on the GPU
// race on the shared buffers and must be ordered by the caller.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/paco.h"
#include "paco_common.cuh"
#include "paco_panel_host.h"

using namespace paco;

namespace {

constexpr int kLg = 14;                                  // N1 = N2 = 2^14
constexpr long long kL = 1LL << kLg;
constexpr long long kN = kL * kL;
constexpr int kP = 64;                                   // panel width (columns)
constexpr long long kPanelsPerBatch = kL / kP;           // 256
constexpr long long kScratchElems = (long long)panel::NBUF * kL * kP;   // 3 * 2^20
constexpr int kCtrWords = (int)(2 * PACO_NOALLOC_MAX_BATCH * kPanelsPerBatch + 1);
// a stage clears and uses 2 * batch * panels + 1 counter words (queue, A and
// B completions per panel): the largest accepted batch must fit
static_assert(2LL * PACO_NOALLOC_MAX_BATCH * kPanelsPerBatch + 1 <= (long long)kCtrWords,
              "counter array too small for PACO_NOALLOC_MAX_BATCH");

__device__ __align__(256) float2 g_scratch[kScratchElems];   // 24 MiB panel ring
__device__ __align__(256) unsigned g_ctr[kCtrWords];         // queue + per-panel counters
__device__ __align__(256) int g_status;                      // PACO_ERR_TIMEOUT from bounded waits
__device__ __align__(256) float2 g_twL[kL];                  // w_{2^14}^{-r}
__device__ __align__(256) float2 g_twN_lo[kL];               // w_{2^28}^{-r}, r < 2^14
__device__ __align__(256) float2 g_twN_hi[kL];               // w_{2^28}^{-r 2^14}

// FP64 twiddles, rounded to FP32: w_M^{-e} = (cos 2 pi e / M, -sin 2 pi e / M).
__global__ void noalloc_tables_kernel(float2 *twL, float2 *lo, float2 *hi)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= kL) return;
    double s, c;
    sincospi(2.0 * (double)r / (double)kL, &s, &c);
    twL[r] = make_float2((float)c, (float)-s);
    sincospi(2.0 * (double)r / (double)kN, &s, &c);
    lo[r] = make_float2((float)c, (float)-s);
    sincospi(2.0 * (double)(r * kL) / (double)kN, &s, &c);
    hi[r] = make_float2((float)c, (float)-s);
}

struct DeviceState {
    bool ready = false;
    float2 *scratch = nullptr, *twL = nullptr, *lo = nullptr, *hi = nullptr;
    unsigned *ctr = nullptr;
    int *status = nullptr;
    int num_sms = 0;
};

constexpr int kMaxDevices = 64;
DeviceState g_state[kMaxDevices];
std::mutex g_mutex;

// paco_debug_noalloc_set_waits: poll limit (0 = default) and the bias added
// to every dependency target of the bounded waits
unsigned g_dbg_spin_limit = 0, g_dbg_wait_bias = 0;

// Set-up for the current device, once: symbol addresses, tables, attributes.
paco_status_t setup(int dev, DeviceState **out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceState &s = g_state[dev];
    if (!s.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return fail(PACO_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed");
        s.scratch = static_cast<float2 *>(p);
        if (cudaGetSymbolAddress(&p, g_ctr) != cudaSuccess) return fail(PACO_ERR_CUDA, "cudaGetSymbolAddress(counters) failed");
        s.ctr = static_cast<unsigned *>(p);
        if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return fail(PACO_ERR_CUDA, "cudaGetSymbolAddress(status) failed");
        s.status = static_cast<int *>(p);
        if (cudaGetSymbolAddress(&p, g_twL) != cudaSuccess) return fail(PACO_ERR_CUDA, "cudaGetSymbolAddress(twL) failed");
        s.twL = static_cast<float2 *>(p);
        if (cudaGetSymbolAddress(&p, g_twN_lo) != cudaSuccess) return fail(PACO_ERR_CUDA, "cudaGetSymbolAddress(twN_lo) failed");
        s.lo = static_cast<float2 *>(p);
        if (cudaGetSymbolAddress(&p, g_twN_hi) != cudaSuccess) return fail(PACO_ERR_CUDA, "cudaGetSymbolAddress(twN_hi) failed");
        s.hi = static_cast<float2 *>(p);
        for (int k = 0; k < 3; ++k) {
            const void *fn = panel_kernel_fn(k == 0 ? 1 : 2, k == 2 ? 4 : 2);
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, panel_smem_bytes()) !=
                cudaSuccess)
                return fail(PACO_ERR_CUDA, "cudaFuncSetAttribute failed");
        }
        if (cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return fail(PACO_ERR_CUDA, "cudaDeviceGetAttribute failed");
        noalloc_tables_kernel<<<(unsigned)(kL / 256), 256>>>(s.twL, s.lo, s.hi);
        if (cudaGetLastError() != cudaSuccess || cudaMemset(s.status, 0, sizeof(int)) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess)
            return fail(PACO_ERR_CUDA, "table set-up failed");
        s.ready = true;
    }
    *out = &s;
    return PACO_OK;
}

} // namespace

extern "C" paco_status_t paco_execute_noalloc(const void *in, void *out, int b, int64_t batch, int dir,
                                              paco_stream_t stream)
{
    if (b != 2 && b != 4) return fail(PACO_ERR_INVALID_ARG, "paco_execute_noalloc: b must be 2 or 4 (N1 = N2 = 2^14)");
    if (batch < 0 || batch > PACO_NOALLOC_MAX_BATCH)
        return fail(PACO_ERR_INVALID_ARG, "paco_execute_noalloc: batch must be in [0, PACO_NOALLOC_MAX_BATCH]");
    if (dir != -1 && dir != 1) return fail(PACO_ERR_INVALID_ARG, "paco_execute_noalloc: dir must be -1 or +1");
    if (batch == 0) return PACO_OK;
    if (!in || !out) return fail(PACO_ERR_INVALID_ARG, "paco_execute_noalloc: NULL buffer");
    if (((uintptr_t)in | (uintptr_t)out) & 15u)
        return fail(PACO_ERR_INVALID_ARG, "paco_execute_noalloc: buffers must be 16-byte aligned");
    const size_t bytes = (size_t)batch * (size_t)kN * 8;
    const char *x = (const char *)in, *y = (const char *)out;
    if (x < y + bytes && y < x + bytes) return fail(PACO_ERR_ALIASING, "paco_execute_noalloc: input and output overlap");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(PACO_ERR_CUDA, "paco_execute_noalloc: no current device");
    DeviceState *s = nullptr;
    paco_status_t st = setup(dev, &s);
    if (st != PACO_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    const long long tiles = 2LL * batch * kPanelsPerBatch * ((long long)panel::L / panel::TILE) * kP;
    const unsigned grid = (unsigned)(s->num_sms < tiles ? s->num_sms : tiles);
    for (int mode = 1; mode <= 2; ++mode) {
        PanelLaunch l;
        memset(&l, 0, sizeof(l));
        l.mode = mode;
        l.b = b;
        l.C = kL;
        l.batch = batch;
        l.N = kN;
        l.P = kP;
        l.in = (mode == 1) ? in : out;
        l.out = out;
        l.scratch = s->scratch;
        l.ctr = s->ctr;
        l.status = s->status;
        l.twL = s->twL;
        l.twN_lo = s->lo;
        l.twN_hi = s->hi;
        l.twN_lo_bits = kLg;
        l.conj = (dir == 1);
        l.spin_limit = g_dbg_spin_limit;
        l.dep_bias = g_dbg_wait_bias;
        PanelArgs a;
        paco_status_t st2 = panel_prepare(l, &a);
        if (st2 != PACO_OK) return st2;
        const size_t words = (size_t)(2 * a.npanels + 1);
        if (cudaMemsetAsync(s->ctr, 0, words * sizeof(unsigned), cs) != cudaSuccess)
            return fail(PACO_ERR_CUDA, "paco_execute_noalloc: counter reset failed");
        void *params[] = {&a};
        if (cudaLaunchKernel(panel_kernel_fn(mode, b), dim3(grid), dim3(panel::NT), params,
                             (size_t)panel_smem_bytes(), cs) != cudaSuccess)
            return fail(PACO_ERR_CUDA, "paco_execute_noalloc: launch failed");
    }
    return PACO_OK;
}

extern "C" paco_status_t paco_noalloc_check(void)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(PACO_ERR_CUDA, "paco_noalloc_check: no current device");
    int *status = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_state[dev].ready) return PACO_OK;          // nothing has run on this device
        status = g_state[dev].status;
    }
    if (cudaDeviceSynchronize() != cudaSuccess)
        return fail(PACO_ERR_CUDA, "paco_noalloc_check: device synchronisation failed");
    int h = 0;
    if (cudaMemcpy(&h, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(status, 0, sizeof(int)) != cudaSuccess)
        return fail(PACO_ERR_CUDA, "paco_noalloc_check: status word read failed");
    if (h == PACO_ERR_TIMEOUT)
        return fail(PACO_ERR_TIMEOUT, "paco_execute_noalloc: a bounded device wait gave up");
    if (h != 0) return fail(PACO_ERR_DEVICE, "paco_execute_noalloc: a device-side check set the status word");
    return PACO_OK;
}

extern "C" void paco_debug_noalloc_set_waits(unsigned spin_limit, unsigned wait_bias)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_dbg_spin_limit = spin_limit;
    g_dbg_wait_bias = wait_bias;
}
