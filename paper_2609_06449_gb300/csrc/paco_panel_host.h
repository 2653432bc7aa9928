// paco_panel_host.h -- host interface of the panel-pipeline stage kernel
// (paco_panel.cu), shared by plans (paco_capi.cu) and the allocation-free
// entry point (paco_noalloc.cu).  Not part of the C ABI.
#pragma once

#include <cstdint>

#include "../../include/paco.h"
#include "paco_panel.cuh"

namespace paco {

// One launch of a length-2^14 stage: mode 1 = Phase I with the fused
// top-level twiddle and digit reversal (X -> W), mode 2 = Phase III (W -> Y).
struct PanelLaunch {
    int mode;                     // 1 or 2
    int b;                        // digit-reversal radix: 2 or 4
    int64_t C;                    // columns of the stage input (mode 1: N2, mode 2: N1)
    int64_t batch;                // transforms
    int64_t N;                    // N1 * N2 (2^14 * C)
    int P;                        // panel width (columns), power of two, 64 <= P <= C
    const void *in;               // stage input
    void *out;                    // stage output (mode 2: may equal in)
    void *scratch;                // NBUF * 2^14 * P complex64 panel buffers
    unsigned *ctr;                // 2 * batch * C / P + 1 counters (cleared before the launch)
    int *status;                  // device status word
    const void *twL;              // w_{2^14}^{-r}
    const void *twN_lo, *twN_hi;  // w_N^{-r} in two levels
    int twN_lo_bits;
    int conj;                     // 1: dir = +1
    unsigned spin_limit;          // 0: default
    unsigned dep_bias;
};

paco_status_t fail(paco_status_t st, const char *fmt, ...);
const void *panel_kernel_fn(int mode, int b);
int panel_smem_bytes();
// Fill the kernel arguments (tensor maps included) for one launch.
paco_status_t panel_prepare(const PanelLaunch &l, PanelArgs *a);

} // namespace paco
