// Panel-pipeline stage kernel (length-2^14 stages, complex64).
#define PACO_PANEL_KERNEL_TU
#include "paco_panel.cuh"

namespace paco {

const void *panel_kernel_fn(int prefetch)
{
    return prefetch ? reinterpret_cast<const void *>(&paco_panel_kernel<true>)
                    : reinterpret_cast<const void *>(&paco_panel_kernel<false>);
}

int panel_smem_bytes() { return panel::A * panel::SP * (int)sizeof(float2); }

const void *panel_tma_kernel_fn() { return reinterpret_cast<const void *>(&paco_panel_tma_kernel); }

int panel_tma_smem_bytes() { return tma::NSTAGE * tma::STAGE_ELEMS * (int)sizeof(float2); }

} // namespace paco
