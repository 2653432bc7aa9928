// Panel-pipeline stage kernel (length-2^14 stages, complex64).
#define PACO_PANEL_KERNEL_TU
#include "paco_panel.cuh"

namespace paco {

const void *panel_kernel_fn() { return reinterpret_cast<const void *>(&paco_panel_kernel); }

int panel_smem_bytes() { return panel::NSTAGE * panel::STAGE_ELEMS * (int)sizeof(float2); }

} // namespace paco
