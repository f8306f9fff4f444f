// rf_shared.cu -- the backward kernels that sum the crossing terms of cells
// shared by many lanes before their atomics (render option
// RF_RENDER_SHARED_CELLS), compiled apart so the four halves of the
// backward build in parallel.
#include "rf_kernels.cuh"

namespace rf {

template void launch_bwd_any<false, true>(int, int, bool, int64_t, const RenderParams &, const BwdIO &, cudaStream_t);

}  // namespace rf
