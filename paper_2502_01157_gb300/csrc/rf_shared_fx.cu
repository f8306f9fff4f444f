// rf_shared_fx.cu -- the shared-cell backward kernels (see rf_shared.cu)
// with the ray-based effects of the paper's Fig. 2.
#include "rf_kernels.cuh"

namespace rf {

template void launch_bwd_any<true, true>(int, int, bool, int64_t, const RenderParams &, const BwdIO &, cudaStream_t);

}  // namespace rf
