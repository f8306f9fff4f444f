// rf_effects.cu -- the renderer's kernels with the analytic sphere in the walk
// (reflection and refraction met by the rays, the ray-based effects of the
// paper's Fig. 2), compiled apart from the plain kernels of rf_render.cu.
#include "rf_kernels.cuh"

namespace rf {

template void launch_fwd_any<true>(int, int, int, int64_t, const RenderParams &, const FwdOut &, cudaStream_t);
template void launch_bwd_any<true, false>(int, int, bool, int64_t, const RenderParams &, const BwdIO &, cudaStream_t);

}  // namespace rf
