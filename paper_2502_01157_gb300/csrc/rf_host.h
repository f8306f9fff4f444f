// rf_host.h -- host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstddef>
#include <cstdint>

#include "../../include/rf.h"
#include "rf_internal.cuh"

struct rf_scene {
    int64_t n_sites = 0;
    int64_t n_edges = 0;
    float4 *cells = nullptr;     // [N]: {x, y, z, first_group << count_bits | n_groups}
    int32_t *off = nullptr;      // [N+1] first face group of each cell
    float4 *faces = nullptr;     // [3 n_groups]: u_x, u_y, u_z of four faces per group
    int32_t *nbr = nullptr;      // [4 n_groups]: neighbour ids (-1: padding)
    int64_t n_groups = 0;
    int32_t count_bits = 4;
    const void *density = nullptr;  // borrowed
    const void *sh = nullptr;       // borrowed
    int32_t sh_degree = 0;
    int32_t attr_dtype = RF_F32;
    float box[6] = {0, 0, 0, 0, 0, 0};
    unsigned long long *start_keys = nullptr;  // workspace [kMaxCamsPerLaunch]
    int32_t *flags = nullptr;                  // workspace [8] (validation counters)
    int32_t sh_v8 = 0;                         // SH rows 32-byte aligned
    float4 *g_acc = nullptr;                   // workspace [N] of the backward (first use)
    size_t bytes = 0;
    int device = 0;
};

namespace rf {

rf_status fail(rf_status code, const char *fmt, ...);
rf_status cuda_fail(cudaError_t e, const char *what);

// per_sm x the current device's SM count (queried once per device), the cap
// of the grid-stride kernels' grids
int grid_cap(int per_sm);

#define RF_CUDA(expr)                                                  \
    do {                                                               \
        cudaError_t e_ = (expr);                                       \
        if (e_ != cudaSuccess) return ::rf::cuda_fail(e_, #expr);      \
    } while (0)

SceneDev scene_dev(const rf_scene *s);
rf_status check_camera(const rf_camera &c, int index);
rf_status check_opts(const rf_render_opts *o, float *eps, int32_t *max_steps, SphereFx *fx);

// Start cells nn(o) of cams[0..n) (n <= kMaxCamsPerLaunch) into keys[0..n).
rf_status launch_nearest_sites(const rf_scene *s, const rf_camera *cams, int n,
                               unsigned long long *keys, cudaStream_t st);

// Fill a LaunchCams for cams[first .. first+count); returns the tile count.
int64_t make_launch_cams(const rf_camera *cams, int first, int count, int64_t ray_begin,
                         LaunchCams *lc);

}  // namespace rf
