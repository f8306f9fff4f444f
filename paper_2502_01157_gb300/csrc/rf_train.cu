// rf_train.cu -- densification and pruning statistics of Radiant Foam
// (arXiv 2502.01157, Sec. 3.3) on the packed foam, sm_103a.
//
//   densify score  s_i = |dL/dp_i| * r_i, r_i = half the mean distance from
//                  p_i to its Delaunay neighbours (the faces of the cell lie
//                  halfway to them): cells that under-fit and are large;
//   multinomial    m draws of sites with probability s_i / sum s; the uniform
//                  numbers are inputs; FP64 inclusive prefix sums, and draw u
//                  takes the first site whose sum exceeds u * total;
//   prune mask     density below a threshold in the cell and in every
//                  neighbour.
#include "rf_host.h"

namespace rf {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;  // elements per block
constexpr int64_t kScanMaxBlocks = kScanTile;          // block sums scanned by one block

__global__ void densify_score_kernel(SceneDev s, int64_t n, const float *__restrict__ g_pos,
                                     float *__restrict__ score) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const CellHdr c = load_cell(s, (int)i);
    float sum = 0.f;
    int cnt = 0;
    for (int sl = 0; sl < 4 * c.gcnt; ++sl) {
        const int j = __ldg(s.nbr + 4 * (size_t)c.gbeg + sl);
        if (j < 0) continue;
        const float4 q = __ldg(s.cells + j);
        const float dx = q.x - c.x, dy = q.y - c.y, dz = q.z - c.z;
        sum += sqrtf(dx * dx + dy * dy + dz * dz);
        ++cnt;
    }
    const float gx = g_pos[3 * i], gy = g_pos[3 * i + 1], gz = g_pos[3 * i + 2];
    const float r = cnt ? 0.5f * sum / (float)cnt : 0.f;
    score[i] = sqrtf(gx * gx + gy * gy + gz * gz) * r;
}

template <typename AT>
__global__ void prune_kernel(SceneDev s, int64_t n, float thr, uint8_t *__restrict__ mask) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const AT *dens = reinterpret_cast<const AT *>(s.density);
    bool prune = to_f(__ldg(dens + i)) < thr;
    if (prune) {
        const CellHdr c = load_cell(s, (int)i);
        for (int sl = 0; sl < 4 * c.gcnt && prune; ++sl) {
            const int j = __ldg(s.nbr + 4 * (size_t)c.gbeg + sl);
            if (j >= 0) prune = to_f(__ldg(dens + j)) < thr;
        }
    }
    mask[i] = prune ? 1 : 0;
}

// inclusive scan of one tile per block (FP64); the tile total goes to sums[b]
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const float *__restrict__ w, int64_t n,
                                                                  double *__restrict__ cdf,
                                                                  double *__restrict__ sums) {
    __shared__ double part[kScanThreads];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    double v[kScanItems];
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t e = base + k;
        acc += e < n ? (double)fmaxf(w[e], 0.f) : 0.0;
        v[k] = acc;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {  // Hillis-Steele over thread totals
        const double add = threadIdx.x >= off ? part[threadIdx.x - off] : 0.0;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    const double before = threadIdx.x ? part[threadIdx.x - 1] : 0.0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t e = base + k;
        if (e < n) cdf[e] = before + v[k];
    }
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = part[threadIdx.x];
}

// exclusive scan of the tile totals in place (one block, <= kScanMaxBlocks)
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(double *__restrict__ sums, int64_t nb) {
    __shared__ double part[kScanThreads];
    const int64_t base = (int64_t)threadIdx.x * kScanItems;
    double v[kScanItems];
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = acc;  // exclusive
        acc += base + k < nb ? sums[base + k] : 0.0;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        const double add = threadIdx.x >= off ? part[threadIdx.x - off] : 0.0;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    const double before = threadIdx.x ? part[threadIdx.x - 1] : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < nb) sums[base + k] = before + v[k];
    if (threadIdx.x == kScanThreads - 1) sums[nb] = part[threadIdx.x];  // grand total
}

__global__ void add_offsets_kernel(double *__restrict__ cdf, int64_t n, const double *__restrict__ sums) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) cdf[e] += sums[e / kScanTile];
}

__global__ void draw_kernel(const double *__restrict__ cdf, int64_t n, const double *__restrict__ total,
                            const float *__restrict__ u, int64_t m, int32_t *__restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const double target = (double)u[k] * total[0];
    int64_t lo = 0, hi = n;  // first e with cdf[e] > target
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cdf[mid] > target) hi = mid; else lo = mid + 1;
    }
    out[k] = (int32_t)(lo < n ? lo : n - 1);
}

}  // namespace
}  // namespace rf

using namespace rf;

RF_API rf_status rf_densify_scores(rf_scene *s, const float *g_pos, float *score, void *stream) {
    if (!s || !g_pos || !score) return fail(RF_ERR_INVALID_ARG, "scene, g_pos and score are required");
    const int threads = 256;
    densify_score_kernel<<<(unsigned)((s->n_sites + threads - 1) / threads), threads, 0, (cudaStream_t)stream>>>(
        scene_dev(s), s->n_sites, g_pos, score);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

RF_API rf_status rf_prune_mask(rf_scene *s, float threshold, uint8_t *mask, void *stream) {
    if (!s || !mask) return fail(RF_ERR_INVALID_ARG, "scene and mask are required");
    const int threads = 256;
    const unsigned blocks = (unsigned)((s->n_sites + threads - 1) / threads);
    cudaStream_t st = (cudaStream_t)stream;
    if (s->attr_dtype == RF_BF16) prune_kernel<__nv_bfloat16><<<blocks, threads, 0, st>>>(scene_dev(s), s->n_sites, threshold, mask);
    else if (s->attr_dtype == RF_F16) prune_kernel<__half><<<blocks, threads, 0, st>>>(scene_dev(s), s->n_sites, threshold, mask);
    else prune_kernel<float><<<blocks, threads, 0, st>>>(scene_dev(s), s->n_sites, threshold, mask);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

RF_API size_t rf_multinomial_workspace_bytes(int64_t n) {
    if (n < 1) return 0;
    return sizeof(double) * (size_t)(n + (n + kScanTile - 1) / kScanTile + 1);
}

RF_API rf_status rf_sample_multinomial(const float *weights, int64_t n, const float *u, int64_t m,
                                       void *workspace, size_t workspace_bytes, int32_t *out,
                                       void *stream) {
    if (!weights || !u || !out || !workspace || n < 1 || m < 0)
        return fail(RF_ERR_INVALID_ARG, "weights, u, out and workspace are required, n >= 1");
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb > kScanMaxBlocks) return fail(RF_ERR_INVALID_ARG, "at most %lld weights", (long long)(kScanMaxBlocks * kScanTile));
    if (workspace_bytes < rf_multinomial_workspace_bytes(n))
        return fail(RF_ERR_INVALID_ARG, "workspace needs %zu bytes", rf_multinomial_workspace_bytes(n));
    if (((uintptr_t)workspace & 7) != 0) return fail(RF_ERR_INVALID_ARG, "workspace must be 8-byte aligned");
    if (m == 0) return RF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    double *cdf = static_cast<double *>(workspace);
    double *sums = cdf + n;  // nb tile totals, then the grand total
    scan_tiles_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(weights, n, cdf, sums);
    scan_sums_kernel<<<1, kScanThreads, 0, st>>>(sums, nb);
    add_offsets_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cdf, n, sums);
    draw_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(cdf, n, sums + nb, u, m, out);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}
