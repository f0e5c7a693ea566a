// Measurement entry points (not on the refinement path).
//
// gs_raster_census counts, for one forward pass, the work the compositing
// kernels must do, so throughput can be stated per unit of algorithmic work
// rather than per unit of whatever a kernel happens to execute:
//   [0] sum over pixels of n_last (every list position up to the pixel's last
//       contributor: an upper bound of the evaluations);
//   [1] (pixel, Gaussian) pairs at positions before the pixel's last
//       contributor whose support box (mean2D +- (rx, ry)) contains the pixel
//       centre: the evaluations Eq. (alpha) needs (outside the box
//       alpha' < alpha_min is known without evaluating);
//   [2] contributing pairs (alpha' >= alpha_min before the pixel stopped);
//   [3] (tile, Gaussian) pairs with at least one contributing pixel: the
//       raster adjoint adds each one's nine gradients to global memory with
//       three atomic instructions (two 4-wide, one scalar);
//   [4] list entries up to each tile's largest n_last (records the adjoint
//       stages).
// The alphas come from the same evaluation as the compositing kernels.
//
// gs_atomic_probe issues the raster adjoint's global atomic pattern - per
// update two float4 and one float reduction into a 48-byte per-Gaussian
// record - at pseudo-random records, to measure the throughput of scattered
// L2 reductions on this GPU (the peak against which the adjoint's atomic
// rate is stated).
#include "common.cuh"

using namespace gsr;

namespace {

template <int TILE>
__global__ void __launch_bounds__(256) census_kernel(const float4 *__restrict__ rec, int64_t n,
                                                     const uint32_t *__restrict__ vals,
                                                     const uint2 *__restrict__ ranges,
                                                     const gs_camera *__restrict__ cams, int n_views,
                                                     gs_raster_config cfg, const int32_t *__restrict__ n_last,
                                                     unsigned long long *__restrict__ counts) {
    constexpr int NT = TILE * TILE;
    constexpr int PT = (NT + 255) / 256;  // pixels per thread
    __shared__ int s_max;
    const int64_t tile = blockIdx.x;
    const int v = view_of_tile(cams, n_views, tile);
    const gs_camera &cam = cams[v];
    const int tiles_x = (cam.width + TILE - 1) / TILE;
    const int64_t lt = tile - cam.tile_offset;
    const int tx = (int)(lt % tiles_x), ty = (int)(lt / tiles_x);
    const uint2 rg = ranges[tile];
    const float4 *recv = rec + (int64_t)v * n * 3;
    int last[PT];
    float px[PT], py[PT];
    int my_max = 0;
    unsigned long long c_last = 0;
#pragma unroll
    for (int k = 0; k < PT; ++k) {
        const int p = threadIdx.x + k * 256;
        last[k] = 0;
        px[k] = py[k] = 0.f;
        if (p < NT) {
            const int x = tx * TILE + p % TILE, y = ty * TILE + p / TILE;
            px[k] = (float)x + 0.5f;
            py[k] = (float)y + 0.5f;
            if (x < cam.width && y < cam.height) last[k] = n_last[cam.pix_offset + (int64_t)y * cam.width + x];
        }
        my_max = max(my_max, last[k]);
        c_last += (unsigned long long)last[k];
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    if (my_max > 0) atomicMax(&s_max, my_max);
    __syncthreads();
    const int max_last = min(s_max, (int)(rg.y - rg.x));
    unsigned long long c_box = 0, c_con = 0, c_pairs = 0;
    for (int j = 0; j < max_last; ++j) {
        const uint32_t g = vals[rg.x + j];
        const float4 a = recv[(int64_t)g * 3], b = recv[(int64_t)g * 3 + 1], c = recv[(int64_t)g * 3 + 2];
        bool any = false;
#pragma unroll
        for (int k = 0; k < PT; ++k) {
            if (j >= last[k]) continue;
            if (fabsf(px[k] - a.x) > c.z || fabsf(py[k] - a.y) > c.w) continue;
            ++c_box;
            const AlphaEval ae = eval_alpha(a, b, px[k], py[k], cfg.alpha_max);
            if (ae.alpha < cfg.alpha_min) continue;
            ++c_con;
            any = true;
        }
        if (__syncthreads_or(any) && threadIdx.x == 0) ++c_pairs;
    }
    // warp sums, then one atomic per warp and counter
    for (int o = 16; o > 0; o >>= 1) {
        c_last += __shfl_xor_sync(0xffffffffu, c_last, o);
        c_box += __shfl_xor_sync(0xffffffffu, c_box, o);
        c_con += __shfl_xor_sync(0xffffffffu, c_con, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&counts[0], c_last);
        atomicAdd(&counts[1], c_box);
        atomicAdd(&counts[2], c_con);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&counts[3], c_pairs);
        atomicAdd(&counts[4], (unsigned long long)max_last);
    }
}

__global__ void census_zero(unsigned long long *counts) {
    if (threadIdx.x < 5) counts[threadIdx.x] = 0ull;
}

// Record index of update u: a multiplicative hash spreads consecutive updates
// over the whole buffer (and so over the L2 slices).
__device__ __forceinline__ int64_t probe_record(uint64_t u, int64_t n_records) {
    const uint64_t h = (u + 1) * 0x9E3779B97F4A7C15ull;
    return (int64_t)((h >> 20) % (uint64_t)n_records);
}

__global__ void __launch_bounds__(256) atomic_probe_kernel(float4 *__restrict__ buf, int64_t n_records,
                                                           int64_t n_updates) {
    const float4 d = make_float4(1e-30f, 1e-30f, 1e-30f, 1e-30f);
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_updates;
         u += (int64_t)gridDim.x * blockDim.x) {
        float4 *dst = buf + probe_record((uint64_t)u, n_records) * 3;
        atomicAdd(dst, d);
        atomicAdd(dst + 1, d);
        atomicAdd(&dst[2].x, d.x);
    }
}

}  // namespace

extern "C" gs_status gs_raster_census(const gs_projected *proj, int64_t n, const uint32_t *vals,
                                      const uint32_t *ranges, const gs_camera *cams, int32_t n_views,
                                      int64_t total_tiles, const gs_raster_config *cfg, const int32_t *n_last,
                                      unsigned long long *counts, cudaStream_t stream) {
    if (!proj || !cfg || !cams || !vals || !ranges || !n_last || !counts || n_views <= 0 || n < 0 ||
        total_tiles <= 0 || total_tiles >= ((int64_t)1 << 31))
        return GS_ERR_INVALID_ARG;
    if (n > 0 && (!proj->rec || ((uintptr_t)proj->rec & 15))) return GS_ERR_INVALID_ARG;
    const float4 *rec = reinterpret_cast<const float4 *>(proj->rec);
    const uint2 *rg = reinterpret_cast<const uint2 *>(ranges);
    census_zero<<<1, 32, 0, stream>>>(counts);
    GS_TRY_LAUNCH();
    const dim3 grid((unsigned)total_tiles);
    switch (cfg->tile) {
        case 8: census_kernel<8><<<grid, 256, 0, stream>>>(rec, n, vals, rg, cams, n_views, *cfg, n_last, counts); break;
        case 16: census_kernel<16><<<grid, 256, 0, stream>>>(rec, n, vals, rg, cams, n_views, *cfg, n_last, counts); break;
        case 32: census_kernel<32><<<grid, 256, 0, stream>>>(rec, n, vals, rg, cams, n_views, *cfg, n_last, counts); break;
        default: return GS_ERR_INVALID_ARG;
    }
    GS_TRY_LAUNCH();
    return GS_OK;
}

extern "C" gs_status gs_atomic_probe(float *buf, int64_t n_records, int64_t n_updates, cudaStream_t stream) {
    if (!buf || n_records <= 0 || n_updates < 0 || ((uintptr_t)buf & 15)) return GS_ERR_INVALID_ARG;
    if (n_updates == 0) return GS_OK;
    const int64_t want = ceil_div(n_updates, 256);
    const int64_t resident = (int64_t)device_sm_count() * 8;  // 8 blocks of 256 threads per SM
    const unsigned blocks = (unsigned)(want < resident ? want : resident);
    atomic_probe_kernel<<<blocks, 256, 0, stream>>>(reinterpret_cast<float4 *>(buf), n_records, n_updates);
    GS_TRY_LAUNCH();
    return GS_OK;
}
