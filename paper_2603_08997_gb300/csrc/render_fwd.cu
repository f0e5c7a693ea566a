// gs_render_fwd: Eq. (blend) / Eq. (alpha), front-to-back compositing.
//
// One CTA per tile, one thread per pixel, each warp an 8 x 4 pixel block that
// skips Gaussians whose support box misses it.  The tile's depth-ordered list is
// consumed `BATCH` Gaussians at a time: the CTA gathers the batch's packed
// records into shared memory (one coalesced 48-byte record per Gaussian),
// then every pixel walks the batch.  At the start of every batch each pixel
// stores its transmittance into the checkpoint slot
//   slot(tile, b) = floor(range_start / BATCH) + tile + b,
// which the backward pass uses to rebuild T without dividing across batches.
// The CTA stops as soon as every pixel has hit the transmittance floor.
#include "common.cuh"

using namespace gsr;

namespace {

template <int TILE, int BATCH>
__global__ void __launch_bounds__(TILE *TILE) render_fwd_kernel(const float4 *__restrict__ rec, int64_t n,
                                                                 const uint32_t *__restrict__ vals,
                                                                 const uint2 *__restrict__ ranges,
                                                                 const gs_camera *__restrict__ cams, int n_views,
                                                                 gs_raster_config cfg, float *__restrict__ image,
                                                                 float *__restrict__ T_final,
                                                                 int32_t *__restrict__ n_last,
                                                                 float *__restrict__ ckpt, int64_t ckpt_slots) {
    constexpr int NT = TILE * TILE;
    __shared__ float4 s_a[BATCH];
    __shared__ float4 s_b[BATCH];
    __shared__ float4 s_c[BATCH];
    const int64_t tile = blockIdx.x;
    const int v = view_of_tile(cams, n_views, tile);
    const gs_camera &cam = cams[v];
    const int tiles_x = (cam.width + TILE - 1) / TILE;
    const int64_t lt = tile - cam.tile_offset;
    const int tx = (int)(lt % tiles_x), ty = (int)(lt / tiles_x);
    int lx, ly;
    tile_pixel<TILE>(threadIdx.x, lx, ly);
    const int x = tx * TILE + lx, y = ty * TILE + ly;
    const bool inside = x < cam.width && y < cam.height;
    const float px = (float)x + 0.5f, py = (float)y + 0.5f;
    const float wx = (float)(tx * TILE + (lx & ~7)) + 0.5f, wy = (float)(ty * TILE + (ly & ~3)) + 0.5f;
    const uint2 rg = ranges[tile];
    const int64_t len = (int64_t)rg.y - rg.x;
    const int64_t nb = ceil_div(len, BATCH);
    const int64_t slot0 = (int64_t)(rg.x / BATCH) + tile;
    const float4 *recv = rec + (int64_t)v * n * 3;
    const float amax = cfg.alpha_max, amin = cfg.alpha_min, tmin = cfg.t_min;

    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    int32_t last = 0;
    bool done = !inside;
    for (int64_t b = 0; b < nb; ++b) {
        if (__syncthreads_count(!done) == 0) break;
        if (inside && slot0 + b < ckpt_slots) ckpt[(slot0 + b) * NT + threadIdx.x] = T;
        const int64_t b0 = (int64_t)rg.x + b * BATCH;
        const int cnt = (int)min((int64_t)BATCH, (int64_t)rg.y - b0);
        for (int k = threadIdx.x; k < cnt; k += NT) {
            const uint32_t g = vals[b0 + k];
            const float4 *r = recv + (int64_t)g * 3;
            s_a[k] = r[0];
            s_b[k] = r[1];
            s_c[k] = r[2];
        }
        __syncthreads();
        if (!done) {
            for (int j = 0; j < cnt; ++j) {
                if (!warp_overlaps(s_a[j], s_c[j], wx, wy)) continue;  // alpha' < alpha_min on all 32 pixels
                const AlphaEval ae = eval_alpha(s_a[j], s_b[j], px, py, amax);
                if (ae.alpha < amin) continue;
                const float testT = __fmul_rn(T, __fsub_rn(1.f, ae.alpha));
                if (testT < tmin) {
                    done = true;
                    break;
                }
                const float w = ae.alpha * T;
                const float4 bb = s_b[j];
                C0 += bb.z * w;
                C1 += bb.w * w;
                C2 += s_c[j].x * w;
                T = testT;
                last = (int32_t)(b * BATCH + j + 1);
            }
        }
    }
    if (inside) {
        const int64_t hw = (int64_t)cam.width * cam.height;
        const int64_t pix = (int64_t)y * cam.width + x;
        float *img = image + 3 * cam.pix_offset;
        img[pix] = C0 + T * cfg.bg[0];
        img[hw + pix] = C1 + T * cfg.bg[1];
        img[2 * hw + pix] = C2 + T * cfg.bg[2];
        T_final[cam.pix_offset + pix] = T;
        n_last[cam.pix_offset + pix] = last;
    }
}

template <int TILE>
gs_status launch_fwd(int batch, int64_t total_tiles, cudaStream_t stream, const float4 *rec, int64_t n,
                     const uint32_t *vals, const uint2 *ranges, const gs_camera *cams, int n_views,
                     const gs_raster_config &cfg, float *image, gs_fwd_saved s) {
    const dim3 grid((unsigned)total_tiles);
    switch (batch) {
        case 64:
            render_fwd_kernel<TILE, 64><<<grid, TILE * TILE, 0, stream>>>(rec, n, vals, ranges, cams, n_views, cfg, image,
                                                                         s.T_final, s.n_last, s.ckpt, s.ckpt_slots);
            break;
        case 128:
            render_fwd_kernel<TILE, 128><<<grid, TILE * TILE, 0, stream>>>(rec, n, vals, ranges, cams, n_views, cfg,
                                                                          image, s.T_final, s.n_last, s.ckpt,
                                                                          s.ckpt_slots);
            break;
        case 256:
            render_fwd_kernel<TILE, 256><<<grid, TILE * TILE, 0, stream>>>(rec, n, vals, ranges, cams, n_views, cfg,
                                                                          image, s.T_final, s.n_last, s.ckpt,
                                                                          s.ckpt_slots);
            break;
        default:
            return GS_ERR_UNSUPPORTED;
    }
    GS_TRY_LAUNCH();
    return GS_OK;
}

}  // namespace

extern "C" gs_status gs_render_fwd(const gs_projected *proj, int64_t n, const uint32_t *vals, const uint32_t *ranges,
                                   const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                                   const gs_raster_config *cfg, float *image, gs_fwd_saved saved,
                                   int32_t *dev_status, cudaStream_t stream) {
    (void)dev_status;
    if (!proj || !cfg || !cams || !vals || !ranges || !image || n_views <= 0 || n < 0 || total_tiles <= 0)
        return GS_ERR_INVALID_ARG;
    if (total_tiles >= ((int64_t)1 << 31)) return GS_ERR_INVALID_ARG;
    if (!saved.T_final || !saved.n_last || !saved.ckpt || saved.ckpt_slots <= 0) return GS_ERR_INVALID_ARG;
    if (n > 0 && !proj->rec) return GS_ERR_INVALID_ARG;
    if ((uintptr_t)proj->rec & 15) return GS_ERR_INVALID_ARG;
    const float4 *rec = reinterpret_cast<const float4 *>(proj->rec);
    const uint2 *rg = reinterpret_cast<const uint2 *>(ranges);
    switch (cfg->tile) {
        case 8: return launch_fwd<8>(cfg->batch, total_tiles, stream, rec, n, vals, rg, cams, n_views, *cfg, image, saved);
        case 16: return launch_fwd<16>(cfg->batch, total_tiles, stream, rec, n, vals, rg, cams, n_views, *cfg, image, saved);
        case 32: return launch_fwd<32>(cfg->batch, total_tiles, stream, rec, n, vals, rg, cams, n_views, *cfg, image, saved);
        default: return GS_ERR_INVALID_ARG;
    }
}
