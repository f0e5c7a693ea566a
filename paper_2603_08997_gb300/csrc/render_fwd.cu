// gs_render_fwd: Eq. (blend) / Eq. (alpha), front-to-back compositing.
//
// One CTA per tile, PPT pixels per thread (1, 2 or 4), each warp an 8 x 4 PPT
// pixel block.  The tile's depth-ordered list is
// consumed `BATCH` Gaussians at a time: the CTA gathers the batch's packed
// records into shared memory (one 48-byte record per Gaussian, copied
// asynchronously one batch ahead into a second buffer) and marks, per warp,
// the records whose support ellipse reaches the warp's pixel block (one ballot
// per warp and 32 records); every warp then walks only its marked records,
// in order.  At the start of every batch but the tile's first (which starts
// at T = 1) each pixel stores its transmittance into the checkpoint slot
//   slot(tile, b) = floor(range_start / BATCH) + tile + b
// (TILE * TILE floats, row-major over the tile's pixels), which the backward pass uses to rebuild T without dividing across batches.
// The CTA stops as soon as every pixel has hit the transmittance floor.
//
// Super-tile form (COARSE): the tile's Gaussian indices come from its
// super-tile's depth-ordered list, filtered by the tile's mask bit while the
// batches are gathered (coarse_gather, one batch ahead of the record copies);
// the batches, and so every output, are the same as with the tile's own list.
// The list position of each batch's first entry goes to batch_pos at the
// batch's checkpoint slot, for the adjoint.
#include "common.cuh"

using namespace gsr;

namespace {

// One pixel per thread (the loop's shape): 5 resident blocks per SM (48
// registers) measured faster than the compiler's own 4 (63).
template <int TILE, int BATCH, int PPT, bool COARSE>
__global__ void __launch_bounds__(TILE *TILE / PPT, PPT == 1 ? 5 : 1) render_fwd_kernel(const float4 *__restrict__ rec, int64_t n,
                                                                       const ListSrc ls,
                                                                       const uint2 *__restrict__ ranges,
                                                                       const gs_camera *__restrict__ cams, int n_views,
                                                                       gs_raster_config cfg, float *__restrict__ image,
                                                                       float *__restrict__ T_final,
                                                                       int32_t *__restrict__ n_last,
                                                                       float *__restrict__ ckpt, int64_t ckpt_slots,
                                                                       const uint32_t *__restrict__ tile_order,
                                                                       uint32_t *queue, int64_t total_tiles) {
    constexpr int NT = TILE * TILE;        // pixels per tile (checkpoint slot size)
    constexpr int NTH = TILE * TILE / PPT; // threads
    constexpr int NW = NTH / 32, NWORD = BATCH / 32;
    constexpr int R = (BATCH + NTH - 1) / NTH;  // batch slots per thread
    constexpr int EPT = gather_ept<NTH>();  // super-tile list entries tested per thread and round
    __shared__ float4 s_a[2][BATCH];  // double buffer: batch b + 1 arrives while batch b is composited
    __shared__ float4 s_b[2][BATCH];
    __shared__ float4 s_c[2][BATCH];
    __shared__ uint32_t s_ov[NW][NWORD];  // per warp: records of the batch that reach its pixel block
    __shared__ uint32_t s_item;
    __shared__ uint32_t s_idx[COARSE ? BATCH : 1];  // a gathered batch's Gaussian indices
    __shared__ uint32_t s_wsum[NW], s_next;
    for (uint32_t item = first_item(queue, &s_item); item < (uint64_t)total_tiles; item = next_item(queue, &s_item)) {
    const int64_t tile = tile_order ? (int64_t)tile_order[item] : (int64_t)item;
    const int v = view_of_tile(cams, n_views, tile);
    const gs_camera &cam = cams[v];
    const int tiles_x = (cam.width + TILE - 1) / TILE;
    const int64_t lt = tile - cam.tile_offset;
    const int tx = (int)(lt % tiles_x), ty = (int)(lt / tiles_x);
    int x[PPT], y[PPT], lp[PPT];
    bool inside[PPT];
    float px[PPT], py[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        int lx, ly;
        tile_pixel<TILE, PPT>(threadIdx.x, k, lx, ly);
        lp[k] = ly * TILE + lx;  // checkpoint slot layout is row-major in the tile
        x[k] = tx * TILE + lx;
        y[k] = ty * TILE + ly;
        inside[k] = x[k] < cam.width && y[k] < cam.height;
        px[k] = (float)x[k] + 0.5f;
        py[k] = (float)y[k] + 0.5f;
    }
    const int warp = threadIdx.x >> 5;
    const uint2 rg = ranges[tile];
    const int64_t len = (int64_t)rg.y - rg.x;
    const int64_t nb = ceil_div(len, BATCH);
    const int64_t slot0 = (int64_t)(rg.x / BATCH) + tile;
    const float4 *recv = rec + (int64_t)v * n * 3;
    const float amax = cfg.alpha_max, amin = cfg.alpha_min, tmin = cfg.t_min;

    float T[PPT], C0[PPT], C1[PPT], C2[PPT];
    int32_t last[PPT];
    bool done[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        T[k] = 1.f; C0[k] = C1[k] = C2[k] = 0.f; last[k] = 0; done[k] = !inside[k];
    }
    // the super-tile list: this tile's bit and the list's unread part
    uint32_t cbit = 0, cpos = 0, cend = 0;
    if constexpr (COARSE) {
        if (len > 0) {
            const int64_t ct = super_tile_of(ls, v, tiles_x, tx, ty, cbit);
            cpos = ls.cstart[ct];
            cend = cpos + ls.ccount[ct];
        }
    }
    // Gaussian indices of this thread's slots of batch bb (0xffffffff past the
    // list); batches are requested in order 0, 1, 2, ... (the super-tile form
    // gathers them with the whole block: uniform calls only)
    auto load_index = [&](int64_t bb, uint32_t (&gi)[R]) {
        if constexpr (COARSE) {
            int got = 0;
            if (bb < nb) {
                if (threadIdx.x == 0 && slot0 + bb < ckpt_slots) ls.batch_pos[slot0 + bb] = cpos;
                got = coarse_gather<NTH, EPT>(ls, cbit, cpos, cend, BATCH, s_idx, s_wsum, &s_next);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int kk = threadIdx.x + r * NTH;
                gi[r] = (kk < got) ? s_idx[kk] : 0xffffffffu;
            }
        } else {
            const int64_t b0 = (int64_t)rg.x + bb * BATCH;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int kk = threadIdx.x + r * NTH;
                gi[r] = (bb < nb && kk < BATCH && b0 + kk < (int64_t)rg.y) ? ls.vals[b0 + kk] : 0xffffffffu;
            }
        }
    };
    // start the copies of this thread's records of a batch into buffer buf
    auto issue = [&](const uint32_t (&gi)[R], int buf) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int kk = threadIdx.x + r * NTH;
            if (kk < BATCH && gi[r] != 0xffffffffu) {
                const float4 *src = recv + (int64_t)gi[r] * 3;
                cp_async16(&s_a[buf][kk], src);
                cp_async16(&s_b[buf][kk], src + 1);
                cp_async16(&s_c[buf][kk], src + 2);
            }
        }
        cp_async_commit();
    };
    // Tile lists: the indices of batch b + 2 load while batch b composites,
    // the records of batch b + 1 copy meanwhile.  Super-tile lists: batch b + 1
    // is gathered (a block-wide step) and its copies issued at the start of
    // batch b, so no batch past the one that finishes the tile is gathered.
    uint32_t gi[R];
    load_index(0, gi);
    issue(gi, 0);
    if constexpr (!COARSE) load_index(1, gi);  // indices of the next batch, one batch ahead of its copies
    for (int64_t b = 0; b < nb; ++b) {
        bool all_done = true;
#pragma unroll
        for (int k = 0; k < PPT; ++k) all_done &= done[k];
        if (__syncthreads_count(!all_done) == 0) break;  // every warp is also past batch b - 1
        if (b > 0 && slot0 + b < ckpt_slots) {  // the first batch starts at T = 1: nothing to store
#pragma unroll
            for (int k = 0; k < PPT; ++k)
                if (inside[k]) ckpt[(slot0 + b) * NT + lp[k]] = T[k];
        }
        const int buf = (int)(b & 1);
        if (b + 1 < nb) {
            if constexpr (COARSE) {
                load_index(b + 1, gi);
                issue(gi, buf ^ 1);
            } else {
                issue(gi, buf ^ 1);
                load_index(b + 2, gi);
            }
            cp_async_wait<1>();  // this thread's copies of batch b have landed
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int64_t b0 = (int64_t)rg.x + b * BATCH;
        const int cnt = (int)min((int64_t)BATCH, (int64_t)rg.y - b0);
        for (int kk = threadIdx.x; kk < BATCH; kk += NTH) {  // whole warps (BATCH, NTH multiples of 32)
            const bool valid = kk < cnt;
            const float4 ra = valid ? s_a[buf][kk] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 rb = valid ? s_b[buf][kk] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 rc = valid ? s_c[buf][kk] : make_float4(0.f, 0.f, 0.f, 0.f);
            overlap_masks<TILE, PPT, NW, NWORD>(s_ov, kk, valid, ra, rb, rc, amin, tx * TILE, ty * TILE);
        }
        __syncthreads();
        const float4 *s_a_b = s_a[buf], *s_b_b = s_b[buf], *s_c_b = s_c[buf];
        if (!all_done) {
            bool alive = true;
            for (int wd = 0; wd < NWORD && alive; ++wd) {
                // only records whose support ellipse reaches the warp's block can have alpha' >= alpha_min there
                uint32_t m = s_ov[warp][wd];
                while (m) {
                    const int j = wd * 32 + __ffs(m) - 1;
                    m &= m - 1;
                    const float4 sa = s_a_b[j], sb = s_b_b[j], sc = s_c_b[j];
                    alive = false;
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        if (done[k]) continue;
                        alive = true;
                        const AlphaEval ae = eval_alpha(sa, sb, px[k], py[k], amax);
                        if (ae.alpha < amin) continue;
                        const float testT = __fmul_rn(T[k], __fsub_rn(1.f, ae.alpha));
                        if (testT < tmin) {
                            done[k] = true;
                            continue;
                        }
                        const float w = ae.alpha * T[k];
                        C0[k] += sb.z * w;
                        C1[k] += sb.w * w;
                        C2[k] += sc.x * w;
                        T[k] = testT;
                        last[k] = (int32_t)(b * BATCH + j + 1);
                    }
                    if (!alive) break;
                }
            }
        }
    }
    cp_async_wait<0>();  // no copy into this block's shared memory outlives it
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (!inside[k]) continue;
        const int64_t hw = (int64_t)cam.width * cam.height;
        const int64_t pix = (int64_t)y[k] * cam.width + x[k];
        float *img = image + 3 * cam.pix_offset;
        img[pix] = C0[k] + T[k] * cfg.bg[0];
        img[hw + pix] = C1[k] + T[k] * cfg.bg[1];
        img[2 * hw + pix] = C2[k] + T[k] * cfg.bg[2];
        T_final[cam.pix_offset + pix] = T[k];
        n_last[cam.pix_offset + pix] = last[k];
    }
    }  // items
}

// Grid of a compositing kernel: a block per tile, or (persistent, with a
// queue) the blocks resident on the device at once (cached per device).
template <typename K>
gs_status item_grid(K kernel, int threads, int64_t total_tiles, bool persistent, int *cache, dim3 &grid) {
    grid = dim3((unsigned)total_tiles);
    if (!persistent) return GS_OK;
    const int dev = cached_device_index();
    if (dev < 0) return GS_ERR_UNSUPPORTED;
    if (cache[dev] <= 0) {
        int per_sm = 0;
        GS_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0));
        cache[dev] = (per_sm > 0 ? per_sm : 1) * device_sm_count();
    }
    if ((int64_t)cache[dev] < total_tiles) grid = dim3((unsigned)cache[dev]);
    return GS_OK;
}

template <int TILE, int PPT, bool CO>
using FwdKernel = decltype(&render_fwd_kernel<TILE, 64, PPT, CO>);

template <int TILE, int PPT, bool CO>
FwdKernel<TILE, PPT, CO> fwd_kernel(int batch) {
    switch (batch) {
        case 64: return render_fwd_kernel<TILE, 64, PPT, CO>;
        case 128: return render_fwd_kernel<TILE, 128, PPT, CO>;
        case 256: return render_fwd_kernel<TILE, 256, PPT, CO>;
        default: return nullptr;
    }
}

template <int TILE, int PPT, bool CO>
gs_status launch_fwd(int batch, int64_t total_tiles, cudaStream_t stream, const float4 *rec, int64_t n,
                     const ListSrc &ls, const uint2 *ranges, const gs_camera *cams, int n_views,
                     const gs_raster_config &cfg, float *image, gs_fwd_saved s) {
    const auto kernel = fwd_kernel<TILE, PPT, CO>(batch);
    if (!kernel) return GS_ERR_UNSUPPORTED;
    constexpr int NTH = TILE * TILE / PPT;
    static int resident[3][kMaxDevices] = {};  // per staging batch size
    const int bi = batch == 64 ? 0 : (batch == 128 ? 1 : 2);
    dim3 grid;
    const gs_status st = item_grid(kernel, NTH, total_tiles, s.queue, resident[bi], grid);
    if (st != GS_OK) return st;
    if (s.queue) GS_TRY(cudaMemsetAsync(s.queue, 0, sizeof(uint32_t), stream));
    kernel<<<grid, NTH, 0, stream>>>(rec, n, ls, ranges, cams, n_views, cfg, image, s.T_final, s.n_last, s.ckpt,
                                     s.ckpt_slots, s.tile_order, s.queue, total_tiles);
    GS_TRY_LAUNCH();
    return GS_OK;
}

template <int TILE, bool CO>
gs_status launch_fwd_ppt(int ppt, int batch, int64_t total_tiles, cudaStream_t stream, const float4 *rec, int64_t n,
                         const ListSrc &ls, const uint2 *ranges, const gs_camera *cams, int n_views,
                         const gs_raster_config &cfg, float *image, gs_fwd_saved s) {
    if constexpr (TILE >= 16)
        if (ppt == 4) return launch_fwd<TILE, 4, CO>(batch, total_tiles, stream, rec, n, ls, ranges, cams, n_views, cfg, image, s);
    if (ppt == 2) return launch_fwd<TILE, 2, CO>(batch, total_tiles, stream, rec, n, ls, ranges, cams, n_views, cfg, image, s);
    return launch_fwd<TILE, 1, CO>(batch, total_tiles, stream, rec, n, ls, ranges, cams, n_views, cfg, image, s);
}

gs_status render_fwd_impl(const gs_projected *proj, int64_t n, const ListSrc &ls, bool coarse,
                          const uint32_t *ranges, const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                          const gs_raster_config *cfg, float *image, gs_fwd_saved saved, cudaStream_t stream) {
    if (!proj || !cfg || !cams || !ranges || !image || n_views <= 0 || n < 0 || total_tiles <= 0)
        return GS_ERR_INVALID_ARG;
    if (total_tiles >= ((int64_t)1 << 31)) return GS_ERR_INVALID_ARG;
    if (!saved.T_final || !saved.n_last || !saved.ckpt || saved.ckpt_slots <= 0) return GS_ERR_INVALID_ARG;
    if (n > 0 && !proj->rec) return GS_ERR_INVALID_ARG;
    if ((uintptr_t)proj->rec & 15) return GS_ERR_INVALID_ARG;
    const float4 *rec = reinterpret_cast<const float4 *>(proj->rec);
    const uint2 *rg = reinterpret_cast<const uint2 *>(ranges);
    const int ppt = cfg->pixels_per_thread;
    if (ppt != 1 && ppt != 2 && ppt != 4) return GS_ERR_INVALID_ARG;
    if (ppt == 4 && cfg->tile < 16) return GS_ERR_INVALID_ARG;  // a warp needs 8 x 16 pixels
    if (cfg->batch != 64 && cfg->batch != 128 && cfg->batch != 256) return GS_ERR_UNSUPPORTED;
    const int b = cfg->batch;
    switch (cfg->tile * 2 + (coarse ? 1 : 0)) {
        case 16: return launch_fwd_ppt<8, false>(ppt, b, total_tiles, stream, rec, n, ls, rg, cams, n_views, *cfg, image, saved);
        case 17: return launch_fwd_ppt<8, true>(ppt, b, total_tiles, stream, rec, n, ls, rg, cams, n_views, *cfg, image, saved);
        case 32: return launch_fwd_ppt<16, false>(ppt, b, total_tiles, stream, rec, n, ls, rg, cams, n_views, *cfg, image, saved);
        case 33: return launch_fwd_ppt<16, true>(ppt, b, total_tiles, stream, rec, n, ls, rg, cams, n_views, *cfg, image, saved);
        case 64: return launch_fwd_ppt<32, false>(ppt, b, total_tiles, stream, rec, n, ls, rg, cams, n_views, *cfg, image, saved);
        case 65: return launch_fwd_ppt<32, true>(ppt, b, total_tiles, stream, rec, n, ls, rg, cams, n_views, *cfg, image, saved);
        default: return GS_ERR_INVALID_ARG;
    }
}

}  // namespace

extern "C" gs_status gs_render_fwd(const gs_projected *proj, int64_t n, const uint32_t *vals, const uint32_t *ranges,
                                   const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                                   const gs_raster_config *cfg, float *image, gs_fwd_saved saved,
                                   int32_t *dev_status, cudaStream_t stream) {
    (void)dev_status;
    if (!vals) return GS_ERR_INVALID_ARG;
    ListSrc ls{};
    ls.vals = vals;
    return render_fwd_impl(proj, n, ls, false, ranges, cams, n_views, total_tiles, cfg, image, saved, stream);
}

extern "C" gs_status gs_render_fwd_coarse(const gs_projected *proj, int64_t n, const gs_coarse_lists *lists,
                                          const uint32_t *ranges, const gs_camera *cams, int32_t n_views,
                                          int64_t total_tiles, const gs_raster_config *cfg, float *image,
                                          gs_fwd_saved saved, int32_t *dev_status, cudaStream_t stream) {
    (void)dev_status;
    ListSrc ls{};
    const gs_status st = coarse_src(lists, saved, ls);
    if (st != GS_OK) return st;
    return render_fwd_impl(proj, n, ls, true, ranges, cams, n_views, total_tiles, cfg, image, saved, stream);
}
