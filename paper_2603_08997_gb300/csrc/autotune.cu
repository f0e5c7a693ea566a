// gs_autotune: launch-shape search for the rasterizer (host code only).
//
// The tile side, the staging batch and the pixels per thread of the
// compositing kernels change how the work maps to the GPU, not what it
// computes (the contribution set does not depend on the tile size, and every
// shape gives the same images and gradients up to the order of float
// atomics), so the choice is made on time alone: each candidate runs
// project -> bin/sort -> tile order -> render -> loss (+ gradient) -> raster
// and projection adjoint on the caller's workload, `reps` timed iterations
// after one untimed one, with CUDA events on the caller's stream.  Every
// buffer is carved from the caller's workspace, sized for the largest
// candidate by gs_autotune_workspace_size.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

using namespace gsr;

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Bufs {
    gs_camera *cams;
    float *rec;
    int32_t *rect, *touched;
    uint32_t *depth_key;
    uint16_t *rect16;
    void *bin_ws;
    size_t bin_ws_bytes;
    uint32_t *vals, *ranges, *tile_order;
    int64_t *pair_count;
    int32_t *status;
    float *image, *T_final;
    int32_t *n_last;
    float *ckpt;
    int64_t ckpt_slots;
    void *loss_ws;
    size_t loss_ws_bytes;
    float *loss, *dL;
    void *g2d;
    size_t g2d_bytes;
    float *grads;
};

// Lays out one candidate's buffers from `base` (nullptr: sizes only) and
// returns the bytes.  cams: host copies with the candidate's tile layout.
size_t layout(int64_t n, int sh_degree, const std::vector<gs_camera> &cams, int tile, int batch,
              int64_t pair_capacity, int64_t T, int64_t P, char *base, Bufs *b) {
    const int64_t V = (int64_t)cams.size(), E = V * n;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += al256(bytes > 0 ? bytes : 1);
        return p;
    };
    Bufs x;
    x.cams = (gs_camera *)take(sizeof(gs_camera) * V);
    x.rec = (float *)take(sizeof(float) * kRecFloats * E);
    x.rect = (int32_t *)take(sizeof(int32_t) * 4 * E);
    x.touched = (int32_t *)take(sizeof(int32_t) * E);
    x.depth_key = (uint32_t *)take(sizeof(uint32_t) * E);
    x.rect16 = (uint16_t *)take(sizeof(uint16_t) * 4 * E);
    x.bin_ws_bytes = gs_bin_sort_workspace_size(n, (int32_t)V, pair_capacity, T);
    x.bin_ws = take(x.bin_ws_bytes);
    x.vals = (uint32_t *)take(sizeof(uint32_t) * pair_capacity);
    x.ranges = (uint32_t *)take(sizeof(uint32_t) * 2 * T);
    x.tile_order = (uint32_t *)take(sizeof(uint32_t) * T);
    x.pair_count = (int64_t *)take(sizeof(int64_t));
    x.status = (int32_t *)take(sizeof(int32_t));
    x.image = (float *)take(sizeof(float) * 3 * P);
    x.T_final = (float *)take(sizeof(float) * P);
    x.n_last = (int32_t *)take(sizeof(int32_t) * P);
    x.ckpt_slots = gs_ckpt_slots(pair_capacity, T, batch);
    x.ckpt = (float *)take(sizeof(float) * (size_t)x.ckpt_slots * tile * tile);
    x.loss_ws_bytes = gs_loss_workspace_size(cams.data(), (int32_t)V);
    x.loss_ws = take(x.loss_ws_bytes);
    x.loss = (float *)take(sizeof(float) * V);
    x.dL = (float *)take(sizeof(float) * 3 * P);
    x.g2d_bytes = gs_render_bwd_workspace_size(n, (int32_t)V);
    x.g2d = take(x.g2d_bytes);
    int64_t o[6];
    param_offsets(n, sh_degree, o);
    x.grads = (float *)take(sizeof(float) * o[5]);
    if (b) *b = x;
    return off;
}

bool valid_shape(const gs_launch_shape &s) {
    const bool tile_ok = s.tile == 8 || s.tile == 16 || s.tile == 32;
    const bool batch_ok = s.batch == 64 || s.batch == 128 || s.batch == 256;
    auto ppt_ok = [&](int p) { return p == 1 || p == 2 || (p == 4 && s.tile >= 16); };
    return tile_ok && batch_ok && ppt_ok(s.pixels_per_thread_fwd) && ppt_ok(s.pixels_per_thread_bwd);
}

// The candidate's host cameras (tile layout filled) and its tile and pixel totals.
gs_status cams_for(const gs_camera *cams_host, int32_t n_views, int tile, std::vector<gs_camera> &out, int64_t &T,
                   int64_t &P) {
    out.assign(cams_host, cams_host + n_views);
    return gs_camera_layout(out.data(), n_views, tile, &T, &P);
}

}  // namespace

extern "C" size_t gs_autotune_workspace_size(int64_t n, int32_t sh_degree, const gs_camera *cams_host,
                                             int32_t n_views, int64_t pair_capacity, const gs_launch_shape *cands,
                                             int32_t n_cands) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3 || !cams_host || n_views <= 0 || pair_capacity < 0 || !cands ||
        n_cands <= 0)
        return 0;
    size_t most = 0;
    for (int c = 0; c < n_cands; ++c) {
        if (!valid_shape(cands[c])) continue;
        std::vector<gs_camera> cams;
        int64_t T = 0, P = 0;
        if (cams_for(cams_host, n_views, cands[c].tile, cams, T, P) != GS_OK) return 0;
        const size_t b = layout(n, sh_degree, cams, cands[c].tile, cands[c].batch, pair_capacity, T, P, nullptr, nullptr);
        if (b > most) most = b;
    }
    return most;
}

extern "C" gs_status gs_autotune(const gs_params *params, const gs_camera *cams_host, int32_t n_views,
                                 const float *target, const gs_raster_config *base, float lambda_ssim,
                                 const gs_launch_shape *cands, int32_t n_cands, int32_t reps,
                                 int64_t pair_capacity, void *workspace, size_t workspace_bytes,
                                 float *ms_per_iter, int32_t *best, cudaStream_t stream) {
    if (!params || !cams_host || n_views <= 0 || !target || !base || !cands || n_cands <= 0 || reps <= 0 ||
        pair_capacity <= 0 || !ms_per_iter || !best)
        return GS_ERR_INVALID_ARG;
    if (params->sh_degree != base->sh_degree) return GS_ERR_INVALID_ARG;
    const int64_t n = params->n;
    if (!workspace || ((uintptr_t)workspace & 255) ||
        workspace_bytes < gs_autotune_workspace_size(n, params->sh_degree, cams_host, n_views, pair_capacity, cands,
                                                     n_cands))
        return GS_ERR_WORKSPACE;
    cudaEvent_t e0, e1;
    GS_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GS_ERR_CUDA;
    }
    gs_status result = GS_OK;
    *best = -1;
    for (int c = 0; c < n_cands && result == GS_OK; ++c) {
        ms_per_iter[c] = INFINITY;
        const gs_launch_shape &s = cands[c];
        if (!valid_shape(s)) continue;
        std::vector<gs_camera> cams;
        int64_t T = 0, P = 0;
        if (cams_for(cams_host, n_views, s.tile, cams, T, P) != GS_OK) continue;
        Bufs b;
        layout(n, params->sh_degree, cams, s.tile, s.batch, pair_capacity, T, P, (char *)workspace, &b);
        gs_raster_config fwd = *base, bwd = *base;
        fwd.tile = bwd.tile = s.tile;
        fwd.batch = bwd.batch = s.batch;
        fwd.pixels_per_thread = s.pixels_per_thread_fwd;
        bwd.pixels_per_thread = s.pixels_per_thread_bwd;
        int64_t mvt = 0;
        for (const gs_camera &cm : cams)
            mvt = std::max(mvt, ceil_div(cm.width, s.tile) * ceil_div(cm.height, s.tile));
        if (cudaMemcpyAsync(b.cams, cams.data(), sizeof(gs_camera) * n_views, cudaMemcpyHostToDevice, stream) !=
                cudaSuccess ||
            cudaMemsetAsync(b.status, 0, sizeof(int32_t), stream) != cudaSuccess) {
            result = GS_ERR_CUDA;
            break;
        }
        gs_projected proj{};
        proj.rec = b.rec;
        proj.rect = b.rect;
        proj.tiles_touched = b.touched;
        proj.depth_key = b.depth_key;
        proj.rect16 = b.rect16;
        gs_fwd_saved saved{};
        saved.T_final = b.T_final;
        saved.n_last = b.n_last;
        saved.ckpt = b.ckpt;
        saved.ckpt_slots = b.ckpt_slots;
        saved.tile_order = b.tile_order;
        int64_t o[6];
        param_offsets(n, params->sh_degree, o);
        gs_grads gr{};
        gr.means = b.grads + o[0];
        gr.log_scales = b.grads + o[1];
        gr.quats = b.grads + o[2];
        gr.opacity_logit = b.grads + o[3];
        gr.sh = b.grads + o[4];
        auto iteration = [&]() -> gs_status {
            gs_status st = gs_project(params, b.cams, n_views, &fwd, proj, b.status, stream);
            if (st == GS_OK)
                st = gs_bin_sort(&proj, b.cams, n_views, n, T, (int32_t)mvt, &fwd, b.bin_ws, b.bin_ws_bytes, nullptr,
                                 b.vals, pair_capacity, b.ranges, b.pair_count, b.status, stream);
            if (st == GS_OK) st = gs_tile_order(b.ranges, T, b.tile_order, stream);
            if (st == GS_OK)
                st = gs_render_fwd(&proj, n, b.vals, b.ranges, b.cams, n_views, T, &fwd, b.image, saved, b.status,
                                   stream);
            if (st == GS_OK)
                st = gs_loss(b.image, target, nullptr, cams.data(), nullptr, nullptr, n_views, lambda_ssim, b.loss_ws,
                             b.loss_ws_bytes, b.loss, b.dL, stream);
            if (st == GS_OK)
                st = gs_render_bwd(params, &proj, b.vals, b.ranges, b.cams, n_views, T, &bwd, saved, b.dL, nullptr,
                                   gr, 0, b.g2d, b.g2d_bytes, b.status, stream);
            return st;
        };
        gs_status st = iteration();  // untimed: warms caches and shows whether the shape runs
        int32_t dev_status = 0;
        if (st == GS_OK && (cudaMemcpyAsync(&dev_status, b.status, sizeof(int32_t), cudaMemcpyDeviceToHost, stream) !=
                                cudaSuccess ||
                            cudaStreamSynchronize(stream) != cudaSuccess))
            st = GS_ERR_CUDA;
        if (st == GS_ERR_CUDA) {
            result = st;
            break;
        }
        if (st != GS_OK || dev_status != 0) continue;  // this workload cannot use the shape (e.g. capacity)
        if (cudaEventRecord(e0, stream) != cudaSuccess) {
            result = GS_ERR_CUDA;
            break;
        }
        for (int r = 0; r < reps && st == GS_OK; ++r) st = iteration();
        float ms = 0.f;
        if (st != GS_OK || cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            result = st != GS_OK ? st : GS_ERR_CUDA;
            break;
        }
        ms_per_iter[c] = ms / (float)reps;
        if (*best < 0 || ms_per_iter[c] < ms_per_iter[*best]) *best = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result == GS_OK && *best < 0) result = GS_ERR_UNSUPPORTED;  // no candidate runs this workload
    return result;
}
