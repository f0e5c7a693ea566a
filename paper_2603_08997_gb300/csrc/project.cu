// gs_project: Eq. (cov), Eq. (proj), SH colour and the conservative tile
// rectangle, one thread per (Gaussian, view).  HBM-bound: ~236 B of parameters
// read and 68 B written per Gaussian at SH degree 3.
#include "common.cuh"

using namespace gsr;

namespace {

template <int DEG>
__global__ void __launch_bounds__(256) project_kernel(gs_params prm, const gs_camera *__restrict__ cams,
                                                      gs_raster_config cfg, float *__restrict__ rec,
                                                      int4 *__restrict__ rect, int32_t *__restrict__ touched,
                                                      uint32_t *__restrict__ depth_key,
                                                      ushort4 *__restrict__ rect16) {
    __shared__ gs_camera s_cam;
    const int v = blockIdx.y;
    if (threadIdx.x == 0) s_cam = cams[v];
    __syncthreads();
    const int64_t n = prm.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const gs_camera &c = s_cam;
    const int64_t e = (int64_t)v * n + i;
    float4 *out = reinterpret_cast<float4 *>(rec + e * kRecFloats);

    const float mu[3] = {prm.means[3 * i], prm.means[3 * i + 1], prm.means[3 * i + 2]};
    const float ls[3] = {prm.log_scales[3 * i], prm.log_scales[3 * i + 1], prm.log_scales[3 * i + 2]};
    const float4 q = reinterpret_cast<const float4 *>(prm.quats)[i];
    ProjState g;
    project_state(mu, ls, q, prm.opacity_logit[i], c, cfg.lowpass, g);
    bool culled = g.culled || !(g.o >= cfg.alpha_min);
    float rx = 0.f, ry = 0.f;
    int x0 = 0, y0 = 0, x1 = -1, y1 = -1;
    if (!culled) {
        // Support of alpha' >= alpha_min: the ellipse dp^T Q dp <= 2 ln(o / alpha_min).
        // Its axis-aligned extents are sqrt(2 ln(o/alpha_min) Sigma2D_xx) and
        // sqrt(2 ln(o/alpha_min) Sigma2D_yy); inflated for float32 rounding.
        const float c2 = 2.f * logf(g.o / cfg.alpha_min);
        rx = sqrtf(c2 * g.s00) * 1.0001f + 1e-3f;
        ry = sqrtf(c2 * g.s11) * 1.0001f + 1e-3f;
        const float fx0 = fmaxf(ceilf(g.mean2d[0] - rx - 0.5f), 0.f);
        const float fx1 = fminf(floorf(g.mean2d[0] + rx - 0.5f), (float)(c.width - 1));
        const float fy0 = fmaxf(ceilf(g.mean2d[1] - ry - 0.5f), 0.f);
        const float fy1 = fminf(floorf(g.mean2d[1] + ry - 0.5f), (float)(c.height - 1));
        if (!(fx0 <= fx1) || !(fy0 <= fy1)) {
            culled = true;
        } else {
            x0 = (int)fx0 / cfg.tile; x1 = (int)fx1 / cfg.tile;
            y0 = (int)fy0 / cfg.tile; y1 = (int)fy1 / cfg.tile;
        }
    }
    if (culled) {
        out[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        out[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        out[2] = make_float4(0.f, __int_as_float(0x7f800000), 0.f, 0.f);
        rect[e] = make_int4(0, 0, -1, -1);
        touched[e] = 0;
        if (depth_key) depth_key[e] = 0xffffffffu;  // culled entries sort last
        if (rect16) rect16[e] = make_ushort4(0, 0, 0, 0);
        return;
    }
    // conic factor U with Q = U^T U (upper Cholesky of Sigma2D^-1)
    const float u11 = 1.0f / sqrtf(g.s11);
    const float u00 = sqrtf(g.s11 / g.det);
    const float u01 = -g.s01 / sqrtf(g.s11 * g.det);
    // colour from SH for the direction camera centre -> mean
    float cp[3];
    cam_center(c, cp);
    float d[3] = {mu[0] - cp[0], mu[1] - cp[1], mu[2] - cp[2]};
    const float dn = 1.0f / sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    d[0] *= dn; d[1] *= dn; d[2] *= dn;
    constexpr int K = (DEG + 1) * (DEG + 1);
    float Y[16];
    sh_basis(DEG, d[0], d[1], d[2], Y);
    float col[3] = {0.5f, 0.5f, 0.5f};
    const float *f = prm.sh + (int64_t)i * (3 * K);
    if constexpr ((3 * K) % 4 == 0) {
        const float4 *f4 = reinterpret_cast<const float4 *>(f);
#pragma unroll
        for (int j = 0; j < (3 * K) / 4; ++j) {
            const float4 t = f4[j];
            const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = 4 * j + u;
                col[idx % 3] += tv[u] * Y[idx / 3];
            }
        }
    } else {
#pragma unroll
        for (int idx = 0; idx < 3 * K; ++idx) col[idx % 3] += f[idx] * Y[idx / 3];
    }
    out[0] = make_float4(g.mean2d[0], g.mean2d[1], u00, u01);
    out[1] = make_float4(u11, g.o, fmaxf(col[0], 0.f), fmaxf(col[1], 0.f));
    out[2] = make_float4(fmaxf(col[2], 0.f), g.p[2], rx, ry);
    rect[e] = make_int4(x0, y0, x1, y1);
    touched[e] = (x1 - x0 + 1) * (y1 - y0 + 1);
    if (depth_key) depth_key[e] = __float_as_uint(g.p[2]);  // positive depth: bit order = value order
    if (rect16)
        rect16[e] = make_ushort4((unsigned short)x0, (unsigned short)y0, (unsigned short)(x1 - x0 + 1),
                                 (unsigned short)(y1 - y0 + 1));
}

}  // namespace

extern "C" {

const char *gs_status_string(int status) {
    switch (status) {
        case GS_OK: return "GS_OK";
        case GS_ERR_INVALID_ARG: return "GS_ERR_INVALID_ARG";
        case GS_ERR_WORKSPACE: return "GS_ERR_WORKSPACE";
        case GS_ERR_CUDA: return "GS_ERR_CUDA";
        case GS_ERR_CAPACITY: return "GS_ERR_CAPACITY";
        case GS_ERR_NONFINITE: return "GS_ERR_NONFINITE";
        case GS_ERR_UNSUPPORTED: return "GS_ERR_UNSUPPORTED";
        default: return "GS_ERR_UNKNOWN";
    }
}

int gs_version(void) { return 100; }

gs_status gs_param_layout(int64_t n, int32_t sh_degree, int64_t *out6) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3 || !out6) return GS_ERR_INVALID_ARG;
    param_offsets(n, sh_degree, out6);
    return GS_OK;
}

gs_status gs_camera_layout(gs_camera *cams, int32_t n_views, int32_t tile, int64_t *total_tiles,
                           int64_t *total_pixels) {
    if (!cams || n_views <= 0 || (tile != 8 && tile != 16 && tile != 32)) return GS_ERR_INVALID_ARG;
    int64_t t = 0, p = 0;
    for (int v = 0; v < n_views; ++v) {
        if (cams[v].width <= 0 || cams[v].height <= 0) return GS_ERR_INVALID_ARG;
        cams[v].tile_offset = (int32_t)t;
        cams[v].pix_offset = p;
        t += ceil_div(cams[v].width, tile) * ceil_div(cams[v].height, tile);
        p += (int64_t)cams[v].width * cams[v].height;
    }
    if (t >= (int64_t)1 << 31) return GS_ERR_INVALID_ARG;
    if (total_tiles) *total_tiles = t;
    if (total_pixels) *total_pixels = p;
    return GS_OK;
}

int64_t gs_ckpt_slots(int64_t pair_capacity, int64_t total_tiles, int32_t batch) {
    if (pair_capacity < 0 || total_tiles < 0 || batch <= 0) return -1;
    // slot of (tile t, batch b) = floor(start_t / batch) + t + b, see render_fwd.cu
    return pair_capacity / batch + total_tiles + 1;
}

gs_status gs_project(const gs_params *params, const gs_camera *cams, int32_t n_views, const gs_raster_config *cfg,
                     gs_projected out, int32_t *dev_status, cudaStream_t stream) {
    (void)dev_status;
    if (!params || !cfg || !cams || n_views <= 0 || n_views > 65535) return GS_ERR_INVALID_ARG;
    if (params->n < 0 || params->n >= ((int64_t)1 << 31)) return GS_ERR_INVALID_ARG;
    if (params->sh_degree < 0 || params->sh_degree > 3 || cfg->sh_degree != params->sh_degree) return GS_ERR_INVALID_ARG;
    if (cfg->tile != 8 && cfg->tile != 16 && cfg->tile != 32) return GS_ERR_INVALID_ARG;
    if (params->n == 0) return GS_OK;
    if (!params->means || !params->log_scales || !params->quats || !params->opacity_logit || !params->sh)
        return GS_ERR_INVALID_ARG;
    if (!out.rec || !out.rect || !out.tiles_touched) return GS_ERR_INVALID_ARG;
    if (((uintptr_t)params->quats & 15) || ((uintptr_t)out.rec & 15) || ((uintptr_t)out.rect & 15))
        return GS_ERR_INVALID_ARG;
    const int K3 = 3 * (params->sh_degree + 1) * (params->sh_degree + 1);
    if ((K3 % 4 == 0) && ((uintptr_t)params->sh & 15)) return GS_ERR_INVALID_ARG;
    dim3 grid((unsigned)ceil_div(params->n, 256), (unsigned)n_views);
    int4 *rect = reinterpret_cast<int4 *>(out.rect);
    if ((uintptr_t)out.rect16 & 7) return GS_ERR_INVALID_ARG;
    ushort4 *r16 = reinterpret_cast<ushort4 *>(out.rect16);
    switch (params->sh_degree) {
        case 0: project_kernel<0><<<grid, 256, 0, stream>>>(*params, cams, *cfg, out.rec, rect, out.tiles_touched, out.depth_key, r16); break;
        case 1: project_kernel<1><<<grid, 256, 0, stream>>>(*params, cams, *cfg, out.rec, rect, out.tiles_touched, out.depth_key, r16); break;
        case 2: project_kernel<2><<<grid, 256, 0, stream>>>(*params, cams, *cfg, out.rec, rect, out.tiles_touched, out.depth_key, r16); break;
        default: project_kernel<3><<<grid, 256, 0, stream>>>(*params, cams, *cfg, out.rec, rect, out.tiles_touched, out.depth_key, r16); break;
    }
    GS_TRY_LAUNCH();
    return GS_OK;
}

}  // extern "C"
