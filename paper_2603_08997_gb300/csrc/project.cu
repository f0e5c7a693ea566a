// gs_project: Eq. (cov), Eq. (proj), SH colour and the conservative tile
// rectangle, one thread per Gaussian over all views.  HBM-bound: ~236 B of
// parameters read once and 80 B written per (Gaussian, view) at SH degree 3.
#include "common.cuh"

using namespace gsr;

namespace {

// One (Gaussian, view): Eq. (cov), Eq. (proj), colour, support rectangle.
// mu, ls, q, logit: the Gaussian's parameters; f: its 3K SH coefficients.
template <int DEG>
__device__ __forceinline__ void project_one(const float (&mu)[3], const float (&ls)[3], float4 q, float logit,
                                            const float *f, const gs_camera &c, const gs_raster_config &cfg,
                                            int64_t e, float *__restrict__ rec, int4 *__restrict__ rect,
                                            int32_t *__restrict__ touched, uint32_t *__restrict__ depth_key,
                                            ushort4 *__restrict__ rect16) {
    float4 *out = reinterpret_cast<float4 *>(rec + e * kRecFloats);
    ProjState g;
    project_state(mu, ls, q, logit, c, cfg.lowpass, g);
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
#pragma unroll
    for (int idx = 0; idx < 3 * K; ++idx) col[idx % 3] += f[idx] * Y[idx / 3];
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

// One block of PB Gaussians: their parameter slices are staged once into
// shared memory with coalesced 16-byte loads, then each thread projects its
// Gaussian into every view (the parameters are read from DRAM once however
// many views there are).  On entry a block also asks L2 for the parameter
// slices of the block `ahead` / PB positions later (one resident wave of
// blocks ahead), so a block's staging loads find their lines in L2 instead
// of waiting on DRAM while the wave before it computes.
template <int DEG>
__global__ void __launch_bounds__(PB) project_kernel(gs_params prm, const gs_camera *__restrict__ cams, int n_views,
                                                     gs_raster_config cfg, float *__restrict__ rec,
                                                     int4 *__restrict__ rect, int32_t *__restrict__ touched,
                                                     uint32_t *__restrict__ depth_key,
                                                     ushort4 *__restrict__ rect16, int64_t ahead) {
    using G = ParamGroups<DEG>;
    extern __shared__ float s_par[];  // [TOT * PB]
    __shared__ gs_camera s_cams[kStagedViews];
    if (threadIdx.x < n_views && threadIdx.x < kStagedViews) s_cams[threadIdx.x] = cams[threadIdx.x];
    const int64_t n = prm.n;
    const int64_t i0 = (int64_t)blockIdx.x * PB;
    const int nb = (int)min((int64_t)PB, n - i0);
    const float *src[5] = {prm.means, prm.log_scales, prm.quats, prm.opacity_logit, prm.sh};
    {
        // slices of a full block start on 16-byte boundaries (groups 256-byte
        // aligned, i0 + ahead a multiple of PB)
        const int64_t j0 = i0 + ahead;
        if (threadIdx.x < 5 && ahead > 0 && j0 + PB <= n) {
            const int g = threadIdx.x;  // selects, not an indexed array (no local copy)
            const float *sp = g == 0 ? prm.means : g == 1 ? prm.log_scales : g == 2 ? prm.quats
                            : g == 3 ? prm.opacity_logit : prm.sh;
            const int sg = g < 2 ? 3 : g == 2 ? 4 : g == 3 ? 1 : 3 * G::K;
            prefetch_l2(sp + (int64_t)sg * j0, (uint32_t)(sizeof(float) * sg * PB));
        }
    }
    if (nb == PB)
        stage_block_full<DEG>(src, i0, s_par);
    else
        stage_partial<DEG>(src, i0, nb, s_par);
    __syncthreads();
    const int t = threadIdx.x;
    if (t >= nb) return;
    const float *P0 = s_par + G::off(0, PB) + G::P(0) * t;
    const float *P1 = s_par + G::off(1, PB) + G::P(1) * t;
    const float *P2 = s_par + G::off(2, PB) + G::P(2) * t;
    const float logit = s_par[G::off(3, PB) + G::P(3) * t];
    const float *f = s_par + G::off(4, PB) + G::P(4) * t;
    const float mu[3] = {P0[0], P0[1], P0[2]};
    const float ls[3] = {P1[0], P1[1], P1[2]};
    const float4 q = make_float4(P2[0], P2[1], P2[2], P2[3]);
    for (int v = 0; v < n_views; ++v) {
        const gs_camera &c = v < kStagedViews ? s_cams[v] : cams[v];
        project_one<DEG>(mu, ls, q, logit, f, c, cfg, (int64_t)v * n + i0 + t, rec, rect, touched, depth_key,
                         rect16);
    }
}

template <int DEG>
gs_status launch_project(const gs_params &prm, const gs_camera *cams, int n_views, const gs_raster_config &cfg,
                         float *rec, int4 *rect, int32_t *touched, uint32_t *depth_key, ushort4 *rect16,
                         cudaStream_t stream) {
    constexpr size_t smem = sizeof(float) * ParamGroups<DEG>::TOT * PB;
    // per device: the shared-memory limit is raised once, and the prefetch
    // distance is one resident wave of blocks, in Gaussians
    static bool attr_set[kMaxDevices] = {};
    static int64_t ahead_of[kMaxDevices] = {};
    const int dev = cached_device_index();
    if (dev < 0) return GS_ERR_UNSUPPORTED;
    if (!attr_set[dev] && smem > 48 * 1024) {
        GS_TRY(cudaFuncSetAttribute(project_kernel<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set[dev] = true;
    }
    int64_t ahead = ahead_of[dev];
    if (ahead <= 0) {
        int per_sm = 0;
        GS_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, project_kernel<DEG>, PB, smem));
        ahead = (int64_t)per_sm * device_sm_count() * PB;
        ahead_of[dev] = ahead;
    }
    project_kernel<DEG><<<(unsigned)ceil_div(prm.n, (int64_t)PB), PB, smem, stream>>>(prm, cams, n_views, cfg, rec, rect,
                                                                                     touched, depth_key, rect16, ahead);
    GS_TRY_LAUNCH();
    return GS_OK;
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
    if (((uintptr_t)params->means | (uintptr_t)params->log_scales | (uintptr_t)params->opacity_logit |
         (uintptr_t)params->sh) & 15)
        return GS_ERR_INVALID_ARG;  // staged with 16-byte loads (gs_param_layout aligns every group)
    int4 *rect = reinterpret_cast<int4 *>(out.rect);
    if ((uintptr_t)out.rect16 & 7) return GS_ERR_INVALID_ARG;
    ushort4 *r16 = reinterpret_cast<ushort4 *>(out.rect16);
    switch (params->sh_degree) {
        case 0: return launch_project<0>(*params, cams, n_views, *cfg, out.rec, rect, out.tiles_touched, out.depth_key, r16, stream);
        case 1: return launch_project<1>(*params, cams, n_views, *cfg, out.rec, rect, out.tiles_touched, out.depth_key, r16, stream);
        case 2: return launch_project<2>(*params, cams, n_views, *cfg, out.rec, rect, out.tiles_touched, out.depth_key, r16, stream);
        default: return launch_project<3>(*params, cams, n_views, *cfg, out.rec, rect, out.tiles_touched, out.depth_key, r16, stream);
    }
}

}  // extern "C"
