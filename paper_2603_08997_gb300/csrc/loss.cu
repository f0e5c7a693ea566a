// gs_loss / gs_loss_backward: Eq. (loss), L = (1 - lambda) L1 + lambda (1 - SSIM).
//
// SSIM uses an 11x11 Gaussian window (sigma 1.5, separable), zero padding,
// C1 = 0.01^2, C2 = 0.03^2.  One CTA computes a 32x16 output tile: it stages
// the tile plus a 5-pixel halo of image and target in shared memory, filters
// rows (a thread computes 4 adjacent outputs of a row, so each staged value
// is loaded once per thread) then columns (2 adjacent rows per thread), and
// evaluates the SSIM map.  Window sums are taken of
// values shifted by the tile's centre value (exact for a window whose weights
// sum to 1, padded pixels included), which keeps the variance terms
// E[x^2] - E[x]^2 well conditioned in float32.
//
// The forward kernel also stores, per pixel and channel, the three partial
// derivatives of the SSIM map that the gradient needs:
//   P1 = dm/dmu_x - 2 mu_x dm/dsxx - mu_y dm/dsxy,  P2 = dm/dsxx,  P3 = dm/dsxy,
// so that d mean(m)/dx = (F(P1) + 2 x F(P2) + y F(P3)) / n with F the same
// window filter.  The gradient kernel only runs when a backward pass does
// (in the refinement step it sits inside the gate's conditional branch).
// Per-view sums are reduced in a fixed order, so the loss is deterministic.
#include "common.cuh"

using namespace gsr;

namespace {

constexpr int LTW = 32, LTH = 16, HALO = 5, LW = LTW + 2 * HALO, LH = LTH + 2 * HALO;
static_assert(LTW == 32 && LTH == 16 && LH * (LTW / 4) <= 256,
              "a 32 x 8 block: 4-column row strips and 2-row column strips cover the tile");
constexpr float SSIM_C1 = 0.0001f;  // (0.01)^2
constexpr float SSIM_C2 = 0.0009f;  // (0.03)^2

// Normalised 1D Gaussian window, sigma 1.5: w[t] = exp(-(t-5)^2 / 4.5) / sum,
// passed by value (kernel parameters), so no upload precedes a graph capture.
struct Win {
    float w[11];
};

Win window_host() {
    Win r;
    double s = 0.0, g[11];
    for (int t = 0; t < 11; ++t) {
        const double d = t - 5.0;
        g[t] = exp(-d * d / 4.5);
        s += g[t];
    }
    for (int t = 0; t < 11; ++t) r.w[t] = (float)(g[t] / s);
    return r;
}

__device__ __forceinline__ const float *target_base(const float *target, const int64_t *target_offsets,
                                                    const int32_t *view_ids, int v, int64_t pix_offset) {
    if (target_offsets && view_ids) return target + target_offsets[view_ids[v]];
    return target + 3 * pix_offset;
}

// The view's size: from the device camera when given (a slot whose camera is
// chosen on the device, at most the launch's capacity), else the launch's.
__device__ __forceinline__ void view_size(const gs_camera *cam_dev, int &W, int &H) {
    if (cam_dev) {
        W = min(W, cam_dev->width);
        H = min(H, cam_dev->height);
    }
}

__global__ void __launch_bounds__(256) ssim_fwd_kernel(const float *__restrict__ img, const float *__restrict__ target,
                                                       const int64_t *__restrict__ target_offsets,
                                                       const int32_t *__restrict__ view_ids, int v,
                                                       int64_t pix_offset, int W, int H,
                                                       const gs_camera *__restrict__ cam_dev, Win win,
                                                       float *__restrict__ dmaps, double2 *__restrict__ partials) {
    __shared__ float sx[LH][LW];
    __shared__ float sy[LH][LW];
    __shared__ __align__(16) float hs[5][LH][LTW];
    __shared__ double red[2][8];
    view_size(cam_dev, W, H);
    const float *tgt = target_base(target, target_offsets, view_ids, v, pix_offset);
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int bx0 = blockIdx.x * LTW, by0 = blockIdx.y * LTH;
    if (bx0 >= W || by0 >= H) {  // past the device camera's size
        if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = make_double2(0.0, 0.0);
        return;
    }
    const int64_t hw = (int64_t)W * H;
    const int ccx = min(bx0 + LTW / 2, W - 1), ccy = min(by0 + LTH / 2, H - 1);
    float ssim_acc = 0.f, l1_acc = 0.f;
    for (int ch = 0; ch < 3; ++ch) {
        const float *X = img + ch * hw, *Yp = tgt + ch * hw;
        const float shx = X[(int64_t)ccy * W + ccx], shy = Yp[(int64_t)ccy * W + ccx];
        for (int r = threadIdx.y; r < LH; r += 8) {
            for (int c = threadIdx.x; c < LW; c += 32) {
                const int gx = bx0 + c - HALO, gy = by0 + r - HALO;
                const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
                const int64_t p = (int64_t)gy * W + gx;
                sx[r][c] = (in ? X[p] : 0.f) - shx;
                sy[r][c] = (in ? Yp[p] : 0.f) - shy;
            }
        }
        __syncthreads();
        // rows: a thread filters 4 adjacent outputs of one row from 14 inputs
        // (each input and its products loaded and formed once)
        if (tid < LH * (LTW / 4)) {
            const int r = tid / (LTW / 4), c0 = 4 * (tid % (LTW / 4));
            float acc[4][5];
#pragma unroll
            for (int o = 0; o < 4; ++o)
#pragma unroll
                for (int q = 0; q < 5; ++q) acc[o][q] = 0.f;
#pragma unroll
            for (int j = 0; j < 14; ++j) {
                const float xv = sx[r][c0 + j], yv = sy[r][c0 + j];
                const float in5[5] = {xv, yv, xv * xv, yv * yv, xv * yv};
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int t = j - o;
                    if (t >= 0 && t < 11) {
#pragma unroll
                        for (int q = 0; q < 5; ++q) acc[o][q] += win.w[t] * in5[q];
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 5; ++q)
                *reinterpret_cast<float4 *>(&hs[q][r][c0]) = make_float4(acc[0][q], acc[1][q], acc[2][q], acc[3][q]);
        }
        __syncthreads();
        // columns: a thread filters 2 adjacent output rows of one column
        {
            const int c = threadIdx.x, r0 = 2 * threadIdx.y;
            float mm[2][5];
#pragma unroll
            for (int o = 0; o < 2; ++o)
#pragma unroll
                for (int q = 0; q < 5; ++q) mm[o][q] = 0.f;
#pragma unroll
            for (int j = 0; j < 12; ++j) {
                float h[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) h[q] = hs[q][r0 + j][c];
#pragma unroll
                for (int o = 0; o < 2; ++o) {
                    const int t = j - o;
                    if (t >= 0 && t < 11) {
#pragma unroll
                        for (int q = 0; q < 5; ++q) mm[o][q] += win.w[t] * h[q];
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const int gx = bx0 + c, gy = by0 + r0 + o;
                if (gx < W && gy < H) {
                    const float m0 = mm[o][0], m1 = mm[o][1], e2 = mm[o][2], f2 = mm[o][3], exy = mm[o][4];
                    const float sxx = e2 - m0 * m0, syy = f2 - m1 * m1, sxy = exy - m0 * m1;
                    const float mx = m0 + shx, my = m1 + shy;
                    const float A1 = 2.f * mx * my + SSIM_C1, A2 = 2.f * sxy + SSIM_C2;
                    const float B1 = mx * mx + my * my + SSIM_C1, B2 = sxx + syy + SSIM_C2;
                    const float iD = 1.f / (B1 * B2);
                    const float m = A1 * A2 * iD;
                    const float P2 = -m / B2;
                    const float P3 = 2.f * A1 * iD;
                    const float dmu = (2.f * my * A2 - 2.f * mx * m * B2) * iD;
                    const float P1 = dmu - 2.f * mx * P2 - my * P3;
                    const int64_t p = (int64_t)gy * W + gx;
                    dmaps[(0 * 3 + ch) * hw + p] = P1;
                    dmaps[(1 * 3 + ch) * hw + p] = P2;
                    dmaps[(2 * 3 + ch) * hw + p] = P3;
                    ssim_acc += m;
                    l1_acc += fabsf(X[p] - Yp[p]);
                }
            }
        }
        __syncthreads();
    }
    double s0 = ssim_acc, s1 = l1_acc;
    for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    }
    if (threadIdx.x == 0) { red[0][threadIdx.y] = s0; red[1][threadIdx.y] = s1; }
    __syncthreads();
    if (tid == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int w = 0; w < 8; ++w) { t0 += red[0][w]; t1 += red[1][w]; }
        partials[blockIdx.y * gridDim.x + blockIdx.x] = make_double2(t0, t1);
    }
}

// Per view: fixed-order sum of the block partials -> loss (n = 3 W H, from
// the device camera when given).
__global__ void loss_reduce_kernel(const double2 *__restrict__ partials, int nblocks, double n,
                                   const gs_camera *__restrict__ cam_dev, float lambda, float *__restrict__ loss_out) {
    if (cam_dev) n = 3.0 * (double)cam_dev->width * (double)cam_dev->height;
    __shared__ double s0[256], s1[256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += 256) {
        const double2 p = partials[i];
        a += p.x;
        b += p.y;
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            s0[threadIdx.x] += s0[threadIdx.x + off];
            s1[threadIdx.x] += s1[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double ssim = s0[0] / n, l1 = s1[0] / n;
        *loss_out = (float)((1.0 - lambda) * l1 + lambda * (1.0 - ssim));
    }
}

__global__ void __launch_bounds__(256) ssim_bwd_kernel(const float *__restrict__ img, const float *__restrict__ target,
                                                       const int64_t *__restrict__ target_offsets,
                                                       const int32_t *__restrict__ view_ids, int v,
                                                       int64_t pix_offset, int W, int H,
                                                       const gs_camera *__restrict__ cam_dev, float lambda, Win win,
                                                       const float *__restrict__ dmaps, float *__restrict__ grad) {
    __shared__ float sp[3][LH][LW];
    __shared__ __align__(16) float hs[3][LH][LTW];
    view_size(cam_dev, W, H);
    const float *tgt = target_base(target, target_offsets, view_ids, v, pix_offset);
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int bx0 = blockIdx.x * LTW, by0 = blockIdx.y * LTH;
    if (bx0 >= W || by0 >= H) return;
    const int64_t hw = (int64_t)W * H;
    const float inv_n = 1.f / (3.f * (float)hw);
    for (int ch = 0; ch < 3; ++ch) {
        for (int r = threadIdx.y; r < LH; r += 8) {
            for (int c = threadIdx.x; c < LW; c += 32) {
                const int gx = bx0 + c - HALO, gy = by0 + r - HALO;
                const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
                const int64_t p = (int64_t)gy * W + gx;
#pragma unroll
                for (int q = 0; q < 3; ++q) sp[q][r][c] = in ? dmaps[(q * 3 + ch) * hw + p] : 0.f;
            }
        }
        __syncthreads();
        // rows: 4 adjacent outputs of one row per thread
        if (tid < LH * (LTW / 4)) {
            const int r = tid / (LTW / 4), c0 = 4 * (tid % (LTW / 4));
            float acc[4][3];
#pragma unroll
            for (int o = 0; o < 4; ++o)
#pragma unroll
                for (int q = 0; q < 3; ++q) acc[o][q] = 0.f;
#pragma unroll
            for (int j = 0; j < 14; ++j) {
                const float in3[3] = {sp[0][r][c0 + j], sp[1][r][c0 + j], sp[2][r][c0 + j]};
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int t = j - o;
                    if (t >= 0 && t < 11) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) acc[o][q] += win.w[t] * in3[q];
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 3; ++q)
                *reinterpret_cast<float4 *>(&hs[q][r][c0]) = make_float4(acc[0][q], acc[1][q], acc[2][q], acc[3][q]);
        }
        __syncthreads();
        // columns: 2 adjacent output rows of one column per thread
        {
            const int c = threadIdx.x, r0 = 2 * threadIdx.y;
            float ff[2][3];
#pragma unroll
            for (int o = 0; o < 2; ++o)
#pragma unroll
                for (int q = 0; q < 3; ++q) ff[o][q] = 0.f;
#pragma unroll
            for (int j = 0; j < 12; ++j) {
                const float h[3] = {hs[0][r0 + j][c], hs[1][r0 + j][c], hs[2][r0 + j][c]};
#pragma unroll
                for (int o = 0; o < 2; ++o) {
                    const int t = j - o;
                    if (t >= 0 && t < 11) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) ff[o][q] += win.w[t] * h[q];
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const int gx = bx0 + c, gy = by0 + r0 + o;
                if (gx < W && gy < H) {
                    const int64_t p = (int64_t)gy * W + gx;
                    const float xv = img[ch * hw + p], yv = tgt[ch * hw + p];
                    const float dssim = (ff[o][0] + 2.f * xv * ff[o][1] + yv * ff[o][2]) * inv_n;
                    const float diff = xv - yv;
                    const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
                    grad[ch * hw + p] = (1.f - lambda) * sgn * inv_n - lambda * dssim;
                }
            }
        }
        __syncthreads();
    }
}

struct LossLayout {
    size_t dmaps_off, partials_off, total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool loss_layout(const gs_camera *cams, int n_views, LossLayout &L, int64_t *block_off /* n_views+1, nullable */) {
    int64_t pixels = 0, blocks = 0;
    for (int v = 0; v < n_views; ++v) {
        if (cams[v].width <= 0 || cams[v].height <= 0) return false;
        if (block_off) block_off[v] = blocks;
        pixels = pixels > cams[v].pix_offset + (int64_t)cams[v].width * cams[v].height
                     ? pixels
                     : cams[v].pix_offset + (int64_t)cams[v].width * cams[v].height;
        blocks += ceil_div(cams[v].width, LTW) * ceil_div(cams[v].height, LTH);
    }
    if (block_off) block_off[n_views] = blocks;
    L.dmaps_off = 0;
    L.partials_off = align256(sizeof(float) * 9 * (size_t)pixels);
    L.total = L.partials_off + align256(sizeof(double2) * (size_t)blocks);
    return true;
}

gs_status check_loss_args(const float *image, const float *target, const gs_camera *cams_host, int32_t n_views,
                          void *workspace, size_t workspace_bytes, LossLayout &L) {
    if (!image || !target || !cams_host || n_views <= 0) return GS_ERR_INVALID_ARG;
    if (!loss_layout(cams_host, n_views, L, nullptr)) return GS_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < L.total || ((uintptr_t)workspace & 255)) return GS_ERR_WORKSPACE;
    return GS_OK;
}

}  // namespace

extern "C" {

size_t gs_loss_workspace_size(const gs_camera *cams_host, int32_t n_views) {
    if (!cams_host || n_views <= 0) return 0;
    LossLayout L;
    if (!loss_layout(cams_host, n_views, L, nullptr)) return 0;
    return L.total;
}

gs_status gs_loss(const float *image, const float *target, const int64_t *target_offsets, const gs_camera *cams_host,
                  const gs_camera *cams_dev, const int32_t *view_ids, int32_t n_views, float lambda_ssim,
                  void *workspace, size_t workspace_bytes, float *loss_per_view, float *dL_dimage,
                  cudaStream_t stream) {
    LossLayout L;
    gs_status st = check_loss_args(image, target, cams_host, n_views, workspace, workspace_bytes, L);
    if (st != GS_OK) return st;
    if (!loss_per_view) return GS_ERR_INVALID_ARG;
    if ((target_offsets == nullptr) != (view_ids == nullptr)) return GS_ERR_INVALID_ARG;
    const Win win = window_host();
    float *dmaps = reinterpret_cast<float *>((char *)workspace + L.dmaps_off);
    double2 *partials = reinterpret_cast<double2 *>((char *)workspace + L.partials_off);
    int64_t boff = 0;
    for (int v = 0; v < n_views; ++v) {
        const gs_camera &c = cams_host[v];
        const dim3 grid((unsigned)ceil_div(c.width, LTW), (unsigned)ceil_div(c.height, LTH));
        ssim_fwd_kernel<<<grid, dim3(32, 8), 0, stream>>>(image + 3 * c.pix_offset, target, target_offsets, view_ids, v,
                                                          c.pix_offset, c.width, c.height,
                                                          cams_dev ? cams_dev + v : nullptr, win,
                                                          dmaps + 9 * c.pix_offset, partials + boff);
        GS_TRY_LAUNCH();
        loss_reduce_kernel<<<1, 256, 0, stream>>>(partials + boff, (int)(grid.x * grid.y),
                                                  3.0 * (double)c.width * c.height, cams_dev ? cams_dev + v : nullptr,
                                                  lambda_ssim, loss_per_view + v);
        GS_TRY_LAUNCH();
        boff += (int64_t)grid.x * grid.y;
    }
    if (dL_dimage)
        return gs_loss_backward(image, target, target_offsets, cams_host, cams_dev, view_ids, n_views, lambda_ssim,
                                workspace, workspace_bytes, dL_dimage, stream);
    return GS_OK;
}

gs_status gs_loss_backward(const float *image, const float *target, const int64_t *target_offsets,
                           const gs_camera *cams_host, const gs_camera *cams_dev, const int32_t *view_ids,
                           int32_t n_views, float lambda_ssim, void *workspace, size_t workspace_bytes,
                           float *dL_dimage, cudaStream_t stream) {
    LossLayout L;
    gs_status st = check_loss_args(image, target, cams_host, n_views, workspace, workspace_bytes, L);
    if (st != GS_OK) return st;
    if (!dL_dimage) return GS_ERR_INVALID_ARG;
    if ((target_offsets == nullptr) != (view_ids == nullptr)) return GS_ERR_INVALID_ARG;
    const Win win = window_host();
    const float *dmaps = reinterpret_cast<const float *>((char *)workspace + L.dmaps_off);
    for (int v = 0; v < n_views; ++v) {
        const gs_camera &c = cams_host[v];
        const dim3 grid((unsigned)ceil_div(c.width, LTW), (unsigned)ceil_div(c.height, LTH));
        ssim_bwd_kernel<<<grid, dim3(32, 8), 0, stream>>>(image + 3 * c.pix_offset, target, target_offsets, view_ids, v,
                                                          c.pix_offset, c.width, c.height,
                                                          cams_dev ? cams_dev + v : nullptr, lambda_ssim, win,
                                                          dmaps + 9 * c.pix_offset, dL_dimage + 3 * c.pix_offset);
        GS_TRY_LAUNCH();
    }
    return GS_OK;
}

}  // extern "C"
