// gs_loss / gs_loss_backward: Eq. (loss), L = (1 - lambda) L1 + lambda (1 - SSIM).
//
// SSIM uses an 11x11 Gaussian window (sigma 1.5, separable), zero padding,
// C1 = 0.01^2, C2 = 0.03^2.  One CTA of 256 threads computes a 32x32 output
// tile of one channel: the tile plus a 5-pixel halo goes to shared memory,
// rows are filtered (a thread computes 4 adjacent outputs of a row, so each
// staged value is loaded once per thread), then columns (a thread computes 4
// adjacent columns of one output row from 16-byte shared loads), pairs of
// sums as packed f32x2 operations, and the
// SSIM map is evaluated.  Window sums are taken of
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

constexpr int LTW = 32, LTH = 32, HALO = 5, LW = LTW + 2 * HALO, LH = LTH + 2 * HALO;
constexpr int LOSS_THREADS = 256;
constexpr int LS = 45;  // staged row stride: = 1 (mod 4), so the 4 rows a warp filters fall in distinct banks
constexpr int STAGE = LW * LH;                                  // staged values per plane
constexpr int SPT = (STAGE + LOSS_THREADS - 1) / LOSS_THREADS;  // of them per thread
constexpr int ROW_TASKS = LH * (LTW / 4);                       // row strips of 4 outputs
static_assert(LS >= LW && LS % 4 == 1, "staged row stride");
static_assert(LOSS_THREADS == LTH * (LTW / 4), "column pass: one output row of 4 columns per thread");
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

// This thread's share of a halo tile of NP planes (value 0 outside the view):
// element e = threadIdx.x + i * LOSS_THREADS of the LH x LW tile.
template <int NP>
__device__ __forceinline__ void halo_load(const float *const (&src)[NP], int W, int H, int bx0, int by0,
                                          float (&reg)[NP][SPT]) {
#pragma unroll
    for (int i = 0; i < SPT; ++i) {
        const int e = threadIdx.x + i * LOSS_THREADS;
        const int r = e / LW, c = e - r * LW;
        const int gx = bx0 + c - HALO, gy = by0 + r - HALO;
        const bool in = e < STAGE && gx >= 0 && gx < W && gy >= 0 && gy < H;
        const int64_t p = (int64_t)gy * W + gx;
#pragma unroll
        for (int q = 0; q < NP; ++q) reg[q][i] = in ? src[q][p] : 0.f;
    }
}

// The registers of halo_load into shared planes [LH][LS], each value minus shift[q].
template <int NP>
__device__ __forceinline__ void halo_store(const float (&reg)[NP][SPT], const float (&shift)[NP],
                                           float (*dst)[LH * LS]) {
#pragma unroll
    for (int i = 0; i < SPT; ++i) {
        const int e = threadIdx.x + i * LOSS_THREADS;
        if (e < STAGE) {
            const int r = e / LW, c = e - r * LW;
#pragma unroll
            for (int q = 0; q < NP; ++q) dst[q][r * LS + c] = reg[q][i] - shift[q];
        }
    }
}

__global__ void __launch_bounds__(LOSS_THREADS, 4) ssim_fwd_kernel(const float *__restrict__ img,
                                                                const float *__restrict__ target,
                                                                const int64_t *__restrict__ target_offsets,
                                                                const int32_t *__restrict__ view_ids, int v,
                                                                int64_t pix_offset, int W, int H,
                                                                const gs_camera *__restrict__ cam_dev, Win win,
                                                                float *__restrict__ dmaps,
                                                                double2 *__restrict__ partials) {
    __shared__ float sxy[2][LH * LS];  // image, target (shifted)
    __shared__ __align__(16) float hs[5][LH][LTW];
    __shared__ double red[2][LOSS_THREADS / 32];
    view_size(cam_dev, W, H);
    const float *tgt = target_base(target, target_offsets, view_ids, v, pix_offset);
    const int tid = threadIdx.x;
    const int bx0 = blockIdx.x * LTW, by0 = blockIdx.y * LTH;
    const int ch = blockIdx.z;
    const int64_t pidx = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (bx0 >= W || by0 >= H) {  // past the device camera's size
        if (tid == 0) partials[pidx] = make_double2(0.0, 0.0);
        return;
    }
    const int64_t hw = (int64_t)W * H;
    const int64_t centre = (int64_t)min(by0 + LTH / 2, H - 1) * W + min(bx0 + LTW / 2, W - 1);
    float ssim_acc = 0.f, l1_acc = 0.f;
    const float *X = img + ch * hw, *Yp = tgt + ch * hw;
    const float shift[2] = {X[centre], Yp[centre]};
    {
        float reg[2][SPT];
        const float *const src[2] = {X, Yp};
        halo_load<2>(src, W, H, bx0, by0, reg);
        halo_store<2>(reg, shift, sxy);
    }
    __syncthreads();
    {
        // rows: a thread filters 4 adjacent outputs of one row from 14 inputs
        // (each input and its products loaded and formed once)
        for (int task = tid; task < ROW_TASKS; task += LOSS_THREADS) {
            const int r = task / (LTW / 4), c0 = 4 * (task % (LTW / 4));
            const float *rx = &sxy[0][r * LS + c0], *ry = &sxy[1][r * LS + c0];
            // per output: (x, y) and (x^2, y^2) as packed pairs, xy alone
            uint64_t a01[4], a23[4];
            float a4[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                a01[o] = a23[o] = 0ull;
                a4[o] = 0.f;
            }
#pragma unroll
            for (int j = 0; j < 14; ++j) {
                const float xv = rx[j], yv = ry[j];
                const uint64_t v01 = pk2(xv, yv), v23 = mul2(v01, v01);
                const float v4 = xv * yv;
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int t = j - o;
                    if (t >= 0 && t < 11) {
                        const uint64_t wt = dup2(win.w[t]);
                        a01[o] = fma2(wt, v01, a01[o]);
                        a23[o] = fma2(wt, v23, a23[o]);
                        a4[o] += win.w[t] * v4;
                    }
                }
            }
            float2 p01[4], p23[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                p01[o] = upk2(a01[o]);
                p23[o] = upk2(a23[o]);
            }
            *reinterpret_cast<float4 *>(&hs[0][r][c0]) = make_float4(p01[0].x, p01[1].x, p01[2].x, p01[3].x);
            *reinterpret_cast<float4 *>(&hs[1][r][c0]) = make_float4(p01[0].y, p01[1].y, p01[2].y, p01[3].y);
            *reinterpret_cast<float4 *>(&hs[2][r][c0]) = make_float4(p23[0].x, p23[1].x, p23[2].x, p23[3].x);
            *reinterpret_cast<float4 *>(&hs[3][r][c0]) = make_float4(p23[0].y, p23[1].y, p23[2].y, p23[3].y);
            *reinterpret_cast<float4 *>(&hs[4][r][c0]) = make_float4(a4[0], a4[1], a4[2], a4[3]);
        }
        __syncthreads();
        // columns: a thread filters 4 adjacent columns of one output row
        {
            const int c0 = 4 * (tid % (LTW / 4)), ro = tid / (LTW / 4);
            uint64_t m01[5], m23[5];  // per quantity: outputs (0, 1) and (2, 3) as packed pairs
#pragma unroll
            for (int q = 0; q < 5; ++q) m01[q] = m23[q] = 0ull;
#pragma unroll
            for (int t = 0; t < 11; ++t) {
                const uint64_t wt = dup2(win.w[t]);
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    const ulonglong2 h = *reinterpret_cast<const ulonglong2 *>(&hs[q][ro + t][c0]);
                    m01[q] = fma2(wt, h.x, m01[q]);
                    m23[q] = fma2(wt, h.y, m23[q]);
                }
            }
            float mm[4][5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const float2 a = upk2(m01[q]), b = upk2(m23[q]);
                mm[0][q] = a.x;
                mm[1][q] = a.y;
                mm[2][q] = b.x;
                mm[3][q] = b.y;
            }
            const int gy = by0 + ro;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int gx = bx0 + c0 + o;
                if (gx < W && gy < H) {
                    const float m0 = mm[o][0], m1 = mm[o][1], e2 = mm[o][2], f2 = mm[o][3], exy = mm[o][4];
                    const float sxx = e2 - m0 * m0, syy = f2 - m1 * m1, sxy = exy - m0 * m1;
                    const float mx = m0 + shift[0], my = m1 + shift[1];
                    const float A1 = 2.f * mx * my + SSIM_C1, A2 = 2.f * sxy + SSIM_C2;
                    const float B1 = mx * mx + my * my + SSIM_C1, B2 = sxx + syy + SSIM_C2;
                    const float iB2 = rcp_approx(B2);  // B1, B2 >= C1, C2 > 0
                    const float iD = rcp_approx(B1) * iB2;
                    const float m = A1 * A2 * iD;
                    const float P2 = -m * iB2;
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
    }
    double s0 = ssim_acc, s1 = l1_acc;
    for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    }
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) { red[0][warp] = s0; red[1][warp] = s1; }
    __syncthreads();
    if (tid == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int w = 0; w < LOSS_THREADS / 32; ++w) { t0 += red[0][w]; t1 += red[1][w]; }
        partials[pidx] = make_double2(t0, t1);
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

__global__ void __launch_bounds__(LOSS_THREADS, 4) ssim_bwd_kernel(const float *__restrict__ img,
                                                                const float *__restrict__ target,
                                                                const int64_t *__restrict__ target_offsets,
                                                                const int32_t *__restrict__ view_ids, int v,
                                                                int64_t pix_offset, int W, int H,
                                                                const gs_camera *__restrict__ cam_dev, float lambda,
                                                                Win win, const float *__restrict__ dmaps,
                                                                float *__restrict__ grad) {
    __shared__ float sp[3][LH * LS];
    __shared__ __align__(16) float hs[3][LH][LTW];
    view_size(cam_dev, W, H);
    const float *tgt = target_base(target, target_offsets, view_ids, v, pix_offset);
    const int tid = threadIdx.x;
    const int bx0 = blockIdx.x * LTW, by0 = blockIdx.y * LTH;
    if (bx0 >= W || by0 >= H) return;
    const int64_t hw = (int64_t)W * H;
    const float inv_n = 1.f / (3.f * (float)hw);
    const float zero[3] = {0.f, 0.f, 0.f};
    const int ch = blockIdx.z;
    {
        float reg[3][SPT];
        const float *const src[3] = {dmaps + ch * hw, dmaps + (3 + ch) * hw, dmaps + (6 + ch) * hw};
        halo_load<3>(src, W, H, bx0, by0, reg);
        halo_store<3>(reg, zero, sp);
    }
    __syncthreads();
    {
        // rows: 4 adjacent outputs of one row per thread
        for (int task = tid; task < ROW_TASKS; task += LOSS_THREADS) {
            const int r = task / (LTW / 4), c0 = 4 * (task % (LTW / 4));
            uint64_t a01[4];  // per output: quantities (0, 1) as a packed pair, 2 alone
            float a2[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                a01[o] = 0ull;
                a2[o] = 0.f;
            }
#pragma unroll
            for (int j = 0; j < 14; ++j) {
                const uint64_t v01 = pk2(sp[0][r * LS + c0 + j], sp[1][r * LS + c0 + j]);
                const float v2 = sp[2][r * LS + c0 + j];
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int t = j - o;
                    if (t >= 0 && t < 11) {
                        a01[o] = fma2(dup2(win.w[t]), v01, a01[o]);
                        a2[o] += win.w[t] * v2;
                    }
                }
            }
            float2 p01[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) p01[o] = upk2(a01[o]);
            *reinterpret_cast<float4 *>(&hs[0][r][c0]) = make_float4(p01[0].x, p01[1].x, p01[2].x, p01[3].x);
            *reinterpret_cast<float4 *>(&hs[1][r][c0]) = make_float4(p01[0].y, p01[1].y, p01[2].y, p01[3].y);
            *reinterpret_cast<float4 *>(&hs[2][r][c0]) = make_float4(a2[0], a2[1], a2[2], a2[3]);
        }
        __syncthreads();
        // columns: 4 adjacent columns of one output row per thread
        {
            const int c0 = 4 * (tid % (LTW / 4)), ro = tid / (LTW / 4);
            uint64_t f01[3], f23[3];  // per quantity: outputs (0, 1) and (2, 3) as packed pairs
#pragma unroll
            for (int q = 0; q < 3; ++q) f01[q] = f23[q] = 0ull;
#pragma unroll
            for (int t = 0; t < 11; ++t) {
                const uint64_t wt = dup2(win.w[t]);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const ulonglong2 h = *reinterpret_cast<const ulonglong2 *>(&hs[q][ro + t][c0]);
                    f01[q] = fma2(wt, h.x, f01[q]);
                    f23[q] = fma2(wt, h.y, f23[q]);
                }
            }
            float ff[4][3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float2 a = upk2(f01[q]), b = upk2(f23[q]);
                ff[0][q] = a.x;
                ff[1][q] = a.y;
                ff[2][q] = b.x;
                ff[3][q] = b.y;
            }
            const int gy = by0 + ro;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int gx = bx0 + c0 + o;
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
        blocks += 3 * ceil_div(cams[v].width, LTW) * ceil_div(cams[v].height, LTH);
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
        const dim3 grid((unsigned)ceil_div(c.width, LTW), (unsigned)ceil_div(c.height, LTH), 3u);
        ssim_fwd_kernel<<<grid, LOSS_THREADS, 0, stream>>>(image + 3 * c.pix_offset, target, target_offsets, view_ids, v,
                                                          c.pix_offset, c.width, c.height,
                                                          cams_dev ? cams_dev + v : nullptr, win,
                                                          dmaps + 9 * c.pix_offset, partials + boff);
        GS_TRY_LAUNCH();
        loss_reduce_kernel<<<1, 256, 0, stream>>>(partials + boff, (int)(grid.x * grid.y * grid.z),
                                                  3.0 * (double)c.width * c.height, cams_dev ? cams_dev + v : nullptr,
                                                  lambda_ssim, loss_per_view + v);
        GS_TRY_LAUNCH();
        boff += (int64_t)grid.x * grid.y * grid.z;
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
        const dim3 grid((unsigned)ceil_div(c.width, LTW), (unsigned)ceil_div(c.height, LTH), 3u);
        ssim_bwd_kernel<<<grid, LOSS_THREADS, 0, stream>>>(image + 3 * c.pix_offset, target, target_offsets, view_ids, v,
                                                          c.pix_offset, c.width, c.height,
                                                          cams_dev ? cams_dev + v : nullptr, lambda_ssim, win,
                                                          dmaps + 9 * c.pix_offset, dL_dimage + 3 * c.pix_offset);
        GS_TRY_LAUNCH();
    }
    return GS_OK;
}

}  // extern "C"
