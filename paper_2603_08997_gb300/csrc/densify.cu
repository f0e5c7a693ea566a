// Adaptive density control (Sec. 3): the densification phase before T_d
// clones small and splits large Gaussians whose view-space positional
// gradient is high, and prunes near-transparent ones (alpha < eps_alpha);
// the same compaction serves an opacity-threshold prune before the
// post-densification phase.
//
//   gs_densify_accumulate  after a backward pass: accum_i += |dL/dmean2D_i|
//                          and denom_i += 1 for every view the Gaussian is
//                          visible in (tiles_touched > 0, gate open).
//   gs_densify_decide      one action per Gaussian (keep / clone / split /
//                          prune) from float32 comparisons only, so the
//                          decisions are reproducible bit for bit; then the
//                          exclusive scan of the output counts (1, 2, 2, 0):
//                          offsets[i] = first output of Gaussian i,
//                          offsets[n] = the new count.
//   gs_densify_apply       writes the output set in input order (stable
//                          compaction): parameters and Adam moments into
//                          buffers laid out for the new count; split children
//                          at mean + R(q) (s * z_k) with the caller's noise.
// Every kernel is a streaming pass (HBM-bound): one thread per Gaussian.
#include "common.cuh"

using namespace gsr;

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;                        // Gaussians per thread in the scan
constexpr int kScanTile = kScanThreads * kScanItems; // Gaussians per scan block

__device__ __forceinline__ int outputs_of(uint8_t a) { return a == GS_DENSIFY_CLONE || a == GS_DENSIFY_SPLIT ? 2 : (a == GS_DENSIFY_KEEP ? 1 : 0); }

__global__ void __launch_bounds__(256) accumulate_kernel(const float4 *__restrict__ g2d,
                                                          const int32_t *__restrict__ touched, int64_t n,
                                                          int n_views, const uint8_t *__restrict__ gate,
                                                          float *__restrict__ accum, int32_t *__restrict__ denom) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a = accum[i];
    int32_t d = denom[i];
    for (int v = 0; v < n_views; ++v) {
        if (gate && !gate[v]) continue;
        const int64_t k = (int64_t)v * n + i;
        if (touched[k] <= 0) continue;
        const float4 g = g2d[k * 3];  // (dL/dmean2D.x, dL/dmean2D.y, ...)
        a += sqrtf(__fmaf_rn(g.x, g.x, __fmul_rn(g.y, g.y)));
        d += 1;
    }
    accum[i] = a;
    denom[i] = d;
}

// Block-wide exclusive scan of one int64 per thread (warp shuffles, then the
// warp totals).  Returns the thread's exclusive prefix; *total = block sum.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t x, int64_t *s_warp, int64_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;  // inclusive prefix of the warp totals
    }
    __syncthreads();
    const int64_t before = warp > 0 ? s_warp[warp - 1] : 0;
    *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();  // s_warp may be reused by the caller
    return before + inc - x;
}

// Decision per Gaussian, and each scan block's output total.
__global__ void __launch_bounds__(kScanThreads) decide_kernel(const float *__restrict__ log_scales,
                                                              const float *__restrict__ logit, int64_t n,
                                                              const float *__restrict__ accum,
                                                              const int32_t *__restrict__ denom,
                                                              gs_densify_config cfg, uint8_t *__restrict__ action,
                                                              int64_t *__restrict__ block_sum) {
    __shared__ int64_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t cnt = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        if (i >= n) break;
        const int32_t d = denom[i];
        const float avg = d > 0 ? __fdiv_rn(accum[i], (float)d) : 0.f;
        const float s0 = log_scales[3 * i], s1 = log_scales[3 * i + 1], s2 = log_scales[3 * i + 2];
        const float smax = fmaxf(s0, fmaxf(s1, s2));
        uint8_t a = GS_DENSIFY_KEEP;
        if (avg >= cfg.grad_thr) a = smax > cfg.log_size_thr ? GS_DENSIFY_SPLIT : GS_DENSIFY_CLONE;
        if (logit[i] < cfg.logit_prune_thr) a = GS_DENSIFY_PRUNE;
        action[i] = a;
        cnt += outputs_of(a);
    }
    int64_t total;
    block_exclusive_scan(cnt, s_warp, &total);
    if (threadIdx.x == 0) block_sum[blockIdx.x] = total;
}

// Exclusive scan of the block totals in place (one block, any count).
__global__ void __launch_bounds__(kScanThreads) scan_block_sums(int64_t *__restrict__ block_sum, int64_t nb) {
    __shared__ int64_t s_warp[32];
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        const int64_t b = b0 + threadIdx.x;
        const int64_t x = b < nb ? block_sum[b] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(x, s_warp, &total);
        if (b < nb) block_sum[b] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads) write_offsets(const uint8_t *__restrict__ action, int64_t n,
                                                              const int64_t *__restrict__ block_base,
                                                              int64_t *__restrict__ offsets) {
    __shared__ int64_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int c[kScanItems];
    int64_t cnt = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        c[k] = i < n ? outputs_of(action[i]) : 0;
        cnt += c[k];
    }
    int64_t total;
    int64_t pos = block_base[blockIdx.x] + block_exclusive_scan(cnt, s_warp, &total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        if (i < n) offsets[i] = pos;
        if (i == n - 1) offsets[n] = pos + c[k];
        pos += c[k];
    }
}

struct Layout {
    int64_t o[6];
};

__host__ __device__ inline Layout layout_of(int64_t n, int sh_degree) {
    Layout l;
    param_offsets(n, sh_degree, l.o);
    return l;
}

// Rotation of a unit quaternion (w, x, y, z) applied to v.
__device__ __forceinline__ float3 rotate(float4 q, float3 v) {
    const float w = q.x, x = q.y, y = q.z, z = q.w;
    const float r00 = 1.f - 2.f * (y * y + z * z), r01 = 2.f * (x * y - w * z), r02 = 2.f * (x * z + w * y);
    const float r10 = 2.f * (x * y + w * z), r11 = 1.f - 2.f * (x * x + z * z), r12 = 2.f * (y * z - w * x);
    const float r20 = 2.f * (x * z - w * y), r21 = 2.f * (y * z + w * x), r22 = 1.f - 2.f * (x * x + y * y);
    return make_float3(r00 * v.x + r01 * v.y + r02 * v.z, r10 * v.x + r11 * v.y + r12 * v.z,
                       r20 * v.x + r21 * v.y + r22 * v.z);
}

__global__ void __launch_bounds__(256) apply_kernel(const float *__restrict__ sp, const float *__restrict__ sm,
                                                     const float *__restrict__ sv, int64_t n, int K3, Layout ls,
                                                     const uint8_t *__restrict__ action,
                                                     const int64_t *__restrict__ offsets,
                                                     const float *__restrict__ noise, float shrink,
                                                     float *__restrict__ dp, float *__restrict__ dm,
                                                     float *__restrict__ dv, int64_t n_out, Layout ld,
                                                     int32_t *__restrict__ status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (offsets[n] != n_out) {  // the destination was sized for another count
        if (i == 0) set_status(status, GS_ERR_INVALID_ARG);
        return;
    }
    const uint8_t a = action[i];
    const int64_t j0 = offsets[i];
    const int cnt = outputs_of(a);
    const int width[5] = {3, 3, 4, 1, K3};
    for (int c = 0; c < cnt; ++c) {
        const int64_t j = j0 + c;
        const bool moments = a == GS_DENSIFY_KEEP || (a == GS_DENSIFY_CLONE && c == 0);
        for (int g = 0; g < 5; ++g) {
            const float *ps = sp + ls.o[g] + (int64_t)width[g] * i;
            const float *ms = sm + ls.o[g] + (int64_t)width[g] * i;
            const float *vs = sv + ls.o[g] + (int64_t)width[g] * i;
            float *pd = dp + ld.o[g] + (int64_t)width[g] * j;
            float *md = dm + ld.o[g] + (int64_t)width[g] * j;
            float *vd = dv + ld.o[g] + (int64_t)width[g] * j;
            for (int e = 0; e < width[g]; ++e) {
                pd[e] = ps[e];
                md[e] = moments ? ms[e] : 0.f;
                vd[e] = moments ? vs[e] : 0.f;
            }
        }
        if (a == GS_DENSIFY_SPLIT) {
            const float *q = sp + ls.o[2] + 4 * i;
            const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
            const float4 qu = make_float4(q[0] / qn, q[1] / qn, q[2] / qn, q[3] / qn);
            const float *l = sp + ls.o[1] + 3 * i;
            const float *z = noise + (i * 2 + c) * 3;
            const float3 off = rotate(qu, make_float3(expf(l[0]) * z[0], expf(l[1]) * z[1], expf(l[2]) * z[2]));
            const float *mu = sp + ls.o[0] + 3 * i;
            float *md = dp + ld.o[0] + 3 * j;
            md[0] = mu[0] + off.x;
            md[1] = mu[1] + off.y;
            md[2] = mu[2] + off.z;
            float *lsd = dp + ld.o[1] + 3 * j;
            lsd[0] = l[0] - shrink;
            lsd[1] = l[1] - shrink;
            lsd[2] = l[2] - shrink;
        }
    }
}

}  // namespace

extern "C" size_t gs_densify_workspace_size(int64_t n) {
    if (n < 0) return 0;
    return sizeof(int64_t) * (size_t)(ceil_div(n, kScanTile) + 1);
}

extern "C" gs_status gs_densify_accumulate(const float *g2d, const int32_t *tiles_touched, int64_t n,
                                           int32_t n_views, const uint8_t *view_gate, float *accum, int32_t *denom,
                                           cudaStream_t stream) {
    if (n < 0 || n_views <= 0) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!g2d || !tiles_touched || !accum || !denom || ((uintptr_t)g2d & 15)) return GS_ERR_INVALID_ARG;
    accumulate_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, stream>>>(reinterpret_cast<const float4 *>(g2d),
                                                                      tiles_touched, n, n_views, view_gate, accum,
                                                                      denom);
    GS_TRY_LAUNCH();
    return GS_OK;
}

extern "C" gs_status gs_densify_decide(const float *flat_params, int64_t n, int32_t sh_degree, const float *accum,
                                       const int32_t *denom, const gs_densify_config *cfg, uint8_t *action,
                                       int64_t *offsets, void *workspace, size_t workspace_bytes,
                                       cudaStream_t stream) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3 || !cfg || !offsets) return GS_ERR_INVALID_ARG;
    if (n == 0) {
        GS_TRY(cudaMemsetAsync(offsets, 0, sizeof(int64_t), stream));
        return GS_OK;
    }
    if (!flat_params || !accum || !denom || !action) return GS_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < gs_densify_workspace_size(n)) return GS_ERR_WORKSPACE;
    const Layout l = layout_of(n, sh_degree);
    const int64_t nb = ceil_div(n, kScanTile);
    int64_t *bsum = static_cast<int64_t *>(workspace);
    decide_kernel<<<(unsigned)nb, kScanThreads, 0, stream>>>(flat_params + l.o[1], flat_params + l.o[3], n, accum,
                                                             denom, *cfg, action, bsum);
    GS_TRY_LAUNCH();
    scan_block_sums<<<1, kScanThreads, 0, stream>>>(bsum, nb);
    GS_TRY_LAUNCH();
    write_offsets<<<(unsigned)nb, kScanThreads, 0, stream>>>(action, n, bsum, offsets);
    GS_TRY_LAUNCH();
    return GS_OK;
}

extern "C" gs_status gs_densify_apply(const float *src_params, const float *src_m, const float *src_v, int64_t n,
                                      int32_t sh_degree, const uint8_t *action, const int64_t *offsets,
                                      const float *noise, const gs_densify_config *cfg, float *dst_params,
                                      float *dst_m, float *dst_v, int64_t n_out, int32_t *dev_status,
                                      cudaStream_t stream) {
    if (n < 0 || n_out < 0 || sh_degree < 0 || sh_degree > 3 || !cfg) return GS_ERR_INVALID_ARG;
    if (n == 0) return n_out == 0 ? GS_OK : GS_ERR_INVALID_ARG;
    if (n_out > 2 * n) return GS_ERR_INVALID_ARG;
    if (!src_params || !src_m || !src_v || !action || !offsets || !noise) return GS_ERR_INVALID_ARG;
    if (n_out > 0 && (!dst_params || !dst_m || !dst_v)) return GS_ERR_INVALID_ARG;
    const int K3 = 3 * (sh_degree + 1) * (sh_degree + 1);
    apply_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, stream>>>(src_params, src_m, src_v, n, K3,
                                                                 layout_of(n, sh_degree), action, offsets, noise,
                                                                 cfg->log_split_shrink, dst_params, dst_m, dst_v,
                                                                 n_out, layout_of(n_out, sh_degree), dev_status);
    GS_TRY_LAUNCH();
    return GS_OK;
}
