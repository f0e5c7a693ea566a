// gs_adam_step: Adam (Kingma & Ba, bias-corrected) over the flat parameter
// buffer, the optimizer step Algorithm 1 runs only when g = 1.
// HBM-bound: 16 B read (p, g, m, v) and 12-16 B written per scalar.
#include "common.cuh"

using namespace gsr;

namespace {

struct Groups {
    int64_t o_scales, o_quats, o_opac, o_sh, total;
    int K3;
};

__device__ __forceinline__ int group_of(int64_t e, const Groups &G) {
    if (e < G.o_scales) return 0;
    if (e < G.o_quats) return 1;
    if (e < G.o_opac) return 2;
    if (e < G.o_sh) return 3;
    return ((e - G.o_sh) % G.K3) < 3 ? 4 : 5;
}

template <bool NORMS>
__global__ void __launch_bounds__(256) adam_kernel(float *__restrict__ p, float *__restrict__ g, float *__restrict__ m,
                                                   float *__restrict__ v, Groups G, gs_adam_config cfg,
                                                   const int32_t *do_step, const int64_t *step, int zero_grad,
                                                   double *__restrict__ norms2) {
    if (do_step && *do_step == 0) return;
    __shared__ float s_lr[6];
    __shared__ float s_ibc2;
    if (threadIdx.x == 0) adam_scalars(cfg, *step, do_step, s_lr, &s_ibc2);
    __syncthreads();
    const float b1 = cfg.beta1, b2 = cfg.beta2, eps = cfg.eps;
    const float ibc2 = s_ibc2;
    const int64_t nvec = G.total / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float sg = 0.f, sd = 0.f;  // sum of g^2 and of (p_new - p_old)^2 over this thread's scalars
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nvec; c += stride) {
        float4 pp = reinterpret_cast<float4 *>(p)[c];
        const float4 gg = reinterpret_cast<const float4 *>(g)[c];
        float4 mm = reinterpret_cast<float4 *>(m)[c];
        float4 vv = reinterpret_cast<float4 *>(v)[c];
        float *pe = &pp.x, *me = &mm.x, *ve = &vv.x;
        const float *ge = &gg.x;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float p0 = pe[u];
            adam_update(pe[u], me[u], ve[u], ge[u], s_lr[group_of(4 * c + u, G)], b1, b2, ibc2, eps);
            if (NORMS) {
                sg += ge[u] * ge[u];
                sd += (pe[u] - p0) * (pe[u] - p0);
            }
        }
        reinterpret_cast<float4 *>(p)[c] = pp;
        reinterpret_cast<float4 *>(m)[c] = mm;
        reinterpret_cast<float4 *>(v)[c] = vv;
        if (zero_grad) reinterpret_cast<float4 *>(g)[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // scalar tail
    for (int64_t e = 4 * nvec + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < G.total; e += stride) {
        float pe = p[e], me = m[e], ve = v[e];
        const float p0 = pe, ge = g[e];
        adam_update(pe, me, ve, ge, s_lr[group_of(e, G)], b1, b2, ibc2, eps);
        if (NORMS) {
            sg += ge * ge;
            sd += (pe - p0) * (pe - p0);
        }
        p[e] = pe;
        m[e] = me;
        v[e] = ve;
        if (zero_grad) g[e] = 0.f;
    }
    if (NORMS) {  // block sums, one double atomic per block and quantity
        __shared__ float s_red[2][8];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sg += __shfl_xor_sync(0xffffffffu, sg, off);
            sd += __shfl_xor_sync(0xffffffffu, sd, off);
        }
        if ((threadIdx.x & 31) == 0) {
            s_red[0][threadIdx.x >> 5] = sg;
            s_red[1][threadIdx.x >> 5] = sd;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < 8; ++w) {
                a += s_red[0][w];
                b += s_red[1][w];
            }
            atomicAdd(norms2, a);
            atomicAdd(norms2 + 1, b);
        }
    }
}

__global__ void adam_count_kernel(const int32_t *do_step, int64_t *step) {
    if (!do_step || *do_step) *step += 1;
}

}  // namespace

extern "C" gs_status gs_adam_step(float *params, float *grads, float *m, float *v, int64_t n, int32_t sh_degree,
                                  const gs_adam_config *cfg, const int32_t *dev_do_step, int64_t *dev_step,
                                  int32_t zero_grad, double *norms2, cudaStream_t stream) {
    if (!params || !grads || !m || !v || !cfg || !dev_step || n < 0 || sh_degree < 0 || sh_degree > 3)
        return GS_ERR_INVALID_ARG;
    if (((uintptr_t)params | (uintptr_t)grads | (uintptr_t)m | (uintptr_t)v) & 15) return GS_ERR_INVALID_ARG;
    if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->eps >= 0.f))
        return GS_ERR_INVALID_ARG;
    const int K = (sh_degree + 1) * (sh_degree + 1);
    int64_t o[6];
    param_offsets(n, sh_degree, o);
    Groups G{o[1], o[2], o[3], o[4], o[5], 3 * K};
    if (n > 0) {
        int64_t blocks = ceil_div(G.total / 4 + 1, 256);
        const int64_t resident = (int64_t)device_sm_count() * 8;  // 8 blocks of 256 threads per SM
        if (blocks > resident) blocks = resident;
        if (norms2)
            adam_kernel<true><<<(unsigned)blocks, 256, 0, stream>>>(params, grads, m, v, G, *cfg, dev_do_step,
                                                                    dev_step, zero_grad, norms2);
        else
            adam_kernel<false><<<(unsigned)blocks, 256, 0, stream>>>(params, grads, m, v, G, *cfg, dev_do_step,
                                                                     dev_step, zero_grad, nullptr);
        GS_TRY_LAUNCH();
    }
    adam_count_kernel<<<1, 1, 0, stream>>>(dev_do_step, dev_step);
    GS_TRY_LAUNCH();
    return GS_OK;
}
