// SkipGS gate (Algorithm 1; Eq. view-ema, deviation, gate, rhocum,
// rhocum_check, rhohat, rhomincalib) as single-thread device kernels.
//
// The state lives in device memory so a captured refinement step never
// returns to the host: skipgs_gate_decide writes the decision where the
// backward kernels (or a graph's conditional node) read it.  All arithmetic is
// binary64 with explicit round-to-nearest intrinsics, one rounding per
// operation in the order the algorithm states, so the decisions are
// reproducible bit for bit from the same float32 losses.
#include "common.cuh"

using namespace gsr;

namespace {

struct GateHeader {
    int32_t W, n_views;
    double beta, eps, rho_lo;
    long long t, b, n_w, n_w1;
    double rho_min;
    int32_t calibrated, errors;
};

constexpr size_t kHeaderBytes = (sizeof(GateHeader) + 15) & ~(size_t)15;

__device__ __forceinline__ double *ema_of(void *st) { return reinterpret_cast<double *>((char *)st + kHeaderBytes); }
__device__ __forceinline__ uint8_t *hist_of(void *st, int n_views) {
    return reinterpret_cast<uint8_t *>((char *)st + kHeaderBytes + sizeof(double) * n_views);
}

__global__ void gate_init_kernel(gs_gate_config cfg, void *st) {
    GateHeader *h = reinterpret_cast<GateHeader *>(st);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        h->W = cfg.W;
        h->n_views = cfg.n_views;
        h->beta = cfg.beta;
        h->eps = cfg.eps;
        h->rho_lo = cfg.rho_lo;
        h->t = h->b = h->n_w = h->n_w1 = 0;
        h->rho_min = cfg.rho_lo >= 0.0 ? cfg.rho_lo : 0.0;  // Algorithm 1: rho_min <- rho_lo
        h->calibrated = 0;
        h->errors = 0;
    }
    double *ema = ema_of(st);
    uint8_t *hist = hist_of(st, cfg.n_views);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < cfg.n_views; v += gridDim.x * blockDim.x) {
        ema[v] = 0.0;  // empty: hist[v] = 0
        hist[v] = 0;
    }
}

__global__ void gate_decide_kernel(void *st, const int32_t *view_ids, const float *losses, int n, uint8_t *g_out,
                                   int32_t *any_out, int has_cond, cudaGraphConditionalHandle cond,
                                   int32_t *dev_status) {
    GateHeader *h = reinterpret_cast<GateHeader *>(st);
    double *ema = ema_of(st);
    uint8_t *hist = hist_of(st, h->n_views);
    int any = 0;
    for (int k = 0; k < n; ++k) {
        const int v = view_ids[k];
        const float Lf = losses[k];
        if (v < 0 || v >= h->n_views) {
            set_status(dev_status, GS_ERR_INVALID_ARG);
            g_out[k] = 0;
            continue;
        }
        if (!isfinite(Lf)) {  // reading (vi): skip, leave the state untouched, report
            set_status(dev_status, GS_ERR_NONFINITE);
            h->errors += 1;
            g_out[k] = 0;
            continue;
        }
        const double L = (double)Lf;
        const long long t = ++h->t;
        int g;
        if (hist[v]) {
            // Eq. (deviation), Eq. (gate)
            const double s = __ddiv_rn(L, __dadd_rn(ema[v], h->eps));
            g = s > 1.0 ? 1 : 0;
        } else {
            g = 1;  // no history: s = +inf
        }
        if (t <= h->W) {
            // warmup: record the skip test for views with history (Eq. rhohat), force backward
            if (hist[v]) {
                h->n_w += 1;
                h->n_w1 += g;
            }
            g = 1;
        } else {
            if (!h->calibrated) {
                // once, at t = W + 1: Eq. (rhohat) and Eq. (rhomincalib)
                if (h->rho_lo >= 0.0 && h->n_w > 0) {
                    const double rho_hat = __ddiv_rn((double)h->n_w1, (double)h->n_w);
                    h->rho_min = __dadd_rn(h->rho_lo, __dmul_rn(__dsub_rn(1.0, h->rho_lo), rho_hat));
                }
                h->calibrated = 1;
            }
            if (h->rho_lo >= 0.0) {
                // Eq. (rhocum) before iteration t, Eq. (rhocum_check)
                const long long den = t - 1 > 1 ? t - 1 : 1;
                const double rho_cum = __ddiv_rn((double)h->b, (double)den);
                if (rho_cum < h->rho_min) g = 1;
            }
        }
        if (g) h->b += 1;
        g_out[k] = (uint8_t)g;
        any += g;  // the number of opened views
    }
    if (any_out) *any_out = any;
    if (has_cond) cudaGraphSetConditional(cond, any ? 1u : 0u);
}

__global__ void gate_update_kernel(void *st, const int32_t *view_ids, const float *losses, int n) {
    GateHeader *h = reinterpret_cast<GateHeader *>(st);
    double *ema = ema_of(st);
    uint8_t *hist = hist_of(st, h->n_views);
    for (int k = 0; k < n; ++k) {
        const int v = view_ids[k];
        const float Lf = losses[k];
        if (v < 0 || v >= h->n_views || !isfinite(Lf)) continue;
        const double L = (double)Lf;
        if (hist[v]) {
            // Eq. (view-ema)
            ema[v] = __dadd_rn(__dmul_rn(h->beta, ema[v]), __dmul_rn(__dsub_rn(1.0, h->beta), L));
        } else {
            ema[v] = L;  // reading (i): the first observation starts the EMA
            hist[v] = 1;
        }
    }
}

}  // namespace

extern "C" {

size_t skipgs_gate_state_size(int32_t n_views) {
    if (n_views <= 0) return 0;
    return (kHeaderBytes + sizeof(double) * (size_t)n_views + (size_t)n_views + 15) & ~(size_t)15;
}

gs_status skipgs_gate_init(const gs_gate_config *cfg, void *dev_state, cudaStream_t stream) {
    if (!cfg || !dev_state || cfg->n_views <= 0 || cfg->W < 0) return GS_ERR_INVALID_ARG;
    if (!(cfg->beta > 0.0 && cfg->beta < 1.0) || !(cfg->eps >= 0.0) || !(cfg->rho_lo <= 1.0))
        return GS_ERR_INVALID_ARG;
    if ((uintptr_t)dev_state & 15) return GS_ERR_INVALID_ARG;
    const int blocks = (int)ceil_div(cfg->n_views, 256);
    gate_init_kernel<<<blocks, 256, 0, stream>>>(*cfg, dev_state);
    GS_TRY_LAUNCH();
    return GS_OK;
}

gs_status skipgs_gate_decide(void *dev_state, const int32_t *dev_view_ids, const float *dev_losses, int32_t n,
                             uint8_t *dev_g, int32_t *dev_any, const cudaGraphConditionalHandle *cond,
                             int32_t *dev_status, cudaStream_t stream) {
    if (!dev_state || !dev_view_ids || !dev_losses || !dev_g || n <= 0) return GS_ERR_INVALID_ARG;
    gate_decide_kernel<<<1, 1, 0, stream>>>(dev_state, dev_view_ids, dev_losses, n, dev_g, dev_any, cond ? 1 : 0,
                                            cond ? *cond : (cudaGraphConditionalHandle)0, dev_status);
    GS_TRY_LAUNCH();
    return GS_OK;
}

gs_status skipgs_gate_update(void *dev_state, const int32_t *dev_view_ids, const float *dev_losses, int32_t n,
                             cudaStream_t stream) {
    if (!dev_state || !dev_view_ids || !dev_losses || n <= 0) return GS_ERR_INVALID_ARG;
    gate_update_kernel<<<1, 1, 0, stream>>>(dev_state, dev_view_ids, dev_losses, n);
    GS_TRY_LAUNCH();
    return GS_OK;
}

gs_status skipgs_gate_read(const void *dev_state, int64_t *out7, double *rho_min, cudaStream_t stream) {
    if (!dev_state || !out7) return GS_ERR_INVALID_ARG;
    GateHeader h;
    GS_TRY(cudaMemcpyAsync(&h, dev_state, sizeof(h), cudaMemcpyDeviceToHost, stream));
    GS_TRY(cudaStreamSynchronize(stream));
    out7[0] = h.t;
    out7[1] = h.b;
    out7[2] = h.n_w;
    out7[3] = h.n_w1;
    out7[4] = h.calibrated;
    out7[5] = h.errors;
    out7[6] = h.n_views;
    if (rho_min) *rho_min = h.rho_min;
    return GS_OK;
}

}  // extern "C"
