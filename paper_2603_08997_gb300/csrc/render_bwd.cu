// gs_render_bwd: analytic adjoint of gs_render_fwd and gs_project.
//
// Raster adjoint (one CTA per tile, PPT = 1, 2 or 4 pixels per thread; each
// warp walks only the staged records whose support ellipse reaches its pixel
// block, marked per batch with one ballot per warp and 32 records).  With
// A_k = sum_{j>k} c_j a_j T_j + T_end bg (the colour behind contributor k),
// Eq. (blend) gives dC/dc_k = a_k T_k and dC/da_k = c_k T_k - A_k / (1 - a_k).
// Batches are visited last to first and each pixel walks back from its last
// contributor, so A_k is a plain suffix sum; a pixel keeps only its product
// with dL/dC (one scalar instead of three).  T is rebuilt by
// T_k = T_{k+1} / (1 - a_k), re-anchored at every batch boundary on the
// transmittance checkpoint the forward pass stored, so division error never
// spans more than one batch.  The alphas come from the same bit-exact
// evaluation as the forward pass, so the contributor set is identical.
//
// Per Gaussian 9 sums over a thread's pixels (sum dG z with z = U dp, the
// three entries of sum dG dp dp^T, dL/d opacity, the 3 colour gradients;
// dG = dL/d alpha G) are reduced across the warp with a halving shuffle
// tree (12 shuffles for 9 values), summed per Gaussian in shared memory, and
// turned into the mean2D and conic gradients (the factors the record fixes:
// opacity, U^T, -1/2) once per (Gaussian, tile), added to a per-view buffer
// with float4 vector atomics.
//
// Projection adjoint: one lane per Gaussian chains those 2D gradients
// through Eq. (proj), Eq. (cov), the SH colour and the sigmoid to the
// parameters, summing the views; each warp stages and sweeps its own 32
// Gaussians.  The sweep either stores the parameter gradients or applies the
// Adam step to them directly (gs_render_bwd_adam, gs_project_bwd_adam).
#include "common.cuh"

using namespace gsr;

namespace {

constexpr unsigned FULL = 0xffffffffu;
// Up to this many contributing lanes of a warp add their 9 gradients to shared
// memory directly instead of reducing over the warp first.
constexpr int kDirectLanes = 1;

// Reduces v[0..9) over the warp.  On return the even lane L with valid index
// `idx` holds the warp total of v[idx]; other lanes get idx = -1.
__device__ __forceinline__ float warp_reduce9(const float (&v)[9], int lane, int &idx) {
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
    float a[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float lo = v[i];
        const float hi = (5 + i < 9) ? v[5 + i] : 0.f;
        a[i] = (h16 ? hi : lo) + __shfl_xor_sync(FULL, h16 ? lo : hi, 16);
    }
    float b[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float lo = a[i];
        const float hi = (3 + i < 5) ? a[3 + i] : 0.f;
        b[i] = (h8 ? hi : lo) + __shfl_xor_sync(FULL, h8 ? lo : hi, 8);
    }
    float c[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float lo = b[i];
        const float hi = (2 + i < 3) ? b[2 + i] : 0.f;
        c[i] = (h4 ? hi : lo) + __shfl_xor_sync(FULL, h4 ? lo : hi, 4);
    }
    float d = (h2 ? c[1] : c[0]) + __shfl_xor_sync(FULL, h2 ? c[0] : c[1], 2);
    d += __shfl_xor_sync(FULL, d, 1);
    const int jb = (h4 ? 2 : 0) + (h2 ? 1 : 0);
    const int ja = (h8 ? 3 : 0) + jb;
    const int j = (h16 ? 5 : 0) + ja;
    idx = ((lane & 1) == 0 && jb < 3 && ja < 5 && j < 9) ? j : -1;
    return d;
}

// Two pixels per thread (the loop's shape): at most 73 registers, so 7 blocks
// fit an SM with no spill (left alone the compiler took 64 and spilled).
template <int TILE, int BATCH, int PPT, bool COARSE>
__global__ void __launch_bounds__(TILE *TILE / PPT, PPT == 2 ? 7 : 1) render_bwd_kernel(
    const float4 *__restrict__ rec, int64_t n, const ListSrc ls, const uint2 *__restrict__ ranges,
    const gs_camera *__restrict__ cams, int n_views, gs_raster_config cfg, const float *__restrict__ T_final,
    const int32_t *__restrict__ n_last, const float *__restrict__ ckpt, int64_t ckpt_slots,
    const float *__restrict__ dL_dimage, const uint8_t *__restrict__ view_gate, float4 *__restrict__ g2d,
    const uint32_t *__restrict__ tile_order, uint32_t *queue, int64_t total_tiles) {
    constexpr int NT = TILE * TILE;
    constexpr int NTH = TILE * TILE / PPT;
    constexpr int NW = NTH / 32, NWORD = BATCH / 32;
    constexpr int EPT = gather_ept<NTH>();  // super-tile list entries tested per thread and round
    __shared__ float4 s_a[BATCH];
    __shared__ float4 s_b[BATCH];
    __shared__ float4 s_c[BATCH];
    __shared__ uint32_t s_g[BATCH];
    __shared__ uint32_t s_ov[NW][NWORD];  // per warp: records of the batch that reach its pixel block
    __shared__ float s_acc[BATCH][9];
    __shared__ int s_max;
    __shared__ uint32_t s_item;
    __shared__ uint32_t s_wsum[NW], s_next;
    for (uint32_t item = first_item(queue, &s_item); item < (uint64_t)total_tiles; item = next_item(queue, &s_item)) {
    const int64_t tile = tile_order ? (int64_t)tile_order[item] : (int64_t)item;
    const int v = view_of_tile(cams, n_views, tile);
    if (view_gate && !view_gate[v]) continue;  // uniform per block
    const gs_camera &cam = cams[v];
    const int tiles_x = (cam.width + TILE - 1) / TILE;
    const int64_t lt = tile - cam.tile_offset;
    const int tx = (int)(lt % tiles_x), ty = (int)(lt / tiles_x);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint2 rg = ranges[tile];
    const int64_t slot0 = (int64_t)(rg.x / BATCH) + tile;
    const float4 *recv = rec + (int64_t)v * n * 3;
    const float amax = cfg.alpha_max, amin = cfg.alpha_min;
    uint32_t cbit = 0, cend = 0;  // the super-tile list: this tile's bit, the list's end
    if constexpr (COARSE) {
        if (rg.y > rg.x) {
            const int64_t ct = super_tile_of(ls, v, tiles_x, tx, ty, cbit);
            cend = ls.cstart[ct] + ls.ccount[ct];
        }
    }

    int lp[PPT], my_last[PPT];
    float px[PPT], py[PPT], dC0[PPT], dC1[PPT], dC2[PPT], T_end[PPT];
    int local_max = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        int lx, ly;
        tile_pixel<TILE, PPT>(threadIdx.x, k, lx, ly);
        lp[k] = ly * TILE + lx;
        const int x = tx * TILE + lx, y = ty * TILE + ly;
        px[k] = (float)x + 0.5f;
        py[k] = (float)y + 0.5f;
        my_last[k] = 0;
        dC0[k] = dC1[k] = dC2[k] = T_end[k] = 0.f;
        if (x < cam.width && y < cam.height) {
            const int64_t hw = (int64_t)cam.width * cam.height;
            const int64_t pix = (int64_t)y * cam.width + x;
            my_last[k] = n_last[cam.pix_offset + pix];
            T_end[k] = T_final[cam.pix_offset + pix];
            const float *g = dL_dimage + 3 * cam.pix_offset;
            dC0[k] = g[pix];
            dC1[k] = g[hw + pix];
            dC2[k] = g[2 * hw + pix];
        }
        local_max = max(local_max, my_last[k]);
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    if (local_max > 0) atomicMax(&s_max, local_max);
    __syncthreads();
    const int max_last = s_max;
    // S = sum_c dL/dC_c A_c (A_c: the colour behind the current contributor),
    // kept instead of the three A_c: dL/da_k needs no more, and the suffix
    // step A_c += c_c w adds (dL/dC . c) w to it
    float S[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k)
        S[k] = T_end[k] * (dC0[k] * cfg.bg[0] + dC1[k] * cfg.bg[1] + dC2[k] * cfg.bg[2]);

    for (int b = (max_last + BATCH - 1) / BATCH - 1; b >= 0; --b) {
        __syncthreads();
        const int64_t b0 = (int64_t)rg.x + (int64_t)b * BATCH;
        const int cnt = (int)min((int64_t)BATCH, (int64_t)rg.y - b0);
        if constexpr (COARSE) {  // the batch's indices from the list, from where the forward pass began it
            const int64_t slot = slot0 + b;
            uint32_t pos = slot < ckpt_slots ? ls.batch_pos[slot] : cend;
            coarse_gather<NTH, EPT>(ls, cbit, pos, cend, cnt, s_g, s_wsum, &s_next);
        }
        for (int kk = threadIdx.x; kk < BATCH; kk += NTH) {  // whole warps (BATCH, NTH multiples of 32)
            const bool valid = kk < cnt;
            float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra, rc = ra;
            if (valid) {
                const uint32_t g = COARSE ? s_g[kk] : ls.vals[b0 + kk];
                const float4 *r = recv + (int64_t)g * 3;
                ra = r[0];
                rb = r[1];
                rc = r[2];
                s_a[kk] = ra;
                s_b[kk] = rb;
                s_c[kk] = rc;
                s_g[kk] = g;
            }
            overlap_masks<TILE, PPT, NW, NWORD>(s_ov, kk, valid, ra, rb, rc, amin, tx * TILE, ty * TILE);
        }
        for (int kk = threadIdx.x; kk < BATCH * 9; kk += NTH) (&s_acc[0][0])[kk] = 0.f;
        __syncthreads();
        const int lo = b * BATCH;
        int jstart[PPT];
        float T[PPT];
        int jmax = -1;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            jstart[k] = -1;
            T[k] = 0.f;
            if (my_last[k] > lo + cnt) {
                jstart[k] = cnt - 1;
                const int64_t slot = slot0 + b + 1;
                T[k] = slot < ckpt_slots ? ckpt[slot * NT + lp[k]] : 0.f;
            } else if (my_last[k] > lo) {
                jstart[k] = my_last[k] - 1 - lo;
                T[k] = T_end[k];
            }
            jmax = max(jmax, jstart[k]);
        }
        const int wj = __reduce_max_sync(FULL, jmax);
        // the warp's marked records at or below wj, last to first
        for (int wd = wj >> 5; wj >= 0 && wd >= 0; --wd) {
          uint32_t m = s_ov[warp][wd];
          if (wd == (wj >> 5)) m &= (2u << (wj & 31)) - 1u;
          while (m) {
            const int bit = 31 - __clz(m);
            m &= ~(1u << bit);
            const int j = wd * 32 + bit;
            const float4 sa = s_a[j], sb = s_b[j], sc = s_c[j];
            float gv[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) gv[q] = 0.f;
            bool contrib = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (j > jstart[k]) continue;
                const AlphaEval ae = eval_alpha(sa, sb, px[k], py[k], amax);
                if (ae.alpha < amin) continue;
                contrib = true;
                const float om = __fsub_rn(1.f, ae.alpha);
                const float inv = rcp_approx(om);  // 1 - alpha >= 0.01
                const float Tk = T[k] * inv;
                const float wgt = ae.alpha * Tk;
                gv[6] += dC0[k] * wgt;
                gv[7] += dC1[k] * wgt;
                gv[8] += dC2[k] * wgt;
                const float dcc = dC0[k] * sb.z + dC1[k] * sb.w + dC2[k] * sc.x;  // dL/dC . c
                const float da = dcc * Tk - S[k] * inv;
                S[k] += dcc * wgt;
                T[k] = Tk;
                if (!ae.clamped) {
                    // dG = dL/da G = dL/d opacity; G dL/dG = o dG.  Per record
                    // the pixels sum dG z (z = U dp) and dG dp dp^T; the flush
                    // applies o, U^T (dL/d mean2D = o U^T sum dG z) and the
                    // conic factors -1/2, -1, -1/2 once per (Gaussian, tile)
                    const float dG = da * ae.G;
                    gv[5] += dG;
                    gv[0] += dG * ae.z0;
                    gv[1] += dG * ae.z1;
                    const float ex = dG * ae.dx, ey = dG * ae.dy;
                    gv[2] += ex * ae.dx;
                    gv[3] += ex * ae.dy;
                    gv[4] += ey * ae.dy;
                }
            }
            const uint32_t cm = __ballot_sync(FULL, contrib);
            if (__popc(cm) > kDirectLanes) {  // many lanes: reduce over the warp first
                int idx;
                const float tot = warp_reduce9(gv, lane, idx);
                if (idx >= 0 && tot != 0.f) atomicAdd(&s_acc[j][idx], tot);
            } else if (contrib) {  // a few lanes: their values go straight to shared memory
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    if (gv[q] != 0.f) atomicAdd(&s_acc[j][q], gv[q]);
            }
          }
        }
        __syncthreads();
        for (int kk = threadIdx.x; kk < cnt; kk += NTH) {
            const float *a = s_acc[kk];
            bool nz = false;
#pragma unroll
            for (int q = 0; q < 9; ++q) nz |= a[q] != 0.f;
            if (!nz) continue;
            // dL/d mean2D = o U^T sum dG z (U = [[u00, u01], [0, u11]] in
            // the record: a.z, a.w, b.x; o = b.y); dL/dQ = -o/2 sum dG dp dp^T
            const float4 ra = s_a[kk], rb = s_b[kk];
            const float o = rb.y, ho = -0.5f * o;
            float4 *dst = g2d + ((int64_t)v * n + s_g[kk]) * 3;
            atomicAdd(dst, make_float4(o * (ra.z * a[0]), o * (ra.w * a[0] + rb.x * a[1]), ho * a[2], -o * a[3]));
            atomicAdd(dst + 1, make_float4(ho * a[4], a[5], a[6], a[7]));
            atomicAdd(&dst[2].x, a[8]);
        }
    }
    }  // items
}

// Optimizer fused into the projection adjoint: the parameters live in one flat
// buffer (param_offsets) with Adam moments m, v in the same layout.
struct AdamFuse {
    float *p, *m, *v;
    int64_t o[6];
    gs_adam_config cfg;
    const int32_t *do_step;
    const int64_t *step;
    double *norms2;  // optional: sum of g^2 and of (p_new - p_old)^2 are added here
};

template <int DEG>
constexpr size_t proj_bwd_smem() { return sizeof(float) * 2 * ParamGroups<DEG>::TOT * PB; }

// Adam over the float4 chunks [0, C4) of a full warp's slice of group g:
// all m and v loads of the lane first, then the updates and stores; the
// lane's sums of g^2 and (p_new - p_old)^2 are added to ng and nd.
template <int DEG, int g, int C4>
__device__ __forceinline__ void adam_full(float *__restrict__ P, float *__restrict__ M, float *__restrict__ V,
                                          const float *sp, const float *sg, const float *lr_t, float ibc2,
                                          const gs_adam_config &cfg, int lane, float &ng, float &nd) {
    using G = ParamGroups<DEG>;
    constexpr int K3 = 3 * G::K;
    constexpr int J = (C4 + 31) / 32;
    float4 m4[J], v4[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int c = lane + j * 32;
        if (c < C4) {
            m4[j] = reinterpret_cast<const float4 *>(M)[c];
            v4[j] = reinterpret_cast<const float4 *>(V)[c];
        }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int c = lane + j * 32;
        if (c < C4) {
            float4 p4;
            float *pm = &m4[j].x, *pv = &v4[j].x, *pp = &p4.x;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = 4 * c + u;
                const int lr = g < 4 ? g : ((k % K3) < 3 ? 4 : 5);
                const int ks = G::pad(g, k);
                const float p0 = sp[ks], gk = sg[ks];
                float p = p0;
                adam_update(p, pm[u], pv[u], gk, lr_t[lr], cfg.beta1, cfg.beta2, ibc2, cfg.eps);
                pp[u] = p;
                ng += gk * gk;
                nd += (p - p0) * (p - p0);
            }
            reinterpret_cast<float4 *>(P)[c] = p4;
            reinterpret_cast<float4 *>(M)[c] = m4[j];
            reinterpret_cast<float4 *>(V)[c] = v4[j];
        }
    }
}

// Projection adjoint, staged through shared memory one warp at a time: each
// warp copies the parameter slices of its WG = 32 Gaussians (contiguous in
// every group) into its own shared region with coalesced loads; each lane
// chains its Gaussian's 2D gradients (all views) to parameter gradients,
// accumulated in its own shared slots; the warp then sweeps its slices again,
// coalesced, to store the gradients (MODE 0 overwrite, 1 add) or to apply
// Adam (MODE 2) without ever storing them.  Warps synchronise only among
// their own lanes, so one warp's sweep overlaps another's chain rule.
constexpr int WG = 32;

template <int DEG, int MODE>
__global__ void __launch_bounds__(PB) proj_bwd_kernel(gs_params prm, const gs_camera *__restrict__ cams, int n_views,
                                                      const uint8_t *__restrict__ view_gate, gs_raster_config cfg,
                                                      const float4 *__restrict__ g2d, gs_grads gr, AdamFuse af) {
    using G = ParamGroups<DEG>;
    constexpr int K = G::K;
    extern __shared__ float smem[];
    __shared__ float s_lr[6];
    __shared__ float s_ibc2;
    __shared__ gs_camera s_cams[kStagedViews];
    if constexpr (MODE == 2) {
        if (af.do_step && *af.do_step == 0) return;  // the same for every block
        if (threadIdx.x == 0) adam_scalars(af.cfg, *af.step, af.do_step, s_lr, &s_ibc2);
    }
    if (threadIdx.x < n_views && threadIdx.x < kStagedViews) s_cams[threadIdx.x] = cams[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t n = prm.n;
    const int64_t i0 = (int64_t)blockIdx.x * PB + WG * (threadIdx.x >> 5);
    float ng = 0.f, nd = 0.f;  // MODE 2: this lane's sums of g^2 and (p_new - p_old)^2
    // the warp's work; a return ends this warp's part, not the block
    [&]() {
    if (i0 >= n) return;
    const int nb = (int)min((int64_t)WG, n - i0);
    float *s_par = smem + (threadIdx.x >> 5) * 2 * G::TOT * WG;  // [TOT * WG], group-major slices
    float *s_grd = s_par + G::TOT * WG;                           // same layout
    if constexpr (MODE == 2) {
        // A full warp asks L2 for its Adam moments (and its 2D gradients) up
        // front, so that the HBM reads of the final sweep overlap the chain
        // rule instead of following it.  Slices are 16-byte aligned: group
        // offsets are 64-float aligned and i0 is a multiple of WG.
        if (nb == WG) {
            if (lane < 10) {
                const int g = lane >> 1;  // selects, not an indexed parameter array (no local copy)
                const int64_t og = g == 0 ? af.o[0] : g == 1 ? af.o[1] : g == 2 ? af.o[2] : g == 3 ? af.o[3] : af.o[4];
                const int sg = g < 2 ? 3 : g == 2 ? 4 : g == 3 ? 1 : 3 * K;
                const float *base = (lane & 1) ? af.v : af.m;
                prefetch_l2(base + og + (int64_t)sg * i0, (uint32_t)(sizeof(float) * sg * WG));
            }
            for (int v = lane - 10; v >= 0 && v < n_views; v += 22)
                if (!view_gate || view_gate[v]) prefetch_l2(g2d + ((int64_t)v * n + i0) * 3, (uint32_t)(3 * sizeof(float4) * WG));
        }
    }
    const float *src[5] = {prm.means, prm.log_scales, prm.quats, prm.opacity_logit, prm.sh};
    if (nb == WG) {
        stage_group_full<DEG, WG>(src, i0, s_par, lane);
    } else {
        stage_group_partial<DEG, WG>(src, i0, nb, s_par, lane);
    }
    for (int k = lane; k < G::TOT * WG / 4; k += 32) reinterpret_cast<float4 *>(s_grd)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();

    const int t = lane;
    if (t < nb) {
        const int64_t i = i0 + t;
        const float *P0 = s_par + G::off(0, WG) + G::P(0) * t;
        const float *P1 = s_par + G::off(1, WG) + G::P(1) * t;
        const float *P2 = s_par + G::off(2, WG) + G::P(2) * t;
        const float logit = s_par[G::off(3, WG) + G::P(3) * t];
        const float *f = s_par + G::off(4, WG) + G::P(4) * t;
        float *D0 = s_grd + G::off(0, WG) + G::P(0) * t;
        float *D1 = s_grd + G::off(1, WG) + G::P(1) * t;
        float *D2 = s_grd + G::off(2, WG) + G::P(2) * t;
        float *D3 = s_grd + G::off(3, WG) + G::P(3) * t;
        float *DF = s_grd + G::off(4, WG) + G::P(4) * t;
        const float mu[3] = {P0[0], P0[1], P0[2]};
        const float ls[3] = {P1[0], P1[1], P1[2]};
        const float4 q4 = make_float4(P2[0], P2[1], P2[2], P2[3]);
        for (int v = 0; v < n_views; ++v) {
            if (view_gate && !view_gate[v]) continue;
            const float4 *gp = g2d + ((int64_t)v * n + i) * 3;
            const float4 ga = gp[0], gb = gp[1];
            const float gc = gp[2].x;
            const float gd[9] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w, gc};
            bool nz = false;
#pragma unroll
            for (int q = 0; q < 9; ++q) nz |= gd[q] != 0.f;
            if (!nz) continue;
            const gs_camera &c = v < kStagedViews ? s_cams[v] : cams[v];
            ProjState g;
            project_state(mu, ls, q4, logit, c, cfg.lowpass, g);
            if (g.culled) continue;
            // opacity = sigmoid(logit)
            D3[0] += gd[5] * g.o * (1.f - g.o);
            // colour = max(0, sum_k f_k Y_k(d) + 0.5), d = (mu - campos) / |mu - campos|
            float cp[3];
            cam_center(c, cp);
            const float dv[3] = {mu[0] - cp[0], mu[1] - cp[1], mu[2] - cp[2]};
            const float inv_n = 1.0f / sqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
            const float d[3] = {dv[0] * inv_n, dv[1] * inv_n, dv[2] * inv_n};
            float Y[16], dY[16][3];
            sh_basis(DEG, d[0], d[1], d[2], Y);
            sh_basis_grad(DEG, d[0], d[1], d[2], dY);
            float ddir[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float pre = 0.5f;
#pragma unroll
                for (int k = 0; k < K; ++k) pre += f[3 * k + ch] * Y[k];
                if (!(pre > 0.f)) continue;
                const float dc = gd[6 + ch];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    DF[3 * k + ch] += dc * Y[k];
                    const float fk = f[3 * k + ch] * dc;
                    ddir[0] += fk * dY[k][0];
                    ddir[1] += fk * dY[k][1];
                    ddir[2] += fk * dY[k][2];
                }
            }
            float dmu[3];
            const float dd = ddir[0] * d[0] + ddir[1] * d[1] + ddir[2] * d[2];
#pragma unroll
            for (int a = 0; a < 3; ++a) dmu[a] = (ddir[a] - d[a] * dd) * inv_n;
            // conic Q = Sigma2D^-1 -> dL/dSigma2D = -Q GQ Q (full symmetric matrices)
            const float idet = 1.f / g.det;
            const float Qa = g.s11 * idet, Qb = -g.s01 * idet, Qc = g.s00 * idet;
            const float Ga = gd[2], Gb = 0.5f * gd[3], Gc = gd[4];
            const float t00 = Ga * Qa + Gb * Qb, t01 = Ga * Qb + Gb * Qc;
            const float t10 = Gb * Qa + Gc * Qb, t11 = Gb * Qb + Gc * Qc;
            const float S00 = -(Qa * t00 + Qb * t10), S01 = -(Qa * t01 + Qb * t11), S11 = -(Qb * t01 + Qc * t11);
            // Sigma2D = M M^T + l I -> dL/dM = 2 S M
            float dM[6];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                dM[k] = 2.f * (S00 * g.M[k] + S01 * g.M[3 + k]);
                dM[3 + k] = 2.f * (S01 * g.M[k] + S11 * g.M[3 + k]);
            }
            // M = T R S: dT = dM (R S)^T, Gp = T^T dM, dR_jk = Gp_jk s_k, ds_k = sum_j Gp_jk R_jk
            float dT[6];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    dT[3 * r + j] = dM[3 * r] * g.R[3 * j] * g.s[0] + dM[3 * r + 1] * g.R[3 * j + 1] * g.s[1] +
                                    dM[3 * r + 2] * g.R[3 * j + 2] * g.s[2];
            float dR[9];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) dR[3 * j + k] = (g.T[j] * dM[k] + g.T[3 + j] * dM[3 + k]) * g.s[k];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float ds = 0.f;
#pragma unroll
                for (int j = 0; j < 3; ++j) ds += (g.T[j] * dM[k] + g.T[3 + j] * dM[3 + k]) * g.R[3 * j + k];
                D1[k] += ds * g.s[k];
            }
            // T = J W: dJ = dT W^T (only J00, J02, J11, J12 are non-zero)
            const float dJ00 = dT[0] * c.R[0] + dT[1] * c.R[1] + dT[2] * c.R[2];
            const float dJ02 = dT[0] * c.R[6] + dT[1] * c.R[7] + dT[2] * c.R[8];
            const float dJ11 = dT[3] * c.R[3] + dT[4] * c.R[4] + dT[5] * c.R[5];
            const float dJ12 = dT[3] * c.R[6] + dT[4] * c.R[7] + dT[5] * c.R[8];
            const float z = g.p[2], iz = 1.f / z, iz2 = iz * iz;
            float dp[3] = {0.f, 0.f, 0.f};
            dp[2] += -dJ00 * c.fx * iz2 - dJ11 * c.fy * iz2;
            if (g.clamp_x == 0) {
                dp[0] += -dJ02 * c.fx * iz2;
                dp[2] += dJ02 * 2.f * c.fx * g.txz * iz2;
            } else {
                dp[2] += dJ02 * c.fx * g.txz * iz2;
            }
            if (g.clamp_y == 0) {
                dp[1] += -dJ12 * c.fy * iz2;
                dp[2] += dJ12 * 2.f * c.fy * g.tyz * iz2;
            } else {
                dp[2] += dJ12 * c.fy * g.tyz * iz2;
            }
            // mean2D = (fx x/z + cx, fy y/z + cy)
            dp[0] += gd[0] * c.fx * iz;
            dp[1] += gd[1] * c.fy * iz;
            dp[2] += -(gd[0] * c.fx * g.p[0] + gd[1] * c.fy * g.p[1]) * iz2;
            // p = W mu + t
#pragma unroll
            for (int a = 0; a < 3; ++a) D0[a] += dmu[a] + c.R[a] * dp[0] + c.R[3 + a] * dp[1] + c.R[6 + a] * dp[2];
            // R(qn): partial derivatives of the rotation matrix entries
            const float w = g.qn[0], qx = g.qn[1], qy = g.qn[2], qz = g.qn[3];
            float dqn[4];
            dqn[0] = 2.f * (-qz * dR[1] + qy * dR[2] + qz * dR[3] - qx * dR[5] - qy * dR[6] + qx * dR[7]);
            dqn[1] = 2.f * (qy * dR[1] + qz * dR[2] + qy * dR[3] - 2.f * qx * dR[4] - w * dR[5] + qz * dR[6] + w * dR[7] -
                            2.f * qx * dR[8]);
            dqn[2] = 2.f * (-2.f * qy * dR[0] + qx * dR[1] + w * dR[2] + qx * dR[3] + qz * dR[5] - w * dR[6] +
                            qz * dR[7] - 2.f * qy * dR[8]);
            dqn[3] = 2.f * (-2.f * qz * dR[0] - w * dR[1] + qx * dR[2] + w * dR[3] - 2.f * qz * dR[4] + qy * dR[5] +
                            qx * dR[6] + qy * dR[7]);
            const float qd = dqn[0] * w + dqn[1] * qx + dqn[2] * qy + dqn[3] * qz;
#pragma unroll
            for (int a = 0; a < 4; ++a) D2[a] += (dqn[a] - g.qn[a] * qd) * g.qinv;
        }
    }
    __syncwarp();
    // coalesced sweep over the warp's slices
    if constexpr (MODE == 2) {
        const float ibc2 = s_ibc2;
        if (nb == WG) {
            adam_full<DEG, 0, 3 * WG / 4>(af.p + af.o[0] + 3 * i0, af.m + af.o[0] + 3 * i0, af.v + af.o[0] + 3 * i0,
                                         s_par + G::off(0, WG), s_grd + G::off(0, WG), s_lr, ibc2, af.cfg, lane, ng, nd);
            adam_full<DEG, 1, 3 * WG / 4>(af.p + af.o[1] + 3 * i0, af.m + af.o[1] + 3 * i0, af.v + af.o[1] + 3 * i0,
                                         s_par + G::off(1, WG), s_grd + G::off(1, WG), s_lr, ibc2, af.cfg, lane, ng, nd);
            adam_full<DEG, 2, WG>(af.p + af.o[2] + 4 * i0, af.m + af.o[2] + 4 * i0, af.v + af.o[2] + 4 * i0,
                                  s_par + G::off(2, WG), s_grd + G::off(2, WG), s_lr, ibc2, af.cfg, lane, ng, nd);
            adam_full<DEG, 3, WG / 4>(af.p + af.o[3] + i0, af.m + af.o[3] + i0, af.v + af.o[3] + i0,
                                      s_par + G::off(3, WG), s_grd + G::off(3, WG), s_lr, ibc2, af.cfg, lane, ng, nd);
            const int64_t o4 = af.o[4] + (int64_t)3 * K * i0;
            adam_full<DEG, 4, 3 * K * WG / 4>(af.p + o4, af.m + o4, af.v + o4, s_par + G::off(4, WG),
                                              s_grd + G::off(4, WG), s_lr, ibc2, af.cfg, lane, ng, nd);
            return;
        }
#pragma unroll
        for (int g = 0; g < 5; ++g) {
            const int cnt = G::S(g) * nb;
            const int64_t e0 = af.o[g] + (int64_t)G::S(g) * i0;
            const float *sp = s_par + G::off(g, WG);
            const float *sg = s_grd + G::off(g, WG);
            // float4 chunks (e0 is 16-byte aligned: group offsets are 64-float aligned, i0 a multiple of WG)
            const int cnt4 = cnt >> 2;
            float4 *P4 = reinterpret_cast<float4 *>(af.p + e0);
            float4 *M4 = reinterpret_cast<float4 *>(af.m + e0);
            float4 *V4 = reinterpret_cast<float4 *>(af.v + e0);
#pragma unroll 2
            for (int c = lane; c < cnt4; c += 32) {
                float4 m4 = M4[c], v4 = V4[c], p4;
                float *pm = &m4.x, *pv = &v4.x, *pp4 = &p4.x;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = 4 * c + u;
                    const int lr = g < 4 ? g : ((k % (3 * K)) < 3 ? 4 : 5);
                    const int ks = G::pad(g, k);
                    const float p0 = sp[ks], gk = sg[ks];
                    float p = p0;
                    adam_update(p, pm[u], pv[u], gk, s_lr[lr], af.cfg.beta1, af.cfg.beta2, ibc2, af.cfg.eps);
                    pp4[u] = p;
                    ng += gk * gk;
                    nd += (p - p0) * (p - p0);
                }
                P4[c] = p4;
                M4[c] = m4;
                V4[c] = v4;
            }
            for (int k = 4 * cnt4 + lane; k < cnt; k += 32) {
                const int lr = g < 4 ? g : ((k % (3 * K)) < 3 ? 4 : 5);
                const int ks = G::pad(g, k);
                const float p0 = sp[ks], gk = sg[ks];
                float p = p0, m = af.m[e0 + k], v = af.v[e0 + k];
                adam_update(p, m, v, gk, s_lr[lr], af.cfg.beta1, af.cfg.beta2, ibc2, af.cfg.eps);
                ng += gk * gk;
                nd += (p - p0) * (p - p0);
                af.p[e0 + k] = p;
                af.m[e0 + k] = m;
                af.v[e0 + k] = v;
            }
        }

    } else {
        float *dst[5] = {gr.means, gr.log_scales, gr.quats, gr.opacity_logit, gr.sh};
#pragma unroll
        for (int g = 0; g < 5; ++g) {
            const int cnt = G::S(g) * nb;
            float *dp = dst[g] + (int64_t)G::S(g) * i0;
            const float *sg = s_grd + G::off(g, WG);
            for (int k = lane; k < cnt; k += 32) {
                if constexpr (MODE == 1) dp[k] += sg[G::pad(g, k)];
                else dp[k] = sg[G::pad(g, k)];
            }
        }
    }
    }();
    if constexpr (MODE == 2) {
        if (af.norms2) {  // block sums, one double atomic per block and quantity
            __shared__ float s_red[2][PB / 32];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                ng += __shfl_xor_sync(0xffffffffu, ng, off);
                nd += __shfl_xor_sync(0xffffffffu, nd, off);
            }
            if (lane == 0) {
                s_red[0][threadIdx.x >> 5] = ng;
                s_red[1][threadIdx.x >> 5] = nd;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double a = 0.0, b = 0.0;
                for (int w = 0; w < PB / 32; ++w) {
                    a += s_red[0][w];
                    b += s_red[1][w];
                }
                atomicAdd(af.norms2, a);
                atomicAdd(af.norms2 + 1, b);
            }
        }
    }
}

template <int TILE, int PPT, bool CO>
using BwdKernel = decltype(&render_bwd_kernel<TILE, 64, PPT, CO>);

template <int TILE, int PPT, bool CO>
BwdKernel<TILE, PPT, CO> bwd_kernel(int batch) {
    switch (batch) {
        case 64: return render_bwd_kernel<TILE, 64, PPT, CO>;
        case 128: return render_bwd_kernel<TILE, 128, PPT, CO>;
        case 256: return render_bwd_kernel<TILE, 256, PPT, CO>;
        default: return nullptr;
    }
}

template <int TILE, int PPT, bool CO>
gs_status launch_bwd(int batch, int64_t total_tiles, cudaStream_t stream, const float4 *rec, int64_t n,
                     const ListSrc &ls, const uint2 *ranges, const gs_camera *cams, int n_views,
                     const gs_raster_config &cfg, gs_fwd_saved s, const float *dL, const uint8_t *gate, float4 *g2d) {
    const auto kernel = bwd_kernel<TILE, PPT, CO>(batch);
    if (!kernel) return GS_ERR_UNSUPPORTED;
    dim3 grid((unsigned)total_tiles);
    constexpr int NTH = TILE * TILE / PPT;
    if (s.queue) {  // persistent: the resident blocks (cached per device and staging batch size)
        static int resident[3][kMaxDevices] = {};
        const int bi = batch == 64 ? 0 : (batch == 128 ? 1 : 2);
        const int dev = cached_device_index();
        if (dev < 0) return GS_ERR_UNSUPPORTED;
        if (resident[bi][dev] <= 0) {
            int per_sm = 0;
            GS_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NTH, 0));
            resident[bi][dev] = (per_sm > 0 ? per_sm : 1) * device_sm_count();
        }
        if ((int64_t)resident[bi][dev] < total_tiles) grid = dim3((unsigned)resident[bi][dev]);
        GS_TRY(cudaMemsetAsync(s.queue, 0, sizeof(uint32_t), stream));
    }
    kernel<<<grid, NTH, 0, stream>>>(rec, n, ls, ranges, cams, n_views, cfg, s.T_final, s.n_last, s.ckpt, s.ckpt_slots,
                                     dL, gate, g2d, s.tile_order, s.queue, total_tiles);
    GS_TRY_LAUNCH();
    return GS_OK;
}

template <int TILE, bool CO>
gs_status launch_bwd_ppt(int ppt, int batch, int64_t total_tiles, cudaStream_t stream, const float4 *rec, int64_t n,
                         const ListSrc &ls, const uint2 *ranges, const gs_camera *cams, int n_views,
                         const gs_raster_config &cfg, gs_fwd_saved s, const float *dL, const uint8_t *gate,
                         float4 *g2d) {
    if constexpr (TILE >= 16)
        if (ppt == 4) return launch_bwd<TILE, 4, CO>(batch, total_tiles, stream, rec, n, ls, ranges, cams, n_views, cfg, s, dL, gate, g2d);
    if (ppt == 2) return launch_bwd<TILE, 2, CO>(batch, total_tiles, stream, rec, n, ls, ranges, cams, n_views, cfg, s, dL, gate, g2d);
    return launch_bwd<TILE, 1, CO>(batch, total_tiles, stream, rec, n, ls, ranges, cams, n_views, cfg, s, dL, gate, g2d);
}

template <int DEG, int MODE>
gs_status launch_proj_bwd_mode(unsigned blocks, cudaStream_t stream, const gs_params &prm, const gs_camera *cams,
                               int n_views, const uint8_t *gate, const gs_raster_config &cfg, const float4 *g2d,
                               const gs_grads &gr, const AdamFuse &af) {
    constexpr size_t smem = proj_bwd_smem<DEG>();
    static bool attr_set[kMaxDevices] = {};  // the shared-memory limit is raised once per device
    const int dev = cached_device_index();
    if (dev < 0) return GS_ERR_UNSUPPORTED;
    if (!attr_set[dev]) {
        GS_TRY(cudaFuncSetAttribute(proj_bwd_kernel<DEG, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set[dev] = true;
    }
    proj_bwd_kernel<DEG, MODE><<<blocks, PB, smem, stream>>>(prm, cams, n_views, gate, cfg, g2d, gr, af);
    GS_TRY_LAUNCH();
    return GS_OK;
}

template <int DEG>
gs_status launch_proj_bwd(int mode, unsigned blocks, cudaStream_t stream, const gs_params &prm, const gs_camera *cams,
                          int n_views, const uint8_t *gate, const gs_raster_config &cfg, const float4 *g2d,
                          const gs_grads &gr, const AdamFuse &af) {
    switch (mode) {
        case 0: return launch_proj_bwd_mode<DEG, 0>(blocks, stream, prm, cams, n_views, gate, cfg, g2d, gr, af);
        case 1: return launch_proj_bwd_mode<DEG, 1>(blocks, stream, prm, cams, n_views, gate, cfg, g2d, gr, af);
        default: return launch_proj_bwd_mode<DEG, 2>(blocks, stream, prm, cams, n_views, gate, cfg, g2d, gr, af);
    }
}

__global__ void adam_step_count_kernel(const int32_t *do_step, int64_t *step) {
    if (!do_step || *do_step) *step += 1;
}

// The staged projection adjoint reads every parameter group with 16-byte loads.
bool proj_params_aligned(const gs_params &p) {
    return !(((uintptr_t)p.means | (uintptr_t)p.log_scales | (uintptr_t)p.quats | (uintptr_t)p.opacity_logit |
              (uintptr_t)p.sh) & 15);
}

// Raster adjoint: zero the per-view 2D gradient buffer, then one CTA per tile
// (tile lists, or super-tile lists when coarse).
gs_status raster_bwd_impl(int64_t n, const gs_projected *proj, const ListSrc &ls, bool coarse,
                          const uint32_t *ranges, const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                          const gs_raster_config *cfg, gs_fwd_saved saved, const float *dL_dimage,
                          const uint8_t *view_gate, float4 *g2d, cudaStream_t stream) {
    const int ppt = cfg->pixels_per_thread, b = cfg->batch;
    if (ppt != 1 && ppt != 2 && ppt != 4) return GS_ERR_INVALID_ARG;
    if (ppt == 4 && cfg->tile < 16) return GS_ERR_INVALID_ARG;  // a warp needs 8 x 16 pixels
    if (b != 64 && b != 128 && b != 256) return GS_ERR_UNSUPPORTED;
    if (cfg->tile != 8 && cfg->tile != 16 && cfg->tile != 32) return GS_ERR_INVALID_ARG;
    GS_TRY(cudaMemsetAsync(g2d, 0, sizeof(float) * kG2d * (size_t)n * n_views, stream));
    const float4 *rec = reinterpret_cast<const float4 *>(proj->rec);
    const uint2 *rg = reinterpret_cast<const uint2 *>(ranges);
    switch (cfg->tile * 2 + (coarse ? 1 : 0)) {
        case 16: return launch_bwd_ppt<8, false>(ppt, b, total_tiles, stream, rec, n, ls, rg, cams, n_views, *cfg, saved, dL_dimage, view_gate, g2d);
        case 17: return launch_bwd_ppt<8, true>(ppt, b, total_tiles, stream, rec, n, ls, rg, cams, n_views, *cfg, saved, dL_dimage, view_gate, g2d);
        case 32: return launch_bwd_ppt<16, false>(ppt, b, total_tiles, stream, rec, n, ls, rg, cams, n_views, *cfg, saved, dL_dimage, view_gate, g2d);
        case 33: return launch_bwd_ppt<16, true>(ppt, b, total_tiles, stream, rec, n, ls, rg, cams, n_views, *cfg, saved, dL_dimage, view_gate, g2d);
        case 64: return launch_bwd_ppt<32, false>(ppt, b, total_tiles, stream, rec, n, ls, rg, cams, n_views, *cfg, saved, dL_dimage, view_gate, g2d);
        default: return launch_bwd_ppt<32, true>(ppt, b, total_tiles, stream, rec, n, ls, rg, cams, n_views, *cfg, saved, dL_dimage, view_gate, g2d);
    }
}

// Projection adjoint (MODE from `fused` / `accumulate`), then the step count when fused.
template <bool FUSED>
gs_status project_bwd_impl(const gs_params *params, const gs_camera *cams, int32_t n_views,
                           const gs_raster_config *cfg, const float4 *g2d, const uint8_t *view_gate, gs_grads grads,
                           int32_t accumulate, const AdamFuse &af, cudaStream_t stream) {
    const int64_t n = params->n;
    const unsigned blocks = (unsigned)ceil_div(n, PB);
    const int mode = FUSED ? 2 : (accumulate ? 1 : 0);
    gs_status st;
    switch (params->sh_degree) {
        case 0: st = launch_proj_bwd<0>(mode, blocks, stream, *params, cams, n_views, view_gate, *cfg, g2d, grads, af); break;
        case 1: st = launch_proj_bwd<1>(mode, blocks, stream, *params, cams, n_views, view_gate, *cfg, g2d, grads, af); break;
        case 2: st = launch_proj_bwd<2>(mode, blocks, stream, *params, cams, n_views, view_gate, *cfg, g2d, grads, af); break;
        default: st = launch_proj_bwd<3>(mode, blocks, stream, *params, cams, n_views, view_gate, *cfg, g2d, grads, af); break;
    }
    if (st != GS_OK) return st;
    if constexpr (FUSED) {
        adam_step_count_kernel<<<1, 1, 0, stream>>>(af.do_step, const_cast<int64_t *>(af.step));
        GS_TRY_LAUNCH();
    }
    return GS_OK;
}

template <bool FUSED>
gs_status render_bwd_impl(const gs_params *params, const gs_projected *proj, const ListSrc &ls, bool coarse,
                          const uint32_t *ranges, const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                          const gs_raster_config *cfg, gs_fwd_saved saved, const float *dL_dimage,
                          const uint8_t *view_gate, gs_grads grads, int32_t accumulate, const AdamFuse &af,
                          void *workspace, cudaStream_t stream) {
    float4 *g2d = reinterpret_cast<float4 *>(workspace);
    gs_status st = raster_bwd_impl(params->n, proj, ls, coarse, ranges, cams, n_views, total_tiles, cfg, saved,
                                   dL_dimage, view_gate, g2d, stream);
    if (st != GS_OK) return st;
    return project_bwd_impl<FUSED>(params, cams, n_views, cfg, g2d, view_gate, grads, accumulate, af, stream);
}

}  // namespace

extern "C" {

size_t gs_render_bwd_workspace_size(int64_t n, int32_t n_views) {
    if (n < 0 || n_views <= 0) return 0;
    return sizeof(float) * kG2d * (size_t)(n > 0 ? n : 1) * (size_t)n_views;
}

}  // extern "C"

namespace {

gs_status render_bwd_entry(const gs_params *params, const gs_projected *proj, const ListSrc &ls, bool coarse,
                           const uint32_t *ranges, const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                           const gs_raster_config *cfg, gs_fwd_saved saved, const float *dL_dimage,
                           const uint8_t *view_gate, gs_grads grads, int32_t accumulate, void *workspace,
                           size_t workspace_bytes, cudaStream_t stream) {
    if (!params || !proj || !cfg || !cams || !ranges || !dL_dimage || n_views <= 0 || total_tiles <= 0)
        return GS_ERR_INVALID_ARG;
    if (params->n < 0 || params->n >= ((int64_t)1 << 31) || params->sh_degree < 0 || params->sh_degree > 3 ||
        cfg->sh_degree != params->sh_degree)
        return GS_ERR_INVALID_ARG;
    if (!saved.T_final || !saved.n_last || !saved.ckpt || saved.ckpt_slots <= 0) return GS_ERR_INVALID_ARG;
    if (!grads.means || !grads.log_scales || !grads.quats || !grads.opacity_logit || !grads.sh) return GS_ERR_INVALID_ARG;
    if (!proj_params_aligned(*params) || ((uintptr_t)proj->rec & 15)) return GS_ERR_INVALID_ARG;
    const int64_t n = params->n;
    if (!workspace || workspace_bytes < gs_render_bwd_workspace_size(n, n_views)) return GS_ERR_WORKSPACE;
    if ((uintptr_t)workspace & 15) return GS_ERR_WORKSPACE;
    if (n == 0) return GS_OK;
    AdamFuse af{};
    return render_bwd_impl<false>(params, proj, ls, coarse, ranges, cams, n_views, total_tiles, cfg, saved,
                                  dL_dimage, view_gate, grads, accumulate, af, workspace, stream);
}

gs_status raster_bwd_entry(const gs_projected *proj, int64_t n, const ListSrc &ls, bool coarse,
                           const uint32_t *ranges, const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                           const gs_raster_config *cfg, gs_fwd_saved saved, const float *dL_dimage,
                           const uint8_t *view_gate, float *g2d, size_t g2d_bytes, cudaStream_t stream) {
    if (!proj || !cfg || !cams || !ranges || !dL_dimage || n_views <= 0 || total_tiles <= 0 || n < 0 ||
        n >= ((int64_t)1 << 31))
        return GS_ERR_INVALID_ARG;
    if (!saved.T_final || !saved.n_last || !saved.ckpt || saved.ckpt_slots <= 0) return GS_ERR_INVALID_ARG;
    if ((uintptr_t)proj->rec & 15) return GS_ERR_INVALID_ARG;
    if (!g2d || g2d_bytes < gs_render_bwd_workspace_size(n, n_views) || ((uintptr_t)g2d & 15)) return GS_ERR_WORKSPACE;
    if (n == 0) return GS_OK;
    return raster_bwd_impl(n, proj, ls, coarse, ranges, cams, n_views, total_tiles, cfg, saved, dL_dimage, view_gate,
                           reinterpret_cast<float4 *>(g2d), stream);
}

}  // namespace

extern "C" {

gs_status gs_render_bwd(const gs_params *params, const gs_projected *proj, const uint32_t *vals,
                        const uint32_t *ranges, const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                        const gs_raster_config *cfg, gs_fwd_saved saved, const float *dL_dimage,
                        const uint8_t *view_gate, gs_grads grads, int32_t accumulate, void *workspace,
                        size_t workspace_bytes, int32_t *dev_status, cudaStream_t stream) {
    (void)dev_status;
    if (!vals) return GS_ERR_INVALID_ARG;
    ListSrc ls{};
    ls.vals = vals;
    return render_bwd_entry(params, proj, ls, false, ranges, cams, n_views, total_tiles, cfg, saved, dL_dimage,
                            view_gate, grads, accumulate, workspace, workspace_bytes, stream);
}

gs_status gs_render_bwd_coarse(const gs_params *params, const gs_projected *proj, const gs_coarse_lists *lists,
                               const uint32_t *ranges, const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                               const gs_raster_config *cfg, gs_fwd_saved saved, const float *dL_dimage,
                               const uint8_t *view_gate, gs_grads grads, int32_t accumulate, void *workspace,
                               size_t workspace_bytes, int32_t *dev_status, cudaStream_t stream) {
    (void)dev_status;
    ListSrc ls{};
    const gs_status st = coarse_src(lists, saved, ls);
    if (st != GS_OK) return st;
    return render_bwd_entry(params, proj, ls, true, ranges, cams, n_views, total_tiles, cfg, saved, dL_dimage,
                            view_gate, grads, accumulate, workspace, workspace_bytes, stream);
}

gs_status gs_raster_bwd(const gs_projected *proj, int64_t n, const uint32_t *vals, const uint32_t *ranges,
                        const gs_camera *cams, int32_t n_views, int64_t total_tiles, const gs_raster_config *cfg,
                        gs_fwd_saved saved, const float *dL_dimage, const uint8_t *view_gate, float *g2d,
                        size_t g2d_bytes, int32_t *dev_status, cudaStream_t stream) {
    (void)dev_status;
    if (!vals) return GS_ERR_INVALID_ARG;
    ListSrc ls{};
    ls.vals = vals;
    return raster_bwd_entry(proj, n, ls, false, ranges, cams, n_views, total_tiles, cfg, saved, dL_dimage, view_gate,
                            g2d, g2d_bytes, stream);
}

gs_status gs_raster_bwd_coarse(const gs_projected *proj, int64_t n, const gs_coarse_lists *lists,
                               const uint32_t *ranges, const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                               const gs_raster_config *cfg, gs_fwd_saved saved, const float *dL_dimage,
                               const uint8_t *view_gate, float *g2d, size_t g2d_bytes, int32_t *dev_status,
                               cudaStream_t stream) {
    (void)dev_status;
    ListSrc ls{};
    const gs_status st = coarse_src(lists, saved, ls);
    if (st != GS_OK) return st;
    return raster_bwd_entry(proj, n, ls, true, ranges, cams, n_views, total_tiles, cfg, saved, dL_dimage, view_gate,
                            g2d, g2d_bytes, stream);
}

gs_status gs_project_bwd(const gs_params *params, const gs_camera *cams, int32_t n_views, const gs_raster_config *cfg,
                         const float *g2d, const uint8_t *view_gate, gs_grads grads, int32_t accumulate,
                         int32_t *dev_status, cudaStream_t stream) {
    (void)dev_status;
    if (!params || !cams || !cfg || !g2d || n_views <= 0) return GS_ERR_INVALID_ARG;
    if (params->n < 0 || params->n >= ((int64_t)1 << 31) || params->sh_degree < 0 || params->sh_degree > 3 ||
        cfg->sh_degree != params->sh_degree)
        return GS_ERR_INVALID_ARG;
    if (!grads.means || !grads.log_scales || !grads.quats || !grads.opacity_logit || !grads.sh) return GS_ERR_INVALID_ARG;
    if ((uintptr_t)g2d & 15) return GS_ERR_INVALID_ARG;
    if (params->n == 0) return GS_OK;
    if (!proj_params_aligned(*params)) return GS_ERR_INVALID_ARG;
    AdamFuse af{};
    return project_bwd_impl<false>(params, cams, n_views, cfg, reinterpret_cast<const float4 *>(g2d), view_gate,
                                   grads, accumulate, af, stream);
}

// The flat-buffer view of the parameters and the fused Adam arguments.
static gs_status fused_args(float *flat_params, float *m, float *v, int64_t n, int32_t sh_degree,
                            const gs_raster_config *cfg, const gs_adam_config *adam, const int32_t *dev_do_step,
                            int64_t *dev_step, double *norms2, gs_params *prm, AdamFuse *af) {
    if (!flat_params || !m || !v || !adam || !dev_step || n < 0 || n >= ((int64_t)1 << 31) || sh_degree < 0 ||
        sh_degree > 3 || cfg == nullptr || cfg->sh_degree != sh_degree)
        return GS_ERR_INVALID_ARG;
    if (((uintptr_t)flat_params | (uintptr_t)m | (uintptr_t)v) & 15) return GS_ERR_INVALID_ARG;
    if (!(adam->beta1 >= 0.f && adam->beta1 < 1.f && adam->beta2 >= 0.f && adam->beta2 < 1.f && adam->eps >= 0.f))
        return GS_ERR_INVALID_ARG;
    *af = AdamFuse{};
    af->p = flat_params;
    af->m = m;
    af->v = v;
    param_offsets(n, sh_degree, af->o);
    af->cfg = *adam;
    af->do_step = dev_do_step;
    af->step = dev_step;
    af->norms2 = norms2;
    prm->means = flat_params + af->o[0];
    prm->log_scales = flat_params + af->o[1];
    prm->quats = flat_params + af->o[2];
    prm->opacity_logit = flat_params + af->o[3];
    prm->sh = flat_params + af->o[4];
    prm->n = n;
    prm->sh_degree = sh_degree;
    return GS_OK;
}

}  // extern "C"

static gs_status render_bwd_adam_entry(float *flat_params, float *m, float *v, int64_t n, int32_t sh_degree,
                                       const gs_projected *proj, const ListSrc &ls, bool coarse,
                                       const uint32_t *ranges, const gs_camera *cams, int32_t n_views,
                                       int64_t total_tiles, const gs_raster_config *cfg, gs_fwd_saved saved,
                                       const float *dL_dimage, const uint8_t *view_gate, const gs_adam_config *adam,
                                       const int32_t *dev_do_step, int64_t *dev_step, double *norms2,
                                       void *workspace, size_t workspace_bytes, cudaStream_t stream) {
    gs_params prm;
    AdamFuse af;
    gs_status st = fused_args(flat_params, m, v, n, sh_degree, cfg, adam, dev_do_step, dev_step, norms2, &prm, &af);
    if (st != GS_OK) return st;
    if (!proj || !cams || !ranges || !dL_dimage || n_views <= 0 || total_tiles <= 0) return GS_ERR_INVALID_ARG;
    if (!saved.T_final || !saved.n_last || !saved.ckpt || saved.ckpt_slots <= 0) return GS_ERR_INVALID_ARG;
    if ((uintptr_t)proj->rec & 15) return GS_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < gs_render_bwd_workspace_size(n, n_views)) return GS_ERR_WORKSPACE;
    if ((uintptr_t)workspace & 15) return GS_ERR_WORKSPACE;
    if (n == 0) return GS_OK;
    gs_grads none{};
    return render_bwd_impl<true>(&prm, proj, ls, coarse, ranges, cams, n_views, total_tiles, cfg, saved, dL_dimage,
                                 view_gate, none, 0, af, workspace, stream);
}

extern "C" {

gs_status gs_render_bwd_adam(float *flat_params, float *m, float *v, int64_t n, int32_t sh_degree,
                             const gs_projected *proj, const uint32_t *vals, const uint32_t *ranges,
                             const gs_camera *cams, int32_t n_views, int64_t total_tiles, const gs_raster_config *cfg,
                             gs_fwd_saved saved, const float *dL_dimage, const uint8_t *view_gate,
                             const gs_adam_config *adam, const int32_t *dev_do_step, int64_t *dev_step,
                             double *norms2, void *workspace, size_t workspace_bytes, int32_t *dev_status,
                             cudaStream_t stream) {
    (void)dev_status;
    if (!vals) return GS_ERR_INVALID_ARG;
    ListSrc ls{};
    ls.vals = vals;
    return render_bwd_adam_entry(flat_params, m, v, n, sh_degree, proj, ls, false, ranges, cams, n_views, total_tiles,
                                 cfg, saved, dL_dimage, view_gate, adam, dev_do_step, dev_step, norms2, workspace,
                                 workspace_bytes, stream);
}

gs_status gs_render_bwd_adam_coarse(float *flat_params, float *m, float *v, int64_t n, int32_t sh_degree,
                                    const gs_projected *proj, const gs_coarse_lists *lists, const uint32_t *ranges,
                                    const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                                    const gs_raster_config *cfg, gs_fwd_saved saved, const float *dL_dimage,
                                    const uint8_t *view_gate, const gs_adam_config *adam,
                                    const int32_t *dev_do_step, int64_t *dev_step, double *norms2, void *workspace,
                                    size_t workspace_bytes, int32_t *dev_status, cudaStream_t stream) {
    (void)dev_status;
    ListSrc ls{};
    const gs_status st = coarse_src(lists, saved, ls);
    if (st != GS_OK) return st;
    return render_bwd_adam_entry(flat_params, m, v, n, sh_degree, proj, ls, true, ranges, cams, n_views, total_tiles,
                                 cfg, saved, dL_dimage, view_gate, adam, dev_do_step, dev_step, norms2, workspace,
                                 workspace_bytes, stream);
}

gs_status gs_project_bwd_adam(float *flat_params, float *m, float *v, int64_t n, int32_t sh_degree,
                              const gs_camera *cams, int32_t n_views, const gs_raster_config *cfg, const float *g2d,
                              const uint8_t *view_gate, const gs_adam_config *adam, const int32_t *dev_do_step,
                              int64_t *dev_step, double *norms2, int32_t *dev_status, cudaStream_t stream) {
    (void)dev_status;
    gs_params prm;
    AdamFuse af;
    gs_status st = fused_args(flat_params, m, v, n, sh_degree, cfg, adam, dev_do_step, dev_step, norms2, &prm, &af);
    if (st != GS_OK) return st;
    if (!cams || !g2d || n_views <= 0 || ((uintptr_t)g2d & 15)) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    gs_grads none{};
    return project_bwd_impl<true>(&prm, cams, n_views, cfg, reinterpret_cast<const float4 *>(g2d), view_gate, none, 0,
                                  af, stream);
}

}  // extern "C"
