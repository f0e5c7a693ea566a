// Internal helpers shared by the sm_103a kernels of libgsr.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gsr.h"

#define GS_TRY_LAUNCH()                                       \
    do {                                                      \
        if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA; \
    } while (0)

#define GS_TRY(call)                                          \
    do {                                                      \
        if ((call) != cudaSuccess) return GS_ERR_CUDA;        \
    } while (0)

namespace gsr {

// Host-side values that the CUDA runtime keeps per device (function
// attributes, occupancy, SM count) are cached per device index.
constexpr int kMaxDevices = 64;

// The current device, or -1 when it cannot be queried or is beyond the cache.
inline int cached_device_index() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
    return dev;
}

// Streaming multiprocessors of the current device (cached per device).
inline int device_sm_count() {
    static int sms[kMaxDevices] = {};
    const int dev = cached_device_index();
    if (dev >= 0 && sms[dev] > 0) return sms[dev];
    int d = dev < 0 ? 0 : dev, n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n <= 0) n = 1;
    if (dev >= 0) sms[dev] = n;
    return n;
}

constexpr int kRecFloats = 12;   // packed projected record (see gsr.h)
constexpr int kG2d = 12;         // per-Gaussian 2D gradient slots: dmean(2) dconic(3) dopac(1) drgb(3) pad(3)

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Offsets (floats) of the parameter groups in the flat buffer: means,
// log_scales, quats, opacity_logit, sh, end.  Each group starts on a 256-byte
// boundary so every group can be read with 16-byte vector loads.
__host__ __device__ inline void param_offsets(int64_t n, int sh_degree, int64_t *o) {
    const int64_t K = (int64_t)(sh_degree + 1) * (sh_degree + 1);
    auto al = [](int64_t x) { return (x + 63) / 64 * 64; };
    o[0] = 0;
    o[1] = al(3 * n);
    o[2] = al(o[1] + 3 * n);
    o[3] = al(o[2] + 4 * n);
    o[4] = al(o[3] + n);
    o[5] = al(o[4] + 3 * K * n);
}

// sqrt and reciprocal on the special-function unit (PTX sqrt.approx /
// rcp.approx, relative error ~2^-22): the optimizer step needs no more.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed float pairs: two floats in one 64-bit register, operated on by one
// f32x2 instruction (fma.rn / mul.rn), each lane rounded as the scalar
// instruction rounds it.  Halves the issued instructions of pairwise
// arithmetic.
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ uint64_t dup2(float a) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float2 upk2(uint64_t r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// One Adam update of a scalar (Kingma & Ba, bias-corrected): lr_t = lr / (1 -
// beta1^t), ibc2 = 1 / sqrt(1 - beta2^t).  Shared by the standalone optimizer
// kernel and the fused adjoint + optimizer kernel so both round alike.
__device__ __forceinline__ void adam_update(float &p, float &m, float &v, float g, float lr_t, float b1, float b2,
                                            float ibc2, float eps) {
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    p -= lr_t * m * rcp_approx(sqrt_approx(v) * ibc2 + eps);
}

// Per-step Adam scalars from the executed-step counter (computed once per
// block).  The bias corrections 1 - beta^t are formed in single precision as
// -expm1(t log1p(beta - 1)): beta - 1 is exact for beta in [0.5, 1), and both
// functions keep the small differences (t = 1, beta2 = 0.999) to a few ulp,
// without the long double-precision pow chain a block would wait on.
// With cfg.lr_scale_den > 0 and a step-gate word, the learning rates of this
// step are multiplied by *do_step / lr_scale_den (the gate writes the number
// of views it opened there: a batched step then moves by each opened view's
// share of the batch).
__device__ __forceinline__ void adam_scalars(const gs_adam_config &cfg, int64_t executed, const int32_t *do_step,
                                             float *lr_t, float *ibc2) {
    const float t = (float)(executed + 1);
    const float bc1 = -expm1f(t * log1pf(cfg.beta1 - 1.f));
    const float bc2 = -expm1f(t * log1pf(cfg.beta2 - 1.f));
    const float scale = (cfg.lr_scale_den > 0 && do_step) ? (float)*do_step / (float)cfg.lr_scale_den : 1.f;
    for (int k = 0; k < 6; ++k) lr_t[k] = cfg.lr[k] * scale / bc1;
    *ibc2 = 1.f / sqrtf(bc2);
}

// First error wins.
__device__ inline void set_status(int32_t *st, int32_t code) {
    if (st) atomicCAS(st, 0, code);
}

// The view a global tile id belongs to (views are few; linear search).
__device__ inline int view_of_tile(const gs_camera *cams, int n_views, int64_t tile) {
    int v = 0;
    while (v + 1 < n_views && cams[v + 1].tile_offset <= tile) ++v;
    return v;
}

// Work items of the compositing kernels (tiles, visited through the
// longest-first tile order).  Without a queue each block takes the item of
// its block index; with a queue (a device word, zero at launch) the kernel
// runs persistently: a grid of resident blocks, each taking the next item
// from the queue until none is left.  Called by every thread of the block.
__device__ __forceinline__ uint32_t first_item(uint32_t *queue, uint32_t *s_item) {
    if (!queue) return blockIdx.x;
    if (threadIdx.x == 0) *s_item = atomicAdd(queue, 1u);
    __syncthreads();
    return *s_item;
}
__device__ __forceinline__ uint32_t next_item(uint32_t *queue, uint32_t *s_item) {
    if (!queue) return 0xffffffffu;
    __syncthreads();  // every thread has read the previous item
    if (threadIdx.x == 0) *s_item = atomicAdd(queue, 1u);
    __syncthreads();
    return *s_item;
}

// Where the compositing kernels find a tile's depth-ordered Gaussians.  Tile
// lists: vals[ranges[tile]].  Super-tile lists (coarse != 0): the binning
// lists each (view, Gaussian) entry once per super-tile of kSup x kSup tiles
// its rectangle meets, in depth order, as its Gaussian index and a 16-bit
// mask of the super-tile's tiles it covers (bit kSup * row + column); a
// tile's list is the subsequence of its super-tile's list with the tile's
// bit set, filtered while the kernels stage it (coarse_gather).
constexpr int kSup = 4;
struct ListSrc {
    const uint32_t *vals;      // tile lists
    const uint32_t *cgid;      // super-tile lists: Gaussian index per entry
    const uint16_t *cmask;     //   covered tiles per entry
    const uint32_t *cstart;    //   first entry of each super-tile
    const uint32_t *ccount;    //   entries of each super-tile
    const int64_t *cview;      //   first super-tile of each view
    uint32_t *batch_pos;       //   per checkpoint slot: list position of the batch's first entry
};

// The ListSrc of a call on super-tile lists (GS_ERR_INVALID_ARG when a buffer is missing).
inline gs_status coarse_src(const gs_coarse_lists *l, const gs_fwd_saved &s, ListSrc &out) {
    if (!l || !l->gid || !l->mask || !l->start || !l->count || !l->view_first || !s.batch_pos)
        return GS_ERR_INVALID_ARG;
    if ((uintptr_t)l->mask & 15) return GS_ERR_INVALID_ARG;  // read with vector loads
    out = ListSrc{};
    out.cgid = l->gid;
    out.cmask = l->mask;
    out.cstart = l->start;
    out.ccount = l->count;
    out.cview = l->view_first;
    out.batch_pos = s.batch_pos;
    return GS_OK;
}

// The super-tile of tile (tx, ty) of view v (tiles_x tiles per row) and the
// tile's bit in its masks.
__device__ __forceinline__ int64_t super_tile_of(const ListSrc &ls, int v, int tiles_x, int tx, int ty,
                                                 uint32_t &bit) {
    const int stx = (tiles_x + kSup - 1) / kSup;
    bit = (uint32_t)((ty % kSup) * kSup + tx % kSup);
    return ls.cview[v] + (int64_t)(ty / kSup) * stx + tx / kSup;
}

// Copies the Gaussian indices of the next `want` (or fewer, at the list's
// end) entries with mask bit `bit` from positions [pos, end) of a super-tile
// list to out[0..), in list order, and returns how many; pos moves past the
// last entry taken.  Per round the block's NTH threads test EPT consecutive
// entries each, from pos rounded down to a multiple of EPT (one vector load
// of masks per thread; entries before pos or from end on are not taken); a
// warp scan and the warps' totals in s_wsum[NTH / 32] rank the covered ones.
// Called by every thread with block-uniform pos, end and want (two barriers
// per round; the last one also publishes out).  mask must be 16-byte aligned.
template <int NTH, int EPT>
__device__ __forceinline__ int coarse_gather(const ListSrc &ls, uint32_t bit, uint32_t &pos, uint32_t end, int want,
                                             uint32_t *out, uint32_t *s_wsum, uint32_t *s_next) {
    static_assert(EPT == 1 || EPT == 2 || EPT == 4 || EPT == 8 || EPT == 16, "masks per thread");
    constexpr int NW = NTH / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int got = 0;
    while (got < want && pos < end) {
        const uint32_t a0 = pos & ~(uint32_t)(EPT - 1);
        const uint32_t base = a0 + (uint32_t)threadIdx.x * EPT;
        uint16_t mk[EPT];
        if (base + EPT <= end) {  // whole vector inside the list
            if constexpr (EPT >= 8) {
#pragma unroll
                for (int q = 0; q < EPT / 8; ++q) {
                    const uint4 x = reinterpret_cast<const uint4 *>(ls.cmask + base)[q];
                    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        mk[8 * q + 2 * e] = (uint16_t)(w[e] & 0xffffu);
                        mk[8 * q + 2 * e + 1] = (uint16_t)(w[e] >> 16);
                    }
                }
            } else if constexpr (EPT == 4) {
                const uint2 x = *reinterpret_cast<const uint2 *>(ls.cmask + base);
                mk[0] = (uint16_t)(x.x & 0xffffu);
                mk[1] = (uint16_t)(x.x >> 16);
                mk[2] = (uint16_t)(x.y & 0xffffu);
                mk[3] = (uint16_t)(x.y >> 16);
            } else if constexpr (EPT == 2) {
                const uint32_t x = *reinterpret_cast<const uint32_t *>(ls.cmask + base);
                mk[0] = (uint16_t)(x & 0xffffu);
                mk[1] = (uint16_t)(x >> 16);
            } else {
                mk[0] = ls.cmask[base];
            }
        } else {
#pragma unroll
            for (int e = 0; e < EPT; ++e) mk[e] = base + e < end ? ls.cmask[base + e] : (uint16_t)0;
        }
        uint32_t mine = 0;
#pragma unroll
        for (int e = 0; e < EPT; ++e)
            if (base + e >= pos && ((mk[e] >> bit) & 1u)) mine |= 1u << e;
        const int c = __popc(mine);
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_wsum[warp] = (uint32_t)inc;
        __syncthreads();
        int before = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int x = (int)s_wsum[w];
            before += w < warp ? x : 0;
            tot += x;
        }
        int r = got + before + inc - c;  // rank of this thread's first covered entry
        while (mine) {
            const int e = __ffs(mine) - 1;
            mine &= mine - 1;
            if (r < want) {
                out[r] = ls.cgid[base + e];
                if (r == want - 1) *s_next = base + e + 1;
            }
            ++r;
        }
        const bool filled = got + tot >= want;
        got = filled ? want : got + tot;
        __syncthreads();
        const uint32_t step = (uint32_t)NTH * EPT;
        pos = filled ? *s_next : (end - a0 > step ? a0 + step : end);
    }
    return got;
}

// Masks each thread tests per gathering round: about 1024 list entries per
// round for a block of NTH threads.
template <int NTH>
__host__ __device__ constexpr int gather_ept() {
    return NTH >= 1024 ? 1 : (NTH >= 512 ? 2 : (NTH >= 256 ? 4 : (NTH >= 128 ? 8 : 16)));
}

// Eq. (alpha) at one pixel, evaluated through the conic's Cholesky factor U
// (Q = U^T U): dp^T Q dp = |U dp|^2 with z0 = u00 dx + u01 dy, z1 = u11 dy.
// A sum of squares keeps the float32 rounding error near eps * sqrt(cond(Q)).
// Explicit round-to-nearest intrinsics pin every operation, so the forward and
// backward kernels obtain bit-identical alphas and contributor sets.
struct AlphaEval {
    float alpha, G, dx, dy, z0, z1;
    bool clamped;
};

// 2^x on the special-function unit (PTX ex2.approx, relative error ~2^-22).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ AlphaEval eval_alpha(float4 a, float4 b, float px, float py, float alpha_max) {
    constexpr float kNegHalfLog2e = -0.72134752044448170f;  // -log2(e) / 2: exp(-q/2) = 2^(q * kNegHalfLog2e)
    AlphaEval r;
    r.dx = __fsub_rn(px, a.x);
    r.dy = __fsub_rn(py, a.y);
    r.z0 = __fmaf_rn(a.z, r.dx, __fmul_rn(a.w, r.dy));
    r.z1 = __fmul_rn(b.x, r.dy);
    const float q = __fmaf_rn(r.z0, r.z0, __fmul_rn(r.z1, r.z1));
    r.G = ex2_approx(__fmul_rn(kNegHalfLog2e, q));
    const float og = __fmul_rn(b.y, r.G);
    r.clamped = og > alpha_max;
    r.alpha = r.clamped ? alpha_max : og;
    return r;
}

// Pixels of thread t in a TILE x TILE tile when each thread owns PPT pixels:
// each warp covers an 8 x (4 PPT) block (pixel k of a thread is 4k rows below
// its first), so a warp can skip a Gaussian whose support misses its block.
// Pixel k of thread t has the in-tile slot t + k * (TILE * TILE / PPT).
template <int TILE, int PPT>
__device__ __forceinline__ void tile_pixel(int t, int k, int &lx, int &ly) {
    const int w = t >> 5, lane = t & 31;
    lx = (w % (TILE / 8)) * 8 + (lane & 7);
    ly = (w / (TILE / 8)) * (4 * PPT) + (lane >> 3) + 4 * k;
}

// Does the support box [m - r, m + r] of a Gaussian reach any pixel centre of
// the warp's 8 x H block whose first pixel centre is (wx, wy)?  Uniform per warp.
template <int H>
__device__ __forceinline__ bool warp_overlaps(float4 a, float4 c, float wx, float wy) {
    constexpr float hy = 0.5f * (H - 1);
    return fabsf(a.x - (wx + 3.5f)) <= c.z + 3.5f && fabsf(a.y - (wy + hy)) <= c.w + hy;
}

// Lower bound of q(dp) = |U dp|^2 (Q = U^T U, U = [[u00, u01], [0, u11]],
// u00, u11 > 0) over the offsets [dx0, dx1] x [dy0, dy1]: 0 when they
// contain dp = 0, else the least of q's minima along the four edges (q is
// convex with its minimum at 0, so over the rectangle it is least on the
// boundary); along an edge q is a quadratic in one offset, minimised in closed
// form and clamped to the edge.  sv = -u00 u01 / (u01^2 + u11^2) and
// sh = -u01 / u00 (the minimising dy at dx = 1 and dx at dy = 1) depend on the
// record only and are passed in.
__device__ __forceinline__ float rect_qmin(float u00, float u01, float u11, float sv, float sh, float dx0,
                                           float dx1, float dy0, float dy1) {
    if (dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f) return 0.f;
    auto at = [&](float dx, float dy) {
        const float z0 = u00 * dx + u01 * dy, z1 = u11 * dy;
        return z0 * z0 + z1 * z1;
    };
    const float qa = at(dx0, fminf(fmaxf(sv * dx0, dy0), dy1)), qb = at(dx1, fminf(fmaxf(sv * dx1, dy0), dy1));
    const float qc = at(fminf(fmaxf(sh * dy0, dx0), dx1), dy0), qd = at(fminf(fmaxf(sh * dy1, dx0), dx1), dy1);
    return fminf(fminf(qa, qb), fminf(qc, qd));
}

// Overlap masks of one staged batch of records: for every warp w of the CTA,
// bit (j % 32) of word j / 32 of row w is set when record j's support box
// reaches w's pixel block (the warp_overlaps test) and so does its support
// ellipse dp^T Q dp <= 2 ln(o / alpha_min): no pixel outside it has
// alpha' >= alpha_min, so a record whose ellipse misses the block (minimum
// of dp^T Q dp over the block's pixel centres above the bound, with a margin
// far beyond float32 rounding) contributes nothing there and is not marked.
// Called by whole warps for batch slots kk = threadIdx.x, threadIdx.x + NTH,
// ... < BATCH; a, b, c are the slot's record (a.x, a.y = mean2D; a.z, a.w,
// b.x = U; b.y = opacity; c.z, c.w = support half-extents), valid false past
// the batch's end.  One ballot per target warp and 32 slots.
template <int TILE, int PPT, int NW, int NWORD>
__device__ __forceinline__ void overlap_masks(uint32_t (*s_ov)[NWORD], int kk, bool valid, float4 a, float4 b,
                                              float4 c, float alpha_min, int tile_x0, int tile_y0) {
    constexpr int H = 4 * PPT;
    const float qcut = valid ? 1.001f * (2.f * __logf(b.y / alpha_min)) + 0.01f : 0.f;
    const float sv = valid ? -a.z * a.w / (a.w * a.w + b.x * b.x) : 0.f;
    const float sh = valid ? -a.w / a.z : 0.f;
#pragma unroll 1
    for (int w = 0; w < NW; ++w) {  // not unrolled: the test's temporaries stay few
        int lx0, ly0;
        tile_pixel<TILE, PPT>(w * 32, 0, lx0, ly0);
        const float wx = (float)(tile_x0 + lx0) + 0.5f, wy = (float)(tile_y0 + ly0) + 0.5f;
        bool hit = valid && warp_overlaps<H>(a, c, wx, wy);
        if (hit) hit = rect_qmin(a.z, a.w, b.x, sv, sh, wx - a.x, wx + 7.f - a.x, wy - a.y, wy + (H - 1) - a.y) <= qcut;
        const uint32_t m = __ballot_sync(0xffffffffu, hit);
        if ((threadIdx.x & 31) == 0) s_ov[w][kk >> 5] = m;
    }
}

// Real spherical harmonics (Condon-Shortley phase) up to degree 3 at a unit
// direction (x, y, z), basis order k = l*l + l + m.  Constants are the
// normalisations sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0)
// folded with the polynomial coefficients of each basis function.
namespace sh {
constexpr float c0 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float c1 = 0.48860251190291992f;   // sqrt(3) / (2 sqrt(pi))
constexpr float c2a = 1.0925484305920792f;   // sqrt(15) / (2 sqrt(pi))
constexpr float c2b = 0.31539156525252005f;  // sqrt(5) / (4 sqrt(pi))
constexpr float c2c = 0.54627421529603959f;  // sqrt(15) / (4 sqrt(pi))
constexpr float c3a = 0.59004358992664352f;  // sqrt(35/2) / (4 sqrt(pi))
constexpr float c3b = 2.8906114426405538f;   // sqrt(105) / (2 sqrt(pi))
constexpr float c3c = 0.45704579946446572f;  // sqrt(21/2) / (4 sqrt(pi))
constexpr float c3d = 0.37317633259011546f;  // sqrt(7) / (4 sqrt(pi))
constexpr float c3e = 1.4453057213202769f;   // sqrt(105) / (4 sqrt(pi))
}  // namespace sh

// Y[0..K) at direction (x,y,z).
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float *Y) {
    Y[0] = sh::c0;
    if (deg < 1) return;
    Y[1] = -sh::c1 * y;
    Y[2] = sh::c1 * z;
    Y[3] = -sh::c1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = sh::c2a * x * y;
    Y[5] = -sh::c2a * y * z;
    Y[6] = sh::c2b * (2.f * zz - xx - yy);
    Y[7] = -sh::c2a * x * z;
    Y[8] = sh::c2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -sh::c3a * y * (3.f * xx - yy);
    Y[10] = sh::c3b * x * y * z;
    Y[11] = -sh::c3c * y * (4.f * zz - xx - yy);
    Y[12] = sh::c3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -sh::c3c * x * (4.f * zz - xx - yy);
    Y[14] = sh::c3e * z * (xx - yy);
    Y[15] = -sh::c3a * x * (xx - 3.f * yy);
}

// Gradient of each basis polynomial above with respect to (x, y, z), taken as
// free variables (the caller projects onto the sphere's tangent plane).
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float (*dY)[3]) {
    dY[0][0] = dY[0][1] = dY[0][2] = 0.f;
    if (deg < 1) return;
    dY[1][0] = 0.f; dY[1][1] = -sh::c1; dY[1][2] = 0.f;
    dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = sh::c1;
    dY[3][0] = -sh::c1; dY[3][1] = 0.f; dY[3][2] = 0.f;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    dY[4][0] = sh::c2a * y; dY[4][1] = sh::c2a * x; dY[4][2] = 0.f;
    dY[5][0] = 0.f; dY[5][1] = -sh::c2a * z; dY[5][2] = -sh::c2a * y;
    dY[6][0] = -2.f * sh::c2b * x; dY[6][1] = -2.f * sh::c2b * y; dY[6][2] = 4.f * sh::c2b * z;
    dY[7][0] = -sh::c2a * z; dY[7][1] = 0.f; dY[7][2] = -sh::c2a * x;
    dY[8][0] = 2.f * sh::c2c * x; dY[8][1] = -2.f * sh::c2c * y; dY[8][2] = 0.f;
    if (deg < 3) return;
    dY[9][0] = -sh::c3a * 6.f * x * y; dY[9][1] = -sh::c3a * (3.f * xx - 3.f * yy); dY[9][2] = 0.f;
    dY[10][0] = sh::c3b * y * z; dY[10][1] = sh::c3b * x * z; dY[10][2] = sh::c3b * x * y;
    dY[11][0] = sh::c3c * 2.f * x * y; dY[11][1] = -sh::c3c * (4.f * zz - xx - 3.f * yy); dY[11][2] = -sh::c3c * 8.f * y * z;
    dY[12][0] = -sh::c3d * 6.f * x * z; dY[12][1] = -sh::c3d * 6.f * y * z; dY[12][2] = sh::c3d * (6.f * zz - 3.f * xx - 3.f * yy);
    dY[13][0] = -sh::c3c * (4.f * zz - 3.f * xx - yy); dY[13][1] = sh::c3c * 2.f * x * y; dY[13][2] = -sh::c3c * 8.f * x * z;
    dY[14][0] = sh::c3e * 2.f * x * z; dY[14][1] = -sh::c3e * 2.f * y * z; dY[14][2] = sh::c3e * (xx - yy);
    dY[15][0] = -sh::c3a * (3.f * xx - 3.f * yy); dY[15][1] = sh::c3a * 6.f * x * y; dY[15][2] = 0.f;
}

// a*b - c*d with one rounding error (Kahan's FMA-based difference of products).
__device__ __forceinline__ float diff_prod(float a, float b, float c, float d) {
    const float w = c * d;
    const float e = __fmaf_rn(-c, d, w);
    const float f = __fmaf_rn(a, b, -w);
    return f + e;
}

// Forward projection state of one Gaussian for one camera (Eq. cov, Eq. proj).
struct ProjState {
    bool culled;
    float qn[4], qinv;      // normalised quaternion, 1/|q|
    float R[9];             // rotation of the Gaussian
    float s[3];             // standard deviations
    float p[3];             // camera-space centre
    int clamp_x, clamp_y;   // J built from x/z, y/z clamped (+1/-1 side) or not (0)
    float txz, tyz;         // the (clamped) x/z, y/z used in J
    float T[6];             // J W (2x3)
    float M[6];             // J W R S (2x3); Sigma2D = M M^T + lowpass I
    float s00, s01, s11;    // Sigma2D
    float det;
    float mean2d[2];
    float o;
};

// Camera centre -R^T t.
__device__ __forceinline__ void cam_center(const gs_camera &c, float *cp) {
    for (int i = 0; i < 3; ++i) cp[i] = -(c.R[i] * c.t[0] + c.R[3 + i] * c.t[1] + c.R[6 + i] * c.t[2]);
}

__device__ __forceinline__ void project_state(const float *mu, const float *ls, float4 q, float logit,
                                              const gs_camera &c, float lowpass, ProjState &g) {
    g.culled = false;
    for (int i = 0; i < 3; ++i) g.p[i] = c.R[3 * i] * mu[0] + c.R[3 * i + 1] * mu[1] + c.R[3 * i + 2] * mu[2] + c.t[i];
    const float x = g.p[0], y = g.p[1], z = g.p[2];
    if (!(z > c.znear)) { g.culled = true; return; }
    const float qq = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    g.qinv = 1.0f / sqrtf(qq);
    const float w = q.x * g.qinv, qx = q.y * g.qinv, qy = q.z * g.qinv, qz = q.w * g.qinv;
    g.qn[0] = w; g.qn[1] = qx; g.qn[2] = qy; g.qn[3] = qz;
    g.R[0] = 1.f - 2.f * (qy * qy + qz * qz); g.R[1] = 2.f * (qx * qy - w * qz); g.R[2] = 2.f * (qx * qz + w * qy);
    g.R[3] = 2.f * (qx * qy + w * qz); g.R[4] = 1.f - 2.f * (qx * qx + qz * qz); g.R[5] = 2.f * (qy * qz - w * qx);
    g.R[6] = 2.f * (qx * qz - w * qy); g.R[7] = 2.f * (qy * qz + w * qx); g.R[8] = 1.f - 2.f * (qx * qx + qy * qy);
    for (int i = 0; i < 3; ++i) g.s[i] = expf(ls[i]);
    const float iz = 1.0f / z;
    const float limx = 1.3f * (0.5f * (float)c.width) / c.fx;
    const float limy = 1.3f * (0.5f * (float)c.height) / c.fy;
    const float xz = x * iz, yz = y * iz;
    g.clamp_x = xz > limx ? 1 : (xz < -limx ? -1 : 0);
    g.clamp_y = yz > limy ? 1 : (yz < -limy ? -1 : 0);
    g.txz = g.clamp_x ? (float)g.clamp_x * limx : xz;
    g.tyz = g.clamp_y ? (float)g.clamp_y * limy : yz;
    // J = [[fx/z, 0, -fx txz/z], [0, fy/z, -fy tyz/z]]; T = J W
    const float j00 = c.fx * iz, j02 = -c.fx * g.txz * iz, j11 = c.fy * iz, j12 = -c.fy * g.tyz * iz;
    for (int k = 0; k < 3; ++k) {
        g.T[k] = j00 * c.R[k] + j02 * c.R[6 + k];
        g.T[3 + k] = j11 * c.R[3 + k] + j12 * c.R[6 + k];
    }
    // M = T R S
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k)
            g.M[3 * r + k] = (g.T[3 * r] * g.R[k] + g.T[3 * r + 1] * g.R[3 + k] + g.T[3 * r + 2] * g.R[6 + k]) * g.s[k];
    const float *m0 = g.M, *m1 = g.M + 3;
    const float n0 = m0[0] * m0[0] + m0[1] * m0[1] + m0[2] * m0[2];
    const float n1 = m1[0] * m1[0] + m1[1] * m1[1] + m1[2] * m1[2];
    g.s00 = n0 + lowpass;
    g.s11 = n1 + lowpass;
    g.s01 = m0[0] * m1[0] + m0[1] * m1[1] + m0[2] * m1[2];
    // det(M M^T + l I) = |m0 x m1|^2 + l (|m0|^2 + |m1|^2) + l^2 (Cauchy-Binet), all terms >= 0
    const float cx_ = diff_prod(m0[1], m1[2], m0[2], m1[1]);
    const float cy_ = diff_prod(m0[2], m1[0], m0[0], m1[2]);
    const float cz_ = diff_prod(m0[0], m1[1], m0[1], m1[0]);
    g.det = (cx_ * cx_ + cy_ * cy_ + cz_ * cz_) + lowpass * (n0 + n1) + lowpass * lowpass;
    if (!(g.det > 0.f) || !(g.s11 > 0.f)) { g.culled = true; return; }
    g.mean2d[0] = c.fx * xz + c.cx;
    g.mean2d[1] = c.fy * yz + c.cy;
    g.o = 1.0f / (1.0f + expf(-logit));
}


// ---------------------------------------------------------------------------
// Per-Gaussian parameters staged through shared memory (projection and its
// adjoint): a block of PB Gaussians copies each parameter group's contiguous
// slice with 16-byte coalesced loads into a padded layout.
// Group strides (floats per Gaussian) and the staged layout in shared memory:
// per Gaussian each group is padded to an odd stride P(g), so the 32 threads
// of a warp touching "their" element k hit 32 different banks.
template <int DEG>
struct ParamGroups {
    static constexpr int K = (DEG + 1) * (DEG + 1);
    __host__ __device__ static constexpr int S(int g) { return g == 0 ? 3 : (g == 1 ? 3 : (g == 2 ? 4 : (g == 3 ? 1 : 3 * K))); }
    __host__ __device__ static constexpr int P(int g) { return S(g) | 1; }
    static constexpr int TOT = P(0) + P(1) + P(2) + P(3) + P(4);  // padded floats per Gaussian
    __host__ __device__ static constexpr int off(int g, int nb) {
        return g == 0 ? 0
             : (g == 1 ? P(0) * nb
             : (g == 2 ? (P(0) + P(1)) * nb : (g == 3 ? (P(0) + P(1) + P(2)) * nb : (P(0) + P(1) + P(2) + P(3)) * nb)));
    }
    // linear index k of a group's contiguous global slice -> padded shared index
    __host__ __device__ static constexpr int pad(int g, int k) { return (k / S(g)) * P(g) + k % S(g); }
};

constexpr int PB = 128;  // Gaussians (and threads) per staged block
constexpr int kStagedViews = 16;  // cameras copied to shared memory per block

// Copy the float4 chunks [0, C4) of a global slice into the padded shared
// layout, NT threads cooperating (this one is `lane`); every load of the
// thread is issued before the first store.
template <int DEG, int g, int C4, int NT>
__device__ __forceinline__ void stage_full(const float *__restrict__ sp, float *dp, int lane) {
    using G = ParamGroups<DEG>;
    constexpr int J = (C4 + NT - 1) / NT;
    float4 x[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int c = lane + j * NT;
        if (c < C4) x[j] = reinterpret_cast<const float4 *>(sp)[c];
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int c = lane + j * NT;
        if (c < C4) {
            dp[G::pad(g, 4 * c)] = x[j].x;
            dp[G::pad(g, 4 * c + 1)] = x[j].y;
            dp[G::pad(g, 4 * c + 2)] = x[j].z;
            dp[G::pad(g, 4 * c + 3)] = x[j].w;
        }
    }
}

// All five groups of NG Gaussians starting at i0 (NG threads, NG a multiple
// of 4 so that every slice is a whole number of float4 chunks).
template <int DEG, int NG>
__device__ __forceinline__ void stage_group_full(const float *const (&src)[5], int64_t i0, float *s_par, int lane) {
    using G = ParamGroups<DEG>;
    constexpr int K = G::K;
    stage_full<DEG, 0, 3 * NG / 4, NG>(src[0] + 3 * i0, s_par + G::off(0, NG), lane);
    stage_full<DEG, 1, 3 * NG / 4, NG>(src[1] + 3 * i0, s_par + G::off(1, NG), lane);
    stage_full<DEG, 2, NG, NG>(src[2] + 4 * i0, s_par + G::off(2, NG), lane);
    stage_full<DEG, 3, NG / 4, NG>(src[3] + i0, s_par + G::off(3, NG), lane);
    stage_full<DEG, 4, 3 * K * NG / 4, NG>(src[4] + (int64_t)3 * K * i0, s_par + G::off(4, NG), lane);
}

// The same for a partial group of nb < NG Gaussians (slices start on 16-byte
// boundaries: i0 is a multiple of NG, NG of 4, and groups are 256-byte aligned).
template <int DEG, int NG>
__device__ __forceinline__ void stage_group_partial(const float *const (&src)[5], int64_t i0, int nb, float *s_par,
                                                    int lane) {
    using G = ParamGroups<DEG>;
#pragma unroll
    for (int g = 0; g < 5; ++g) {
        const int cnt = G::S(g) * nb;
        const float *sp = src[g] + (int64_t)G::S(g) * i0;
        float *dp = s_par + G::off(g, NG);
        const int cnt4 = cnt >> 2;
#pragma unroll 4
        for (int c = lane; c < cnt4; c += NG) {
            const float4 x = reinterpret_cast<const float4 *>(sp)[c];
            dp[G::pad(g, 4 * c)] = x.x;
            dp[G::pad(g, 4 * c + 1)] = x.y;
            dp[G::pad(g, 4 * c + 2)] = x.z;
            dp[G::pad(g, 4 * c + 3)] = x.w;
        }
        for (int k = 4 * cnt4 + lane; k < cnt; k += NG) dp[G::pad(g, k)] = sp[k];
    }
}

// A whole block of PB Gaussians, PB threads.
template <int DEG>
__device__ __forceinline__ void stage_block_full(const float *const (&src)[5], int64_t i0, float *s_par) {
    stage_group_full<DEG, PB>(src, i0, s_par, threadIdx.x);
}
template <int DEG>
__device__ __forceinline__ void stage_partial(const float *const (&src)[5], int64_t i0, int nb, float *s_par) {
    stage_group_partial<DEG, PB>(src, i0, nb, s_par, threadIdx.x);
}


// Asynchronous 16-byte global -> shared copies (cp.async, bypassing L1) and
// their group bookkeeping, for staging the next batch while the current one
// is processed.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Bulk prefetch of a global range into L2 (no completion to wait on).  The
// address must be 16-byte aligned and `bytes` a multiple of 16.
__device__ __forceinline__ void prefetch_l2(const void *gmem, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gmem), "r"(bytes) : "memory");
}

}  // namespace gsr
