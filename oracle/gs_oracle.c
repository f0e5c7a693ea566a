/*
 * FP64 CPU oracle for the 3DGS tile rasterizer that SkipGS gates.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline / reference arm may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it and shares no code
 * with it.
 *
 * What it computes, step by step, in the order and notation of the paper's
 * Sec. 3 (Preliminaries):
 *   - Eq. (cov):   Sigma = R S S^T R^T from a unit quaternion and per-axis
 *                  standard deviations s = exp(log_s).
 *   - Eq. (proj):  Sigma2D = J W Sigma W^T J^T (+ lowpass * I, reading R1),
 *                  conic Q = Sigma2D^-1, mean2D = pinhole projection.
 *   - SH colour:   c = max(0, sum_k f_k Y_k(d) + 0.5) with Y_k the real
 *                  spherical harmonics (Condon-Shortley phase), built here from
 *                  their definition (Legendre polynomials and normalisation).
 *   - Tile binning + depth order: key = (global tile id << 32) | float32 bits
 *                  of depth, stable sort (reading R3).
 *   - Eq. (blend) / Eq. (alpha): front-to-back compositing of depth-sorted
 *                  Gaussians, alpha' = min(0.99, o G), skip alpha' < 1/255,
 *                  stop before a Gaussian that would drive T below 1e-4.
 *   - The analytic adjoint of all of the above down to the 59 parameters per
 *                  Gaussian (derived here; the paper only says "fully
 *                  differentiable").
 * Readings where the paper is silent (lowpass dilation, near plane, 1.3x
 * frustum clamp of J, SH offset/clamp, pixel centres at i+0.5, black
 * background, the tile-size-invariant contribution set) are stated at the
 * point of use.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.  No FMA contraction,
 * so every double operation rounds once.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    double R[9];      /* world -> camera rotation, row-major */
    double t[3];      /* world -> camera translation: x_c = R x + t */
    double fx, fy, cx, cy;
    int32_t width, height;
    double znear;
} orc_camera;

typedef struct {
    double lowpass;   /* isotropic dilation of Sigma2D (px^2) */
    double alpha_max; /* 0.99 */
    double alpha_min; /* 1/255 */
    double t_min;     /* 1e-4 */
    double bg[3];
    int32_t tile;
} orc_raster;

/* ------------------------------------------------------------------ SH --
 * Real spherical harmonics up to degree 3, index k = l*l + l + m.
 *   m > 0: sqrt2 K_l^m cos(m phi) P_l^m(cos theta)
 *   m < 0: sqrt2 K_l^|m| sin(|m| phi) P_l^|m|(cos theta)
 *   m = 0: K_l^0 P_l^0(cos theta)
 * K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_l^m with the Condon-Shortley
 * phase: P_l^m(z) = (-1)^m (1-z^2)^(m/2) d^m/dz^m P_l(z).
 * With d = (sin t cos p, sin t sin p, cos t):
 *   cos(m p) sin^m t = Re (x + i y)^m,  sin(m p) sin^m t = Im (x + i y)^m,
 * so each basis function is  norm * Re/Im((x+iy)^|m|) * Qlm(z),
 * Qlm(z) = (-1)^m d^m P_l/dz^m, a polynomial: no trigonometry, and the
 * gradient in (x, y, z) follows by differentiating the two polynomial factors.
 */
static double fact(int n) { double r = 1.0; for (int i = 2; i <= n; ++i) r *= i; return r; }

/* Legendre polynomial coefficients (ascending powers) via Bonnet's recurrence
 * (n+1) P_{n+1} = (2n+1) z P_n - n P_{n-1}. */
static void legendre_coeffs(int l, double c[4]) {
    double p0[4] = {1, 0, 0, 0}, p1[4] = {0, 1, 0, 0}, p2[4];
    if (l == 0) { memcpy(c, p0, sizeof p0); return; }
    for (int n = 1; n < l; ++n) {
        for (int i = 0; i < 4; ++i) {
            double zp = (i > 0) ? p1[i - 1] : 0.0;
            p2[i] = ((2 * n + 1) * zp - n * p0[i]) / (n + 1);
        }
        memcpy(p0, p1, sizeof p0);
        memcpy(p1, p2, sizeof p1);
    }
    memcpy(c, p1, sizeof p1);
}

static double poly_eval(const double *c, int n, double z) {
    double r = 0.0;
    for (int i = n - 1; i >= 0; --i) r = r * z + c[i];
    return r;
}

/* Values Y[k] and gradients dY[k][3] wrt (x,y,z), treated as free variables. */
static void sh_basis(int deg, const double d[3], double *Y, double (*dY)[3]) {
    const double x = d[0], y = d[1], z = d[2];
    for (int l = 0; l <= deg; ++l) {
        double P[4];
        legendre_coeffs(l, P);
        for (int m = -l; m <= l; ++m) {
            const int am = m < 0 ? -m : m;
            /* Qlm = (-1)^am d^am P_l / dz^am */
            double Q[4] = {0, 0, 0, 0};
            for (int i = am; i < 4; ++i) {
                double f = 1.0;
                for (int j = 0; j < am; ++j) f *= (double)(i - j);
                Q[i - am] = P[i] * f * ((am & 1) ? -1.0 : 1.0);
            }
            double dQ[4] = {0, 0, 0, 0};
            for (int i = 1; i < 4; ++i) dQ[i - 1] = Q[i] * i;
            const double q = poly_eval(Q, 4, z), dq = poly_eval(dQ, 4, z);
            /* (x + i y)^am and its derivative am (x + i y)^(am-1) */
            double re = 1.0, im = 0.0, dre = 0.0, dim = 0.0;
            for (int j = 0; j < am; ++j) {
                if (j == am - 1) { dre = re * am; dim = im * am; }
                const double nre = re * x - im * y, nim = re * y + im * x;
                re = nre; im = nim;
            }
            double K = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * fact(l - am) / fact(l + am));
            if (m != 0) K *= sqrt(2.0);
            const int k = l * l + l + m;
            double a, da_dx, da_dy;
            if (m > 0) { a = re; da_dx = dre; da_dy = -dim; }        /* d/dy Re((x+iy)^m) = -m Im((x+iy)^(m-1)) */
            else if (m < 0) { a = im; da_dx = dim; da_dy = dre; }   /* d/dy Im((x+iy)^m) =  m Re((x+iy)^(m-1)) */
            else { a = 1.0; da_dx = 0.0; da_dy = 0.0; }
            Y[k] = K * a * q;
            if (dY) {
                dY[k][0] = K * da_dx * q;
                dY[k][1] = K * da_dy * q;
                dY[k][2] = K * a * dq;
            }
        }
    }
}

/* exported for the SH pin tests */
void orc_sh_basis(int deg, const double *d, double *Y, double *dY) {
    sh_basis(deg, d, Y, (double (*)[3])dY);
}

/* ------------------------------------------------------- quaternion -- */
/* Rotation matrix of a unit quaternion (w,x,y,z), row-major. */
static void quat_to_rot(const double q[4], double R[9]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* dR/dq_c for c in {w,x,y,z}: the entrywise partial derivatives of quat_to_rot. */
static void quat_to_rot_grad(const double q[4], double dR[4][9]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double Dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    const double Dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    const double Dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    const double Dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    memcpy(dR[0], Dw, sizeof Dw); memcpy(dR[1], Dx, sizeof Dx);
    memcpy(dR[2], Dy, sizeof Dy); memcpy(dR[3], Dz, sizeof Dz);
}

/* ------------------------------------------------------- projection --
 * Per-Gaussian state shared by the forward projection and its adjoint. */
typedef struct {
    int culled;
    double qn[4], qnorm, R[9], s[3], Sigma[9];
    double p[3];          /* camera-space centre */
    int clamp_x, clamp_y; /* 0, +1 or -1: which side of the 1.3x frustum limit */
    double xt, yt;        /* clamped x, y used in J */
    double J[6];          /* 2x3 */
    double T[6];          /* J Rc, 2x3 */
    double cov[3];        /* Sigma2D (a, b, c) incl. lowpass */
    double conic[3];      /* Q = Sigma2D^-1 (a, b, c) */
    double mean2d[2];
    double o;
    double dir[3], vnorm; /* unit view direction and |mu - campos| */
    double Y[16];
    double pre[3];        /* colour before the clamp at 0 */
    double rgb[3];
    double radius, radius_x, radius_y;
    int rect[4];          /* tile x0, y0, x1, y1 (inclusive) */
    int touched;
} orc_gauss;

static void project_one(const double *mu, const double *log_s, const double *q, double logit,
                        const double *f, int K, const orc_camera *cam, const orc_raster *rc,
                        orc_gauss *g) {
    memset(g, 0, sizeof *g);
    /* Eq. (cov): R from the normalised quaternion, S = diag(exp(log_s)). */
    g->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) g->qn[i] = q[i] / g->qnorm;
    quat_to_rot(g->qn, g->R);
    for (int i = 0; i < 3; ++i) g->s[i] = exp(log_s[i]);
    double RS2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) RS2[3 * i + j] = g->R[3 * i + j] * g->s[j] * g->s[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += RS2[3 * i + k] * g->R[3 * j + k];
            g->Sigma[3 * i + j] = s;
        }
    /* Viewing transform W (the camera pose). */
    for (int i = 0; i < 3; ++i)
        g->p[i] = cam->R[3 * i] * mu[0] + cam->R[3 * i + 1] * mu[1] + cam->R[3 * i + 2] * mu[2] + cam->t[i];
    const double x = g->p[0], y = g->p[1], z = g->p[2];
    /* Reading: near plane; Gaussians at or behind it are culled. */
    if (!(z > cam->znear)) { g->culled = 1; return; }
    /* Reading: J uses x, y clamped to 1.3x the half field of view. */
    const double limx = 1.3 * (0.5 * cam->width) / cam->fx;
    const double limy = 1.3 * (0.5 * cam->height) / cam->fy;
    g->xt = x; g->yt = y;
    if (x / z > limx) { g->clamp_x = 1; g->xt = limx * z; }
    else if (x / z < -limx) { g->clamp_x = -1; g->xt = -limx * z; }
    if (y / z > limy) { g->clamp_y = 1; g->yt = limy * z; }
    else if (y / z < -limy) { g->clamp_y = -1; g->yt = -limy * z; }
    /* J: Jacobian of the local affine approximation of the projection. */
    g->J[0] = cam->fx / z; g->J[1] = 0.0; g->J[2] = -cam->fx * g->xt / (z * z);
    g->J[3] = 0.0; g->J[4] = cam->fy / z; g->J[5] = -cam->fy * g->yt / (z * z);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += g->J[3 * i + k] * cam->R[3 * k + j];
            g->T[3 * i + j] = s;
        }
    /* Eq. (proj): Sigma2D = T Sigma T^T, T = J W; plus the lowpass dilation. */
    double TS[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += g->T[3 * i + k] * g->Sigma[3 * k + j];
            TS[3 * i + j] = s;
        }
    double C2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += TS[3 * i + k] * g->T[3 * j + k];
            C2[2 * i + j] = s;
        }
    g->cov[0] = C2[0] + rc->lowpass;
    g->cov[1] = 0.5 * (C2[1] + C2[2]);
    g->cov[2] = C2[3] + rc->lowpass;
    const double det = g->cov[0] * g->cov[2] - g->cov[1] * g->cov[1];
    if (!(det > 0.0)) { g->culled = 1; return; }
    g->conic[0] = g->cov[2] / det;
    g->conic[1] = -g->cov[1] / det;
    g->conic[2] = g->cov[0] / det;
    g->mean2d[0] = cam->fx * x / z + cam->cx;
    g->mean2d[1] = cam->fy * y / z + cam->cy;
    g->o = 1.0 / (1.0 + exp(-logit));
    /* SH colour for the direction from the camera centre to the Gaussian. */
    double campos[3];
    for (int i = 0; i < 3; ++i)
        campos[i] = -(cam->R[i] * cam->t[0] + cam->R[3 + i] * cam->t[1] + cam->R[6 + i] * cam->t[2]);
    double v[3] = {mu[0] - campos[0], mu[1] - campos[1], mu[2] - campos[2]};
    g->vnorm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int i = 0; i < 3; ++i) g->dir[i] = v[i] / g->vnorm;
    int deg = 0;
    while ((deg + 1) * (deg + 1) < K) ++deg;
    sh_basis(deg, g->dir, g->Y, NULL);
    for (int ch = 0; ch < 3; ++ch) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += f[3 * k + ch] * g->Y[k];
        g->pre[ch] = s + 0.5;
        g->rgb[ch] = g->pre[ch] > 0.0 ? g->pre[ch] : 0.0;
    }
    /* Reading R2: a pixel can only receive alpha' >= 1/255 if o >= 1/255, and
     * only inside the ellipse dp^T Q dp <= c with c = 2 ln(255 o); its
     * axis-aligned extents are sqrt(c Sigma2D_xx) and sqrt(c Sigma2D_yy) (the
     * support function of an ellipse).  The tile rectangle covers every pixel
     * centre (i + 0.5) inside those extents. */
    if (g->o < rc->alpha_min) { g->culled = 1; return; }
    const double cth = 2.0 * log(g->o / rc->alpha_min);
    g->radius_x = sqrt(cth * g->cov[0]);
    g->radius_y = sqrt(cth * g->cov[2]);
    /* The rectangle may be any superset of the support (no pixel depends on
     * it); a slight inflation keeps every pair whose alpha' lies near the
     * cut-off in the tile lists, where the margin flags of orc_render see it. */
    g->radius_x = g->radius_x * 1.001 + 0.01;
    g->radius_y = g->radius_y * 1.001 + 0.01;
    g->radius = g->radius_x > g->radius_y ? g->radius_x : g->radius_y;
    double fx0 = ceil(g->mean2d[0] - g->radius_x - 0.5), fx1 = floor(g->mean2d[0] + g->radius_x - 0.5);
    double fy0 = ceil(g->mean2d[1] - g->radius_y - 0.5), fy1 = floor(g->mean2d[1] + g->radius_y - 0.5);
    if (fx0 < 0.0) fx0 = 0.0;
    if (fy0 < 0.0) fy0 = 0.0;
    if (fx1 > cam->width - 1) fx1 = cam->width - 1;
    if (fy1 > cam->height - 1) fy1 = cam->height - 1;
    if (!(fx0 <= fx1) || !(fy0 <= fy1)) { g->culled = 1; return; }
    const int px0 = (int)fx0, px1 = (int)fx1, py0 = (int)fy0, py1 = (int)fy1;
    g->rect[0] = px0 / rc->tile; g->rect[1] = py0 / rc->tile;
    g->rect[2] = px1 / rc->tile; g->rect[3] = py1 / rc->tile;
    g->touched = (g->rect[2] - g->rect[0] + 1) * (g->rect[3] - g->rect[1] + 1);
}

/* Projection of n Gaussians for one camera.  Outputs (per Gaussian):
 * mean2d[2], cov2d[3], conic[3], depth, rgb[3], opacity, radius[2] (x and y
 * extents of the support before clipping to the image), rect[4],
 * touched (0 = culled), flags (bit0/1: x/y frustum clamp of J active,
 * bits2-4: colour channel clamped at 0, bit5: culled). */
void orc_project(int64_t n, int K, const double *means, const double *log_scales,
                 const double *quats, const double *opac_logit, const double *sh,
                 const orc_camera *cam, const orc_raster *rc,
                 double *mean2d, double *cov2d, double *conic, double *depth, double *rgb,
                 double *opacity, double *radius, int32_t *rect, int32_t *touched, int32_t *flags) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        orc_gauss g;
        project_one(means + 3 * i, log_scales + 3 * i, quats + 4 * i, opac_logit[i], sh + 3 * K * i, K,
                    cam, rc, &g);
        mean2d[2 * i] = g.mean2d[0]; mean2d[2 * i + 1] = g.mean2d[1];
        for (int k = 0; k < 3; ++k) {
            cov2d[3 * i + k] = g.cov[k];
            conic[3 * i + k] = g.conic[k];
            rgb[3 * i + k] = g.rgb[k];
        }
        depth[i] = g.p[2];
        opacity[i] = g.o;
        radius[2 * i] = g.culled ? 0.0 : g.radius_x;
        radius[2 * i + 1] = g.culled ? 0.0 : g.radius_y;
        int fl = 0;
        if (g.clamp_x) fl |= 1;
        if (g.clamp_y) fl |= 2;
        for (int ch = 0; ch < 3; ++ch) if (!(g.pre[ch] > 0.0)) fl |= 4 << ch;
        if (g.culled) {
            fl |= 32;
            rect[4 * i] = 0; rect[4 * i + 1] = 0; rect[4 * i + 2] = -1; rect[4 * i + 3] = -1;
            touched[i] = 0;
        } else {
            for (int k = 0; k < 4; ++k) rect[4 * i + k] = g.rect[k];
            touched[i] = g.touched;
        }
        flags[i] = fl;
    }
}

/* ---------------------------------------------------------- binning --
 * Reading R3: one (key, value) pair per Gaussian x overlapped tile,
 * key = (global tile id << 32) | float32 bits of the depth, value = Gaussian
 * index, global tile id = view's tile offset + ty * tiles_x + tx.  Pairs are
 * emitted view-major, Gaussian index ascending, tiles row-major, then stably
 * sorted by key, so equal keys keep ascending index. */
typedef struct { uint64_t key; uint32_t val; int64_t pos; } orc_pair;

static int pair_cmp(const void *a, const void *b) {
    const orc_pair *x = (const orc_pair *)a, *y = (const orc_pair *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->pos < y->pos ? -1 : (x->pos > y->pos ? 1 : 0);
}

/* rect/depth_bits/touched are [n_views][n]; returns the pair count.
 * ranges has total_tiles * 2 entries ([start, end), empty tiles [0, 0)). */
int64_t orc_bin_sort(int64_t n, int n_views, const int32_t *rect, const uint32_t *depth_bits,
                     const int32_t *touched, const int32_t *tile_offset, const int32_t *tiles_x,
                     int64_t total_tiles, uint64_t *keys, uint32_t *vals, uint32_t *ranges) {
    int64_t P = 0;
    for (int v = 0; v < n_views; ++v)
        for (int64_t i = 0; i < n; ++i) P += touched[(int64_t)v * n + i];
    orc_pair *pairs = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(P > 0 ? P : 1));
    int64_t w = 0;
    for (int v = 0; v < n_views; ++v)
        for (int64_t i = 0; i < n; ++i) {
            const int64_t gi = (int64_t)v * n + i;
            if (touched[gi] == 0) continue;
            const int32_t *r = rect + 4 * gi;
            for (int ty = r[1]; ty <= r[3]; ++ty)
                for (int tx = r[0]; tx <= r[2]; ++tx) {
                    const uint64_t tile = (uint64_t)(tile_offset[v] + ty * tiles_x[v] + tx);
                    pairs[w].key = (tile << 32) | (uint64_t)depth_bits[gi];
                    pairs[w].val = (uint32_t)i;
                    pairs[w].pos = w;
                    ++w;
                }
        }
    qsort(pairs, (size_t)P, sizeof(orc_pair), pair_cmp);
    for (int64_t t = 0; t < 2 * total_tiles; ++t) ranges[t] = 0;
    for (int64_t k = 0; k < P; ++k) {
        keys[k] = pairs[k].key;
        vals[k] = pairs[k].val;
        const int64_t tile = (int64_t)(pairs[k].key >> 32);
        if (k == 0 || (pairs[k - 1].key >> 32) != (uint64_t)tile) ranges[2 * tile] = (uint32_t)k;
        if (k == P - 1 || (pairs[k + 1].key >> 32) != (uint64_t)tile) ranges[2 * tile + 1] = (uint32_t)(k + 1);
    }
    free(pairs);
    return P;
}

/* ------------------------------------------------------- compositing -- */
static inline uint64_t mix64(uint64_t h) {
    h ^= h >> 33; h *= 0xff51afd7ed558ccdULL; h ^= h >> 33; h *= 0xc4ceb9fe1a85ec53ULL; h ^= h >> 33;
    return h;
}

/* Eq. (alpha): alpha'(p) = min(alpha_max, o exp(-1/2 dp^T Q dp)). */
static inline double eval_alpha(const double *m2, const double *Q, double o, double px, double py,
                                double amax, double *G_out, int *clamped, double *dx_out, double *dy_out) {
    const double dx = px - m2[0], dy = py - m2[1];
    const double power = -0.5 * (Q[0] * dx * dx + 2.0 * Q[1] * dx * dy + Q[2] * dy * dy);
    const double G = exp(power);
    const double a = o * G;
    *G_out = G; *dx_out = dx; *dy_out = dy;
    *clamped = a > amax;
    return a > amax ? amax : a;
}

/* Margin test: is x within rel * |thr| of a threshold thr? */
static inline int near_thr(double x, double thr, double rel) { return fabs(x - thr) <= rel * fabs(thr); }

/* Tiled front-to-back compositing, Eq. (blend), of one view.
 * image is [3][H][W]; T_final, n_last (1 + position in the tile list of the
 * last contributor, 0 if none), n_contrib (number of contributors) and margin
 * (1 where some decision of the pixel lies within margin_rel of its
 * threshold) are [H][W].  Returns a hash of every discrete decision (each
 * contributor's list position, clamp state and the stop position). */
uint64_t orc_render(int W, int H, int32_t tile_offset, const double *mean2d, const double *conic,
                    const double *rgb, const double *opacity, const uint32_t *vals,
                    const uint32_t *ranges, const orc_raster *rc, double margin_rel,
                    double *image, double *T_final, int32_t *n_last, int32_t *n_contrib,
                    uint8_t *margin) {
    const int ts = rc->tile;
    const int tiles_x = (W + ts - 1) / ts, tiles_y = (H + ts - 1) / ts;
    uint64_t hash = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : hash)
    for (int tid = 0; tid < tiles_x * tiles_y; ++tid) {
        const int tx = tid % tiles_x, ty = tid / tiles_x;
        const uint32_t start = ranges[2 * (tile_offset + tid)], end = ranges[2 * (tile_offset + tid) + 1];
        for (int j = ty * ts; j < (ty + 1) * ts && j < H; ++j)
            for (int i = tx * ts; i < (tx + 1) * ts && i < W; ++i) {
                const double px = i + 0.5, py = j + 0.5; /* reading: pixel centres */
                double T = 1.0, C[3] = {0, 0, 0};
                int last = 0, cnt = 0, mg = 0;
                uint64_t h = mix64((uint64_t)(j * W + i) + 1);
                for (uint32_t k = start; k < end; ++k) {
                    const uint32_t gi = vals[k];
                    double G, dx, dy;
                    int cl;
                    const double a = eval_alpha(mean2d + 2 * gi, conic + 3 * gi, opacity[gi], px, py,
                                                rc->alpha_max, &G, &cl, &dx, &dy);
                    if (near_thr(a, rc->alpha_min, margin_rel)) mg = 1;
                    if (a < rc->alpha_min) continue;
                    const double testT = T * (1.0 - a);
                    if (near_thr(testT, rc->t_min, margin_rel)) mg = 1;
                    if (testT < rc->t_min) { h = mix64(h ^ (0x5700000000ULL + k)); break; }
                    for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * gi + ch] * a * T;
                    T = testT;
                    last = (int)(k - start) + 1;
                    ++cnt;
                    h = mix64(h ^ ((uint64_t)k << 1 | (uint64_t)cl));
                }
                for (int ch = 0; ch < 3; ++ch) image[(size_t)ch * W * H + (size_t)j * W + i] = C[ch] + T * rc->bg[ch];
                T_final[(size_t)j * W + i] = T;
                n_last[(size_t)j * W + i] = last;
                n_contrib[(size_t)j * W + i] = cnt;
                margin[(size_t)j * W + i] = (uint8_t)mg;
                hash += h;
            }
    }
    return hash;
}

/* Brute-force compositing: every pixel tests every non-culled Gaussian
 * (touched > 0), keeps those with alpha' >= alpha_min, orders them by
 * (float32 depth bits, index) and composites with the same stop rule.
 * No tiles, no rectangles: the definition of the contribution set. */
typedef struct { uint32_t dbits; uint32_t idx; double a; } orc_contrib;

static int contrib_cmp(const void *a, const void *b) {
    const orc_contrib *x = (const orc_contrib *)a, *y = (const orc_contrib *)b;
    if (x->dbits != y->dbits) return x->dbits < y->dbits ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

void orc_render_brute(int W, int H, int64_t n, const double *mean2d, const double *conic,
                      const double *rgb, const double *opacity, const uint32_t *depth_bits,
                      const int32_t *touched, const orc_raster *rc, double *image, double *T_final) {
#pragma omp parallel
    {
        orc_contrib *list = (orc_contrib *)malloc(sizeof(orc_contrib) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic)
        for (int pix = 0; pix < W * H; ++pix) {
            const int i = pix % W, j = pix / W;
            const double px = i + 0.5, py = j + 0.5;
            int64_t m = 0;
            for (int64_t g = 0; g < n; ++g) {
                if (touched[g] == 0) continue;
                double G, dx, dy;
                int cl;
                const double a = eval_alpha(mean2d + 2 * g, conic + 3 * g, opacity[g], px, py, rc->alpha_max,
                                            &G, &cl, &dx, &dy);
                if (a < rc->alpha_min) continue;
                list[m].dbits = depth_bits[g];
                list[m].idx = (uint32_t)g;
                list[m].a = a;
                ++m;
            }
            qsort(list, (size_t)m, sizeof(orc_contrib), contrib_cmp);
            double T = 1.0, C[3] = {0, 0, 0};
            for (int64_t k = 0; k < m; ++k) {
                const double testT = T * (1.0 - list[k].a);
                if (testT < rc->t_min) break;
                for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * list[k].idx + ch] * list[k].a * T;
                T = testT;
            }
            for (int ch = 0; ch < 3; ++ch) image[(size_t)ch * W * H + pix] = C[ch] + T * rc->bg[ch];
            T_final[pix] = T;
        }
        free(list);
    }
}

/* ---------------------------------------------------------- adjoint --
 * Raster adjoint of one view.  With A_k = sum_{j>k} c_j a_j T_j + T_end bg
 * (the colour behind contributor k), Eq. (blend) gives
 *   dC/dc_k = a_k T_k,   dC/da_k = c_k T_k - A_k / (1 - a_k).
 * Through Eq. (alpha): a = o G unless clamped (then the true derivative, 0),
 *   dG/dmean2d = G Q dp,  dG/dQ = -1/2 G dp dp^T.
 * Per Gaussian output g2d[9]: dL/dmean2d (2), dL/dQ (a, b, c with b the
 * shared off-diagonal parameter), dL/dopacity, dL/drgb (3).  Accumulated. */
static inline void atomic_addd(double *p, double v) {
#pragma omp atomic
    *p += v;
}

void orc_raster_bwd(int W, int H, int32_t tile_offset, const double *mean2d, const double *conic,
                    const double *rgb, const double *opacity, const uint32_t *vals,
                    const uint32_t *ranges, const orc_raster *rc, const double *dL_dimage,
                    double *g2d) {
    const int ts = rc->tile;
    const int tiles_x = (W + ts - 1) / ts, tiles_y = (H + ts - 1) / ts;
#pragma omp parallel
    {
        int cap = 1024;
        uint32_t *idx = (uint32_t *)malloc(sizeof(uint32_t) * cap);
        double *al = (double *)malloc(sizeof(double) * cap), *Gs = (double *)malloc(sizeof(double) * cap);
        double *Ts = (double *)malloc(sizeof(double) * cap), *dxs = (double *)malloc(sizeof(double) * cap);
        double *dys = (double *)malloc(sizeof(double) * cap);
        int *cls = (int *)malloc(sizeof(int) * cap);
#pragma omp for schedule(dynamic)
        for (int tid = 0; tid < tiles_x * tiles_y; ++tid) {
            const int tx = tid % tiles_x, ty = tid / tiles_x;
            const uint32_t start = ranges[2 * (tile_offset + tid)], end = ranges[2 * (tile_offset + tid) + 1];
            for (int j = ty * ts; j < (ty + 1) * ts && j < H; ++j)
                for (int i = tx * ts; i < (tx + 1) * ts && i < W; ++i) {
                    const double px = i + 0.5, py = j + 0.5;
                    /* forward replay: the contributor list with a, G, T */
                    double T = 1.0;
                    int m = 0;
                    for (uint32_t k = start; k < end; ++k) {
                        const uint32_t gi = vals[k];
                        double G, dx, dy;
                        int cl;
                        const double a = eval_alpha(mean2d + 2 * gi, conic + 3 * gi, opacity[gi], px, py,
                                                    rc->alpha_max, &G, &cl, &dx, &dy);
                        if (a < rc->alpha_min) continue;
                        const double testT = T * (1.0 - a);
                        if (testT < rc->t_min) break;
                        if (m == cap) {
                            cap *= 2;
                            idx = (uint32_t *)realloc(idx, sizeof(uint32_t) * cap);
                            al = (double *)realloc(al, sizeof(double) * cap);
                            Gs = (double *)realloc(Gs, sizeof(double) * cap);
                            Ts = (double *)realloc(Ts, sizeof(double) * cap);
                            dxs = (double *)realloc(dxs, sizeof(double) * cap);
                            dys = (double *)realloc(dys, sizeof(double) * cap);
                            cls = (int *)realloc(cls, sizeof(int) * cap);
                        }
                        idx[m] = gi; al[m] = a; Gs[m] = G; Ts[m] = T; dxs[m] = dx; dys[m] = dy; cls[m] = cl;
                        ++m;
                        T = testT;
                    }
                    double dC[3], A[3];
                    for (int ch = 0; ch < 3; ++ch) {
                        dC[ch] = dL_dimage[(size_t)ch * W * H + (size_t)j * W + i];
                        A[ch] = T * rc->bg[ch];
                    }
                    for (int k = m - 1; k >= 0; --k) {
                        const uint32_t gi = idx[k];
                        const double a = al[k], Tk = Ts[k];
                        double dL_da = 0.0;
                        for (int ch = 0; ch < 3; ++ch) {
                            const double c = rgb[3 * gi + ch];
                            atomic_addd(&g2d[9 * (size_t)gi + 6 + ch], dC[ch] * a * Tk);
                            dL_da += dC[ch] * (c * Tk - A[ch] / (1.0 - a));
                        }
                        for (int ch = 0; ch < 3; ++ch) A[ch] += rgb[3 * gi + ch] * a * Tk;
                        if (cls[k]) continue;
                        const double G = Gs[k], o = opacity[gi], dx = dxs[k], dy = dys[k];
                        atomic_addd(&g2d[9 * (size_t)gi + 5], dL_da * G);
                        const double dL_dG = dL_da * o;
                        const double *Q = conic + 3 * gi;
                        /* dp = p - mean2d, so d(dp)/d(mean2d) = -I and dG/dmean2d = +G Q dp */
                        atomic_addd(&g2d[9 * (size_t)gi + 0], dL_dG * G * (Q[0] * dx + Q[1] * dy));
                        atomic_addd(&g2d[9 * (size_t)gi + 1], dL_dG * G * (Q[1] * dx + Q[2] * dy));
                        atomic_addd(&g2d[9 * (size_t)gi + 2], dL_dG * (-0.5 * G * dx * dx));
                        atomic_addd(&g2d[9 * (size_t)gi + 3], dL_dG * (-G * dx * dy));
                        atomic_addd(&g2d[9 * (size_t)gi + 4], dL_dG * (-0.5 * G * dy * dy));
                    }
                }
        }
        free(idx); free(al); free(Gs); free(Ts); free(dxs); free(dys); free(cls);
    }
}

/* Projection adjoint: from g2d (see orc_raster_bwd) to the parameters.
 * Gradients are accumulated into the outputs (so views sum). */
void orc_project_bwd(int64_t n, int K, const double *means, const double *log_scales,
                     const double *quats, const double *opac_logit, const double *sh,
                     const orc_camera *cam, const orc_raster *rc, const double *g2d,
                     double *d_means, double *d_log_scales, double *d_quats, double *d_opac_logit,
                     double *d_sh) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        orc_gauss g;
        project_one(means + 3 * i, log_scales + 3 * i, quats + 4 * i, opac_logit[i], sh + 3 * K * i, K,
                    cam, rc, &g);
        if (g.culled) continue;
        const double *gd = g2d + 9 * i;
        double dmu[3] = {0, 0, 0};
        /* opacity: o = sigmoid(logit) */
        d_opac_logit[i] += gd[5] * g.o * (1.0 - g.o);
        /* colour: c = max(0, sum f Y + 0.5); the clamp passes no gradient */
        int deg = 0;
        while ((deg + 1) * (deg + 1) < K) ++deg;
        double Y[16], dY[16][3];
        sh_basis(deg, g.dir, Y, dY);
        double ddir[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            if (!(g.pre[ch] > 0.0)) continue;
            const double dc = gd[6 + ch];
            for (int k = 0; k < K; ++k) {
                d_sh[3 * K * i + 3 * k + ch] += dc * Y[k];
                for (int a = 0; a < 3; ++a) ddir[a] += dc * sh[3 * K * i + 3 * k + ch] * dY[k][a];
            }
        }
        /* dir = v / |v|: d dir / dv = (I - dir dir^T) / |v| */
        const double dd = ddir[0] * g.dir[0] + ddir[1] * g.dir[1] + ddir[2] * g.dir[2];
        for (int a = 0; a < 3; ++a) dmu[a] += (ddir[a] - g.dir[a] * dd) / g.vnorm;
        /* conic -> Sigma2D: dL/dSigma2D = -Q GQ Q (full symmetric matrices) */
        const double GQ[4] = {gd[2], 0.5 * gd[3], 0.5 * gd[3], gd[4]};
        const double Q[4] = {g.conic[0], g.conic[1], g.conic[1], g.conic[2]};
        double tmp[4], GS2[4];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) tmp[2 * r + c] = GQ[2 * r] * Q[c] + GQ[2 * r + 1] * Q[2 + c];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) GS2[2 * r + c] = -(Q[2 * r] * tmp[c] + Q[2 * r + 1] * tmp[2 + c]);
        /* Sigma2D = T Sigma T^T: dL/dT = 2 GS2 T Sigma, dL/dSigma = T^T GS2 T */
        double TS[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += g.T[3 * r + k] * g.Sigma[3 * k + c];
                TS[3 * r + c] = s;
            }
        double dT[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) dT[3 * r + c] = 2.0 * (GS2[2 * r] * TS[c] + GS2[2 * r + 1] * TS[3 + c]);
        double dSig[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) s += g.T[3 * a + r] * GS2[2 * a + b] * g.T[3 * b + c];
                dSig[3 * r + c] = s;
            }
        /* T = J Rc: dL/dJ = dL/dT Rc^T */
        double dJ[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += dT[3 * r + k] * cam->R[3 * c + k];
                dJ[3 * r + c] = s;
            }
        /* J(p) and mean2d(p) -> camera-space p */
        const double x = g.p[0], y = g.p[1], z = g.p[2], fx = cam->fx, fy = cam->fy;
        double dp[3] = {0, 0, 0};
        dp[2] += dJ[0] * (-fx / (z * z)) + dJ[4] * (-fy / (z * z));
        if (g.clamp_x == 0) {
            dp[0] += dJ[2] * (-fx / (z * z));
            dp[2] += dJ[2] * (2.0 * fx * x / (z * z * z));
        } else {
            const double lim = g.xt / z; /* +-limx */
            dp[2] += dJ[2] * (fx * lim / (z * z));
        }
        if (g.clamp_y == 0) {
            dp[1] += dJ[5] * (-fy / (z * z));
            dp[2] += dJ[5] * (2.0 * fy * y / (z * z * z));
        } else {
            const double lim = g.yt / z;
            dp[2] += dJ[5] * (fy * lim / (z * z));
        }
        dp[0] += gd[0] * fx / z;
        dp[1] += gd[1] * fy / z;
        dp[2] += -gd[0] * fx * x / (z * z) - gd[1] * fy * y / (z * z);
        /* p = Rc mu + t */
        for (int a = 0; a < 3; ++a) dmu[a] += cam->R[a] * dp[0] + cam->R[3 + a] * dp[1] + cam->R[6 + a] * dp[2];
        for (int a = 0; a < 3; ++a) d_means[3 * i + a] += dmu[a];
        /* Sigma = sum_k s_k^2 r_k r_k^T (r_k = column k of R) */
        double dR[9];
        for (int k = 0; k < 3; ++k) {
            double rk[3] = {g.R[k], g.R[3 + k], g.R[6 + k]};
            double Gr[3];
            for (int a = 0; a < 3; ++a) Gr[a] = dSig[3 * a] * rk[0] + dSig[3 * a + 1] * rk[1] + dSig[3 * a + 2] * rk[2];
            const double ds = 2.0 * g.s[k] * (rk[0] * Gr[0] + rk[1] * Gr[1] + rk[2] * Gr[2]);
            d_log_scales[3 * i + k] += ds * g.s[k];
            for (int a = 0; a < 3; ++a) dR[3 * a + k] = 2.0 * g.s[k] * g.s[k] * Gr[a];
        }
        /* R(qn), qn = q / |q| */
        double dRq[4][9], dqn[4];
        quat_to_rot_grad(g.qn, dRq);
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int e = 0; e < 9; ++e) s += dR[e] * dRq[c][e];
            dqn[c] = s;
        }
        const double qd = dqn[0] * g.qn[0] + dqn[1] * g.qn[1] + dqn[2] * g.qn[2] + dqn[3] * g.qn[3];
        for (int c = 0; c < 4; ++c) d_quats[4 * i + c] += (dqn[c] - g.qn[c] * qd) / g.qnorm;
    }
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
