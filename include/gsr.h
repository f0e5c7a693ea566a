/*
 * gsr.h - C ABI of the GB300 (sm_103a) 3DGS rasterizer and SkipGS gate.
 *
 * The calls follow the paper's statement of the problem:
 *   Sec. 3 (Preliminaries), Eq. (gaussian), (cov), (proj), (blend), (alpha),
 *   (loss); Sec. 3.1-3.3 and Algorithm 1 (SkipGS gating) with Eq. (view-ema),
 *   (deviation), (gate), (rhocum), (rhocum_check), (rhohat), (rhomincalib).
 *
 * Conventions shared by every call
 *   - Every function returns gs_status (GS_OK = 0).  Argument checks run on the
 *     host before anything is launched and return GS_ERR_INVALID_ARG or
 *     GS_ERR_WORKSPACE; a failed launch returns GS_ERR_CUDA.
 *   - Work is enqueued asynchronously on the given stream; the call does not
 *     synchronise.  Failures found on the device (pair capacity exceeded, a
 *     non-finite loss given to the gate) are written into the caller's device
 *     word `dev_status` (0 = no error; the first error wins) and the kernel
 *     skips the affected work.  Read it after synchronising.
 *   - All memory is owned by the caller: every pointer is a device pointer
 *     unless marked "host", arrays are dense, row-major, float32 unless stated.
 *     The library allocates no device memory; scratch space is passed in as a
 *     workspace whose size the matching *_workspace_size call returns.
 *   - No call reads back from the device, so every call can be captured into
 *     a CUDA graph; sizes that depend on data (the number of Gaussian x tile
 *     pairs) stay on the device.
 *
 * Layouts
 *   - Parameters of N Gaussians (gs_params): means [N,3], log_scales [N,3]
 *     (per-axis standard deviation s = exp(log_scale), Eq. cov), quats [N,4]
 *     (w,x,y,z; normalised inside), opacity_logit [N] (opacity =
 *     sigmoid(logit)), sh [N,K,3] with K = (sh_degree+1)^2 real SH
 *     coefficients per colour channel.  gs_param_layout gives the offsets of
 *     these groups inside one flat buffer (59 floats per Gaussian at degree 3
 *     plus alignment padding; means | log_scales | quats | opacity_logit | sh),
 *     the layout the optimizer step works on.  quats, and sh when 3K is a
 *     multiple of 4, must be 16-byte aligned.
 *   - Views: an array of gs_camera in device memory.  View v's tiles occupy
 *     global tile ids [tile_offset, tile_offset + tiles_x * tiles_y) and its
 *     pixels the image range starting at pix_offset, stored planar
 *     [3][height][width].  gs_camera_layout fills both offsets.
 *   - Projected Gaussians (gs_projected), per view and Gaussian, at index
 *     v * N + i: a 12-float record rec = (mean2d.x, mean2d.y, u00, u01, u11,
 *     opacity, r, g, b, depth, rx, ry), where U = [[u00, u01], [0, u11]] is
 *     the upper Cholesky factor of the conic Q = Sigma2D^-1 (Q = U^T U) and
 *     (rx, ry) bound the support (alpha' >= alpha_min only where
 *     |p.x - mean2d.x| <= rx and |p.y - mean2d.y| <= ry);
 *     rect = tile rectangle (x0, y0, x1, y1) inclusive; tiles_touched = its
 *     tile count (0 = culled).
 *   - Pixel centres are at (i + 0.5, j + 0.5); the principal point (cx, cy) is
 *     in the same continuous coordinates.
 */
#ifndef GSR_H
#define GSR_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,  /* a pointer, size or configuration value is invalid */
    GS_ERR_WORKSPACE = 2,    /* the workspace is missing or smaller than required */
    GS_ERR_CUDA = 3,         /* a CUDA runtime call failed (launch or capture) */
    GS_ERR_CAPACITY = 4,     /* device: more Gaussian x tile pairs than pair_capacity */
    GS_ERR_NONFINITE = 5,    /* device: the gate was given a NaN or infinite loss */
    GS_ERR_UNSUPPORTED = 6   /* a configuration this build does not provide */
} gs_status;

/* Human-readable name of a status code (static storage, never NULL). */
const char *gs_status_string(int status);

/* Library version as major * 10000 + minor * 100 + patch. */
int gs_version(void);

/* ---------------------------------------------------------------- types */

/* Pinhole camera of one view, Eq. (proj): world -> camera x_c = R x + t
 * (x right, y down, z forward); fx, fy, cx, cy in pixels; znear: Gaussians with
 * z <= znear are culled.  tile_offset / pix_offset: see Layouts above. */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear;
    int32_t tile_offset;
    int64_t pix_offset;
} gs_camera;

/* Rasterizer constants.  lowpass: isotropic dilation added to Sigma2D (px^2);
 * alpha_max (0.99), alpha_min (1/255) and t_min (1e-4): Eq. (alpha) clamp, the
 * cut-off below which a Gaussian is skipped at a pixel, and the transmittance
 * floor (a pixel stops before a Gaussian that would take T below it);
 * bg: background colour added with the final transmittance; tile: 8, 16 or
 * 32 (pixels per tile side); batch: Gaussians staged in shared memory per step
 * (64, 128 or 256); sh_degree: 0..3; pixels_per_thread: 1, 2, or 4 with tile
 * >= 16 (block shape of the compositing kernels; results do not depend on it). */
typedef struct {
    float lowpass, alpha_max, alpha_min, t_min;
    float bg[3];
    int32_t tile;
    int32_t batch;
    int32_t sh_degree;
    int32_t pixels_per_thread;
} gs_raster_config;

typedef struct {
    const float *means, *log_scales, *quats, *opacity_logit, *sh;
    int64_t n;
    int32_t sh_degree;
} gs_params;

typedef struct {
    float *means, *log_scales, *quats, *opacity_logit, *sh;
} gs_grads;

typedef struct {
    float *rec;              /* [V*N][12] */
    int32_t *rect;           /* [V*N][4]  */
    int32_t *tiles_touched;  /* [V*N]     */
    uint32_t *depth_key;     /* [V*N] or NULL: float32 bits of the depth, 0xffffffff when culled */
    uint16_t *rect16;        /* [V*N][4] or NULL (8-byte aligned): rect as (x0, y0, width, height) in tiles,
                                all 0 when culled */
} gs_projected;

/* State the forward pass saves for the backward pass (caller-owned):
 *   T_final [total pixels]: transmittance after the pixel's last contributor;
 *   n_last  [total pixels]: 1 + position, in its tile's list, of the pixel's
 *            last contributor (0 = none);
 *   ckpt    [ckpt_slots][tile*tile]: transmittance of every pixel at the
 *            start of each staging batch the forward pass processed after the
 *            tile's first (which starts at T = 1; its slot is not written)
 *            (per-tile transmittance checkpoints); gs_ckpt_slots gives
 *            ckpt_slots. */
typedef struct {
    float *T_final;
    int32_t *n_last;
    float *ckpt;
    int64_t ckpt_slots;
    const uint32_t *tile_order;  /* [total_tiles] visiting order of the tiles (gs_tile_order), or NULL for
                                    ascending tile id; a permutation of 0..total_tiles-1; results do not
                                    depend on it */
    uint32_t *queue;             /* NULL: one block per tile; else a device word (4-byte aligned) through
                                    which a persistent grid of resident blocks takes the tiles in
                                    tile_order (reset by each compositing call, so the calls that share it
                                    must be ordered on one stream); results do not depend on it */
    uint32_t *batch_pos;         /* [ckpt_slots] for the *_coarse calls (else ignored, may be NULL): per
                                    checkpoint slot, the super-tile list position of the batch's first
                                    Gaussian (written by gs_render_fwd_coarse, read by the adjoints) */
} gs_fwd_saved;

/* Super-tile lists, the output of gs_bin_sort_coarse and the input of the
 * *_coarse compositing calls.  The (view, Gaussian) entries are listed once
 * per super-tile of 4 x 4 tiles that their tile rectangle meets, in depth
 * order, each as its Gaussian index and a 16-bit mask of the super-tile's
 * tiles the rectangle covers (bit 4 * row + column, rows and columns counted
 * from the super-tile's first tile).  A view's super-tiles cover its tile grid
 * row-major in steps of 4 tiles (the last row and column may be partial);
 * views follow one another.  A tile's list as gs_bin_sort writes it is
 * exactly the entries of its super-tile's list with the tile's bit set, in
 * the same order: the compositing kernels filter it out as they stage it and
 * only as far as the tile's pixels need, so the tile lists are never
 * written.  Caller-owned device buffers:
 *   gid        [capacity] Gaussian index within its view;
 *   mask       [capacity] covered tiles (16-byte aligned);
 *   start      [total_tiles / 4 + n_views] first list entry of each super-tile;
 *   count      [total_tiles / 4 + n_views] its number of entries (0 past the last super-tile);
 *   view_first [n_views + 1] first super-tile of each view, then the super-tile total;
 *   total      [1] number of entries of all lists (written also when above capacity);
 *   capacity   at most 2^32 - 65536. */
typedef struct {
    uint32_t *gid;
    uint16_t *mask;
    uint32_t *start;
    uint32_t *count;
    int64_t *view_first;
    int64_t *total;
    int64_t capacity;
} gs_coarse_lists;

/* --------------------------------------------------------------- layout */

/* Offsets (in floats) of the parameter groups inside one flat buffer for N
 * Gaussians: out[0..5] = means, log_scales, quats, opacity_logit, sh, end.
 * Each group starts on a 256-byte boundary (padding floats between groups are
 * ignored by the kernels and stay zero under the optimizer). */
gs_status gs_param_layout(int64_t n, int32_t sh_degree, int64_t *out6 /* host */);

/* Fills tile_offset and pix_offset of n_views host-side cameras for `tile`,
 * and returns the total tile and pixel counts (host pointers). */
gs_status gs_camera_layout(gs_camera *cams /* host */, int32_t n_views, int32_t tile,
                           int64_t *total_tiles, int64_t *total_pixels);

/* Number of per-tile transmittance checkpoint slots needed for pair_capacity
 * pairs over total_tiles tiles at staging batch `batch`. */
int64_t gs_ckpt_slots(int64_t pair_capacity, int64_t total_tiles, int32_t batch);

/* ------------------------------------------------------------ projection */

/* Eq. (cov) and Eq. (proj) for n_views views: Sigma = R S S^T R^T, camera
 * transform, EWA Jacobian J (x/z, y/z clamped to 1.3x the half field of view),
 * Sigma2D = J W Sigma W^T J^T + lowpass I, conic factor U, mean2D, depth,
 * opacity = sigmoid(logit), colour = max(0, sum_k f_k Y_k(d) + 0.5) for the
 * direction d from the camera centre (real SH, Condon-Shortley phase), and
 * the conservative tile rectangle of the region where alpha' >= alpha_min
 * can hold: the bounding box of the ellipse dp^T Q dp <= c with
 * c = 2 ln(opacity / alpha_min), i.e. half-extents r_x = sqrt(c Sigma2D_xx),
 * r_y = sqrt(c Sigma2D_yy), inflated by x1.0001 + 0.001 px for float32
 * rounding (stored in the record's last two floats).  Every parameter array
 * must start on a 16-byte boundary (the groups of gs_param_layout do). */
gs_status gs_project(const gs_params *params /* host */, const gs_camera *cams, int32_t n_views, const gs_raster_config *cfg /* host */, gs_projected out,
                     int32_t *dev_status, cudaStream_t stream);

/* ------------------------------------------------------ binning and sort */

/* Scratch bytes gs_bin_sort needs for n Gaussians x n_views views over
 * total_tiles tiles and pair_capacity pairs (about 6 bytes per pair of
 * capacity: the entries listed by super-tile of 4 x 4 tiles, at most one per
 * pair, as a Gaussian index and a mask of covered tiles). */
size_t gs_bin_sort_workspace_size(int64_t n, int32_t n_views, int64_t pair_capacity, int64_t total_tiles);

/* Tile binning + depth order ("depth-sorted Gaussians overlapping a pixel",
 * Sec. 3): every (Gaussian, tile of its rectangle) pair, ordered by
 * (global tile id, float32 bits of depth, Gaussian index) - the stable sort
 * of the 64-bit keys (tile << 32 | depth bits) in emission order.  Writes
 * vals[pair] = Gaussian index, ranges[tile] = [start, end) (empty = [0,0)),
 * *dev_pair_count, and - if keys is not NULL - the 64-bit keys.
 * max_view_tiles: the largest tile count of one view (0 = total_tiles); at
 * most 20480, else GS_ERR_UNSUPPORTED; a view with more tiles than given
 * sets GS_ERR_INVALID_ARG in dev_status and emits no pairs.  Rectangles are
 * clipped to the view's tile grid; entries with tiles_touched <= 0 emit
 * nothing.  More pairs than pair_capacity: GS_ERR_CAPACITY in dev_status,
 * the full count in *dev_pair_count, ranges left empty, vals untouched.
 * Only the tile geometry of cams is read.  If proj->depth_key and
 * proj->rect16 are set (written by gs_project with the same cfg) the sort
 * reads them instead of deriving them from rec, rect and tiles_touched. */
gs_status gs_bin_sort(const gs_projected *proj /* host */, const gs_camera *cams, int32_t n_views, int64_t n,
                      int64_t total_tiles, int32_t max_view_tiles, const gs_raster_config *cfg /* host */,
                      void *workspace, size_t workspace_bytes, uint64_t *keys, uint32_t *vals,
                      int64_t pair_capacity, uint32_t *ranges, int64_t *dev_pair_count,
                      int32_t *dev_status, cudaStream_t stream);

/* The super-tile form of gs_bin_sort: the same depth order and tile
 * rectangles, written as the super-tile lists of `lists` (gs_coarse_lists, a
 * host struct of device pointers) instead of per-tile lists; the pairs are
 * counted but not placed.  ranges[tile] = the [start, end) that gs_bin_sort
 * writes (where the tile's pairs would lie in its vals; the *_coarse
 * compositing calls take their checkpoint slots from them, gs_tile_order its
 * order).  max_view_super_tiles: the largest super-tile count of one view,
 * ceil(tiles_x / 4) * ceil(tiles_y / 4), or 0 to bound it by
 * max_view_tiles / 4 + 1 (the bound of the skinniest grid); a tighter bound
 * lets more of the placement's warps share an SM; a view with more super-tiles
 * than it sets GS_ERR_INVALID_ARG in dev_status and emits nothing.
 * *dev_pair_count as gs_bin_sort (the pairs are counted from the
 * lists' masks; 0 when the lists did not fit); more pairs than
 * pair_capacity, or more list entries than lists->capacity (at most one per
 * pair): GS_ERR_CAPACITY in dev_status, ranges left empty.  workspace: at least
 * gs_bin_sort_coarse_workspace_size(n, n_views, total_tiles) bytes, 256-byte
 * aligned.  Other arguments and errors as gs_bin_sort. */
size_t gs_bin_sort_coarse_workspace_size(int64_t n, int32_t n_views, int64_t total_tiles);
gs_status gs_bin_sort_coarse(const gs_projected *proj /* host */, const gs_camera *cams, int32_t n_views, int64_t n,
                             int64_t total_tiles, int32_t max_view_tiles, int32_t max_view_super_tiles,
                             const gs_raster_config *cfg /* host */,
                             void *workspace, size_t workspace_bytes, const gs_coarse_lists *lists /* host */,
                             int64_t pair_capacity, uint32_t *ranges, int64_t *dev_pair_count, int32_t *dev_status,
                             cudaStream_t stream);

/* gs_bin_sort without a caller-provided workspace, for callers that cannot
 * allocate device memory: work issued while a CUDA graph is being captured
 * (cudaMalloc cannot be captured), plugins whose host application owns all
 * device memory, real-time loops that must not block on the allocator.  The
 * paper has no counterpart; it is a deployment variant of gs_bin_sort.
 * The scratch is a fixed 16 MB array in the library's device memory (on
 * every GPU that loads the library, until the process exits), so the sizes
 * are capped: n * n_views <= 262144 entries and
 * gs_bin_sort_workspace_size(...) <= 16 MB; larger requests return
 * GS_ERR_WORKSPACE and launch nothing.
 * Each call outside stream capture looks up the array's device address with
 * the device current; a call during capture reuses the address of the last
 * call outside capture on that device, so make one call before any stream
 * capture, and again after the device's context was reset (cudaDeviceReset
 * invalidates the address a captured graph holds: capture again).  Every call
 * shares the one array: calls that overlap on the GPU (different streams, or
 * other threads) race and must be serialised by the caller.  Nothing in the
 * array needs to start at zero: each call overwrites all scratch it reads.
 * Other arguments, outputs and errors as gs_bin_sort. */
gs_status gs_bin_sort_noalloc(const gs_projected *proj /* host */, const gs_camera *cams, int32_t n_views, int64_t n,
                              int64_t total_tiles, int32_t max_view_tiles, const gs_raster_config *cfg /* host */,
                              uint64_t *keys, uint32_t *vals, int64_t pair_capacity, uint32_t *ranges,
                              int64_t *dev_pair_count, int32_t *dev_status, cudaStream_t stream);

/* --------------------------------------------------------------- forward */

/* Visiting order of the tiles for the compositing kernels, longest list
 * first: tiles grouped by x = list length + 1 (ranges from gs_bin_sort) into
 * 8 (bit length of x - 1) + (the three bits of x after its leading one),
 * eight groups per doubling, longest group first; the order within a group
 * is unspecified.  Writes tile_order[total_tiles], a
 * permutation of 0..total_tiles-1, for gs_fwd_saved.tile_order.  The paper
 * has no counterpart: it is a scheduling choice (one CTA per tile, launched
 * in this order) that changes no result. */
gs_status gs_tile_order(const uint32_t *ranges, int64_t total_tiles, uint32_t *tile_order, cudaStream_t stream);

/* Eq. (blend) and Eq. (alpha): per tile, Gaussians staged `batch` at a time in
 * shared memory; per pixel front to back alpha' = min(alpha_max, o exp(-1/2
 * dp^T Q dp)), skip alpha' < alpha_min, stop before a Gaussian with
 * T (1 - alpha') < t_min, C += c alpha' T, T *= 1 - alpha'; C += T bg.
 * image: planar float [3][H][W] per view at pix_offset.  Saves state for
 * gs_render_bwd. */
gs_status gs_render_fwd(const gs_projected *proj /* host */, int64_t n, const uint32_t *vals,
                        const uint32_t *ranges, const gs_camera *cams, int32_t n_views,
                        int64_t total_tiles, const gs_raster_config *cfg /* host */, float *image, gs_fwd_saved saved, int32_t *dev_status, cudaStream_t stream);

/* gs_render_fwd reading the super-tile lists of gs_bin_sort_coarse (lists:
 * host struct, device buffers; ranges from the same call) instead of tile
 * lists: every output bit for bit as gs_render_fwd on gs_bin_sort's lists of
 * the same projection (the same Gaussians in the same order per tile), and
 * saved.batch_pos (required) receives, per processed batch, the list position
 * of its first Gaussian for the *_coarse adjoints. */
gs_status gs_render_fwd_coarse(const gs_projected *proj /* host */, int64_t n, const gs_coarse_lists *lists /* host */,
                               const uint32_t *ranges, const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                               const gs_raster_config *cfg /* host */, float *image, gs_fwd_saved saved,
                               int32_t *dev_status, cudaStream_t stream);

/* ------------------------------------------------------------------ loss */

/* Scratch bytes of gs_loss for these views (host cameras; width, height and
 * pix_offset are read). */
size_t gs_loss_workspace_size(const gs_camera *cams_host, int32_t n_views);

/* Eq. (loss): L_v = (1 - lambda) mean|C - C_hat| + lambda (1 - mean SSIM) per
 * view (11x11 Gaussian window, sigma 1.5, C1 = 0.01^2, C2 = 0.03^2, zero
 * padding, 'same' size, means over 3HW).  cams_host: the views' cameras in
 * host memory (only width, height and pix_offset are read); cams_dev (device
 * memory, nullable): when given, view v's actual width and height are read
 * from cams_dev[v] on the device - at most cams_host[v]'s, which then give
 * the launch size and the slot's capacity (views chosen on the device, e.g.
 * by gs_select_views inside a captured step).  image: as
 * written by gs_render_fwd; target: same layout, or - when target_offsets is
 * given - view slot v's target starts at target + target_offsets[view_ids[v]]
 * (floats; view_ids in device memory).  Writes
 * loss_per_view[n_views] (the gate's input) and keeps the SSIM partial
 * derivatives in the workspace for gs_loss_backward.  If dL_dimage is not NULL
 * the gradient is written too (as gs_loss_backward would). */
gs_status gs_loss(const float *image, const float *target, const int64_t *target_offsets,
                  const gs_camera *cams_host, const gs_camera *cams_dev, const int32_t *view_ids, int32_t n_views,
                  float lambda_ssim, void *workspace, size_t workspace_bytes, float *loss_per_view,
                  float *dL_dimage, cudaStream_t stream);

/* dL/dimage from the state gs_loss left in the workspace (same arguments). */
gs_status gs_loss_backward(const float *image, const float *target, const int64_t *target_offsets,
                           const gs_camera *cams_host, const gs_camera *cams_dev, const int32_t *view_ids,
                           int32_t n_views, float lambda_ssim, void *workspace, size_t workspace_bytes,
                           float *dL_dimage, cudaStream_t stream);

/* -------------------------------------------------------------- backward */

size_t gs_render_bwd_workspace_size(int64_t n, int32_t n_views);

/* Analytic adjoint of gs_render_fwd and gs_project (the paper's
 * differentiable rasterizer, Sec. 3).  Per tile, pixels walk their list back
 * to front from their last contributor, rebuilding T from the per-batch
 * checkpoints; per-pair gradients of (mean2D, conic, opacity, colour) are
 * reduced across the warp with shuffles, across the block in shared memory,
 * and added to a per-view, per-Gaussian buffer with vector float atomics;
 * a per-Gaussian pass then chains them to the parameters.  view_gate
 * (nullable, device u8[n_views]): views with 0 contribute nothing.  grads are
 * overwritten (accumulate = 0) or added to (accumulate = 1); views are summed. */
gs_status gs_render_bwd(const gs_params *params /* host */, const gs_projected *proj /* host */,
                        const uint32_t *vals, const uint32_t *ranges, const gs_camera *cams,
                        int32_t n_views, int64_t total_tiles,
                        const gs_raster_config *cfg /* host */, gs_fwd_saved saved, const float *dL_dimage,
                        const uint8_t *view_gate, gs_grads grads, int32_t accumulate, void *workspace,
                        size_t workspace_bytes, int32_t *dev_status, cudaStream_t stream);

/* The two passes of gs_render_bwd as separate calls (gs_render_bwd = the
 * first followed by the second on the same g2d buffer):
 * gs_raster_bwd - the raster adjoint: per view and Gaussian the gradients of
 *   the loss with respect to (mean2D.x, mean2D.y, conic a, b, c, opacity, r, g,
 *   b) into g2d [n_views][n][12] floats (3 padding; zeroed first; 16-byte
 *   aligned; g2d_bytes >= gs_render_bwd_workspace_size(n, n_views)), where
 *   the conic Q = [[a, b], [b, c]] is parameterised by its three entries;
 * gs_project_bwd - the projection adjoint from g2d to the parameters, views
 *   summed; grads overwritten (accumulate = 0) or added to.
 * Parameter pointers must be 16-byte aligned (as inside gs_param_layout). */
gs_status gs_raster_bwd(const gs_projected *proj /* host */, int64_t n, const uint32_t *vals, const uint32_t *ranges,
                        const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                        const gs_raster_config *cfg /* host */, gs_fwd_saved saved, const float *dL_dimage,
                        const uint8_t *view_gate, float *g2d, size_t g2d_bytes, int32_t *dev_status,
                        cudaStream_t stream);
gs_status gs_project_bwd(const gs_params *params /* host */, const gs_camera *cams, int32_t n_views,
                         const gs_raster_config *cfg /* host */, const float *g2d, const uint8_t *view_gate,
                         gs_grads grads, int32_t accumulate, int32_t *dev_status, cudaStream_t stream);

/* gs_render_bwd and gs_raster_bwd over the super-tile lists (lists and
 * ranges of gs_bin_sort_coarse, saved from gs_render_fwd_coarse, whose
 * batch_pos they read): the same gradients up to the order of float atomics. */
gs_status gs_render_bwd_coarse(const gs_params *params /* host */, const gs_projected *proj /* host */,
                               const gs_coarse_lists *lists /* host */, const uint32_t *ranges, const gs_camera *cams,
                               int32_t n_views, int64_t total_tiles, const gs_raster_config *cfg /* host */,
                               gs_fwd_saved saved, const float *dL_dimage, const uint8_t *view_gate, gs_grads grads,
                               int32_t accumulate, void *workspace, size_t workspace_bytes, int32_t *dev_status,
                               cudaStream_t stream);
gs_status gs_raster_bwd_coarse(const gs_projected *proj /* host */, int64_t n, const gs_coarse_lists *lists /* host */,
                               const uint32_t *ranges, const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                               const gs_raster_config *cfg /* host */, gs_fwd_saved saved, const float *dL_dimage,
                               const uint8_t *view_gate, float *g2d, size_t g2d_bytes, int32_t *dev_status,
                               cudaStream_t stream);

/* ----------------------------------------------------------------- Adam */
/* (gs_adam_config and gs_adam_step below; gs_render_bwd_adam after them.) */

/* Adam (Kingma & Ba, bias-corrected), the optimizer step of Algorithm 1.
 * lr[6]: means, log_scales, quats, opacity, SH DC, SH higher bands.
 * lr_scale_den: 0, or (with a step-gate word dev_do_step) the learning rates
 * of a step are multiplied by *dev_do_step / lr_scale_den - for a batched
 * step whose gate word holds the number of views the gate opened
 * (skipgs_gate_decide's dev_any) out of lr_scale_den, so the step moves by
 * the opened views' share of the batch (a reading of Algorithm 1 for
 * several views per step; the paper decides one view per step). */
typedef struct {
    float lr[6];
    float beta1, beta2, eps;
    int32_t lr_scale_den;
} gs_adam_config;

/* One fused update of every scalar of the flat parameter buffer (layout of
 * gs_param_layout): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr m_hat / (sqrt(v_hat) + eps); zero_grad != 0 also sets g = 0.
 * dev_step (int64, device) counts executed steps and is incremented.
 * dev_do_step (nullable, int32 device): when it holds 0 nothing changes.
 * norms2 (nullable, 2 doubles, device): the step adds sum g^2 and
 * sum (p_new - p_old)^2 over all scalars to norms2[0] and norms2[1]
 * (telemetry of gradient and update norms; the caller resets them). */
gs_status gs_adam_step(float *params, float *grads, float *m, float *v, int64_t n, int32_t sh_degree,
                       const gs_adam_config *cfg /* host */, const int32_t *dev_do_step, int64_t *dev_step,
                       int32_t zero_grad, double *norms2, cudaStream_t stream);

/* The backward pass and the optimizer step of Algorithm 1 in one call: the
 * adjoint of gs_render_bwd, after which every parameter of the flat buffer
 * (gs_param_layout) takes one Adam step with the gradient just computed,
 * without storing the gradient.  Equal to gs_render_bwd (accumulate = 0)
 * followed by gs_adam_step; dev_do_step, dev_step and norms2 (nullable) as in
 * gs_adam_step, view_gate as in gs_render_bwd.  The projection adjoint and the
 * Adam step run in one kernel, so the parameter gradients never reach DRAM.
 * flat_params, m and v: device, caller-owned, gs_param_layout(n, sh_degree)
 * floats each, 16-byte aligned, updated in place.  workspace: device, at least
 * gs_render_bwd_workspace_size(n, n_views) bytes, 16-byte aligned (the 2D
 * gradients).  Returns GS_ERR_INVALID_ARG (null or unaligned pointers,
 * sh_degree outside 0..3 or unlike cfg->sh_degree, beta outside [0, 1),
 * eps < 0) or GS_ERR_WORKSPACE before any launch. */
gs_status gs_render_bwd_adam(float *flat_params, float *m, float *v, int64_t n, int32_t sh_degree,
                             const gs_projected *proj /* host */, const uint32_t *vals, const uint32_t *ranges,
                             const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                             const gs_raster_config *cfg /* host */, gs_fwd_saved saved, const float *dL_dimage,
                             const uint8_t *view_gate, const gs_adam_config *adam /* host */,
                             const int32_t *dev_do_step, int64_t *dev_step, double *norms2, void *workspace,
                             size_t workspace_bytes, int32_t *dev_status, cudaStream_t stream);

/* gs_render_bwd_adam over the super-tile lists (as gs_render_bwd_coarse). */
gs_status gs_render_bwd_adam_coarse(float *flat_params, float *m, float *v, int64_t n, int32_t sh_degree,
                                    const gs_projected *proj /* host */, const gs_coarse_lists *lists /* host */,
                                    const uint32_t *ranges, const gs_camera *cams, int32_t n_views,
                                    int64_t total_tiles, const gs_raster_config *cfg /* host */, gs_fwd_saved saved,
                                    const float *dL_dimage, const uint8_t *view_gate,
                                    const gs_adam_config *adam /* host */, const int32_t *dev_do_step,
                                    int64_t *dev_step, double *norms2, void *workspace, size_t workspace_bytes,
                                    int32_t *dev_status, cudaStream_t stream);

/* The second half of gs_render_bwd_adam on its own: the projection adjoint of
 * the 2D gradients that gs_raster_bwd left in g2d (device, layout and
 * alignment as there), fused with the Adam step as above.  gs_raster_bwd
 * followed by this call equals gs_render_bwd_adam.  Argument checks as for
 * gs_render_bwd_adam (GS_ERR_INVALID_ARG before any launch). */
gs_status gs_project_bwd_adam(float *flat_params, float *m, float *v, int64_t n, int32_t sh_degree,
                              const gs_camera *cams, int32_t n_views, const gs_raster_config *cfg /* host */,
                              const float *g2d, const uint8_t *view_gate, const gs_adam_config *adam /* host */,
                              const int32_t *dev_do_step, int64_t *dev_step, double *norms2, int32_t *dev_status,
                              cudaStream_t stream);

/* ----------------------------------------------------------- SkipGS gate */

/* Gate hyperparameters (Sec. 4.1): W = 500, beta = 0.95, eps = 1e-8,
 * rho_lo = 0.5.  rho_lo < 0 selects the ablation without budget control
 * (Table 4). */
typedef struct {
    int32_t W;
    double beta, eps, rho_lo;
    int32_t n_views;
} gs_gate_config;

/* Bytes of device state for a gate over n_views training views. */
size_t skipgs_gate_state_size(int32_t n_views);

/* Initialise the state (Algorithm 1: EMA table empty, rho_min = rho_lo, b = 0). */
gs_status skipgs_gate_init(const gs_gate_config *cfg /* host */, void *dev_state, cudaStream_t stream);

/* Algorithm 1, per loss in order (reading: each one is its own iteration t, and
 * all losses of one call are compared with the EMA as it stood before the
 * call - they come from the same parameters; skipgs_gate_update then applies
 * their EMA updates in order):
 * deviation score s = L / (EMA + eps) or +inf without history (Eq. deviation),
 * skip test g = [s > 1] (Eq. gate); during warmup (t <= W) the test is recorded
 * for views with history and g is forced to 1; at t = W + 1 rho_min = rho_lo +
 * (1 - rho_lo) rho_hat (Eq. rhohat, rhomincalib); after warmup g is forced to 1
 * when b / max(t-1, 1) < rho_min (Eq. rhocum_check); b += g.  All arithmetic
 * in binary64 with one rounding per operation.  Writes g[n] (u8) and, if
 * given, *dev_any = OR of g (int32) and the graph conditional `cond` (host
 * pointer to a handle created for the graph being captured; NULL outside a
 * graph).  A non-finite loss: g = 0, state untouched, GS_ERR_NONFINITE.
 * *dev_any holds the number of g = 1 (nonzero exactly when any view opened). */
gs_status skipgs_gate_decide(void *dev_state, const int32_t *dev_view_ids, const float *dev_losses, int32_t n,
                             uint8_t *dev_g, int32_t *dev_any, const cudaGraphConditionalHandle *cond,
                             int32_t *dev_status, cudaStream_t stream);

/* Eq. (view-ema), unconditional after the decision: EMA_v = beta EMA_v +
 * (1 - beta) L, or L on the view's first observation. */
gs_status skipgs_gate_update(void *dev_state, const int32_t *dev_view_ids, const float *dev_losses, int32_t n,
                             cudaStream_t stream);

/* Copies the scalar part of the state to host memory for inspection:
 * out[0..6] = t, b, n_w, n_w1, calibrated, errors, n_views (int64, host) and
 * rho_min (double, host).  Synchronises the stream. */
gs_status skipgs_gate_read(const void *dev_state, int64_t *out7 /* host */, double *rho_min /* host */,
                           cudaStream_t stream);

/* ------------------------------------------------------------ step graph */

/* Small helpers that build one refinement step as a CUDA graph whose backward
 * branch is a conditional IF node set on the device by skipgs_gate_decide.
 * Capture is stream capture: between gs_graph_begin and gs_graph_end only gs_*
 * calls (and other capturable work) may be issued on `stream`. */
typedef struct gs_graph_s *gs_graph;

gs_status gs_graph_begin(cudaStream_t stream);
/* Creates a conditional handle in the graph being captured on `stream`
 * (default value 0). */
gs_status gs_graph_cond_create(cudaStream_t stream, cudaGraphConditionalHandle *out /* host */);
/* Adds an IF node on `cond` after the work captured so far on `stream`, and
 * starts capturing `body_stream` into its body. */
gs_status gs_graph_if_begin(cudaStream_t stream, cudaGraphConditionalHandle cond, cudaStream_t body_stream);
/* Ends the body capture; later work on `stream` runs after the IF node. */
gs_status gs_graph_if_end(cudaStream_t stream, cudaStream_t body_stream);
gs_status gs_graph_end(cudaStream_t stream, gs_graph *out /* host */);
gs_status gs_graph_launch(gs_graph graph, cudaStream_t stream);
/* Kernel nodes of the graph: out2[0] outside, out2[1] inside the IF bodies
 * (host pointer).  One replay launches out2[0] kernels, plus out2[1] when the
 * gate opens the branch. */
gs_status gs_graph_kernel_counts(gs_graph graph, int64_t *out2 /* host */);
gs_status gs_graph_destroy(gs_graph graph);

/* Device-side view selection for graph replay: view_ids[k] =
 * seq[(*iter * n + k) mod seq_len] for k < n, then *iter += 1 (int64, device).
 * If pose_src and slots are given, slot k takes the pose, intrinsics, size and
 * near plane of pose_src[view_ids[k]] and keeps its own pix_offset, so a
 * captured step renders the selected views; a view larger than the slot's
 * capacity is the caller's error.  tile = 0: each slot keeps its tile_offset
 * (every slot a grid of the largest view's size); tile = 8, 16 or 32: each
 * slot's tile_offset is recomputed so the selected views' own tile grids
 * follow one another from slot 0's offset (the slots' total tile count still
 * bounds them; the tiles past the last view's grid render nothing). */
gs_status gs_select_views(const int32_t *seq, int64_t seq_len, int64_t *iter, int32_t n, int32_t *view_ids,
                          const gs_camera *pose_src, gs_camera *slots, int32_t tile, cudaStream_t stream);

/* Per-view optimizer steps of a batched iteration (one reading of Algorithm 1
 * for several views per step: the views of a batch are consecutive
 * iterations whose forward passes share the batch's parameters, and each
 * opened view takes its own Adam step, in slot order, on its own gradient).
 * From the gate's decisions g[n] (device u8; may be NULL with all_open)
 * writes gates[k][j] = 1 exactly when j == k and view k opened (or
 * all_open), as the view_gate of slot k's gs_project_bwd_adam call, and
 * do_steps[k] (int32) = whether view k opened (or all_open), as its
 * dev_do_step.  n <= 1024.  The paper has no counterpart (it decides one
 * view per iteration). */
gs_status gs_view_steps(const uint8_t *g, int32_t n, int32_t all_open, uint8_t *gates, int32_t *do_steps,
                        cudaStream_t stream);

/* Per-iteration log for graph replay: with k = (*iter - 1) mod cap (iter as
 * advanced by gs_select_views), writes loss_log[k n + j] = loss[j] and
 * g_log[k n + j] = g[j] for j < n; if norms2 and norm_log are given, also
 * norm_log[2k .. 2k+1] = norms2[0..1] and then norms2 = 0 (the telemetry of
 * gs_adam_step for this iteration; 0 when no step ran).  All device memory. */
gs_status gs_log_step(const int64_t *iter, int32_t n, const float *loss, const uint8_t *g, double *norms2,
                      float *loss_log, uint8_t *g_log, double *norm_log, int64_t cap, cudaStream_t stream);

/* ------------------------------------------------------------- autotuning */

/* A launch shape of the rasterizer: tile side (8, 16, 32), staging batch (64,
 * 128, 256) and pixels per thread of the forward and adjoint compositing
 * kernels (1, 2, or 4 with tile >= 16).  Shapes change how the work maps to
 * the GPU, not the results (the contribution set does not depend on the tile
 * size; gradients equal up to the order of float atomics). */
typedef struct {
    int32_t tile, batch, pixels_per_thread_fwd, pixels_per_thread_bwd;
} gs_launch_shape;

/* Scratch bytes gs_autotune needs: the buffers of one rasterization
 * pipeline over these views for the largest candidate (invalid candidates
 * are ignored).  0 for invalid arguments. */
size_t gs_autotune_workspace_size(int64_t n, int32_t sh_degree, const gs_camera *cams_host, int32_t n_views,
                                  int64_t pair_capacity, const gs_launch_shape *cands, int32_t n_cands);

/* Times each candidate shape on the caller's workload: one untimed, then
 * `reps` timed iterations of gs_project -> gs_bin_sort -> gs_tile_order ->
 * gs_render_fwd -> gs_loss (with its gradient, lambda_ssim) -> gs_render_bwd
 * over all n_views views in one call, with CUDA events on `stream`
 * (synchronises; not capturable).  params: device parameters (as gs_project);
 * cams_host: the views (host; tile_offset and pix_offset are filled per
 * candidate, the input is not modified); target: device, planar [3][H][W]
 * per view in view order (the layout of gs_render_fwd's image, which does
 * not depend on the tile); base: the rasterizer constants (tile, batch and
 * pixels per thread are taken from each candidate).  Writes ms_per_iter[c]
 * (host; +infinity for a candidate this workload cannot use: an invalid
 * shape, a view with more tiles than the binning holds, more pairs than
 * pair_capacity) and *best (host) = the fastest candidate's index.  All
 * buffers are carved from `workspace` (device, 256-byte aligned, at least
 * gs_autotune_workspace_size bytes, else GS_ERR_WORKSPACE); the library
 * allocates nothing.  GS_ERR_UNSUPPORTED when no candidate runs. */
gs_status gs_autotune(const gs_params *params /* host */, const gs_camera *cams_host, int32_t n_views,
                      const float *target, const gs_raster_config *base /* host */, float lambda_ssim,
                      const gs_launch_shape *cands /* host */, int32_t n_cands, int32_t reps, int64_t pair_capacity,
                      void *workspace, size_t workspace_bytes, float *ms_per_iter /* host */,
                      int32_t *best /* host */, cudaStream_t stream);

/* ------------------------------------------------- adaptive density control */

/* Adaptive density control (Sec. 3, Preliminaries): during the densification
 * phase (iterations 0..T_d) Gaussians with a high view-space positional
 * gradient are cloned when small and split when large, and near-transparent
 * ones (alpha < eps_alpha) are pruned; after T_d the set is fixed.  The paper
 * states the rules qualitatively; the thresholds are the caller's.
 * Thresholds in the units the decision compares, so it is a float32
 * comparison only: grad_thr on the mean view-space gradient norm (pixels),
 * log_size_thr on the largest log-scale, logit_prune_thr on the opacity logit
 * (opacity < eps_alpha <=> logit < log(eps_alpha / (1 - eps_alpha)));
 * log_split_shrink: split children's log-scales are reduced by it (log 1.6 in
 * the vanilla scheme). */
typedef struct {
    float grad_thr, log_size_thr, logit_prune_thr, log_split_shrink;
} gs_densify_config;

enum { GS_DENSIFY_KEEP = 0, GS_DENSIFY_CLONE = 1, GS_DENSIFY_SPLIT = 2, GS_DENSIFY_PRUNE = 3 };

/* The gradient statistic, after a backward pass: for every view v (with
 * view_gate[v] != 0 when view_gate, device u8[n_views], is given) and every
 * Gaussian i visible in v (tiles_touched[v * n + i] > 0, as gs_project wrote),
 * accum[i] += |(g2d.x, g2d.y)| - the norm of dL/dmean2D that gs_raster_bwd or
 * gs_render_bwd_adam left in g2d (device, [n_views][n][12] floats, 16-byte
 * aligned) - and denom[i] += 1.  accum: device float[n], denom: device
 * int32[n], both caller-owned and updated in place (zero them to start). */
gs_status gs_densify_accumulate(const float *g2d, const int32_t *tiles_touched, int64_t n, int32_t n_views,
                                const uint8_t *view_gate, float *accum, int32_t *denom, cudaStream_t stream);

/* Scratch bytes of gs_densify_decide for n Gaussians. */
size_t gs_densify_workspace_size(int64_t n);

/* One action per Gaussian into action[n] (device u8): with avg = accum /
 * denom (one float32 division; 0 when denom = 0): GS_DENSIFY_PRUNE when the
 * opacity logit < logit_prune_thr; else, when avg >= grad_thr,
 * GS_DENSIFY_SPLIT if the largest log-scale > log_size_thr and
 * GS_DENSIFY_CLONE otherwise; else GS_DENSIFY_KEEP.  Then offsets[n + 1]
 * (device int64): the exclusive scan of the outputs per Gaussian (keep 1,
 * clone 2, split 2, prune 0), so offsets[n] is the new count - read it to
 * size the buffers of gs_densify_apply.  flat_params: gs_param_layout(n,
 * sh_degree).  GS_ERR_WORKSPACE below gs_densify_workspace_size(n). */
gs_status gs_densify_decide(const float *flat_params, int64_t n, int32_t sh_degree, const float *accum,
                            const int32_t *denom, const gs_densify_config *cfg /* host */, uint8_t *action,
                            int64_t *offsets, void *workspace, size_t workspace_bytes, cudaStream_t stream);

/* The output set, in input order (a Gaussian's outputs consecutive, at
 * offsets[i]): keep copies the Gaussian with its Adam moments; clone writes
 * the Gaussian (moments kept) and then an identical copy (moments zero);
 * split writes two children (moments zero) at mean + R(q / |q|) (exp(log_s)
 * * z_k), k = 0, 1, with z = noise[i][k][0..3) (device float [n][2][3],
 * standard normal draws, the caller's), log-scales reduced by
 * log_split_shrink, rotation, opacity and SH copied; prune writes nothing.
 * src_*: gs_param_layout(n, sh_degree) floats each; dst_*: caller-allocated
 * gs_param_layout(n_out, sh_degree) floats each, n_out = offsets[n] (else
 * GS_ERR_INVALID_ARG in dev_status and nothing is written).  The step count
 * of the optimizer is the caller's and carries on; the statistics of the new
 * set start at zero (the caller's arrays for n_out). */
gs_status gs_densify_apply(const float *src_params, const float *src_m, const float *src_v, int64_t n,
                           int32_t sh_degree, const uint8_t *action, const int64_t *offsets, const float *noise,
                           const gs_densify_config *cfg /* host */, float *dst_params, float *dst_m, float *dst_v,
                           int64_t n_out, int32_t *dev_status, cudaStream_t stream);

/* ----------------------------------------------------------- measurement */

/* Work census of one forward pass (not on the refinement path; for stating
 * throughput per unit of algorithmic work).  Inputs as gs_render_fwd after
 * it ran (records, vals, ranges, cams, n_last = saved.n_last), cfg->tile and
 * the alpha constants as used there.  Writes counts[5] (device, uint64,
 * overwritten): [0] sum over pixels of n_last; [1] (pixel, Gaussian) pairs
 * before the pixel's last contributor whose support box (mean2D +- (rx, ry))
 * contains the pixel centre - the evaluations of Eq. (alpha) the pass needs;
 * [2] contributing pairs (alpha' >= alpha_min, Eq. blend); [3] (tile,
 * Gaussian) pairs with a contributing pixel - the raster adjoint issues
 * three global atomic instructions for each; [4] list entries up to each
 * tile's largest n_last.  GS_ERR_INVALID_ARG for null or unaligned pointers
 * before any launch.  The paper has no counterpart. */
gs_status gs_raster_census(const gs_projected *proj /* host */, int64_t n, const uint32_t *vals,
                           const uint32_t *ranges, const gs_camera *cams, int32_t n_views, int64_t total_tiles,
                           const gs_raster_config *cfg /* host */, const int32_t *n_last,
                           unsigned long long *counts, cudaStream_t stream);

/* Throughput probe of scattered global reductions: n_updates updates, each
 * two float4 and one float atomic add into one of n_records 48-byte records
 * of buf (device, 16-byte aligned, [n_records][12] floats, contents
 * perturbed by ~1e-30 per update) chosen by a multiplicative hash of the
 * update's index - the pattern the raster adjoint uses for its per-Gaussian
 * 2D gradients.  Timing it gives the atomic peak the adjoint's rate is
 * compared with.  The paper has no counterpart. */
gs_status gs_atomic_probe(float *buf, int64_t n_records, int64_t n_updates, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GSR_H */
