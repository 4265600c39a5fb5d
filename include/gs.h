/*
 * gs.h -- C ABI of libgs, the CUDA (sm_103a) library for differentiable
 * rendering of an anchor-grid Gaussian map, forward and backward.
 *
 * The mapping iteration of the paper (Sec. III-B "System Overview": the
 * Gaussian mapper runs refinement against Eq. 3 on keyframes sampled as in
 * Sec. IV-A) renders its anchor map (Sec. III-A, Scaffold-GS anchors with the
 * partitioned decoders of Sec. III-D / Eq. 6) with a differentiable tile
 * rasterizer (Eq. 1) and back-propagates the photometric loss.  The calls
 * below are the steps of that pass:
 *
 *   gs_decode      visible (view, anchor) rows -> k 3D Gaussians per row
 *   gs_project     3D Gaussians -> 2D splats (EWA conic, depth, tile rect)
 *   gs_bin_sort    splats -> (tile, depth)-sorted splat ids + tile ranges
 *   gs_render_fwd  Eq. 1 per 16x16 tile, front to back
 *   gs_l1_loss     L1 term of Eq. 3 and its gradient
 *   gs_photometric_loss  full Eq. 3 (L1 + SSIM terms) and its gradient
 *   gs_render_bwd  reverse of Eq. 1 and of the projection
 *   gs_decode_bwd  reverse of the decoders (Eq. 6, Eq. 2), summed over views
 *   gs_adam_step, gs_densify_stats, gs_densify_masks  optimizer step and
 *                  growth / pruning statistics after the reverse pass
 *   gs_voxelize, gs_loop_closure  map maintenance (Eq. 4, Eq. 7)
 *   gs_flow_triangulate  epipolar filtering (Eq. 5) and triangulation of flow
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every pointer inside the structs is a DEVICE pointer unless it says HOST.
 *   Buffers are caller-owned, contiguous and laid out as documented; the
 *   library never allocates, frees or synchronises, and every call is
 *   enqueued on the given CUDA stream (`stream` is a cudaStream_t; NULL is
 *   the legacy default stream).  Every call is safe to capture in a CUDA
 *   graph.
 * - Sizes that depend on data (visible rows, pairs) live in device memory;
 *   capacities are fixed by the caller.  A kernel that would exceed a
 *   capacity writes nothing past it, records GS_ERR_CAPACITY and the size it
 *   needed in the caller's device `gs_status`, and every later call that is
 *   given the same status word returns early on the device.  Zero the status
 *   word (cudaMemsetAsync) before a pass and read it after the stream
 *   synchronises; on GS_ERR_CAPACITY grow the buffers and run the pass again.
 * - Return value: GS_OK, or a host-detected error (bad argument, launch
 *   failure) in which case nothing was enqueued or the enqueue failed.
 * - Views: a HOST array of gs_view (resolution) plus a DEVICE array of
 *   gs_camera (intrinsics and world->camera pose), V <= GS_MAX_VIEWS.  Pixel
 *   (u, v) is sampled at integer coordinates.  Views are tiled in 16x16
 *   tiles; tiles and pixels of all views are numbered view-major (view v's
 *   tiles start at the sum of the tile counts of views 0..v-1, row-major
 *   inside a view).  Images are FP32, view-major, each view planar [3][H][W].
 * - Rows and candidates: decoding emits one row per visible (view, anchor)
 *   pair, view-major and in anchor order inside a view.  Row r carries k
 *   candidate Gaussians with ids r*k + i (i < k).  Explicit Gaussians use
 *   k = 1 and one row per Gaussian.  `view_start[v]` (device, int32[V+1]) is
 *   the first row of view v and view_start[V] the number of rows.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_OK 0
#define GS_ERR_INVALID_ARG (-1)
#define GS_ERR_CAPACITY (-2)
#define GS_ERR_CUDA (-3)
#define GS_ERR_TIMEOUT (-4)
#define GS_ERR_UNSUPPORTED (-5)

#define GS_TILE 16
#define GS_MAX_VIEWS 64

/* decoder arithmetic */
#define GS_PREC_FP32 0   /* FP32 SIMT decode */
#define GS_PREC_BF16 1   /* BF16 tensor-core decode, FP32 accumulation */

/* Intrinsics and world->camera pose (p_cam = R x_world + t, R row-major). */
typedef struct gs_camera {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
} gs_camera; /* 64 bytes */

/* Resolution of one view (HOST). */
typedef struct gs_view {
    int32_t width, height;
} gs_view;

/* Device status word.  code: 0 or a GS_ERR_* recorded on the device;
 * where: the call that recorded it (1 decode, 2 project, 3 bin_sort,
 * 4 render_fwd, 5 render_bwd, 6 decode_bwd); needed: the capacity that
 * would have sufficed (rows for decode, pairs for bin_sort). */
typedef struct gs_status {
    int32_t code;
    int32_t where;
    int64_t needed;
} gs_status;

/* Anchor map (Sec. III-A): N anchors with position x_a, feature f_a (F
 * floats), log-scaling l_a (6 floats: [0:3] scale the offsets, [3:6] bound the
 * Gaussian scales), k offsets each, and a partition id (Eq. 6), anchors
 * sorted by partition.  MLP sets: M packed FP32 vectors of
 * gs_mlp_floats(F, k, hidden) floats each; per partition the heads
 * (opacity: k outputs, colour: 3k, covariance: 7k) follow each other, each as
 * W1[hidden][F+4], b1[hidden], W2[dout][hidden], b2[dout], row-major.  The
 * decoder input is [f_a, (x_a - x_c)/|x_a - x_c|, |x_a - x_c|] (Eq. 2). */
typedef struct gs_anchors {
    int32_t N, F, k, hidden, M;
    const float *xyz;          /* [N][3] */
    const float *feat;         /* [N][F] */
    const float *log_scaling;  /* [N][6] */
    const float *offsets;      /* [N][k][3] */
    const int32_t *part;       /* [N], non-decreasing, < M */
    const float *mlp;          /* [M][gs_mlp_floats] */
} gs_anchors;

/* 3D Gaussians, candidate-indexed (id = row*k + i), capacity cap_rows*k. */
typedef struct gs_gauss3d {
    int32_t k;
    int64_t cap_rows;
    int32_t *row_anchor;   /* [cap_rows] anchor of each row (NULL for explicit Gaussians) */
    int32_t *view_start;   /* [V+1] */
    float *mu;             /* [C][3] */
    float *scale;          /* [C][3] */
    float *quat;           /* [C][4] (w, x, y, z), unit */
    float *opacity;        /* [C]; <= 0 marks a candidate that decoding culled */
    float *colour;         /* [C][3] */
} gs_gauss3d;

/* Gradients w.r.t. the 3D Gaussians, same indexing. */
typedef struct gs_gauss3d_grad {
    float *dmu, *dscale, *dquat, *dopacity, *dcolour;
} gs_gauss3d_grad;

/* Projected splats, candidate-indexed.  `rec` holds one 48-byte record per
 * candidate: float[12] = mean_x, mean_y, A, B, C, L, r, g, b, depth, then two
 * uint32 words x0 | x1 << 16 and y0 | y1 << 16 (the tile rectangle [x0,x1) x
 * [y0,y1) inside the candidate's view).  With the conic (a, b, c) = Sigma2^-1
 * and the opacity o: A = -a log2(e)/2, B = -b log2(e), C = -c log2(e)/2,
 * L = log2(o), so that the power of pixel p is power = (A dx^2 + B dx dy +
 * C dy^2) ln 2 with (dx, dy) = mean - p, and o exp(power) = 2^(A dx^2 + B dx dy
 * + C dy^2 + L).  `tiles` is the number of tiles the rectangle covers, 0 for
 * a culled candidate. */
typedef struct gs_splats {
    int64_t cap;      /* capacity C in records */
    float *rec;       /* [C][12], 16-byte aligned */
    int32_t *tiles;   /* [C] */
} gs_splats;

/* Per-splat gradients of the rendering (view space), nine per candidate:
 * d mean_x, d mean_y, d conic_a, d conic_b, d conic_c, d opacity, d r, d g,
 * d b.  Two layouts:
 *   GS_SGRAD_CANDIDATE  g[9 c + v] for candidate c = row k + i ([C][9]);
 *   GS_SGRAD_ROW_TILES  g[((t k + i) 9 + v) 128 + r] for row 128 t + r: rows
 *                       in tiles of 128, each value of a tile's rows
 *                       contiguous (what the tensor-core reverse decoder reads
 *                       one row per thread); g holds ceil(cap_rows / 128) 128
 *                       k 9 floats.
 * gs_render_bwd writes either (with out = NULL); gs_decode_project_bwd at
 * GS_PREC_BF16 reads either; every other reader takes GS_SGRAD_CANDIDATE. */
#define GS_SGRAD_CANDIDATE 0
#define GS_SGRAD_ROW_TILES 1
typedef struct gs_splat_grad {
    float *g;
    int32_t layout;   /* GS_SGRAD_* */
} gs_splat_grad;

/* Sorted binning of splats into tiles. */
typedef struct gs_bins {
    int64_t cap_pairs;
    uint32_t *vals;      /* [cap_pairs] splat id of each (tile, splat) pair, sorted */
    uint64_t *keys;      /* [cap_pairs] or NULL: (global tile << 32) | float bits of depth */
    uint32_t *ranges;    /* [T_total][2] pair range [start, end) of each tile */
    uint32_t *n_pairs;   /* [1] number of pairs */
} gs_bins;

/* Gradients w.r.t. the anchor map (accumulated over all views). */
typedef struct gs_anchor_grad {
    float *dxyz, *dfeat, *dlog_scaling, *doffsets; /* like the inputs */
    float *dmlp;                                    /* [M][gs_mlp_floats] */
} gs_anchor_grad;

/* --- sizes ------------------------------------------------------------- */
/* Floats in one packed partition MLP set. */
int64_t gs_mlp_floats(int32_t F, int32_t k, int32_t hidden);
/* Total 16x16 tiles / pixels of a view set. */
int64_t gs_total_tiles(const gs_view *views, int32_t V);
int64_t gs_total_pixels(const gs_view *views, int32_t V);
/* Workspace bytes of each call that takes one (0 for the others). */
size_t gs_decode_workspace(int32_t N, int32_t V, int32_t M, int64_t cap_rows);
size_t gs_bin_sort_workspace(const gs_view *views, int32_t V, int64_t cap_cand, int64_t cap_pairs);
size_t gs_decode_bwd_workspace(int32_t N, int32_t V, int32_t M, int64_t cap_rows);
/* Render workspace (shared by gs_render_fwd and gs_render_bwd): the chunk
 * plan and per-chunk state of the tiles whose list is longer than `chunk`. */
size_t gs_render_workspace(const gs_view *views, int32_t V, int64_t cap_pairs, int32_t chunk);
const char *gs_status_string(int32_t code);
/* Number of kernels this library has enqueued since it was loaded (host
 * counter, all devices and threads); a diagnostic for launch accounting. */
uint64_t gs_kernel_launches(void);
/* Failure-detection hook (no counterpart in the paper).  Sets the limit, in
 * nanoseconds, of the waits of the tensor-core kernels (GS_PREC_BF16
 * gs_decode / gs_decode_noalloc / gs_decode_bwd) for their MMAs to complete,
 * for the calls enqueued after it (the value is read on the host at launch):
 * a wait that runs out records GS_ERR_TIMEOUT in the status word, and the
 * kernel then waits (with the default limit) for its MMAs still in flight,
 * frees its tensor memory and returns, leaving the context usable.  0 makes
 * the first completion wait give up at once (how a test drives that path);
 * ns < 0 restores the default of 1 s.  Process-wide; returns GS_OK. */
int gs_set_wait_limit(int64_t ns);
/* Launch shapes (no counterpart in the paper; set by the autotuner of the
 * Python layer): CTAs per SM of the persistent forward and reverse
 * compositing kernels, of the radix-sort and compaction passes and of the pair
 * emission.  0 keeps the library's choice (as many as fit on an SM for the
 * persistent kernels, 4 for the sort passes and the emission); the
 * persistent kernels clamp larger values to what fits, the sort passes take
 * at most 1024 CTAs and the emission at most 8 per SM.  None of them
 * changes a result bit except through
 * the order of the reverse pass's floating-point atomics.  Process-wide and
 * read when a call enqueues its kernels (a captured CUDA graph keeps the
 * shapes of its capture).  gs_set_tuning(NULL) restores the defaults;
 * negative values are GS_ERR_INVALID_ARG. */
typedef struct gs_tuning {
    int32_t fwd_ctas_per_sm;
    int32_t bwd_ctas_per_sm;
    int32_t sort_ctas_per_sm;
    int32_t emit_ctas_per_sm;
} gs_tuning;
int gs_set_tuning(const gs_tuning *t);
int gs_get_tuning(gs_tuning *t);

/* --- the pass ---------------------------------------------------------- */

/* Anchor visibility and decoding (Sec. III-A, Eq. 2, Eq. 6).  A row is made
 * for every (view, anchor) whose centre is in front of z = 0.2 and projects
 * inside the image grown by 15 % per side.  Each row's partition MLP gives, for
 * i < k: opacity = tanh(z_o), colour = sigmoid(z_c), scale = exp(l[3:6]) *
 * sigmoid(z_s), quat = z_q / |z_q|, mu = x_a + offset_i * exp(l[0:3]).
 * precision: GS_PREC_FP32 or GS_PREC_BF16 (features and weights rounded to
 * BF16 for the two MLP layers, FP32 accumulation and epilogue).  Capacity:
 * out->cap_rows rows; overflow -> GS_ERR_CAPACITY with the row count needed.
 * Workspace: gs_decode_workspace bytes, 256-byte aligned. */
int gs_decode(const gs_anchors *A, const gs_camera *cams, const gs_view *views, int32_t V,
              int32_t precision, gs_gauss3d *out, void *ws, size_t ws_bytes, gs_status *status,
              void *stream);

/* Same as gs_decode, for callers that cannot allocate device memory (for
 * example a real-time thread that must not enter the driver's allocator, or a
 * plug-in whose host framework owns all device memory): there is no workspace
 * argument.  The scratch lives in a static device array of 512 KiB that every
 * GPU loading this library keeps until the process exits; calls needing more
 * than ceil(N / 2048) * V <= 131072 counts return GS_ERR_CAPACITY at once and
 * enqueue nothing.  The array used is the one of the CURRENT device
 * (cudaGetDevice): `stream` must belong to that device.  The first call on
 * each device looks the array's device address up (cudaGetSymbolAddress) with
 * that device current and keeps it for the life of the process; make that
 * first call before any stream capture, and do not use this entry point on a
 * device after cudaDeviceReset of that device in the same process (the kept
 * address then refers to the old context).  All calls on a device share the
 * array, so calls that overlap on the GPU race on it.  Nothing is allocated.
 * The paper has no counterpart of this entry point. */
int gs_decode_noalloc(const gs_anchors *A, const gs_camera *cams, const gs_view *views, int32_t V,
                      int32_t precision, gs_gauss3d *out, gs_status *status, void *stream);

/* EWA projection of every candidate (3DGS preliminaries, Sec. III-A): p = R mu
 * + t, culled if opacity <= 0 or p_z <= 0.2; Sigma3 = R_q S^2 R_q^T; Sigma2 =
 * J R Sigma3 R^T J^T + 0.3 I with x/z, y/z clamped to 1.3x the half field of
 * view; culled if det <= 0; conic = Sigma2^-1 (FP64 when det < 1e-3 a c);
 * radius ceil(3 sqrt(lambda_max)), lambda_max = m + sqrt(max(0.1, m^2 - det));
 * rect x0 = floor((mx - r)/16), x1 = floor((mx + r)/16) + 1 clamped to the
 * view, same in y; culled if empty.  Reads the row count from
 * g->view_start[V] on the device; writes cap_rows*k records at most. */
int gs_project(const gs_gauss3d *g, const gs_camera *cams, const gs_view *views, int32_t V,
               gs_splats *out, gs_status *status, void *stream);

/* gs_decode followed by gs_project in one call: visible rows, then each
 * candidate's splat record (same arithmetic, same records).  With
 * GS_PREC_BF16 the tensor-core decoder projects each candidate in its
 * epilogue and writes the records directly: the 3D Gaussians never reach
 * device memory and g's candidate arrays (mu, scale, quat, opacity, colour)
 * are left untouched -- g->row_anchor and g->view_start are written, as the
 * reverse pass (gs_decode_project_bwd) needs them.  With GS_PREC_FP32 the two
 * calls run one after the other and g's candidate arrays hold the decoded
 * Gaussians.  Arguments as in gs_decode and gs_project (sp->rec 16-byte
 * aligned, sp->cap >= g->cap_rows k); workspace: gs_decode_workspace. */
int gs_decode_project(const gs_anchors *A, const gs_camera *cams, const gs_view *views, int32_t V,
                      int32_t precision, gs_gauss3d *g, gs_splats *sp, void *ws, size_t ws_bytes,
                      gs_status *status, void *stream);

/* Tile binning and sort of the tile-based differentiable rasterizer the
 * paper renders with (Sec. II, the 3DGS rasterizer it builds on; Sec. III-A,
 * Eq. 1 composites each pixel's splats front to back, so every tile needs
 * its splats in depth order): one pair per (covered tile, splat), ordered by
 * (global tile, float bits of depth, splat id) -- exactly the order of a sort
 * on the 64-bit key (tile << 32 | depth bits) with ties broken by id.  Also
 * writes [start, end) per tile (empty tiles [0, 0)).  The covering splats
 * (tiles > 0) contribute the tiles of their rectangle (record floats 10-11);
 * one whose rectangle is empty records GS_ERR_INVALID_ARG.  k and view_start
 * as in gs_gauss3d.  Capacity: bins->cap_pairs; overflow -> GS_ERR_CAPACITY with the
 * pair count needed.  Workspace: gs_bin_sort_workspace bytes. */
int gs_bin_sort(const gs_splats *sp, int32_t k, const int32_t *view_start, int64_t cap_rows,
                const gs_view *views, int32_t V, gs_bins *bins, void *ws, size_t ws_bytes,
                gs_status *status, void *stream);

/* Eq. 1 per pixel over its tile's sorted list: T = 1; for each splat,
 * alpha = min(0.99, o exp(power)), skipped if power > 0 or alpha < 1/255;
 * stop before a splat whose T(1 - alpha) < 1e-4; C += c alpha T; T *= 1 -
 * alpha.  image = C + T bg.  bg: HOST float[3].
 * Work items: each tile's list is cut into chunks of `chunk` splats (0 selects
 * 384; otherwise 256 .. 2^24), and every 16x4 pixel block of every chunk is a
 * work unit that persistent warps take from a device counter, so that a few
 * very long tiles do not serialise the launch.  Later chunks of a tile are
 * composited on their own transmittance and scaled by the transmittance in
 * front of them; a chunk that holds a pixel's stop is composited again from
 * its entering transmittance, which reproduces the front-to-back order and
 * the stop rule exactly.  ws / ws_bytes: gs_render_workspace bytes,
 * 256-byte aligned; gs_render_bwd needs the same workspace, untouched, and
 * the same `chunk`.  T_final (float per pixel) and last (int32 per pixel:
 * 1-based list position of the last composited splat) are optional outputs
 * (NULL to skip).  n_eval (device int64[4], NULL to skip) receives the number
 * of (pixel, splat) pairs examined (every list position up to the pixel's
 * stop), the number composited, and the same two counts over the tiles whose
 * list forms a single work item (a counting variant of the kernels runs when
 * it is given). */
int gs_render_fwd(const gs_splats *sp, const gs_bins *bins, const gs_view *views, int32_t V,
                  const float *bg, int32_t chunk, void *ws, size_t ws_bytes, float *image,
                  float *T_final, int32_t *last, int64_t *n_eval, gs_status *status, void *stream);

/* L = sum over views of mean |C - C_target| (L1 term of Eq. 3), written to
 * loss (device float[1], overwritten); dL/dC = sign(C - C_target)/(3 H W)
 * written to d_image (same layout as image). */
int gs_l1_loss(const float *image, const float *target, const gs_view *views, int32_t V,
               float *loss, float *d_image, void *stream);

/* The full photometric objective of Eq. 3 (Sec. III-A), which the paper takes
 * from the 3DGS work it cites: L = lambda L1 + (1 - lambda) L_SSIM with
 * L_SSIM = 1 - SSIM.  SSIM of a view is the mean over pixels and channels of
 * the SSIM map computed per channel with an 11x11 Gaussian window (sigma 1.5,
 * normalised), zero padding outside the image, C1 = 0.01^2, C2 = 0.03^2 (the
 * paper states none of these; lambda = 0.8 is the usual choice).  Both terms
 * are per-view means summed over the views, as in gs_l1_loss.
 * image, target: device float, [V][3][H][W] planar (the layout of
 * gs_render_fwd's image).  lambda in [0, 1].  loss: device float[3],
 * overwritten with (L, L1, L_SSIM).  d_image: dL/dimage, same layout,
 * overwritten; it is the input gs_render_bwd takes.  ws: caller-owned device
 * workspace of gs_photometric_workspace bytes, 256-byte aligned (8 bytes per
 * work unit of 32 columns x 64 rows of one channel).  Errors: GS_ERR_INVALID_ARG for null pointers,
 * a bad view set, lambda outside [0, 1] or a small / unaligned workspace. */
size_t gs_photometric_workspace(const gs_view *views, int32_t V);
int gs_photometric_loss(const float *image, const float *target, const gs_view *views, int32_t V,
                        float lambda, void *ws, size_t ws_bytes, float *loss, float *d_image,
                        void *stream);

/* ---- After the reverse pass: optimizer step and densification statistics.
 * The paper refines, densifies and prunes the anchor map to minimise Eq. 3
 * (Sec. III, "System Overview") with the training of the incremental
 * Scaffold-GS it adopts; it states neither the optimizer nor its settings.
 *
 * gs_adam_step: one Adam step with bias correction (t = step >= 1) over up
 * to GS_ADAM_MAX_GROUPS float tensors in one launch, in place:
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
 *   p -= lr / (1 - b1^t) * m / (sqrt(v) / sqrt(1 - b2^t) + eps).
 * groups: HOST array of n_groups descriptors; param / m / v are device
 * arrays of n floats updated in place (m, v start at zero), grad is read.
 * beta1, beta2, eps are doubles so that 1 - beta is formed without the
 * cancellation a single-precision 0.999 would bring (it is off by 1.3e-5).
 * Anchor positions are not in the paper's optimised set: they change only at
 * loop closures (ibid.), so callers leave them out.  Errors:
 * GS_ERR_INVALID_ARG for n_groups outside 1..GS_ADAM_MAX_GROUPS, step < 1, a
 * null pointer with n > 0, n < 0, or b1, b2 outside [0, 1), eps < 0. */
#define GS_ADAM_MAX_GROUPS 16
typedef struct gs_adam_group {
    float *param;
    const float *grad;
    float *m;
    float *v;
    int64_t n;
    float lr;
} gs_adam_group;
int gs_adam_step(const gs_adam_group *groups, int32_t n_groups, int64_t step, double beta1, double beta2,
                 double eps, void *stream);

/* gs_densify_stats: adds one iteration's statistics of the Scaffold-GS
 * growth and pruning rules into caller-owned accumulators (zero them at the
 * start of an interval):
 *   every decoded row (view, anchor a):  anchor_denom[a] += 1,
 *       opacity_accum[a] += sum over its k Gaussians of max(opacity, 0);
 *   every rendered Gaussian (row, i), tiles[row k + i] > 0:
 *       grad_accum[a k + i] += |dL/d mean2d| (pixel units, the first two
 *       values of its gs_render_bwd splat gradient), offset_denom[a k + i] += 1.
 * g: the decoded rows (row_anchor, view_start, opacity, k, cap_rows); V its
 * views; tiles: gs_splats.tiles; sgrad: the splat gradients [C][9] of
 * gs_render_bwd.  Accumulators: device float [N k], int32 [N k], float [N],
 * int32 [N].  An anchor index outside [0, N) is reported through status.
 *
 * gs_densify_masks: growth candidates grow[a k + i] = (offset_denom >=
 * min_count and grad_accum / offset_denom >= grad_thr) and pruning candidates
 * prune[a] = (anchor_denom >= min_count and opacity_accum / anchor_denom <
 * opacity_thr), the means in single precision (device uint8 outputs). */
int gs_densify_stats(const gs_gauss3d *g, int32_t V, const int32_t *tiles, const float *sgrad, int32_t N,
                     float *grad_accum, int32_t *offset_denom, float *opacity_accum, int32_t *anchor_denom,
                     gs_status *status, void *stream);
int gs_densify_masks(int64_t N, int32_t k, const float *grad_accum, const int32_t *offset_denom,
                     const float *opacity_accum, const int32_t *anchor_denom, float grad_thr,
                     float opacity_thr, int32_t min_count, uint8_t *grow, uint8_t *prune, void *stream);

/* ---- Map maintenance.
 *
 * gs_voxelize (Eq. 4, Sec. III "System Overview": the fused point cloud is
 * discretised onto the anchor voxel grid, keeping unique entries): the voxel
 * index of a point is rint(p / eps) per axis (one correctly rounded single
 * precision division, ties to even), packed into the 64-bit key
 * ((i + 2^20) << 42) | ((j + 2^20) << 21) | (l + 2^20).  Writes, in ascending
 * key order, the distinct keys that are not in `existing` and their centres
 * index * eps.  points: device float [P][3], 0 <= P < 2^31; existing: device
 * uint64 [n_existing], sorted ascending (the keys of the anchors already in
 * the map; NULL when n_existing = 0); keys_out [cap_out] uint64 and
 * centers_out [cap_out][3] float: device outputs; n_out: device uint32, the
 * number written.  ws: gs_voxelize_workspace(P) bytes, 256-byte aligned.
 * Errors in status: GS_ERR_INVALID_ARG (site 80) for an index outside
 * (-2^20, 2^20); GS_ERR_CAPACITY with the needed count when it exceeds
 * cap_out (nothing written, *n_out = 0). */
size_t gs_voxelize_workspace(int64_t P);
int gs_voxelize(const float *points, int64_t P, float eps, const uint64_t *existing, int64_t n_existing,
                uint64_t *keys_out, float *centers_out, int64_t cap_out, uint32_t *n_out, void *ws,
                size_t ws_bytes, gs_status *status, void *stream);

/* gs_loop_closure (Eq. 7, Sec. III "Loop Closures"): for each corrected
 * keyframe i with old and new world-to-camera poses, Delta T_i = T_new,i^-1
 * T_old,i moves an anchor x to R_new^T (R_old x + t_old - t_new).  It applies
 * to the anchors inside keyframe i's view frustum under its old pose -- in
 * front of the near plane 0.2, inside the image grown by 15 % per side (the
 * decoder's visibility rule), no deeper than z_far -- and an anchor inside
 * several frusta takes the nearest keyframe (distance to the old camera
 * centre; lowest index on ties; the paper leaves this open).  Other anchors
 * keep their position.  xyz: device float [N][3], updated in place;
 * old_cams / new_cams: device gs_camera [K]; wh: device int32 [K][2] (width,
 * height); assigned: device int32 [N] (the keyframe used, -1 for none) or
 * NULL.  Offsets, features and scalings are left as they are. */
int gs_loop_closure(float *xyz, int32_t N, const gs_camera *old_cams, const gs_camera *new_cams,
                    const int32_t *wh, int32_t K, float z_far, int32_t *assigned, void *stream);

/* ---- Flow densification geometry (Sec. III, Flow Densification; Eq. 5).
 * For keyframes 1 and 2 with known poses, F = [e2]x P2 P1^+ with P_i =
 * K_i [R_i | t_i], e2 = P2 C1 and C1 the centre of keyframe 1.  Each sampled
 * pixel x = (px, py, 1) of keyframe 1 and its flow correspondence x' = x +
 * flow(x) is kept iff |x'^T F x| < tau (F and the residual in double
 * precision); kept pairs are triangulated by linear least squares on the four
 * DLT rows with the homogeneous coordinate fixed to 1 (double precision).
 * The paper states neither tau nor N: they are the caller's, and so is the
 * random choice of the N samples (passed in).
 * cam1, cam2: device gs_camera (one each); flow: device float [H][W][2]
 * (x, y displacement in pixels, pixels at integer coordinates); samples:
 * device int32 [N] pixel indices py W + px; residual: device float [N] or
 * NULL; kept: device int32 [cap] sample positions of the kept pairs in sample
 * order; points: device float [cap][3] their world points; n_kept: device
 * uint32.  A kept pair without parallax (its two rays parallel, e.g. a pixel
 * at the epipole with zero flow) has a singular system and a non-finite
 * point; callers drop such points.  ws: gs_flow_workspace(N) bytes, 256-byte
 * aligned.  Errors in status: GS_ERR_INVALID_ARG (site 90) for a sample
 * outside the image;
 * GS_ERR_CAPACITY with the needed count when the kept pairs exceed cap
 * (nothing written, *n_kept = 0). */
size_t gs_flow_workspace(int32_t N);
int gs_flow_triangulate(const gs_camera *cam1, const gs_camera *cam2, int32_t width, int32_t height,
                        const float *flow, const int32_t *samples, int32_t N, double tau, float *residual,
                        int32_t *kept, float *points, int64_t cap, uint32_t *n_kept, void *ws, size_t ws_bytes,
                        gs_status *status, void *stream);

/* Reverse of Eq. 1 and of the projection.  With w_i = alpha_i T_i and B_i
 * the colour composited behind splat i (plus T_final bg), dL/dc_i = w_i g and
 * dL/dalpha_i = g.(c_i T_i - B_i/(1 - alpha_i)), then through alpha = o
 * exp(power) (no gradient where the 0.99 clamp is active) to mean and conic;
 * per-splat sums are reduced across each warp before global atomics.  Then
 * (unless out is NULL) the projection chain rule of gs_project_bwd.  Each
 * pixel's list is walked front to back again: T_i and the colour composited
 * up to splat i are recomputed with the forward's arithmetic (the forward's
 * skip and stop decisions), and B_i is the pixel's final colour minus that
 * prefix, so the forward stores nothing per pixel.  image: the forward's
 * output (device, same layout as d_image).  last: the forward's optional
 * per-pixel output (1-based position of the last composited splat), or NULL
 * to decide the stop rule again.  chunk and ws must be those of the forward,
 * ws untouched since: tiles cut into several chunks start each chunk from
 * the transmittance and colour prefix the forward left there.  sgrad:
 * per-splat view-space gradients in either layout, overwritten for every
 * candidate up to the row count (zeros for the ones that cover no tile; in
 * the row-tiled layout the whole last tile of rows).  out: NULL, or
 * overwritten for every candidate (zeros for culled ones); it needs
 * GS_SGRAD_CANDIDATE. */
int gs_render_bwd(const gs_gauss3d *g, const gs_camera *cams, const gs_splats *sp,
                  const gs_bins *bins, const gs_view *views, int32_t V, int32_t chunk, void *ws,
                  size_t ws_bytes, const float *image, const float *d_image, const int32_t *last,
                  gs_splat_grad *sgrad, gs_gauss3d_grad *out, gs_status *status, void *stream);

/* Chain rule of the EWA projection (3DGS preliminaries, Sec. III-A): from the
 * splat gradients of gs_render_bwd (d mean2d, d conic, d opacity, d colour)
 * to d mu, d scale, d quat of the 3D Gaussians, with the FP64 inverse
 * derivative (on the compensated covariance) for near-degenerate splats as in
 * gs_project; d opacity and d colour pass through.  Candidates with
 * sp->tiles == 0 get zeros.  out is overwritten for every candidate up to the
 * row count.  sgrad: GS_SGRAD_CANDIDATE. */
int gs_project_bwd(const gs_gauss3d *g, const gs_camera *cams, const gs_splats *sp, const gs_view *views,
                   int32_t V, const gs_splat_grad *sgrad, gs_gauss3d_grad *out, gs_status *status,
                   void *stream);

/* Reverse of gs_decode, summed over views: through the activations (only for
 * candidates with opacity > 0), both MLP layers (hidden activations
 * recomputed, not stored) and the view inputs of Eq. 2.  out is overwritten.
 * precision as in gs_decode.  Workspace: gs_decode_bwd_workspace bytes. */
int gs_decode_bwd(const gs_anchors *A, const gs_camera *cams, const gs_view *views, int32_t V,
                  int32_t precision, const gs_gauss3d *g, const gs_gauss3d_grad *dg,
                  gs_anchor_grad *out, void *ws, size_t ws_bytes, gs_status *status,
                  void *stream);

/* Reverse of the projection and of the decoders in one call, from the splat
 * gradients of gs_render_bwd (called with out = NULL): the result of
 * gs_project_bwd followed by gs_decode_bwd, without the 3D-Gaussian
 * gradients in between.  With GS_PREC_BF16 the tensor-core reverse decoder
 * applies the projection's chain rule (the near-degenerate branch included)
 * to each candidate it recomputes -- mean x_a + offset exp(l[0:3]), scale
 * exp(l[3:6]) sigmoid, unit quaternion, evaluated with the reverse pass's
 * recomputed decoder activations, reading the splat gradients one row per
 * thread: GS_SGRAD_ROW_TILES directly (no workspace needed: ws may be NULL),
 * GS_SGRAD_CANDIDATE after rearranging them in the workspace.  With
 * GS_PREC_FP32 (GS_SGRAD_CANDIDATE only) the two steps run one after the
 * other through the workspace.  Workspace: gs_decode_project_bwd_workspace
 * bytes, 256-byte aligned.  sp->tiles marks the candidates that cover a tile
 * (the others get no gradient).  out is overwritten. */
size_t gs_decode_project_bwd_workspace(int32_t k, int64_t cap_rows, int32_t precision);
int gs_decode_project_bwd(const gs_anchors *A, const gs_camera *cams, const gs_view *views, int32_t V,
                          int32_t precision, const gs_gauss3d *g, const gs_splats *sp,
                          const gs_splat_grad *sgrad, gs_anchor_grad *out, void *ws, size_t ws_bytes,
                          gs_status *status, void *stream);

/* Measurement helper (no counterpart in the paper): launches `blocks` CTAs of
 * 256 threads, each running 8 independent chains of `iters` dependent
 * operations -- kind 0: FP32 fused multiply-add, kind 1: SFU ex2.approx --
 * and stores the number of operations issued in *ops (host).  The caller
 * times the launch on `stream` to get the device's FP32-pipe or SFU issue
 * rate, the denominators of the compositing kernels' rooflines.  sink: a
 * device buffer of `blocks` floats (written only in a case that does not
 * occur).  Returns GS_ERR_INVALID_ARG for another kind, blocks < 1 or
 * iters < 1. */
int gs_probe_peak(int32_t kind, int32_t blocks, int32_t iters, float *sink, int64_t *ops, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
