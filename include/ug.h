/*
 * ug.h — C ABI of the GB300 UltraGauss plane rasterizer.
 *
 * UltraGauss (arXiv 2505.05643) renders an ultrasound image as the
 * intersection of anisotropic 3D Gaussians with a probe plane (Sec. 4.1):
 * each pixel x of the plane is lifted to x_|0 = [x1, x2, 0] in the probe frame
 * and takes
 *
 *     C(x) = (sum_i w_i(x) c_i + a_bg c_bg) / (sum_i w_i(x) + a_bg),
 *     w_i(x) = alpha_i exp(-1/2 (x_|0 - mu3D_i)^T (Sigma3D_i)^-1 (x_|0 - mu3D_i))
 *
 * (Eq. alpha-combine, Eq. colour-combine, Eq. us-render, Eq. mahalanobis-3d),
 * summed only over pixels inside each Gaussian's chi^2 bounding box
 * (Sec. 4.3, Eq. ellipsoid and Eq. boundary) and only for Gaussians whose
 * box meets the plane (Sec. 4.4). Covariances use the paper's triangular
 * precision factor Sigma^-1 = L L^T with diagonal l_kk^2 + beta (Sec. 4.2,
 * Eq. tri-param) or, as a second front-end, Sigma = R diag(s^2) R^T.
 *
 * Conventions shared by every call:
 *  - All array pointers are DEVICE pointers unless a parameter says "host".
 *    The caller owns all memory; the library never allocates or frees and
 *    never synchronises the stream.
 *  - Gaussian parameters are structure-of-arrays, "row" layout: a parameter
 *    with k components is a row-major [k][n] float32 array (component r of
 *    Gaussian g at index r * n + g), n = ug_plan.n.
 *  - Argument errors are returned synchronously. Data-dependent errors
 *    (capacity overflow, an invalid plane pose in device memory, an internal
 *    inconsistency) are written to the workspace status word by the kernels;
 *    every later kernel of the same workspace then does nothing, the outputs
 *    are invalid, and ug_read_status reports the error and the sizes needed.
 *  - Every call only enqueues work on `stream` and can be captured in a CUDA
 *    graph.
 *  - Outputs are overwritten, not accumulated.
 */
#ifndef UG_H
#define UG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (0 = the legacy default stream). */
typedef struct CUstream_st* ug_stream;

typedef enum {
  UG_OK = 0,
  UG_ERR_INVALID_ARGUMENT = 1,    /* bad pointer, size, config or host plane */
  UG_ERR_WORKSPACE_TOO_SMALL = 2, /* ws_bytes < ug_plan.workspace_bytes */
  UG_ERR_CAPACITY = 3,            /* device: more records/instances than the plan holds */
  UG_ERR_CUDA = 4,                /* a CUDA launch or copy failed */
  UG_ERR_TIMEOUT = 5,             /* device: a bounded wait gave up */
  UG_ERR_NOT_SUPPORTED = 6,       /* config value not compiled in (e.g. tile shape) */
  UG_ERR_INVALID_PLANE = 7,       /* device: a plane in device memory is not a valid pose */
  UG_ERR_INTERNAL = 8             /* device: two passes disagreed (a bug) */
} ug_status;

enum { UG_COV_TRI = 0, UG_COV_SCALE_ROT = 1 };
enum { UG_CUTOFF_BOX = 0, UG_CUTOFF_BOX_AND_ELLIPSOID = 1 };

/* Gaussian parameters (device, row layout, float32). For UG_COV_TRI `tri` is
 * [6][n] = l11, l21, l31, l22, l32, l33 and log_scale/quat are unused; for
 * UG_COV_SCALE_ROT `log_scale` is [3][n] (s = exp(log_scale)) and `quat` is
 * [4][n] = w, x, y, z (normalised inside; need not be unit). mean is [3][n];
 * opacity_logit and intensity are [n] (alpha = sigmoid(logit), Sec. 4.5). */
typedef struct {
  const float* mean;
  const float* tri;
  const float* log_scale;
  const float* quat;
  const float* opacity_logit;
  const float* intensity;
} ug_gaussians;

/* Gradient outputs, same layout as ug_gaussians (written, not accumulated).
 * Rows of the unused front-end may be NULL. */
typedef struct {
  float* mean;
  float* tri;
  float* log_scale;
  float* quat;
  float* opacity_logit;
  float* intensity;
} ug_gaussian_grads;

/* One probe plane (64 bytes). The probe frame has rows u, v, n = u x v and
 * origin `origin` at the plane centre; u, v must be orthonormal to 1e-4.
 * Pixel (i, j), 0 <= i < height, 0 <= j < width, has its centre at
 *   x1 = (j + 1/2 - width/2) * pitch_u,  x2 = (i + 1/2 - height/2) * pitch_v
 * and is stored at image[pixel_offset + i * width + j]. */
typedef struct {
  float origin[3];
  float u[3];
  float v[3];
  float pitch_u, pitch_v;
  int32_t width, height; /* 1 .. 16384 */
  int32_t reserved;      /* must be 0 */
  int64_t pixel_offset;
} ug_plane;

/* Cut-off and image-formation constants, tile shape and kernel variant. */
typedef struct {
  float chi2;        /* chi^2_3 bound of the cut-off ellipsoid; 7.815 (p = 95 %, Sec. 4.3) */
  float beta;        /* diagonal offset of Eq. tri-param, > 0; default 1e-4 */
  float alpha_bg;    /* background coefficient a_bg > 0 (Eq. alpha-combine); default 1e-3 */
  float c_bg;        /* background intensity; default 0 */
  int32_t cutoff;    /* UG_CUTOFF_BOX (paper) or UG_CUTOFF_BOX_AND_ELLIPSOID */
  int32_t cov_param; /* UG_COV_TRI (paper) or UG_COV_SCALE_ROT */
  int32_t tile;      /* square tile edge in pixels: 8 or 16 (default 16) */
  int32_t variant;   /* forward rasterizer variant, 0 .. ug_num_variants(tile) - 1: lane
                        groups per 8x8 footprint (pixels per lane), stages in the record
                        ring and records per stage: 0 = 4 groups, 3 stages of 128 (default),
                        1 = 2 groups, 2 = 1 group; tile 16 also 3 = stages of 64 records,
                        4 = 2 stages of 256, 5 = 4 stages of 128 */
  float fp64_ratio;  /* axis-ratio proxy above which the per-(plane, Gaussian) geometry runs
                        in extended (double-word, ~48-bit) precision; default 1e3 */
  int32_t variant_bwd; /* backward rasterizer variant, 0 .. ug_num_variants_bwd(tile) - 1:
                          0 = 8-row footprints, 4 stages of 128 records (default), 1 = 4-row
                          footprints; tile 16 also 2 = 3 stages of 128 (more resident
                          blocks), 3 = 4 stages of 64, 4 = 3 stages of 256, 5 = 4 stages
                          of 128 with three resident blocks (more registers a thread) */
  float fp32_reach;  /* the geometry also runs in extended precision when ||F||_F (|mu| +
                        max |o|) exceeds this (F the Gaussian's precision factor, o the plane
                        origins): FP32 differences mu - o then lose the bits that thin or
                        distant Gaussians need; default 20. Both this and fp64_ratio +inf:
                        FP32 geometry throughout */
  int32_t reserved;
} ug_config;

/* Sizes, capacities and the workspace layout of one rendering problem.
 * Filled by ug_plan_init; treat as read-only afterwards. */
typedef struct {
  ug_config cfg;
  int64_t n;                 /* Gaussians */
  int32_t num_planes;
  int32_t total_tiles;
  int64_t total_pixels;      /* length of the image buffers */
  int64_t record_capacity;   /* visible (plane, Gaussian) pairs the workspace holds */
  int64_t instance_capacity; /* (tile, record) pairs the workspace holds, < 2^31 */
  int32_t key_bits;          /* bits of the tile key */
  int32_t sort_passes;       /* 8-bit LSD passes */
  int64_t chunks;            /* ceil(n / 32) */
  size_t workspace_bytes;
  size_t off[32];            /* internal section offsets (unused entries 0) */
} ug_plan;

/* Workspace status (64 bytes), copied out by ug_read_status. */
typedef struct {
  int32_t status;       /* ug_status of the first data-dependent failure, 0 if none */
  int32_t detail;       /* e.g. the index of an invalid plane */
  int64_t records;      /* record slots of the last preprocess: the visible (plane, Gaussian)
                           pairs plus the FP64 candidates that the exact test rejected */
  int64_t instances;    /* (tile, record) instances found by the last preprocess */
  int64_t fp64_records; /* visible records whose covariance inverse ran in FP64 */
  int64_t box_pixels;   /* sum over records of their clipped pixel-box area: the number
                           of (pixel, Gaussian) pairs the box cut-off includes */
  int64_t evaluated_pairs; /* (pixel, record) pairs the last ug_render evaluated: warp
                              footprints x records that reach them; pairs whose weight is
                              provably an FP32 zero are not evaluated */
  int64_t evaluated_pairs_bwd; /* the same count for the last backward rasterizer launch */
  int64_t reserved[1];
} ug_ws_status;

/* Adam learning-rate schedule of one parameter row (device array entry):
 * lr(t) = lr_init * (lr_final / lr_init)^min(t / decay_steps, 1); decay_steps
 * <= 0 keeps lr_init (Sec. 4.5: 0.05 for all rows, the means' rows decay from
 * 1.6e-4). */
typedef struct {
  float lr_init, lr_final;
  int32_t decay_steps;
  int32_t reserved;
} ug_adam_row;

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t ug_version(void);

/* Human-readable name of a status code (static string). */
const char* ug_status_string(ug_status status);

/* Number of forward (ug_num_variants) and backward (ug_num_variants_bwd)
 * rasterizer variants compiled in for `tile` (0 if the tile size is
 * unsupported). The variants compute the same result; they differ in how the
 * work is laid out (see ug_config.variant and .variant_bwd), and the fastest
 * depends on the workload. */
int32_t ug_num_variants(int32_t tile);
int32_t ug_num_variants_bwd(int32_t tile);

/* Fill *cfg with the defaults listed above. */
ug_status ug_config_default(ug_config* cfg);

/* Validate a configuration and the HOST copy of the planes (sizes, pixel
 * offsets, finite orthonormal poses) and fill *plan: tile counts, key bits,
 * and the workspace size for the given capacities. record_capacity and
 * instance_capacity must be >= 1; instance_capacity < 2^31. The planes may
 * hold at most 2^24 tiles in all (UG_ERR_NOT_SUPPORTED beyond: a sort key
 * keeps its top byte for the instance's footprint tests). The plane poses
 * may change later in device memory; their sizes may not. */
ug_status ug_plan_init(const ug_config* cfg, int64_t n, const ug_plane* host_planes,
                       int32_t num_planes, int64_t record_capacity,
                       int64_t instance_capacity, ug_plan* plan);

/* Rows a1-a3 (Sec. 4.2-4.4): per (plane, Gaussian) activation, probe-frame
 * mean, Sigma3D by forward substitution, chi^2 box, phase-1 rejection, pixel
 * box, in-plane conic and peak weight; then the records of the visible pairs
 * in (Gaussian chunk, plane, Gaussian) order and their (tile, record)
 * instances. d_planes: device array of plan->num_planes ug_plane with the
 * sizes given to ug_plan_init. Resets the status word first. */
ug_status ug_preprocess(const ug_plan* plan, const ug_gaussians* gaussians,
                        const ug_plane* d_planes, void* ws, size_t ws_bytes, ug_stream stream);

/* Row a4: stable LSD radix sort of the instances on their tile key (so each
 * tile lists its records in ascending (plane, Gaussian) order) and the
 * [start, end) range of every tile. */
ug_status ug_bin_sort(const ug_plan* plan, void* ws, size_t ws_bytes, ug_stream stream);

/* Row a5 (Eq. us-render with Eq. alpha-combine / colour-combine): writes
 * image[total_pixels] = C and alpha[total_pixels] = sum_i w_i + a_bg (the
 * rendered opacity, kept for the backward pass). Pixels not covered by any
 * plane are left untouched. */
ug_status ug_render(const ug_plan* plan, void* ws, size_t ws_bytes, float* image,
                    float* alpha, ug_stream stream);

/* Evaluation metrics of rendered slices (Sec. 5): for P images of W x H pixels
 * stored one after the other (row-major, device memory), the mean SSIM of
 * image against target (Wang et al.: 11 x 11 Gaussian window, sigma 1.5,
 * C1 = 0.01^2, C2 = 0.03^2, data range 1, every position where the window lies
 * inside the image) into ssim[P] and PSNR = 10 log10(1 / MSE) into psnr[P]
 * (either may be NULL, not both). scratch is caller-owned device memory of at
 * least ug_ssim_scratch_floats(P, W, H) floats. Deterministic. Returns
 * UG_ERR_INVALID_ARGUMENT for W or H below 11, UG_ERR_WORKSPACE_TOO_SMALL for
 * too little scratch. ug_ssim_scratch_floats returns 0 for invalid sizes. */
size_t ug_ssim_scratch_floats(int32_t P, int32_t W, int32_t H);
ug_status ug_ssim(const float* image, const float* target, int32_t P, int32_t W, int32_t H,
                  float* scratch, size_t scratch_floats, float* ssim, float* psnr,
                  ug_stream stream);

/* The paper's own phase 2 (Sec. 4.4), kept as an ablation of ug_render: every
 * visible record of the last ug_preprocess adds its weight and weighted
 * intensity to each pixel of its box with atomics (no binning or sort needed),
 * then C and alpha are formed as in ug_render. Same records and per-pixel
 * weights as ug_render; the sums run in a different (unspecified) order, so the
 * result agrees with ug_render to FP32 rounding and is not bit-reproducible.
 * image and alpha are written as in ug_render (they serve as the accumulators). */
ug_status ug_render_scatter(const ug_plan* plan, void* ws, size_t ws_bytes, float* image,
                            float* alpha, ug_stream stream);

/* Floats of device memory the `loss` argument of ug_mse_loss_grad points to. */
#define UG_MSE_LOSS_FLOATS 1025

/* Row a6: mean squared error over n pixels. Writes grad_image[n] =
 * 2 (image - target) / n (if grad_image != NULL) and loss[0] = mean((image -
 * target)^2). `loss` points to UG_MSE_LOSS_FLOATS device floats: loss[0] gets
 * the value, the rest holds per-block partial sums, so the result does not
 * depend on scheduling (deterministic). */
ug_status ug_mse_loss_grad(const float* image, const float* target, int64_t n,
                           float* grad_image, float* loss, ug_stream stream);

/* Row a6 for one part of a larger set of images (the planes one rank of a
 * plane-split run renders): writes grad_image[n] = 2 (image - target) / n_total
 * and loss[0] = sum((image - target)^2) / n_total over this part's n pixels,
 * so that the parts' gradients and losses, summed over all parts (one
 * all-reduce of the per-Gaussian gradients), are those of the mean squared
 * error over all n_total pixels. Same buffers and determinism as
 * ug_mse_loss_grad, which equals this call with n_total = n. Returns
 * UG_ERR_INVALID_ARGUMENT for a NULL input, n < 1 or n_total < n. */
ug_status ug_mse_loss_grad_part(const float* image, const float* target, int64_t n,
                                int64_t n_total, float* grad_image, float* loss,
                                ug_stream stream);

/* Largest n accepted by ug_mse_loss_grad_static (2^30 pixels). */
#define UG_MSE_STATIC_MAX_N (1LL << 30)

/* The same loss and gradient as ug_mse_loss_grad for callers that cannot
 * allocate device memory. The paper has no counterpart; this exists for code
 * that may not call cudaMalloc where it runs (inside a stream capture, in a
 * plugin that is handed only the buffers it works on, under a memory budget
 * owned by someone else). The caller passes only the inputs, grad_image (or
 * NULL) and `loss`, which here is ONE device float. The per-block partial sums
 * live in a 64 KiB array inside this library that stays allocated on every
 * GPU that loads it until the process exits. Returns UG_ERR_INVALID_ARGUMENT
 * for n < 1 or n > UG_MSE_STATIC_MAX_N. The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture. All calls share
 * the array: calls whose kernels may overlap on the GPU (unordered streams)
 * race on it and must be serialised by the caller. Allocates nothing. */
ug_status ug_mse_loss_grad_static(const float* image, const float* target, int64_t n,
                                  float* grad_image, float* loss, ug_stream stream);

/* Rows a7-a8: gradient of a scalar loss with respect to the Gaussian
 * parameters, given dL/dC per pixel (grad_image) and the image and alpha that
 * ug_render wrote for the same workspace. The box cut-off is a constant of the
 * derivative. Gradients are summed over planes and written to *grads. */
ug_status ug_render_backward(const ug_plan* plan, const ug_gaussians* gaussians,
                             const ug_plane* d_planes, void* ws, size_t ws_bytes,
                             const float* image, const float* alpha, const float* grad_image,
                             const ug_gaussian_grads* grads, ug_stream stream);

/* Row a7 alone (the first half of ug_render_backward): per tile, recompute
 * every included weight and reduce dL/d(record) over the tile's pixels into the
 * workspace's per-record gradient buffer (8 floats per record: dL/dc, dL/d lw2,
 * and the sums that give dL/dx*, dL/d(r11, r12, r22)), zeroed first by this
 * call. image, alpha and grad_image are device arrays of plan->total_pixels
 * floats laid out as for ug_render. Returns UG_ERR_INVALID_ARGUMENT for a NULL
 * pointer; device-side failures of the preceding calls propagate through the
 * workspace status (the kernels then return without work). */
ug_status ug_render_backward_raster(const ug_plan* plan, void* ws, size_t ws_bytes,
                                    const float* image, const float* alpha,
                                    const float* grad_image, ug_stream stream);

/* Row a8 alone (the second half of ug_render_backward): chain the per-record
 * gradients left in the workspace by ug_render_backward_raster through the
 * preprocess of rows a1-a2 (plane projection, Sec. 4.1; Eq. tri-param or the
 * scale-rotation front-end, Sec. 4.2; the cut-off box is a constant) and the
 * activations (Sec. 4.5), and sum them over planes into *grads (written, not
 * accumulated; one thread per Gaussian, no atomics). `gaussians` must be the
 * parameters ug_preprocess ran on. */
ug_status ug_preprocess_backward(const ug_plan* plan, const ug_gaussians* gaussians, void* ws,
                                 size_t ws_bytes, const ug_gaussian_grads* grads,
                                 ug_stream stream);

/* Row a9: one Adam step on `rows` parameter rows of n floats each, all in one
 * contiguous [rows][n] buffer (param, grad, exp_avg, exp_avg_sq alike):
 *   m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
 *   p <- p - lr_r(t) / (1 - b1^t) * m / (sqrt(v) / sqrt(1 - b2^t) + eps)
 * where t = *d_step + 1 is read from device memory and *d_step is then
 * incremented on the device (so a captured graph advances by itself), and
 * lr_r(t) follows d_rows[r] (device array of `rows` ug_adam_row). */
ug_status ug_adam_step(float* param, const float* grad, float* exp_avg, float* exp_avg_sq,
                       int32_t rows, int64_t n, const ug_adam_row* d_rows, int32_t* d_step,
                       float beta1, float beta2, float eps, ug_stream stream);

/* Copy the workspace status to `out` (host pinned or device memory) on
 * `stream`; the caller synchronises before reading it. */
ug_status ug_read_status(const ug_plan* plan, const void* ws, size_t ws_bytes, ug_ws_status* out,
                         ug_stream stream);

/* Device pointers into the workspace, for inspection and tests: the sorted
 * tile keys and record ids (instance order; a key's low 24 bits are the
 * (plane, tile) id, its top byte the instance's tests against the tile's 8x8
 * footprints in row-major order: bit 2f set if the record can have a non-zero
 * FP32 weight in footprint f, bit 2f + 1 if its box also covers the whole
 * footprint), the tile ranges (uint32 pairs
 * [start, end) per tile), and per record slot its pixel box (uint32 pairs:
 * j0 | j1 << 16, i0 | i1 << 16; an empty box marks a rejected candidate), its
 * render data as 4 floats each: a = (X, Y, r11, kappa), b = (r22, lw2, c,
 * ellipsoid threshold), c = (X', Y', kappa', 0), the low parts of X, Y, kappa,
 * where (X + X', Y + Y') is the in-plane peak in pixel units relative to the
 * box's first column and row (pixel (i, j) centred at (j - j0 + 1/2, i - i0 +
 * 1/2)) and the weight at a pixel is 2^(lw2 - t1^2 - t2^2), t1 = r11 (dx +
 * kappa dy), t2 = r22 dy; and its plane index. Valid after ug_bin_sort; any
 * argument may be NULL. A record is binned only to the tiles of its box in
 * which some weight can be non-zero in FP32. */
ug_status ug_debug_views(const ug_plan* plan, void* ws, size_t ws_bytes, uint32_t** sorted_keys,
                         uint32_t** sorted_records, uint32_t** tile_ranges,
                         uint32_t** record_boxes, float** record_a, float** record_b,
                         float** record_c, uint32_t** record_planes);

/* Row f4 (the loss half): the training loss of Kerbl et al., which Sec. 4.5
 * takes over, for P planes of W x H pixels stored one after the other:
 *   L = (1 - lambda) mean|x - y| + lambda (1 - SSIM),
 * SSIM the mean over the planes of each plane's mean SSIM (the ug_ssim
 * definition), and dL/dx for every pixel (the L1 term's derivative is taken
 * as 0 where x = y). *loss and grad are device memory; scratch holds at least
 * ug_l1_dssim_scratch_floats(P, W, H) floats. Deterministic. Returns
 * UG_ERR_INVALID_ARGUMENT for W or H below 11 or lambda outside [0, 1],
 * UG_ERR_WORKSPACE_TOO_SMALL for too little scratch. */
size_t ug_l1_dssim_scratch_floats(int32_t P, int32_t W, int32_t H);
ug_status ug_l1_dssim_loss_grad(const float* image, const float* target, int32_t P, int32_t W,
                                int32_t H, float lambda, float* scratch, size_t scratch_floats,
                                float* grad, float* loss, ug_stream stream);

/* Row f2: resampling and the densify / prune step (Sec. 4.2 sampling
 * y = mu + L^-T z; Sec. 4.5 takes the densification heuristics over from Kerbl
 * et al. without stating them, so the decision quantities below are this
 * library's reading). Parameters are one [rows][n] FP32 buffer in the packed
 * row order (mean 3, then tri 6 = l11 l21 l31 l22 l32 l33, or log_scale 3 +
 * quat 4, then opacity logit, intensity), as ug_adam_step takes them. */
typedef struct {
  float grad_threshold; /* densify when the mean |dL/dmu| over the counted steps exceeds
                           this; default 2e-4 */
  float min_opacity;    /* prune when sigmoid(logit) < this (decided on the logit);
                           default 0.005 */
  float size_threshold; /* split when the extent exceeds this, else clone; the extent is
                           sqrt(trace Sigma) (TRI) or the largest scale (SCALE_ROT);
                           default 0.01 */
  float split_factor;   /* phi > 1: a split's two children have covariance Sigma / phi^2;
                           default 1.6 */
  int32_t reserved[4];
} ug_densify_config;

ug_status ug_densify_config_default(ug_densify_config* dc);

/* y = mu + L^-T z (TRI, by back substitution with L^T, L_kk = l_kk^2 + beta) or
 * y = mu + R S z (SCALE_ROT) for the m Gaussians idx[k] of the [rows][n]
 * parameter buffer; z and y are [3][m] (z: standard normal draws supplied by
 * the caller). cfg gives cov_param and beta. Device pointers; m = 0 is a no-op. */
ug_status ug_sample(const ug_config* cfg, const float* params, int64_t n, const int32_t* idx,
                    int64_t m, const float* z, float* y, ug_stream stream);

/* Densify statistics of one step: for every Gaussian with dL/dmu != 0,
 * stats[0][i] += |dL/dmu_i| and stats[1][i] += 1 (grad_mean: [3][n], the mean
 * rows of the gradient; stats: [2][n], zeroed by the caller when a new
 * interval starts). */
ug_status ug_densify_stats(const float* grad_mean, int64_t n, float* stats, ug_stream stream);

/* Bytes of device scratch ug_densify needs for n Gaussians. */
size_t ug_densify_scratch_bytes(int64_t n);

/* One densify / prune step, in input order: a Gaussian with sigmoid(logit) <
 * min_opacity is removed; else, with mean |dL/dmu| = stats[0][i] / stats[1][i]
 * (0 when never counted) above grad_threshold, it is cloned (itself and an
 * identical copy) when its extent is at most size_threshold and split into two
 * children otherwise (means mu + L^-T z with z = z_rows[0..2][i] and
 * z_rows[3..5][i], covariance Sigma / phi^2, same opacity and intensity);
 * the rest are kept. Kept Gaussians keep their Adam moments, clones and
 * children get zero moments. Outputs are [rows][capacity] buffers (params,
 * exp_avg, exp_avg_sq); *n_out (device) receives the number of outputs, and
 * when it exceeds capacity nothing past capacity is written. z: [6][n].
 * Device pointers; scratch of ug_densify_scratch_bytes(n) bytes. */
ug_status ug_densify(const ug_config* cfg, const ug_densify_config* dc, const float* params,
                     const float* exp_avg, const float* exp_avg_sq, int64_t n, const float* stats,
                     const float* z, int64_t capacity, float* params_out, float* exp_avg_out,
                     float* exp_avg_sq_out, int64_t* n_out, void* scratch, size_t scratch_bytes,
                     ug_stream stream);

/* Gaussian split across ranks (row a5; Sec. 4.1, Eq. alpha-combine and Eq.
 * colour-combine): S_a = sum_i w_i and S_c = sum_i w_i c_i are sums over
 * Gaussians in no particular order, so the partial sums of shards of the
 * Gaussians add up to the full ones. ug_shard_sums turns a shard's ug_render
 * output (image, alpha of n pixels, rendered with the given alpha_bg and c_bg)
 * into its partial sums: sums[2 i] = alpha[i] - alpha_bg, sums[2 i + 1] =
 * image[i] alpha[i] - alpha_bg c_bg (an interleaved [n][2] float array, 8-byte
 * aligned). After the caller sums `sums` over the shards (one all-reduce of two
 * floats per pixel), ug_composite writes alpha[i] = sums[2 i] + alpha_bg and
 * image[i] = (sums[2 i + 1] + alpha_bg c_bg) / alpha[i], the image and alpha of
 * all Gaussians, which each rank's ug_render_backward for its own shard then
 * takes as inputs (its gradients need no further exchange). Returns
 * UG_ERR_INVALID_ARGUMENT for a NULL pointer, n < 1, a misaligned `sums` or
 * alpha_bg <= 0. */
ug_status ug_shard_sums(const float* image, const float* alpha, int64_t n, float alpha_bg,
                        float c_bg, float* sums, ug_stream stream);
ug_status ug_composite(const float* sums, int64_t n, float alpha_bg, float c_bg, float* image,
                       float* alpha, ug_stream stream);

/* Test hook for the rasterizers' bounded waits (rows a5, a7). With on != 0
 * the producer warps of ug_render and ug_render_backward_raster issue no
 * stage, so every consumer wait runs out after its time limit (about one
 * second): the launch then ends with UG_ERR_TIMEOUT in the workspace status,
 * and the context stays usable. on = 0 restores normal operation, and so does
 * ug_preprocess, which clears the flag: set it after the preprocess of the
 * launch to be tested. Written on `stream`. */
ug_status ug_debug_stall_pipeline(const ug_plan* plan, void* ws, size_t ws_bytes, int32_t on,
                                  ug_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* UG_H */
