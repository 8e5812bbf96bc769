/*
 * fastergs.h -- C ABI of libfastergs.so: one 3D Gaussian Splatting training
 * step on an NVIDIA GB300 (sm_103a), as described by Faster-GS (arXiv
 * 2602.09999): preprocess, duplicate + radix sort + tile ranges, tile
 * blending, L1 + D-SSIM loss, blend backward, preprocess backward, Adam.
 *
 * Conventions shared by every entry point
 *  - All data pointers are DEVICE pointers unless a comment says "host".
 *  - The caller owns every buffer: parameters, gradients, Adam moments,
 *    images, targets and the workspace.  The library never allocates,
 *    frees or synchronises, except fgs_get_error (which synchronises).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy stream).
 *    Every call is asynchronous on it and may be captured in a CUDA graph
 *    as long as the view sizes stay the same between replays.
 *  - Return value: FGS_OK (0) or a negative FGS_ERR_* code for an error the
 *    host can see (bad pointer, shape, degree, dtype, workspace size, launch
 *    failure).  Errors found on the device (instance capacity exceeded,
 *    non-finite loss or Adam update) set sticky bits in the workspace header
 *    read by fgs_get_error; no kernel traps.
 *  - Gradients are overwritten, never accumulated.
 *  - Layouts are row-major; a [n,3] array is n consecutive triples.
 *
 * Gaussian parameters (Sec. 2.1 of the paper; fgs_params.data[] order):
 *   0 means       [n,3]  float32
 *   1 log_scales  [n,3]  float32   (scale = exp, Sec. 2.1 activations)
 *   2 quats       [n,4]  float32   (w,x,y,z; normalised in the kernel; the
 *                                    buffer 16-byte aligned, else FGS_ERR_ALIGN)
 *   3 opacity     [n]    float32   (logit; sigmoid in the kernel)
 *   4 sh_dc       [n,3]  float32 / bf16 / fp16 (SH band 0, separate buffer
 *                                               as in Sec. 3.2 "Rasterization
 *                                               Kernel Fusion")
 *   5 sh_rest     [n,15,3] same dtype as sh_dc (bands 1..3)
 *   6 velocity    [n,3]  float32   (optional: dynamic Gaussians, below)
 *   7 t0          [n]    float32   (optional: temporal centre)
 *
 * Dynamic (4D) Gaussians (Sec. 3.4, the conditional Gaussian of Yang et al.
 * in its linear-velocity form): when groups 6 and 7 are set, a view taken at
 * time t (fgs_camera.time) sees the mean mu + v (t - t0) -- the conditional
 * mean with Sigma_{1:3,4} Sigma_{4,4}^-1 = v and mu_4 = t0 -- and the
 * opacity multiplied by the temporal marginal exp(-(t - t0)^2 / (2
 * sigma_t^2)) (fgs_params.sigma_t); the 3D covariance is used as is.  With
 * both NULL the Gaussians are static (3D) and time is ignored.
 */
#ifndef FASTERGS_H
#define FASTERGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FGS_TILE 16          /* tile edge in pixels (Sec. 3.1) */
#define FGS_MAX_VIEWS 16     /* views per batched call */
#define FGS_NUM_GROUPS 8     /* parameter groups in fgs_params (6 and 7 optional) */

enum fgs_status {
    FGS_OK = 0,
    FGS_ERR_NULL = -1,       /* a required pointer is NULL */
    FGS_ERR_SHAPE = -2,      /* n <= 0, n too large, or bad image size */
    FGS_ERR_SH_DEGREE = -3,  /* SH degree outside 0..3 */
    FGS_ERR_WORKSPACE = -4,  /* workspace layout does not match the call or is too small */
    FGS_ERR_DTYPE = -5,      /* unsupported storage type for a group */
    FGS_ERR_CUDA = -6,       /* a kernel launch failed */
    FGS_ERR_VIEWS = -7,      /* n_views outside 1..FGS_MAX_VIEWS */
    FGS_ERR_ALIGN = -8,      /* a pointer is not 16-byte aligned */
    FGS_ERR_ARG = -9,        /* another argument is out of range */
    FGS_ERR_TOO_LARGE = -10  /* more pairs than fgs_sort_pairs_static can hold */
};

/* Sticky bits set on the device, read by fgs_get_error.  Setting one never
 * stops a kernel: the outputs of that call hold whatever the arithmetic gave
 * (dropped instances, NaN or infinity), and the caller decides. */
enum fgs_device_flags {
    FGS_FLAG_CAPACITY = 1u,  /* instances exceeded k_max; the extra ones were dropped */
    FGS_FLAG_NONFINITE = 2u  /* a NaN or infinity reached the loss (a per-view sum or
                                dL/dimages, set by fgs_loss_l1_dssim) or an Adam update
                                (a new parameter or moment, set by the fused
                                fgs_render_backward_adam) */
};

enum fgs_dtype { FGS_F32 = 0, FGS_BF16 = 1, FGS_F16 = 2 };

/* Pinhole camera, OpenCV axes (x right, y down, z forward).
 * R: world->camera rotation, row-major; t: translation (Eq. 1, W = [R|t]).
 * fx, fy, cx, cy: intrinsics in pixels (Eq. 1-2; Suppl. B.1 uses the
 * intrinsics directly instead of a projection matrix).  Pixel (u, v) is
 * sampled at (u + 0.5, v + 0.5).  near_plane: Gaussians with camera depth
 * <= near_plane are not rendered.  cam_pos: camera centre in world space,
 * used for the SH view direction.  time: the view's timestamp, used by
 * dynamic Gaussians only. */
typedef struct fgs_camera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_plane;
    float cam_pos[3];
    float time;
} fgs_camera;

/* One tensor per parameter group (order above), each with its storage
 * type.  Used for parameters, gradients (always FGS_F32) and the two Adam
 * moments.  Groups 6 and 7 are both set or both NULL, and the gradient and
 * moment structs follow the parameters.  sigma_t: temporal standard
 * deviation of dynamic Gaussians (> 0 when groups 6 and 7 are set). */
typedef struct fgs_params {
    int64_t n;
    void *data[FGS_NUM_GROUPS];
    int32_t dtype[FGS_NUM_GROUPS];
    float sigma_t;
} fgs_params;

/* Sub-arrays of the caller-allocated workspace (byte offsets from its
 * start; every offset is 256-byte aligned).  Offset 0 always holds the
 * header: uint32 flags, uint32 reserved, uint64 instance count of the last
 * forward (may exceed k_max), uint32 counters. */
enum fgs_ws_slot {
    FGS_WS_HEADER = 0,
    FGS_WS_SCREEN,      /* 48-byte records [n_views*n]: float4 (mu2D, conic eigenvalues lb >= ls),
                           float4 (major-axis direction cos, sin, o, depth),
                           float4 (rgb, bits: clamp mask 0..2, visible 3); written only for the
                           pairs the forward renders (FGS_WS_RECT count > 0), the others keep
                           whatever they held */
    FGS_WS_RECT,        /* 16-byte records [n_views*n]: tile rectangle x0, y0, x1, y1 (uint16,
                           inclusive; x0 > x1 when not rendered), then for rectangles of at most
                           32 tiles the uint32 mask of tiles kept by culling (bit t = row-major
                           tile t), then the uint32 number of kept tiles (0: not rendered) */
    FGS_WS_LOCAL_OFF,   /* uint32 [n_views*n]: CTA-local exclusive prefix of the rendered flags */
    FGS_WS_BLOCK_SUM,   /* uint32 [n_views*ceil(n/128)+1]: prefix of the CTA totals */
    FGS_WS_KEYS,        /* uint32 [k_max]: global tile id of each instance (tile sort keys) */
    FGS_WS_VALS,        /* uint32 [k_max]: Gaussian index */
    FGS_WS_KEYS_ALT,    /* uint32 [k_max]: sort ping-pong buffer */
    FGS_WS_VALS_ALT,    /* uint32 [k_max] */
    FGS_WS_SORT_HIST,   /* uint32 radix histograms (shared by both sorts) */
    FGS_WS_RANGES,      /* uint2 [total_tiles]: [start, end) of each tile's list */
    FGS_WS_T_FINAL,     /* float [total_pixels]: final transmittance */
    FGS_WS_N_CONTRIB,   /* uint32 [total_pixels]: list position of the last blended entry */
    FGS_WS_SCREEN_GRAD, /* 48-byte records [n_views*n]: float4 (dL/dmu2D, dL/dSigma2D 00, 01),
                           float4 (dL/dSigma2D 11, dL/do, dL/dr, dL/dg), float4 (dL/db, 0, 0, 0);
                           dL/dSigma2D is the full symmetric gradient.  The backward clears
                           only the records of 128-Gaussian blocks with a rendered pair in
                           that view; the others keep whatever they held */
    FGS_WS_LOSS_MAPS,   /* float [9*total_pixels]: SSIM partial-derivative maps */
    FGS_WS_LOSS_PART,   /* double [loss blocks*2]: per-CTA L1 / SSIM sums */
    FGS_WS_N_BLENDED,   /* uint32 [total_pixels]: fragments blended into each pixel */
    FGS_WS_TILE_QUEUE,  /* uint32 [4 + total_tiles]: work-queue counters (forward head and
                           exits, backward head and exits), then every tile of every view in
                           descending order of list length (written by each forward) */
    FGS_WS_DEPTH_KEYS,  /* uint32 [n_views*n]: depth bits of the rendered (view, Gaussian) pairs;
                           after the depth sort, the split duplication order's list of pairs
                           with large rectangles */
    FGS_WS_DEPTH_VALS,  /* uint32 [n_views*n]: view * n + Gaussian index of those pairs */
    FGS_WS_DEPTH_KEYS_ALT, /* uint32 [n_views*n]: depth-sort ping-pong buffers */
    FGS_WS_DEPTH_VALS_ALT,
    FGS_WS_SORTED_OFF,  /* uint32 [n_views*n]: instance offsets in depth order (CTA-local) */
    FGS_WS_SORTED_BLOCK, /* uint32 [ceil(n_views*n/512)+1]: prefix of those CTA totals */
    /* per-Gaussian backward only (FGS_WS_PER_GAUSSIAN; empty otherwise).  A bucket is 32
       consecutive entries of one tile's list; buckets are numbered tile by tile. */
    FGS_WS_BUCKET_OFF,   /* uint32 [total_tiles+1]: first bucket of each tile; the last entry
                            holds the number of buckets */
    FGS_WS_BUCKET_TILE,  /* uint32 [k_max/32 + total_tiles]: tile of each bucket */
    FGS_WS_BUCKET_STATE, /* float4 [256 per bucket]: (T, C.r, C.g, C.b) of each pixel of the
                            tile in front of the bucket's first entry, written by the forward
                            for the pixels still blending there (pixel ly*16 + lx) */
    FGS_WS_PIXEL_FINAL,  /* float4 [total_pixels]: output colour C + T bg of each pixel */
    FGS_WS_NUM_SLOTS
};

/* Launch choices that change speed, never results: pixels each blend thread
 * owns (1, 2 or 4; the CTA of a 16x16 tile has 256 / that many threads) and
 * list entries staged per shared-memory batch (64, 128 or 256).  Supported
 * pairs: (1,256) (2,128) (2,256) (4,64) (4,128) (4,256).  The per-pixel
 * blend backward may take its own pair (backward_pixels_per_thread,
 * backward_batch; both 0, the default: the forward's pair).  The radix
 * digit width of each of the two sorts (Sec. 3.2 "Sorting": a pass per
 * digit) is 8 or 11 bits: 11 takes 3 passes instead of 4 over the 32 depth
 * bits, with 2048 digit counters per CTA instead of 256.
 * fgs_workspace_size fills the defaults; an autotuner may overwrite them in
 * the layout before the calls that use it.  The forward and the backward
 * that share a workspace must run with the same layout. */
typedef struct fgs_tuning {
    int32_t blend_pixels_per_thread;
    int32_t blend_batch;
    int32_t blend_schedule;  /* FGS_SCHEDULE_QUEUE (default) or FGS_SCHEDULE_GRID */
    int32_t blend_backward;  /* FGS_BACKWARD_PER_PIXEL (default) or FGS_BACKWARD_PER_GAUSSIAN */
    int32_t backward_pixels_per_thread;  /* 0: blend_pixels_per_thread */
    int32_t backward_batch;              /* 0: blend_batch */
    int32_t depth_sort_digit_bits;       /* radix digit of the depth sort: 8 or 11 (0: 8) */
    int32_t tile_sort_digit_bits;        /* radix digit of the tile sort: 8 or 11 (0: 8); the
                                            layout's sorted_in_alt must then be the parity of
                                            ceil(sort_bits / digit bits) */
    int32_t duplicate_order;             /* FGS_DUPLICATE_STRIDED (default) or FGS_DUPLICATE_SPLIT */
} fgs_tuning;

/* How the duplication step (Sec. 3.2 "Sorting": one key per kept tile of
 * every rendered Gaussian, in depth order) assigns rendered pairs to
 * threads; the emitted instances are the same either way.  STRIDED: one
 * kernel, lane l of warp w taking pair l * W + w, so the near splats with
 * large rectangles (first in depth order) spread over all warps, each
 * culled by its whole warp; a warp's stores land in 32 far-apart runs.
 * SPLIT: consecutive threads take consecutive pairs (one contiguous run of
 * stores per warp) and list the large rectangles, which a second kernel
 * culls one warp per entry; it pays where the instance arrays exceed L2
 * (batches of many views). */
enum { FGS_DUPLICATE_STRIDED = 0, FGS_DUPLICATE_SPLIT = 1 };

/* Order of the blend backward (the same gradients up to float32 rounding).
 * PER_PIXEL: one thread per pixel walks its tile's list back to front,
 * recovering T by division; per-fragment gradients are summed over the warp
 * and the CTA before one set of atomics per (entry, CTA).  PER_GAUSSIAN
 * (Sec. 3.2 "Per-Gaussian Backward", after Mallick et al.): the list is cut
 * into buckets of 32 entries, one warp per bucket and one lane per entry;
 * starting from each pixel's (T, C) in front of the bucket, stored by the
 * forward, the lanes replay the blend front to back, passing the state from
 * lane to lane with shuffles, and each lane adds its entry's gradient with
 * one set of atomics per bucket.  Pixel states are staged per warp in
 * shared memory, 32 at a time (the paper's refinement).  Needs a workspace
 * made with FGS_WS_PER_GAUSSIAN. */
enum { FGS_BACKWARD_PER_PIXEL = 0, FGS_BACKWARD_PER_GAUSSIAN = 1 };

/* How the blend kernels visit tiles.  QUEUE: one resident CTA set per SM
 * (SMs x occupancy CTAs) takes tiles from a work queue, longest list first
 * (a longest-processing-time order, so no long tile starts last).  GRID: one
 * CTA per tile, tiles in row-major order of each view. */
enum { FGS_SCHEDULE_QUEUE = 0, FGS_SCHEDULE_GRID = 1 };

typedef struct fgs_workspace_layout {
    size_t total_bytes;
    size_t offset[FGS_WS_NUM_SLOTS];
    size_t bytes[FGS_WS_NUM_SLOTS];
    int64_t n;
    int64_t k_max;
    int32_t n_views;
    int32_t total_tiles;
    int64_t total_pixels;
    int32_t sort_bits;       /* tile-id bits the tile sort orders (the depth sort: 32) */
    int32_t sorted_in_alt;   /* 1: the tile-sorted keys/values end in the *_ALT slots (an odd
                                number of passes of tuning.tile_sort_digit_bits) */
    int32_t flags;           /* the FGS_WS_* options the layout was made with */
    fgs_tuning tuning;       /* launch choices (defaults filled in) */
} fgs_workspace_layout;

/* Workspace size and layout for n Gaussians, n_views host cameras and an
 * instance capacity k_max ((Gaussian, tile) pairs summed over all views;
 * the paper's model is about 8 tiles per visible Gaussian, Suppl. B.2).
 * Pure host arithmetic.  The caller allocates at least total_bytes of
 * 256-byte aligned device memory and passes the same layout (host struct)
 * to the forward, loss and backward calls that share the workspace; each
 * call checks it against its cameras.  Returns FGS_ERR_* on bad arguments
 * (n outside 1..2^31-1, n_views outside 1..FGS_MAX_VIEWS, n_views * n
 * above 2^32-1, a camera size outside 1..65535, k_max outside 0..2^31-1). */
int fgs_workspace_size(int64_t n, const fgs_camera *cams_host, int32_t n_views, int64_t k_max,
                       fgs_workspace_layout *out_host);

/* The same with options: flags & FGS_WS_PER_GAUSSIAN also reserves the
 * buffers of the per-Gaussian backward (4 KB of pixel states per bucket of
 * 32 instances: about 128 k_max + 4096 total_tiles bytes more).
 * fgs_workspace_size(...) is fgs_workspace_size_ex(..., 0, ...). */
enum { FGS_WS_PER_GAUSSIAN = 1 };
int fgs_workspace_size_ex(int64_t n, const fgs_camera *cams_host, int32_t n_views, int64_t k_max,
                          int32_t flags, fgs_workspace_layout *out_host);

/* Forward pass for layout->n_views views (Eq. 1-4; Sec. 3.2 bounds, culling and
 * sorting; Suppl. B.1 clamp, early stop and degeneracy tests):
 *   preprocess -> per-CTA scan -> duplicate into (tile << 32 | depth) keys
 *   -> LSD radix sort -> tile ranges -> front-to-back blending.
 * cams_host gives the view sizes (grids and layout); cams_device holds the
 * same n_views cameras in device memory and is what the kernels read, so a
 * captured graph may be replayed with new poses.  bg: host float[3]
 * background colour.  images: float32, the n_views images [3,H_v,W_v]
 * concatenated.  The rendered colour is not clipped (Suppl. B.1).
 * The workspace keeps what the backward needs (screen state, sorted lists,
 * final transmittance, last-contributor positions). */
int fgs_render_forward(void *ws, const fgs_workspace_layout *layout, const fgs_params *params,
                       int32_t sh_degree, const fgs_camera *cams_host,
                       const fgs_camera *cams_device, const float bg[3], float *images,
                       void *stream);

/* Loss of Suppl. A for each view: (1 - lambda) mean|C - C_gt| + lambda
 * (1 - mean SSIM) with an 11x11 Gaussian window (sigma 1.5, zero padding,
 * C1 = 0.01^2, C2 = 0.03^2), averaged over the views.  Writes the scalar
 * loss (device float, loss_out[0]) and dL/dimages (same layout as images).
 * Uses the workspace loss slots; call after fgs_render_forward with the
 * same workspace. */
int fgs_loss_l1_dssim(void *ws, const fgs_workspace_layout *layout, const fgs_camera *cams_host,
                      const float *images, const float *targets, float lambda, float *loss_out,
                      float *dl_dimages, void *stream);

/* Backward pass: zero the screen-gradient accumulators of the blocks of
 * 128 Gaussians with a rendered pair in the forward, re-traverse every
 * tile back to front from each pixel's last contributor (recovering T by
 * division, Suppl. B.1), reduce per-Gaussian gradients across each warp
 * and CTA before global atomics, then the chain rule of the preprocessing
 * (fused activation gradients, Sec. 3.2).  grads: float32 tensors for every
 * group the parameters have (6, or 8 for dynamic Gaussians); written for
 * every Gaussian (zero where invisible), summed over the views.  Needs the
 * workspace of the matching forward. */
int fgs_render_backward(void *ws, const fgs_workspace_layout *layout, const fgs_params *params,
                        int32_t sh_degree, const fgs_camera *cams_host,
                        const fgs_camera *cams_device, const float bg[3],
                        const float *dl_dimages, const fgs_params *grads, void *stream);

/* Adam (Suppl. A; Sec. 3.3 own fused Adam matching PyTorch): for every
 * element of every group, m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr/(1-b1^t) * m / (sqrt(v)/sqrt(1-b2^t) + eps), step t >= 1.
 * As in PyTorch, 1 - b1, 1 - b2 and the bias corrections are formed in
 * double precision and rounded to float once.
 * lr: host float[8] in group order (6 and 7 used only when those groups
 * are set).  Every Gaussian is updated, including
 * those with zero gradient (Sec. 3.3 "Fusing Backward and Optimizer").
 * params groups 4..5 and both moments may be FGS_BF16 or FGS_F16 (math in
 * float32, rounded to nearest on store); grads are float32. */
int fgs_adam_step(const fgs_params *params, const fgs_params *grads, const fgs_params *exp_avg,
                  const fgs_params *exp_avg_sq, const float lr[8], double beta1, double beta2,
                  double eps, int32_t step, void *stream);

/* Adam state kept in device memory, so that a captured graph can replay
 * training steps without host involvement: each fgs_adam_step_device call
 * first increments `step` on the device, derives the step sizes and the
 * bias correction, then updates every group. */
typedef struct fgs_adam_state {
    double beta1, beta2, eps;  /* exact hyper-parameters (0.999 is not a float32) */
    float lr[8];            /* base learning rates in group order (Suppl. A) */
    float lr_means_final;   /* exponential decay target of lr[0] (Suppl. A); <= 0: constant */
    int32_t decay_steps;    /* steps over which lr[0] decays to lr_means_final */
    int32_t step;           /* steps taken so far; the call uses step + 1 and stores it */
    float step_size[8];     /* written by the call: lr_t / (1 - beta1^t) */
    float inv_bc2_sqrt;     /* written by the call: 1 / sqrt(1 - beta2^t) */
    float beta1_f, beta2_f, one_minus_beta1_f, one_minus_beta2_f, eps_f; /* written by the call */
} fgs_adam_state;

/* Same update as fgs_adam_step with the hyper-parameters and step counter
 * read from (and the counter written back to) `state_device`. */
int fgs_adam_step_device(const fgs_params *params, const fgs_params *grads,
                         const fgs_params *exp_avg, const fgs_params *exp_avg_sq,
                         fgs_adam_state *state_device, void *stream);

/* Backward pass fused with the Adam step (Sec. 3.3 "Fusing Backward and
 * Optimizer"): the blend backward of fgs_render_backward, then one kernel
 * that forms each Gaussian's parameter gradients (summed over the views)
 * and applies the fgs_adam_step_device update to all of its values right
 * away, so the gradients never round-trip through memory.  Every Gaussian
 * is updated, zero-gradient ones included.  params are updated in place
 * (the same buffers the forward read).  exp_avg / exp_avg_sq: one moment
 * dtype for all groups; supported pairs (SH dtype, moment dtype): (F32,
 * F32), (BF16, F32), (BF16, BF16), (F16, F32), (F16, F16); others return
 * FGS_ERR_DTYPE.  An FP16 second moment is stored as sqrt(v), as in
 * fgs_adam_step.  grads: optional (NULL skips them); when given, float32
 * groups that receive the gradients used.  state_device as for
 * fgs_adam_step_device (its step is incremented).  Results equal
 * fgs_render_backward followed by fgs_adam_step_device up to the order of
 * the float32 atomic additions in the blend backward. */
int fgs_render_backward_adam(void *ws, const fgs_workspace_layout *layout, const fgs_params *params,
                             int32_t sh_degree, const fgs_camera *cams_host,
                             const fgs_camera *cams_device, const float bg[3],
                             const float *dl_dimages, const fgs_params *exp_avg,
                             const fgs_params *exp_avg_sq, fgs_adam_state *state_device,
                             const fgs_params *grads, void *stream);

/* Stable LSD radix sort of (uint64 key, uint32 value) pairs on the low
 * `bits` key bits (1..64), 8 bits per pass (Sec. 3.2 "Sorting": a single
 * radix sort of the combined keys).  keys/vals hold the input; keys_alt /
 * vals_alt are same-sized scratch.  The sorted result ends in keys/vals
 * when *result_in_alt (host) is 0, else in the *_alt buffers.  scratch:
 * device buffer of fgs_sort_scratch_bytes(n) bytes, 256-byte aligned.
 * Key buffers must be 8-byte and value buffers 4-byte aligned, else
 * FGS_ERR_ALIGN before any launch. */
size_t fgs_sort_scratch_bytes(int64_t n);
int fgs_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                   int64_t n, int32_t bits, void *scratch, size_t scratch_bytes,
                   int32_t *result_in_alt, void *stream);

/* The same stable radix sort for callers that cannot allocate device
 * memory on the path where they sort -- for instance a host framework that
 * owns every device allocation through its own pool and forbids raw
 * cudaMalloc from plug-ins, or latency-critical code that cannot afford the
 * device-wide synchronisation cudaMalloc and cudaFree imply.  The paper has
 * no counterpart; this is a deployment variant of fgs_sort_pairs.
 *
 * keys[n] / vals[n] (device) are sorted in place on their low `bits` bits.
 * All scratch is one library-owned array of FGS_STATIC_SORT_MAX_PAIRS pairs
 * (about 12.3 MB: keys and values ping-pong buffers plus histograms), held
 * by every GPU that loads the library until the process exits; the call
 * allocates nothing.  n > FGS_STATIC_SORT_MAX_PAIRS returns
 * FGS_ERR_TOO_LARGE before any launch; n == 0 returns FGS_OK.
 * keys must be 8-byte and vals 4-byte aligned, else FGS_ERR_ALIGN.
 * The first call on a device looks up the array's device address (with that
 * device current), so make it before any stream capture on that device.
 * The address is cached per device number for the CUDA runtime's primary
 * context; after cudaDeviceReset, or under another context made current
 * through the driver API, the cached address is stale and must not be used.
 * Every call uses the same array: calls whose kernels overlap on the GPU
 * (different streams, or different host threads, without ordering between
 * them) race on it and corrupt each other's results. */
#define FGS_STATIC_SORT_MAX_PAIRS (1 << 20)
int fgs_sort_pairs_static(uint64_t *keys, uint32_t *vals, int64_t n, int32_t bits, void *stream);

/* Locality-preserving order (Sec. 3.3 "Locality-preserving
 * densification"): the z-order (Morton) permutation of the Gaussians, so
 * that Gaussians close in 3D sit close in the parameter buffers.  The paper
 * applies it every few thousand iterations; apply the permutation to every
 * buffer indexed by Gaussian (parameters, Adam moments) with
 * fgs_permute_params.
 *
 * means: [n,3] float32 (device), finite.  The bounding box [lo, hi] of the
 * means is found on the device; each coordinate maps to 10 bits,
 *   q_a = min(1023, floor((x_a - lo_a) * s_a)),  s_a = 1024 / (hi_a - lo_a)
 * (s_a = 0 when hi_a == lo_a), evaluated in float32 with round-to-nearest
 * and no fused multiply-add, so that the codes are reproducible bit for
 * bit.  The code interleaves the bits: bit 3b + a of the code is bit b of
 * q_a (a = 0, 1, 2 for x, y, z), 30 bits in all.
 * order: [n] uint32 (device, output): order[i] is the index of the Gaussian
 * at position i of the stable sort of the codes (equal codes keep index
 * order).  codes: [n] uint32 (device, output) receiving the sorted codes,
 * or NULL.  scratch: device buffer of fgs_morton_scratch_bytes(n) bytes,
 * 256-byte aligned.  n == 0 is a no-op; n > 2^31 - 1 is FGS_ERR_SHAPE. */
size_t fgs_morton_scratch_bytes(int64_t n);
int fgs_morton_order(const float *means, int64_t n, uint32_t *order, uint32_t *codes,
                     void *scratch, size_t scratch_bytes, void *stream);

/* Gathers every group present in *src into *dst by a permutation:
 * row i of each dst group = row order[i] of the src group (order: [n]
 * uint32, device, a permutation of 0..n-1 as fgs_morton_order writes it),
 * or row i itself when order is NULL (a plain copy).  Works for parameters
 * and for Adam moments alike: any storage type, groups 0..5 always, 6 and 7
 * both or neither; *dst must hold the same n, groups and types, and no dst
 * group may share memory with its src group.  Rows of an index outside
 * 0..n-1 are left unwritten (a bad order is the caller's bug; nothing
 * faults). */
int fgs_permute_params(const fgs_params *src, const fgs_params *dst, const uint32_t *order,
                       void *stream);

/* Microbenchmarks of the rates that bound the blend kernels (measurement
 * only; the caller times each call with events on `stream`).  Each returns
 * through *grid_out the number of 256-thread CTAs it launched; out is a
 * device float[*grid_out] the kernels never write in practice (it keeps
 * their work from being optimised away).
 *   fgs_peak_fma:     grid * 256 * iters * 8 FP32 fused multiply-adds.
 *   fgs_peak_ex2:     grid * 256 * iters * 8 evaluations of ex2.approx.
 *   fgs_peak_l2_read: reps passes of 16-byte reads over buf (n4 words,
 *                     16-byte aligned; sized to stay in L2). */
int fgs_peak_fma(int32_t iters, float *out, int32_t *grid_out, void *stream);
int fgs_peak_ex2(int32_t iters, float *out, int32_t *grid_out, void *stream);
int fgs_peak_l2_read(const void *buf, int64_t n4, int32_t reps, float *out, int32_t *grid_out,
                     void *stream);

/* Synchronises `stream`, then reads the workspace header: sticky device
 * flags (FGS_FLAG_*) and the instance count of the last forward.  Either
 * output pointer may be NULL.  clear != 0 resets the flags afterwards. */
int fgs_get_error(void *ws, uint32_t *flags_host, uint64_t *instances_host, int32_t clear,
                  void *stream);

/* Optional per-kernel timing.  After fgs_profile_attach(events, labels,
 * capacity) with `capacity` caller-created cudaEvent_t handles (host array,
 * passed as void*) and a host array of as many label pointers, every entry
 * point records the next event on its stream after each kernel it launches
 * (and one before its first) and stores a static label naming the kernel;
 * recording stops when the array is full.  The elapsed time between two
 * consecutive events is the device time of the kernel the second one
 * names.  fgs_profile_attach(NULL, NULL, 0) detaches; fgs_profile_count
 * returns the number of events recorded since the last attach.  Not meant
 * for stream capture.  Host state: one attachment per process. */
int fgs_profile_attach(void **events, const char **labels, int32_t capacity);
int32_t fgs_profile_count(void);

/* Static description of a status code. */
const char *fgs_strerror(int code);

/* Static description of one device flag bit (FGS_FLAG_*); "unknown flag"
 * for any other value, including 0 and combinations of bits. */
const char *fgs_flag_string(uint32_t flag);

#ifdef __cplusplus
}
#endif
#endif /* FASTERGS_H */
