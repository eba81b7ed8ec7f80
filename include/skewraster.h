/* skewraster.h — C ABI of the GB300 (sm_103a) tile rasterizer for 3D skew
 * Gaussians (3D Skew Gaussian Splatting).
 *
 * The library renders N skew Gaussians into one or more views and computes
 * gradients of a scalar loss with respect to every Gaussian attribute.  A
 * frame is four calls, in this order, on one CUDA stream:
 *
 *   sr_preprocess   project each Gaussian into each view (Preliminaries,
 *                   Eq. 1 and the EWA local-affine projection; Appendix
 *                   "Forward Pass": dilation, compensation, conic (a,b,c)
 *                   and o' = d; Alg. 1 inputs beta_x, beta_y; Eq. alpha for
 *                   the enhanced opacity; SH colour), plus a conservative
 *                   tile rectangle and the FP32 depth key;
 *   sr_bin_sort     one (tile | depth) key per touched tile, radix-sorted
 *                   so each tile's Gaussians are in depth order (Preliminaries:
 *                   "tile-based ... sorted in depth"), and per-tile ranges;
 *   sr_render_fwd   per pixel, front-to-back alpha blending of the skew
 *                   kernel alpha = d G'(x) (1 + erf z) with early stop
 *                   (Alg. 1, Eq. 2, Eq. color);
 *   sr_render_bwd   reverse replay of the blend (Alg. 2, Appendix "Backward
 *                   Pass") and the chain rule back through the projection.
 *
 * Conventions shared by every entry point
 *  - Memory: the library never allocates device memory.  Every device buffer
 *    (attributes, cameras, workspace, images, gradients) is allocated and
 *    owned by the caller; pointers must stay valid until the stream work
 *    that uses them has completed.  Host structs are read during the call
 *    only.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  All device work is enqueued asynchronously on it;
 *    only sr_bin_sort with a non-NULL keys_needed, sr_read_status,
 *    sr_frame_counters, sr_selftest_bounded_wait and sr_sort_keys_noalloc
 *    block the host (they read a few bytes back from the device).
 *  - Errors: every call returns an sr_status; nothing is thrown across the
 *    ABI.  Host-side argument checks run first and leave the device
 *    untouched on failure.  Device-side failures (key capacity exceeded, a
 *    bounded wait that gave up) set bits in a status word in the workspace,
 *    read by sr_read_status (or returned by sr_bin_sort when it syncs).
 *  - Coordinates: cameras use the OpenCV convention (+Z forward, +Y down,
 *    +X right).  Pixel (px, py) has its centre at (px + 0.5, py + 0.5).
 *  - Images are planar FP32, [3][H][W] per view; views are concatenated in
 *    view order at plan.image_offset[v] floats.  Per-pixel state (t_final,
 *    n_contrib) is [H][W] per view at plan.pixel_offset[v].
 */
#ifndef SKEWRASTER_H
#define SKEWRASTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SR_MAX_VIEWS 256
#define SR_ABI_VERSION 3

typedef enum sr_status {
  SR_OK = 0,
  SR_ERR_INVALID = 1,     /* bad argument: sizes, NULL pointers, degree > 3, dtype tag */
  SR_ERR_CAPACITY = 2,    /* more tile keys than the plan's key capacity */
  SR_ERR_CUDA = 3,        /* a CUDA runtime call failed (launch, copy) */
  SR_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
  SR_ERR_UNSUPPORTED = 5  /* a valid request this build does not implement */
} sr_status;

/* Storage type of the SH coefficients, log-scales and skew/split vectors.
 * Arithmetic is FP32 whatever the storage. */
typedef enum sr_dtype { SR_F32 = 0, SR_BF16 = 1, SR_F16 = 2 } sr_dtype;

/* N Gaussians, structure of arrays, device pointers, caller-owned.
 * Row-major, element i of an [n,k] array at ptr + i*k.  Alignment: each
 * pointer 16-byte aligned. */
typedef struct sr_gaussians {
  const void* means;          /* [n,3] f32 world-space centre mu (Eq. 1) */
  const void* log_scales;     /* [n,3] dt_scale; S = diag(exp(log_scales)) (Eq. 1) */
  const void* quats;          /* [n,4] f32 (w,x,y,z), any norm > 0; R from q/|q| (Eq. 1) */
  const void* opacity_logits; /* [n] f32, or [n,2] f32 when two_opacities: alpha_1, alpha_2 = sigmoid (Eq. alpha) */
  const void* skew;           /* [n,3] dt_skew: skew eta in the Gaussian's standardised local frame */
  const void* split_dir;      /* [n,3] dt_skew or NULL: direction d of the enhanced opacity (Eq. alpha) */
  const void* sh;             /* [n,(deg+1)^2,3] dt_sh: SH colour coefficients (Preliminaries) */
  int64_t n;                  /* number of Gaussians, >= 0 */
  int32_t sh_degree;          /* 0..3 */
  int32_t two_opacities;      /* 0: one opacity per Gaussian; 1: alpha_1, alpha_2 */
  int32_t dt_sh, dt_scale, dt_skew; /* sr_dtype tags */
  int32_t reserved_;
} sr_gaussians;

/* One view, OpenCV convention, FP32 (see sr_camera_from_gl). */
typedef struct sr_camera {
  float w2c[12];              /* row-major 3x4 world-to-camera [R | t] */
  float fx, fy, cx, cy;       /* intrinsics K (pixels) */
  float tan_fovx, tan_fovy;   /* tan(FoV/2), bound the local-affine Jacobian */
  float campos[3];            /* camera centre (world), for the SH view direction */
  int32_t width, height;      /* pixels, 1..32768 */
} sr_camera;

/* Rasterizer constants.  sr_config_default fills the values used by the
 * paper's 3DGS baseline and this library's tests. */
typedef struct sr_config {
  int32_t tile_w, tile_h;     /* 16x16 (only size in this build) */
  float alpha_min;            /* gate: pairs with alpha < alpha_min are skipped (1/255) */
  float alpha_max;            /* clamp on alpha (0.99) */
  float t_stop;               /* stop before the Gaussian that takes T below t_stop (1e-4) */
  float dilation;             /* s of Sigma' + sI (0.3 px^2) */
  float fov_clamp;            /* |x/z| <= fov_clamp * tan_fovx in the Jacobian (1.3) */
  float near_z;               /* cull camera z <= near_z (0.2) */
  float bg[3];                /* background colour */
  int32_t antialias_comp;     /* 1: d = o * sqrt(det Sigma' / det(Sigma' + sI)); 0: d = o */
  int32_t fwd_batch;          /* 128, 256 or 512 (0 = 256): records sr_render_fwd stages in shared memory per batch */
  int32_t sort_spin_limit;    /* 0 = auto; bound on each look-back wait of the sort */
  int32_t fwd_pixels_per_thread; /* 1, 2 or 4 (0 = 2): pixels each thread of sr_render_fwd owns */
  int32_t bwd_pixels_per_thread; /* 1, 2 or 4 (0 = 2): pixels each thread of sr_render_bwd owns */
  int32_t forward_only;       /* plans made with 1 record no per-pixel blend masks (less workspace);
                                 sr_render_bwd on them returns SR_ERR_UNSUPPORTED */
  int32_t bwd_batch;          /* 128 or 256 (0 = 128): records sr_render_bwd stages per batch */
  int32_t recompute_keys;     /* plans made with 1 keep no per-pixel blend masks; sr_render_bwd then
                                 rebuilds the frame's records and tile key lists (sr_preprocess and a
                                 non-blocking sr_bin_sort) and replays every position up to each pixel's
                                 n_contrib with the alpha gate (Alg. 2), so the workspace may serve other
                                 frames between a forward and its backward.  Not with forward_only. */
  int32_t persistent;         /* bit 0: sr_render_fwd, bit 1: the backward composite launch as many blocks
                                 as fit on the GPU, each taking tile after tile (longest key lists first)
                                 from a counter, instead of one block per tile; results are the same */
  int32_t fwd_blocks_per_sm;  /* 0..32 (0 = as many as fit): cap on the blocks of sr_render_fwd resident on
                                 an SM (each block then reserves a matching share of shared memory) */
  int32_t bwd_blocks_per_sm;  /* the same for the backward composite */
} sr_config;

/* Gradients of the loss w.r.t. the attributes, FP32, device, caller-owned,
 * same layouts as sr_gaussians (FP32 whatever the storage type).  Fully
 * overwritten by sr_render_bwd (summed over all views of the plan).
 * split_dir may be NULL iff the scene has none.  means2d_abs (optional, [n])
 * receives sum over views of |dL/dmu_2| and depth_grad (optional, [n]) the
 * sum over views of dL/dz of the camera-space centre. */
typedef struct sr_grads {
  float* means;
  float* log_scales;
  float* quats;
  float* opacity_logits;
  float* skew;
  float* split_dir;
  float* sh;
  float* means2d_abs;
  float* depth_grad;
} sr_grads;

/* Host-side plan: sizes and workspace layout for one (N, cameras) set-up.
 * Caller-owned plain struct filled by sr_plan_init; read-only afterwards. */
typedef struct sr_plan {
  int32_t abi_version;
  int32_t n_views;
  int64_t n;
  int32_t sh_degree;
  int32_t tile_w, tile_h;
  int32_t sort_passes;        /* 8-bit radix passes over the tile ids (after a 4-pass depth sort of the records) */
  int32_t sort_bits;          /* width of the (tile | depth) order: 32 depth bits + tile-id bits */
  int32_t render_mode;        /* 0: one opacity; 1: two opacities; 2: two opacities + split direction */
  int32_t two_opacities;      /* copied from the sr_gaussians the plan was made for */
  int32_t has_split;          /* 1 if split_dir was non-NULL */
  int32_t forward_only;       /* from the config: no blend masks, no backward */
  int32_t recompute_keys;     /* from the config: no blend masks; the backward rebuilds the key lists */
  int64_t key_capacity;       /* keys the workspace can hold */
  int64_t total_tiles;
  int64_t total_pixels;
  int64_t tile_base[SR_MAX_VIEWS + 1];    /* first global tile id of view v */
  int64_t image_offset[SR_MAX_VIEWS + 1]; /* float offset of view v's [3][H][W] image */
  int64_t pixel_offset[SR_MAX_VIEWS + 1]; /* element offset of view v's [H][W] state */
  int32_t width[SR_MAX_VIEWS], height[SR_MAX_VIEWS];
  size_t ws_bytes;            /* workspace size to allocate (256-byte aligned base) */
  size_t off[32];             /* internal offsets into the workspace */
} sr_plan;

/* Version of this ABI (SR_ABI_VERSION). */
int32_t sr_abi_version(void);

/* Human-readable name of a status code; never NULL. */
const char* sr_status_string(sr_status s);

/* Fill *cfg with the defaults listed in sr_config.  Returns SR_ERR_INVALID on NULL. */
sr_status sr_config_default(sr_config* cfg);

/* Camera set-up of Alg. 3: c2w_gl is the row-major 4x4 camera-to-world pose in
 * the OpenGL/Blender convention (-Z forward, +Y up).  Applies
 * M_cv = M_gl diag(1,-1,-1,1) (Eq. coord_transform), inverts it to W2C, and
 * builds K with fx = W / (2 tan(fovx/2)), fy = H / (2 tan(fovy/2)),
 * (cx, cy) = (W/2, H/2) (the K matrix).  Computed in FP64, rounded once to
 * FP32.  Host only.  SR_ERR_INVALID on NULL, non-positive size, or a FoV
 * outside (0, pi). */
sr_status sr_camera_from_gl(const double c2w_gl[16], int32_t width, int32_t height, double fovx, double fovy,
                            sr_camera* out);

/* Plan the Gaussians described by g (only n, sh_degree, two_opacities,
 * the dtype tags and whether split_dir is non-NULL are read; the data
 * pointers may be NULL here) into n_views views (host array cams_host, used
 * for sizes only) with room for key_capacity tile keys.  Later calls must
 * pass Gaussians with the same description.  SR_ERR_INVALID on bad sizes
 * (n < 0, n_views outside 1..SR_MAX_VIEWS, degree > 3, a view size outside
 * 1..32768, tile size other than 16x16, key_capacity outside 0..2^32-1, or
 * n * n_views >= 2^31). */
sr_status sr_plan_init(sr_plan* plan, const sr_config* cfg, const sr_gaussians* g, const sr_camera* cams_host,
                       int32_t n_views, int64_t key_capacity);

/* Workspace bytes for the plan (same as plan->ws_bytes). */
size_t sr_workspace_size(const sr_plan* plan);

/* Project every Gaussian into every view.  cams_dev: device array of
 * plan->n_views sr_camera whose sizes match the plan.  ws: device workspace
 * of plan->ws_bytes bytes, 256-byte aligned.  Writes the per-(view,
 * Gaussian) records, depth keys, tile rectangles and tile counts into ws. */
sr_status sr_preprocess(const sr_plan* plan, const sr_gaussians* g, const sr_camera* cams_dev, const sr_config* cfg,
                        void* ws, void* stream);

/* Tile binning and depth sort.  The records are first sorted by their FP32
 * depth bits (4 stable 8-bit LSD radix passes over the records, ties in
 * record-index order); an exclusive scan of the tile counts, taken in that
 * depth order, places each record's keys; one 32-bit global tile id per
 * touched tile (row-major within the record) is emitted in depth order with
 * the record index as value; a stable LSD radix sort over the tile-id bits
 * only then leaves every tile's keys in (depth bits, record index) order.
 * The result is the list a stable sort of 64-bit (global tile << 32 | depth
 * bits) keys emitted in record-index order would give, with per-tile
 * [start, end) ranges.  If keys_needed is non-NULL the call blocks until
 * the key emission is done, stores the number of keys the frame needs and
 * returns SR_ERR_CAPACITY (nothing to render) if it exceeds
 * plan->key_capacity; the tile sort is queued behind the count's readback
 * (a kernel writes it into mapped pinned host memory, so it never waits for
 * the caller's own copies) and the device does not idle meanwhile; where no
 * mapped pinned memory can be had the sort waits for the count and skips
 * radix passes whose digit is the same for every key.  If NULL, the call
 * never blocks (for CUDA-graph capture): every pass runs and an overflow is
 * reported through the status word (sr_read_status). */
sr_status sr_bin_sort(const sr_plan* plan, const sr_config* cfg, void* ws, int64_t* keys_needed, void* stream);

/* Forward composite of all views.  images: plan->image_offset[n_views]
 * floats; t_final: final transmittance per pixel; n_contrib: per pixel, one
 * past the position (within its tile's sorted range) of the last blended
 * Gaussian.  t_final and n_contrib are plan->total_pixels elements and are
 * needed by sr_render_bwd. */
sr_status sr_render_fwd(const sr_plan* plan, const sr_config* cfg, void* ws, float* images, float* t_final,
                        uint32_t* n_contrib, void* stream);

/* Backward of L with dL/dimage = d_images (same layout as images): reverse
 * replay per pixel (Alg. 2; the d/dx bracket is read with delta = x - mu,
 * giving -sqrt(2/pi) beta e^{-z^2} inside the bracket of dL/dmu), FP32
 * gradients reduced per warp before global atomics, then the chain rule
 * through the projection into *out (overwritten).  Needs the ws, t_final and
 * n_contrib of the matching forward call and the same g and cams_dev.  May be
 * called again for the same frame (another d_images): the workspace's 2D
 * gradients, zeroed by sr_preprocess for its frame, are cleared again on the
 * device when a backward has used them since.  On a recompute_keys plan the
 * workspace need not hold the frame any more: the call first re-runs
 * sr_preprocess and sr_bin_sort (non-blocking) for g and cams_dev, then
 * replays without blend masks; only t_final and n_contrib of the forward are
 * needed. */
sr_status sr_render_bwd(const sr_plan* plan, const sr_gaussians* g, const sr_camera* cams_dev, const sr_config* cfg,
                        void* ws, const float* d_images, const float* t_final, const uint32_t* n_contrib,
                        const sr_grads* out, void* stream);

/* Stable radix sort of (key, value) pairs that allocates nothing: the same
 * onesweep passes as sr_bin_sort, for callers that cannot allocate device
 * memory at all (a runtime that hands out only fixed, pre-assigned buffers,
 * a plugin that receives just its input and output pointers, or a frame
 * loop that must never call cudaMalloc).  The paper has no counterpart.
 *
 * keys_in/vals_in: n input pairs (device, read only); keys_out/vals_out: n
 * output pairs (device, must not alias the inputs), sorted by the key's low
 * ceil(sort_bits / 8) bytes, ties in input order; key bits above sort_bits
 * are expected to be zero.  n at most SR_NOALLOC_MAX_KEYS (2^20), else
 * SR_ERR_CAPACITY; sort_bits in 1..64 and non-NULL distinct pointers, else
 * SR_ERR_INVALID.
 *
 * Scratch: one fixed array of about 16 MiB in the library's device memory,
 * present on every GPU that loads the library until the process exits.
 * Each call looks up that array's device address on the current device
 * (cudaGetSymbolAddress; the address can change after a cudaDeviceReset).
 * Every call reuses the same array and the work it enqueues clears what
 * must start at zero; calls whose work overlaps on the GPU (different
 * streams, or several host threads) race on it and must be serialised by the
 * caller.
 *
 * Completion: the call ends by reading the sort's 4-byte status word back
 * and synchronising the stream, so the output is ready when it returns.  It
 * returns SR_ERR_TIMEOUT if one of the sort's bounded look-back waits gave
 * up (the output is then not sorted), and SR_ERR_CUDA only when one of its
 * own launches or its readback failed (errors left pending by earlier,
 * unrelated calls are neither reported nor cleared). */
#define SR_NOALLOC_MAX_KEYS (1u << 20)
sr_status sr_sort_keys_noalloc(const uint64_t* keys_in, const uint32_t* vals_in, int64_t n, int32_t sort_bits,
                               uint64_t* keys_out, uint32_t* vals_out, void* stream);

/* Diagnostics: number of kernels this library has launched in this process
 * (all devices and streams), and the last frame's work counters (pairs of
 * pixel and Gaussian tested and blended by sr_render_fwd), read from the
 * workspace with a stream synchronisation.  Either output may be NULL. */
uint64_t sr_kernel_launches(void);
sr_status sr_frame_counters(const sr_plan* plan, void* ws, uint64_t* pairs_tested, uint64_t* pairs_blended,
                            void* stream);

/* The two halves of sr_render_bwd, for callers that time or overlap them:
 * sr_render_bwd_composite runs the reverse replay (Alg. 2) and leaves the
 * per-(view, Gaussian) gradients of the 2D quantities (mu_2, conic,
 * projected skew, opacity terms, colour) in the workspace;
 * sr_render_bwd_project then applies the chain rule through the projection
 * (Appendix "Backward Pass", deferred to 3DGS in the paper) into *out.
 * Same arguments and rules as sr_render_bwd, except that on a recompute_keys
 * plan sr_render_bwd_composite does not rebuild the key lists: the
 * workspace must hold the frame (its sr_preprocess and sr_bin_sort). */
sr_status sr_render_bwd_composite(const sr_plan* plan, const sr_config* cfg, void* ws, const float* d_images,
                                  const float* t_final, const uint32_t* n_contrib, void* stream);
sr_status sr_render_bwd_project(const sr_plan* plan, const sr_gaussians* g, const sr_camera* cams_dev,
                                const sr_config* cfg, void* ws, const sr_grads* out, void* stream);

/* Measured instruction throughput of this GPU for the arithmetic the blend
 * loops of Alg. 1 and Alg. 2 are bound by (the roofline of the composites):
 * FP32 fused multiply-add, packed FP32x2 fused multiply-add, FP32 min/max
 * (the gate and clamp), and the multi-function unit's ex2 and rcp (the
 * exponentials and the reciprocal of each skew-kernel evaluation).  Each
 * rate is the best of three launches that fill every SM with independent
 * dependency chains of that one kind, timed with CUDA events on the stream;
 * the rates hold at the SM clock of the run (sample it alongside).
 * scratch: 128 bytes of device memory, 16-byte aligned, never read (a sink
 * that keeps the chains live).  Synchronises the stream; takes about 0.1 s. */
typedef struct sr_alu_peaks {
  double fma_lane_ops_per_s;    /* FP32 FMA results per second (one per lane) */
  double ffma2_lane_ops_per_s;  /* FP32 FMA results per second from packed FP32x2 instructions */
  double minmax_lane_ops_per_s; /* FP32 min or max results per second */
  double ex2_per_s;             /* ex2.approx results per second */
  double rcp_per_s;             /* rcp.approx results per second */
  double seconds;               /* device time of the timed launches */
} sr_alu_peaks;
sr_status sr_measure_alu_peaks(void* scratch, sr_alu_peaks* out, void* stream);

/* Self-test of the sort's bounded waits (failure detection without a GPU
 * fault): runs one radix pass over zero keys in the workspace in which no
 * block takes partition 0, so the block of partition 1 waits for a
 * look-back word that is never written.  The wait gives up after spin_limit
 * polls, flags the status word and lets the pass finish.  Synchronises the
 * stream; returns SR_ERR_TIMEOUT (the expected outcome) with the partition
 * that gave up in *gave_up_partition, SR_OK if no wait gave up.  Clobbers
 * the workspace's sort buffers and status word: call it between frames.
 * Needs key_capacity >= 8192 and at least one tile pass (>1 tile). */
sr_status sr_selftest_bounded_wait(const sr_plan* plan, void* ws, int32_t spin_limit, int64_t* gave_up_partition,
                                   void* stream);

/* Synchronise the stream and read the device status word.  Returns SR_OK,
 * SR_ERR_CAPACITY or SR_ERR_TIMEOUT (first set bit), clears the word, and
 * stores the last frame's key count in *keys_needed if non-NULL. */
sr_status sr_read_status(const sr_plan* plan, void* ws, int64_t* keys_needed, void* stream);

/* ---- Training step ------------------------------------------------------
 * The paper optimises its skew Gaussians inside the 3DGS framework
 * (Preliminaries: gradient descent "driven by photometric loss"; Appendix
 * "Implementation": the 3DGS protocol, learning rate 1e-4 for the skew
 * parameters).  These two calls are that loop's other steps. */

/* Bytes of device scratch sr_loss_l1_dssim needs for a plan's views. */
size_t sr_loss_scratch_size(const sr_plan* plan);

/* Photometric loss of all views of a plan and its gradient:
 *   L = (1 - lambda) mean |C - T| + lambda (1 - mean SSIM(C, T)),
 * means over the 3 channels and all pixels of all views; SSIM per channel
 * with an 11 x 11 Gaussian window (sigma 1.5, normalised, zero padding),
 * C1 = 0.01^2, C2 = 0.03^2 (values in [0, 1]).
 * images, targets, d_images: device FP32, plan->image_offset[n_views] floats,
 * each view [3][H][W] at its image offset (the layout of sr_render_fwd);
 * d_images receives dL/dC (it may be the d_images of sr_render_bwd).
 * loss: device float[1]; ssim_l1: optional device float[2] receiving the
 * mean SSIM and the mean |C - T|.  ws: the plan's workspace after
 * sr_preprocess (its view table).  scratch: device, sr_loss_scratch_size
 * bytes, 256-byte aligned, overwritten.  lambda in [0, 1].
 * Errors: SR_ERR_INVALID for NULL pointers, misalignment or lambda out of
 * range; SR_ERR_CUDA if a launch fails. */
sr_status sr_loss_l1_dssim(const sr_plan* plan, void* ws, const float* images, const float* targets, float lambda,
                           float* d_images, float* loss, float* ssim_l1, void* scratch, void* stream);

/* One Adam step (Kingma & Ba 2015, the update of torch.optim.Adam) over up to
 * SR_ADAM_MAX_GROUPS parameter groups in one launch:
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   p -= lr / (1 - b1^step) * m / (sqrt(v) / sqrt(1 - b2^step) + eps).
 * Each group: FP32 device arrays param (updated in place), grad, m, v (the
 * moment states, zero before step 1, updated in place) of n elements; lr,
 * and lr_rest for the elements whose index modulo period (> 0) is at least
 * split_at (the higher-order SH coefficients of an [N][K][3] array:
 * period 3K, split_at 3).  step >= 1.
 * Errors: SR_ERR_INVALID for n_groups out of range, NULL arrays with n > 0,
 * step < 1, betas outside [0, 1) or eps <= 0; SR_ERR_CUDA if the launch fails. */
#define SR_ADAM_MAX_GROUPS 16
typedef struct sr_adam_group {
  float* param;
  const float* grad;
  float* m;
  float* v;
  int64_t n;
  float lr;
  float lr_rest;
  int32_t period;
  int32_t split_at;
} sr_adam_group;
sr_status sr_adam_step(const sr_adam_group* groups, int32_t n_groups, int64_t step, float beta1, float beta2,
                       float eps, void* stream);

/* Densification statistics over iterations (Sec. "Depth-Aware Densification
 * Strategy"), from one backward's sr_grads.means2d_abs (g^(uv) of this step)
 * and sr_grads.depth_grad (dL/dz of the centre): for each of the n Gaussians
 * with a nonzero g^(uv), uv_sum += g^(uv) and seen += 1 (the 3DGS average
 * is uv_sum / seen); z_max = max(z_max, |dL/dz|), the paper's g^(z).  All
 * arrays device, [n], the accumulators updated in place (zero them to start).
 * Errors: SR_ERR_INVALID for n < 0 or NULL arrays with n > 0. */
sr_status sr_densify_stats(const float* means2d_abs, const float* depth_grad, int64_t n, float* uv_sum,
                           int32_t* seen, float* z_max, void* stream);

/* ---- Densification (Sec. "Depth-Aware Densification Strategy"; Fig. "split") ----
 * From the statistics sr_densify_stats collects, each of the n Gaussians is
 * (decisions in FP32):
 *   removed  if its largest opacity logit < logit_prune;
 *   else split or cloned if uv_sum / seen >= grad_uv (g^(uv); 0 when seen is
 *            0) or z_max >= grad_z (g^(z), Eq. depth_grad): split if its
 *            largest log-scale > log_scale_split, cloned otherwise;
 *   else kept.
 * A split cuts the skew Gaussian at its centre across its largest axis k
 * (first of equal maxima); each child stands for one half and takes that
 * half's mean and variance along the axis (centre moved by s_k m along the
 * axis, log-scale log s_k + log(v) / 2 on it), skew component 0 on the axis
 * and eta_j / sqrt(1 + eta_k^2) on the others (the parent's marginal skew);
 * rotation, opacities, SH and split direction are copied.
 * Output order: the kept Gaussians (cloned ones included) in index order,
 * then the clones' copies in index order, then for each split Gaussian in
 * index order its child on the + side of the axis and its child on the -
 * side.  There are at most 2n outputs. */
typedef struct sr_densify_config {
  float grad_uv;              /* threshold on uv_sum / seen */
  float grad_z;               /* threshold on z_max */
  float log_scale_split;      /* largest log-scale above which a densified Gaussian is split */
  float logit_prune;          /* Gaussians whose largest opacity logit is below are removed */
} sr_densify_config;

/* FP32 attribute arrays of a scene (the outputs of sr_densify), caller-owned,
 * same layouts as sr_gaussians; split_dir NULL iff the input has none. */
typedef struct sr_scene_arrays {
  float* means;
  float* log_scales;
  float* quats;               /* 16-byte aligned */
  float* opacity_logits;
  float* skew;
  float* split_dir;
  float* sh;
} sr_scene_arrays;

/* Bytes of device scratch sr_densify needs for n Gaussians. */
size_t sr_densify_scratch_size(int64_t n);

/* g: FP32 attributes (dt_sh = dt_scale = dt_skew = SR_F32), 0 <= n < 2^30;
 * uv_sum, seen, z_max: [n] device statistics; out: device arrays with room
 * for 2n Gaussians; src_map (optional, [2n] device): per output, its source
 * index | kind << 30 with kind 0 kept, 1 clone copy, 2 child on the + side,
 * 3 child on the - side; counts: device int64[4] = kept, cloned, split,
 * total outputs (read them back to learn the new size); scratch:
 * sr_densify_scratch_size(n) device bytes.  Asynchronous on stream.
 * Errors: SR_ERR_INVALID for NULL pointers, other dtypes, n out of range or
 * misaligned quaternion arrays; SR_ERR_CUDA if a launch fails. */
sr_status sr_densify(const sr_gaussians* g, const float* uv_sum, const int32_t* seen, const float* z_max,
                     const sr_densify_config* cfg, const sr_scene_arrays* out, uint32_t* src_map, int64_t* counts,
                     void* scratch, void* stream);

/* Per-Gaussian state after sr_densify (e.g. Adam moments), width floats per
 * Gaussian: for each output j < min(counts[3], cap), out[j] = in[source(j)]
 * if j is a kept Gaussian, zeros for clone copies and children.  in: [n,
 * width], out: [cap, width], src_map and counts from sr_densify (device).
 * Errors: SR_ERR_INVALID for NULL pointers or negative sizes. */
sr_status sr_densify_remap(const float* in, int32_t width, const uint32_t* src_map, const int64_t* counts,
                           int64_t cap, float* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SKEWRASTER_H */
