/*
 * vrs.h - C-ABI of libvrs, a GB300 (sm_103a) tile-based 3D Gaussian Splatting
 * rasterizer for the periphery of VR-Splatting (Franke, Fink, Stamminger,
 * "VR-Splatting: Foveated Radiance Field Rendering via 3D Gaussian Splatting
 * and Neural Points", arXiv 2410.17932).
 *
 * What it computes.  Sec. 3.1 ("Naive Method") renders the periphery with 3D
 * Gaussian splats: each splat has an opacity alpha, a colour C and a 3D
 * covariance Sigma built from a per-splat scale and rotation; the splats are
 * projected and blended to screen into the full-resolution image P.  Sec. 3.2
 * renders that image for the whole frame and, in the same pass, the
 * approximate depth buffer of Eq. 1,
 *      d = sum_i d_i alpha_i prod_{m<i} (1 - alpha_m),
 * which the foveal renderer uses to cull occluded neural points.  Sec. 1 names
 * the cost that grows with the number of primitives: tiling and sorting them.
 *
 * The path behind this header:
 *   vrs_plan_batch  host: sizes, tile grid, record/tile/pixel offsets, workspace bytes
 *   vrs_preprocess  per Gaussian x view: EWA projection with the 0.3 px dilation,
 *                   3-sigma screen radius, view-dependent SH colour, tile rectangle,
 *                   and emission of (tile, depth) keys for every touched tile
 *   vrs_bin_sort    LSD radix sort of the keys, equal-key order by record index,
 *                   per-tile [start, end) ranges
 *   vrs_render_fwd  per tile, front-to-back compositing of RGB, Eq. 1 depth and
 *                   final transmittance
 *   vrs_render_bwd  the adjoint of the three steps above: gradients w.r.t. the
 *                   Gaussian parameters (the method is trained end to end by
 *                   gradient descent, Sec. 3.5 and Sec. 4 "Training")
 *
 * Conventions shared by every call:
 *  - All pointers named device_* or documented as device memory must point to
 *    memory of the current CUDA device; host structs are read during the call
 *    only and may be freed afterwards.
 *  - The caller owns every buffer, including the workspace of
 *    plan.workspace_bytes bytes (256-byte aligned).  The library allocates and
 *    frees nothing and never synchronises the stream, except vrs_query_status,
 *    which synchronises the stream it is given.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Every call is stream ordered and launches a fixed set of kernels
 *    whose shapes depend on the plan only, so a sequence of calls can be
 *    captured into a CUDA graph and replayed.
 *  - Errors detectable on the host (bad sizes, null pointers, a camera that
 *    does not match the plan) return a status at once and launch nothing.
 *    Errors detectable only on the device (instance capacity exceeded, a
 *    non-finite parameter, an all-zero quaternion) set bits in a status word
 *    inside the workspace; kernels after a capacity overflow skip their work.
 *    vrs_query_status reads that word.  No kernel spins on a flag or a counter
 *    that another kernel sets; the only waits are those of programmatic
 *    dependent launch (a kernel's first instruction waits until the kernel
 *    before it in the stream has completed), so no call can hang on the
 *    device.
 *
 * Parameterisation (Sec. 3.1: opacity, colour, scale and rotation per splat):
 *  means [n][3], log_scales [n][3] (log of the per-axis standard deviation),
 *  quats [n][4] (w, x, y, z; normalised inside), opacity_logits [n]
 *  (opacity = 1 / (1 + exp(-logit))), sh [n][(deg+1)^2][3] real spherical
 *  harmonics coefficients in (l, m = -l..l) order, deg in {0, 1, 2, 3}.  The
 *  rendered colour is max(0, sum_k Y_k(dir) sh_k + 0.5) with dir the unit
 *  vector from the camera centre to the mean.
 *
 * Cameras are pinholes: x_cam = R x_world + t, +z forward, +y down, pixel
 * (i, j) centred at (i + 0.5, j + 0.5), u = fx x/z + cx, v = fy y/z + cy.  A
 * foveal crop (Sec. 3.3: a subfrustum through an adapted projection) is an
 * off-axis view with cx, cy shifted by the crop origin and tan_fov copied
 * from the full frame.
 */
#ifndef VRS_H
#define VRS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VRS_MAX_VIEWS 64
#define VRS_MAX_SCENES 16

typedef enum {
    VRS_OK = 0,
    VRS_ERR_INVALID = 1,     /* bad argument; on the device: an all-zero quaternion */
    VRS_ERR_CAPACITY = 2,    /* more tile instances than plan.max_instances */
    VRS_ERR_CUDA = 3,        /* a CUDA runtime call failed (launch, copy) */
    VRS_ERR_TIMEOUT = 4,     /* reserved: no call of this version waits on the device */
    VRS_ERR_NONFINITE = 5    /* a Gaussian parameter was NaN or Inf (that Gaussian is skipped) */
} vrs_status;

/* One scene of Gaussians: device pointers, structure of arrays, float32. */
typedef struct {
    const float *means;          /* [n][3] */
    const float *log_scales;     /* [n][3] */
    const float *quats;          /* [n][4] (w, x, y, z) */
    const float *opacity_logits; /* [n] */
    const float *sh;             /* [n][(sh_degree+1)^2][3]; IEEE half values when sh_half = 1 */
    int32_t n;                   /* number of Gaussians, >= 0 */
    int32_t sh_degree;           /* 0..3 */
    const float *baked;          /* nullable: [n][VRS_BAKED_FLOATS] written by vrs_bake; when set,
                                    vrs_preprocess reads the Gaussian's scales, rotation and opacity
                                    from it and ignores log_scales, quats and opacity_logits */
    int32_t sh_half;             /* 1: sh holds IEEE binary16 values (inference only) */
    int32_t reserved;
} vrs_scene;

/* Floats per Gaussian in a baked attribute array (see vrs_bake). */
#define VRS_BAKED_FLOATS 16

/* A pinhole view (host struct). */
typedef struct {
    float R[9];        /* world -> camera rotation, row-major */
    float t[3];        /* translation: x_cam = R x_world + t */
    float fx, fy;      /* focal lengths in pixels */
    float cx, cy;      /* principal point in pixels */
    float znear;       /* splats with z_cam <= znear are culled (0.2 in the reference setting) */
    float tan_fovx;    /* half-FOV tangents bounding the projection-Jacobian clamp at 1.3x; */
    float tan_fovy;    /*   0 means width/(2 fx) and height/(2 fy) */
    int32_t width, height;   /* >= 1 */
    int32_t scene;           /* index into the scene array */
} vrs_camera;

typedef struct {
    int32_t tile;          /* tile edge in pixels: 8, 16 or 32 (0 = 16) */
    int32_t persistent;    /* 0 = one CTA per tile; 1 = blend every tile of every view in
                              one persistent launch (a resident wave of CTAs pulling tiles),
                              heaviest tiles first; 2 = the same launch, tiles in tile order
                              (view by view, row by row); any value gives the same images */
    int32_t backward;      /* 1 = reserve the workspace that vrs_render_bwd needs */
    int32_t sort;          /* 0 = bucket by tile, then sort each tile's bucket (default);
                              1 = one global LSD radix sort of all keys;
                              2 = bucket by tile and sort only the tiles larger than one blend
                                  batch (tile^2 / 2 instances); vrs_render_fwd orders the others
                                  while staging them and writes their sorted lists back.  The
                                  same result; mode 2 needs resort = 0. */
    int64_t max_instances; /* capacity of the (tile, Gaussian) instance list; 0 = 4 x records + 65536 */
    int32_t count_pairs;   /* 1 = vrs_render_fwd also counts the Gaussian-pixel pairs it evaluated
                              and blended into the status block (a slower, measuring variant) */
    int32_t resort;        /* 0 = every pixel blends its tile's list in the list's depth order;
                              4, 8 or 16 = per-pixel depth order (the popping fix of Sec. 3.2)
                              through a sorting window of that many splats per pixel (see
                              vrs_render_fwd); forward only (backward must be 0) */
    int32_t half_out;      /* 1 = vrs_render_fwd writes rgb, depth and T_final as IEEE binary16
                              (half the output bytes; inference only, backward must be 0) */
    int32_t key_bits;      /* 0 = the minimal radix-sort key width (tile-id bits + 32); otherwise a
                              width of at least that, up to 64 (more passes, the same order) */
    int32_t tiles_per_pull;/* persistent blend: work-order items a CTA claims per atomic (1..64;
                              0 = 1); any value gives the same images */
    int32_t reserved;
} vrs_plan_opts;

/* Sizes and workspace layout, filled by vrs_plan_batch.  Treat as read-only. */
typedef struct {
    int32_t n_views, n_scenes;
    int32_t tile;              /* tile edge */
    int32_t key_bits;          /* significant bits of the sort key: tile-id bits + 32 */
    int32_t sort_passes;       /* 8-bit LSD passes */
    int32_t persistent, backward;
    int32_t sort_ctas;         /* CTAs of each radix pass */
    int64_t max_instances;
    int64_t n_records;         /* sum over views of the view's scene size */
    int64_t n_tiles;           /* sum over views of gw * gh */
    int64_t n_pixels;          /* sum over views of width * height */
    int64_t workspace_bytes;
    /* byte offsets inside the workspace */
    int64_t off_status;        /* device status block (see vrs_run_info) */
    int64_t off_records;       /* [n_records][3] float4 projected-splat records */
    int64_t off_keys[2];       /* [max_instances] uint64 ping-pong key buffers */
    int64_t off_vals[2];       /* [max_instances] uint32 ping-pong record-index buffers */
    int64_t off_hist;          /* radix scratch */
    int64_t off_ranges;        /* [n_tiles] uint2 {start, end} into the sorted list; {0, 0} if empty */
    int64_t off_ncontrib;      /* [n_pixels] uint32 last blended position + 1, written by
                                  vrs_render_fwd for plans made with backward = 1 (the
                                  reverse pass starts there); untouched otherwise */
    int64_t off_order;         /* [n_tiles] uint32 tile work order, heaviest first (persistent
                                  blend; reverse pass), then its bucket scratch.  Backward plans
                                  also keep, in the workspace's last
                                  ceil(n_tiles * tile^2 / 64 * 4 / 256) * 256 bytes, each 8x8
                                  block's largest last blended position (uint32 [n_tiles][tile^2/64]),
                                  written by vrs_render_fwd */
    int64_t off_grad2d;        /* [n_records][10] float 2D gradients (backward only) */
    int64_t off_tilesort;      /* uint32 [n_tiles] counts, [n_tiles] cursors, [n_tiles] list of
                                  tiles sorted by a whole CTA, [ceil(n_tiles / 1024)] block sums
                                  (bucketed sort) */
    int64_t off_pairs;         /* [n_records] 32-byte visible (Gaussian, view) pairs, the
                                  preprocess step's scratch; scene s's list starts at entry
                                  sum over s' < s of scene_n[s'] * (views of s') */
    int32_t sorted_buf;        /* which ping-pong buffer holds the sorted list */
    int32_t n_sms;
    int32_t sort_mode;         /* vrs_plan_opts.sort */
    int32_t count_pairs;       /* vrs_plan_opts.count_pairs; may be toggled between calls */
    /* per scene */
    int32_t scene_n[VRS_MAX_SCENES];
    int32_t scene_deg[VRS_MAX_SCENES];
    /* per view */
    int32_t view_scene[VRS_MAX_VIEWS];
    int32_t view_w[VRS_MAX_VIEWS], view_h[VRS_MAX_VIEWS];
    int32_t view_gw[VRS_MAX_VIEWS], view_gh[VRS_MAX_VIEWS];
    int64_t view_rec_base[VRS_MAX_VIEWS];   /* record index of (view v, Gaussian g) = view_rec_base[v] + g */
    int64_t view_tile_base[VRS_MAX_VIEWS];  /* global tile id = view_tile_base[v] + ty * gw + tx */
    int64_t view_pix_base[VRS_MAX_VIEWS];   /* view v's pixels start at element view_pix_base[v] */
    int32_t resort;            /* vrs_plan_opts.resort */
    int32_t half_out;          /* vrs_plan_opts.half_out */
    int32_t tiles_per_pull;    /* vrs_plan_opts.tiles_per_pull (>= 1) */
    int32_t reserved;
    int64_t off_raydepth;      /* resort plans: [n_records][3] float4, per record the terms of the
                                  per-pixel depth (see vrs_render_fwd); 0 otherwise */
    int64_t off_resort_flags;  /* resort plans: [n_pixels] uint8, 1 where the pixel's sorting
                                  window could not restore the per-pixel order; 0 otherwise */
} vrs_plan;

/* Device status block, copied to the host by vrs_query_status. */
typedef struct {
    uint32_t flags;            /* bit 0: all-zero quaternion, 1: non-finite parameter,
                                  2: capacity exceeded, 3: reserved */
    uint32_t reserved;
    uint64_t instances;        /* tile instances requested by the last vrs_preprocess
                                  (may exceed max_instances on overflow) */
    uint64_t pair_evals;       /* with plan.count_pairs: Gaussian-pixel pairs vrs_render_fwd
                                  evaluated by definition since the last vrs_preprocess (per
                                  pixel, its tile-list position where it stopped, else the list
                                  length) */
    uint64_t pair_blends;      /* of those, pairs that were blended */
    uint64_t block_evals;      /* with plan.count_pairs: (instance, 8x8 pixel block) pairs the
                                  blend kernel evaluated after its culling (each covers 64
                                  Gaussian-pixel evaluations) */
    uint64_t visible_pairs[VRS_MAX_SCENES]; /* (Gaussian, view) pairs of each scene that the last
                                  vrs_preprocess found visible (one 48-byte record each) */
    uint64_t resort_flagged;   /* resort plans: pixels whose sorting window overflowed in the last
                                  vrs_render_fwd (their flag is set in the resort flag plane) */
} vrs_run_info;

/* Sizes a batch of n_views views over n_scenes scenes and lays out the
 * workspace.  Reads scenes[*].n and .sh_degree and the views' sizes and scene
 * indices only; the pointers may be NULL here.  Re-plan when any size changes;
 * a plan stays valid for any poses and parameter values of the same sizes.
 * Errors: VRS_ERR_INVALID for n_views outside 1..VRS_MAX_VIEWS, n_scenes outside
 * 1..VRS_MAX_SCENES, a view with width or height < 1 or > 16384, a bad scene
 * index or SH degree, or a tile size other than 0/8/16/32. */
vrs_status vrs_plan_batch(const vrs_scene *scenes, int32_t n_scenes, const vrs_camera *views,
                          int32_t n_views, const vrs_plan_opts *opts, vrs_plan *plan);

/* Step 1, per Gaussian and per view of its scene (Sec. 3.1 projection).
 * Projects every Gaussian, writes its record (2D mean, Cholesky factors of the
 * conic, log2 opacity, colour, depth) and appends one (key, record index)
 * instance per touched tile:  key = (global tile id << 32) | float bits of z_cam.
 * Instances beyond plan.max_instances are dropped and flag VRS_ERR_CAPACITY.
 * scenes: n_scenes entries with device pointers, sizes as planned.
 * views: n_views host cameras, sizes and scene indices as planned.
 * Returns VRS_ERR_INVALID if sizes differ from the plan or a pointer is NULL
 * for a non-empty scene, VRS_ERR_CUDA on a launch failure. */
vrs_status vrs_preprocess(const vrs_plan *plan, const vrs_scene *scenes, const vrs_camera *views,
                          void *workspace, void *stream);

/* Step 2 (Sec. 1: tiling and sorting of all primitives).  Sorts the instances
 * into (tile, depth, record index) order and writes each tile's [start, end)
 * range.  plan.sort_mode 0 scans the per-tile counts taken at emission,
 * scatters the instances into tile buckets and sorts every bucket on its own
 * (a warp per tile of <= 256 instances, a CTA otherwise); mode 1 runs an 8-bit
 * LSD radix sort over plan.key_bits bits and orders runs of equal keys by
 * record index.  Both give the same list.
 * After it (after vrs_render_fwd for sort mode 2), the sorted keys and record
 * indices are at workspace + plan.off_keys[plan.sorted_buf] / off_vals[plan.sorted_buf]. */
vrs_status vrs_bin_sort(const vrs_plan *plan, void *workspace, void *stream);

/* Step 3 (Sec. 3.1 blending to screen; Sec. 3.2 Eq. 1).  For every pixel,
 * front to back over its tile's sorted list: alpha = min(0.99, o exp(power)),
 * skipped below 1/255; the pixel stops before a splat that would bring T under
 * 1e-4; otherwise C += rgb alpha T, D += z alpha T, T *= 1 - alpha.
 *
 * Per-pixel order (plans with resort = K; the popping fix of Sec. 3.2, which
 * sorts Gaussian contributions per pixel instead of per primitive).  Each pixel
 * orders the splats it blends by the depth of each 3D Gaussian's density
 * maximum along the pixel's ray, t* = r^T Sigma_c^-1 mu / r^T Sigma_c^-1 r with
 * r = ((x - cx)/fx, (y - cy)/fy, 1) (exact ties in list order), and Eq. 1 takes
 * d_i = t* at the pixel.  In these plans vrs_preprocess keys each instance by
 * t* at its tile's centre (moved into the splat's alpha >= 1/255 box where the
 * centre lies outside it) instead of by the mean's depth, so the tile list
 * arrives in an order close to every pixel's own; every pixel
 * keeps the K nearest splats it has not blended yet in a window in shared
 * memory and blends the nearest one whenever the window is full.  A splat that
 * arrives nearer than one the pixel has already blended (or than the one it
 * stopped at) breaks the per-pixel order: the pixel's byte in the resort flag
 * plane (workspace + plan.off_resort_flags) is set to 1 and
 * vrs_run_info.resort_flagged counts it.  Unflagged pixels are blended exactly
 * in per-pixel order.  The per-tile early exit is not taken in this mode, so
 * that every splat is checked.
 * Outputs (device, float32, written for every pixel of every view):
 *   rgb     [3][H][W] per view, view v at rgb + 3 * plan.view_pix_base[v]
 *   depth   [H][W] per view at depth + plan.view_pix_base[v]   (Eq. 1, not normalised)
 *   T_final [H][W] per view at T_final + plan.view_pix_base[v]
 * Colour is premultiplied with no background; composite with T_final.
 * For a plan made with half_out = 1 the three outputs are arrays of IEEE
 * binary16 values (pass their addresses as float*): the same results, each
 * rounded to half precision at the store.
 * For a plan made with backward = 1 it also writes each pixel's last blended
 * list position at workspace + plan.off_ncontrib, where vrs_render_bwd starts. */
vrs_status vrs_render_fwd(const vrs_plan *plan, void *workspace, float *rgb, float *depth,
                          float *T_final, void *stream);

/* Adjoint of steps 1-3 for the upstream gradients dL/drgb, dL/ddepth and
 * (nullable) dL/dT_final, laid out like the forward outputs; T_final is the
 * forward output.  Needs a plan made with opts.backward = 1 and the workspace
 * left by vrs_render_fwd for the same scenes and views.  Gradients are
 * ACCUMULATED (+=) into per-scene device arrays shaped like the parameters:
 * grads[s] holds g_means, g_log_scales, g_quats, g_opacity_logits, g_sh for
 * scene s in the fields of a vrs_scene (const is cast away; n and sh_degree
 * must match).  Each call starts from zeroed record gradients, so it may be
 * repeated after one forward; it also writes the call's record (2D)
 * gradients at workspace + plan.off_grad2d, [n_records][10] floats: dL/d of
 * (u, v, Sigma'_xx, Sigma'_xy, Sigma'_yy, opacity, r, g, b, depth).  When every
 * scene has one view only the rows of the visible (Gaussian, view) pairs are
 * cleared and written; the other rows keep whatever they held. */
vrs_status vrs_render_bwd(const vrs_plan *plan, void *workspace, const vrs_scene *scenes,
                          const vrs_camera *views, const float *T_final, const float *dL_drgb,
                          const float *dL_ddepth, const float *dL_dT, const vrs_scene *grads,
                          void *stream);

/* Baked attributes for inference (Sec. 4 "Inference": opacities, features and
 * covariances are baked into the point cloud to minimise runtime cost).  For
 * each Gaussian of `scene` (parameter form, device pointers) writes
 * VRS_BAKED_FLOATS floats to `baked` (device, [n][16], 16-byte aligned): the
 * scales exp(log_s) (3), the rotation of the normalised quaternion (9,
 * row-major), the opacity sigmoid(logit) and its log2 (2), a status word (1:
 * all-zero quaternion, 2: non-finite parameter; as float bits) and one unused
 * float.  Each value is computed by the same sequence of FP32 operations the
 * preprocess applies to the parameters, so a scene whose `baked` pointer is
 * set renders bit for bit the same images as its parameter form, with the
 * activations skipped.  The SH coefficients stay as they are (the colour
 * depends on the view).  Re-bake after the parameters change.  Stream
 * ordered; VRS_ERR_INVALID for a NULL pointer with n > 0. */
vrs_status vrs_bake(const vrs_scene *scene, float *baked, void *stream);

/* ------------------------------------------------------------------------ */
/* Training-loop pieces (Sec. 3.5, Sec. 4 "Training").
 *
 * vrs_image_loss: the Gaussian branch's loss L = (1 - lambda) L1 +
 * lambda (1 - SSIM) of `image` against `target` (Sec. 3.5: the first two terms
 * of the loss are those of 3DGS, with lambda = 0.2), and optionally dL/dimage,
 * the upstream colour gradient vrs_render_bwd takes.  L1 is the mean absolute
 * difference over the C H W values; SSIM is the mean over channels and pixels
 * of Wang et al.'s structural similarity with an 11 x 11 Gaussian window of
 * standard deviation 1.5, zero outside the image, C1 = 0.01^2, C2 = 0.03^2
 * (images in [0, 1]).  Where image and target are equal, the L1 term's
 * gradient is 0.
 *   image, target: device float32 [C][H][W] (one view's planes, e.g. a view of
 *     vrs_render_fwd's rgb output); dL_dimage: nullable device [C][H][W]
 *     (overwritten, not accumulated);
 *   loss_out: device float[3] = (L, L1, SSIM), reduced in FP64 in a fixed order;
 *   scratch: device, 16-byte aligned, at least vrs_image_loss_scratch bytes.
 * VRS_ERR_INVALID for sizes < 1, lambda outside [0, 1], NULL pointers or short
 * scratch. */
vrs_status vrs_image_loss_scratch(int32_t C, int32_t H, int32_t W, int64_t *bytes);
vrs_status vrs_image_loss(const float *image, const float *target, int32_t C, int32_t H, int32_t W,
                          float lambda, float *loss_out, float *dL_dimage, void *scratch,
                          int64_t scratch_bytes, void *stream);

/* vrs_opacity_decay: the opacity decay and pruning test of training (Sec. 4:
 * opacities are multiplied by 0.999 at intervals; Gaussians below 0.005 are
 * pruned).  In place on device `opacity_logits` [n]: o = factor sigmoid(logit),
 * logit <- ln(o / (1 - o)); keep[i] = 1 where o >= threshold (device uint8 [n]);
 * *n_kept (device uint32) = the number kept.  factor in (0, 1], threshold in
 * [0, 1). */
vrs_status vrs_opacity_decay(float *opacity_logits, int64_t n, float factor, float threshold,
                             uint8_t *keep, uint32_t *n_kept, void *stream);

/* Synchronises `stream`, copies the device status block to *info (nullable)
 * and returns the most severe device status: CAPACITY, then (reserved) TIMEOUT, then
 * NONFINITE, then INVALID, else VRS_OK. */
vrs_status vrs_query_status(const vrs_plan *plan, const void *workspace, vrs_run_info *info,
                            void *stream);

/* Clears the device status block (stream ordered). */
vrs_status vrs_reset_status(const vrs_plan *plan, void *workspace, void *stream);

/* Largest n that vrs_sort_pairs_noalloc accepts: its static scratch holds this many pairs. */
#define VRS_NOALLOC_MAX_PAIRS (1 << 20)

/* Stable LSD radix sort of n (key, value) pairs by the low key_bits bits of
 * each key (8 bits per pass; a last pass that ends inside a byte sorts only the
 * bits left, so bits above key_bits may hold anything), the same sort
 * vrs_bin_sort runs on the tile instances, for callers that must not allocate
 * device memory: real-time frame loops that must not risk the device-wide
 * synchronisation an allocation can cause, and plug-ins that live inside
 * another application's fixed memory budget.  The paper has no counterpart;
 * this is a service of the library.
 *
 * It allocates nothing.  Its scratch is a static device array of about
 * 13.6 MB (VRS_NOALLOC_MAX_PAIRS pairs of ping-pong storage plus digit counts)
 * that every GPU loading the library holds until the process exits.  The
 * first call on a device, with that device current, looks the array's device
 * address up and caches it; make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents (each call
 * resets what must start at zero), so calls that overlap on the GPU - on
 * different streams with no ordering between them - race and must not be
 * issued.
 *
 * keys_in, vals_in: device, n entries, read only.  keys_out, vals_out: device,
 * n entries, must not overlap the inputs.  Pairs with equal sort bits keep
 * their input order.  Returns VRS_ERR_CAPACITY for n > VRS_NOALLOC_MAX_PAIRS
 * (nothing is launched), VRS_ERR_INVALID for n < 0, key_bits outside 1..64,
 * a NULL pointer or an output equal to its input, VRS_ERR_CUDA on a launch or
 * set-up failure; n == 0 returns VRS_OK at once.  Stream ordered on `stream`
 * (a cudaStream_t as void*). */
vrs_status vrs_sort_pairs_noalloc(const uint64_t *keys_in, const uint32_t *vals_in,
                                  uint64_t *keys_out, uint32_t *vals_out, int64_t n,
                                  int32_t key_bits, void *stream);

/* ------------------------------------------------------------------------ */
/* Occlusion culling of the foveal neural points (Sec. 3.3).  After the
 * periphery is rendered, the fovea's subfrustum camera (the eye camera with its
 * principal point moved to a crop window, an "adapted projection matrix")
 * projects the neural point cloud; points outside the subfrustum are
 * discarded, and points hidden behind the Gaussians are culled against the
 * approximate depth buffer of Eq. 1 (Sec. 3.2) that vrs_render_fwd wrote.
 *
 * The paper does not spell the test out; the library's reading: Eq. 1 is
 * unnormalised, so a pixel's surface depth is depth / (1 - T_final), and a
 * pixel occludes only where its accumulated opacity 1 - T_final is at least
 * alpha_min.  A point at view depth z on that pixel is occluded when
 *   z > depth / (1 - T_final) * (1 + rel_margin) + abs_margin.
 * Every step is a correctly rounded FP32 operation in a fixed order: camera
 * space x = ((R0 px + R1 py) + R2 pz) + t0 (and y, z alike); outside when not
 * z > znear or x, y non-finite; u = fx (x (1/z)) + cx, v alike; inside when
 * 0 <= u < width and 0 <= v < height; map pixel (trunc(u) + x0, trunc(v) + y0). */
typedef struct {
    float alpha_min;           /* default 0.5 */
    float rel_margin;          /* default 0.02 */
    float abs_margin;          /* default 0.05 (scene units) */
    int32_t reserved;          /* 0 */
} vrs_cull_opts;

/* points: device, [n_points][3] float world positions (4-byte aligned; 16-byte
 * aligned bases load faster).  fovea: host, the subfrustum camera; its pixel
 * (i, j) is pixel (i + x0, j + y0) of the depth map.  depth, T_final: device,
 * [map_h][map_w] float (one view of vrs_render_fwd's outputs).  opts: host,
 * NULL for the defaults.  Outputs, all device and written in full:
 *   mask[n_points]   0 outside the subfrustum, 1 occluded, 2 kept;
 *   kept[n_points]   (nullable) indices of the kept points, first *n_kept
 *                    entries, in no particular order;
 *   n_kept           one uint64, the number of kept points (set, not added).
 * Returns VRS_ERR_INVALID for n_points < 0 or >= 2^32, a NULL required pointer,
 * a camera or map size below 1, or a reserved field that is not 0;
 * VRS_ERR_CUDA on a launch failure.  n_points == 0 writes *n_kept = 0.  No
 * allocation, no synchronisation; stream ordered on `stream` and capturable. */
vrs_status vrs_cull_points(const float *points, int64_t n_points, const vrs_camera *fovea,
                           int32_t x0, int32_t y0, const float *depth, const float *T_final,
                           int32_t map_w, int32_t map_h, const vrs_cull_opts *opts, uint8_t *mask,
                           uint32_t *kept, uint64_t *n_kept, void *stream);

/* ------------------------------------------------------------------------ */
/* Combination of the peripheral image P and the foveal image F (Sec. 3.4).
 * Over the foveal crop window [x0, x0 + w) x [y0, y0 + h) of P, for crop pixel
 * (i, j) at P-frame position (u, v) = (x0 + i + 0.5, y0 + j + 0.5):
 *   r_norm = clamp(|(u, v) - (ex, ey)| / d_f, 0, 1),  f_p = (r_norm - m) / (1 - m),
 *   f_e    = magnitude of the Sobel gradient of F's channel mean (3x3 kernels
 *            weighted 1-2-1, divided by 8; the crop's border replicated),
 *   c      = 1 - S2(clamp(f_p + gamma f_e, 0, 1)),  S2(x) = 6x^5 - 15x^4 + 10x^3,
 *   out    = (1 - c) p + c f per channel.
 * The library's readings where the paper is silent: the Sobel filter acts on the
 * mean of F's three channels, is normalised so that a unit-slope ramp gives 1,
 * and replicates the border; S2's argument is clamped to [0, 1].  FP32. */
typedef struct {
    float d_f;                 /* fovea radius in pixels, default 256 */
    float m;                   /* start of the blending interval, default 0.75 */
    float gamma;               /* edge weight, default 0.2 */
    int32_t reserved;          /* 0 */
} vrs_combine_opts;

/* P: device [3][ph][pw] float (one view of vrs_render_fwd's RGB).  F: device
 * [3][h][w] float, the foveal image of the crop.  (ex, ey): the fixation in P's
 * pixel frame.  opts: host, NULL for the defaults.  out: device [3][h][w], must
 * not overlap F.  c_out: device [h][w] (nullable), the factor c.  Returns
 * VRS_ERR_INVALID for NULL required pointers, sizes below 1, a window not
 * inside P, out overlapping F, d_f <= 0, m >= 1 or a reserved field that is
 * not 0; VRS_ERR_CUDA on a launch failure.  No allocation; stream ordered. */
vrs_status vrs_foveal_combine(const float *P, int32_t pw, int32_t ph, const float *F, int32_t w, int32_t h,
                              int32_t x0, int32_t y0, float ex, float ey, const vrs_combine_opts *opts,
                              float *out, float *c_out, void *stream);

/* Reverse pass of vrs_foveal_combine, for the end-to-end training of Sec. 3.5.
 * With out = p + c (f - p) and c = 1 - S2(x), x = clamp(f_p + gamma f_e, 0, 1):
 * dL/dp = (1 - c) g and dL/df = c g directly, and dL/dc = sum_ch g (f - p) flows
 * through dc/dx = -S2'(x) (0 where x is clamped), gamma, f_e = |grad| (0 where
 * f_e = 0), the Sobel taps (border replicated) and the channel mean into F.
 * dL_dout: device [3][h][w].  dL_dP: device [3][ph][pw], accumulated (+=) on
 * the window.  dL_dF: device [3][h][w], accumulated (+=).  scratch: device
 * [h][w] float, overwritten.  Other arguments and errors as vrs_foveal_combine;
 * also VRS_ERR_INVALID for a NULL gradient or scratch pointer.  The edge
 * path's taps are summed with atomics, so its last bits may vary from run to
 * run.  No allocation; stream ordered. */
vrs_status vrs_foveal_combine_bwd(const float *P, int32_t pw, int32_t ph, const float *F, int32_t w,
                                  int32_t h, int32_t x0, int32_t y0, float ex, float ey,
                                  const vrs_combine_opts *opts, const float *dL_dout, float *dL_dP,
                                  float *dL_dF, float *scratch, void *stream);

/* A static, human-readable name of a status. */
const char *vrs_status_string(vrs_status status);

#ifdef __cplusplus
}
#endif

#endif /* VRS_H */
