/*
 * cicero.h - C ABI of the GB300 (sm_103a) voxel-grid NeRF renderer with sparse radiance
 * warping (SpaRW), after "Cicero: Addressing Algorithmic and Architectural Bottlenecks in
 * Neural Rendering by Radiance Warping and Memory Optimizations" (arXiv 2404.11852).
 *
 * Conventions shared by every call
 *   - Every array pointer is a DEVICE pointer owned by the caller, unless the parameter says
 *     otherwise.  Descriptor structs (cicero_grid, cicero_mlp, cicero_camera, cicero_sampling,
 *     cicero_options) are read on the host during the call and may be freed afterwards.
 *   - Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream).  The
 *     host validates the arguments and returns a status before anything is launched; no call
 *     synchronises the stream or allocates device memory.
 *   - Scratch memory is the caller's `workspace` of `ws_bytes` bytes (size it with the matching
 *     cicero_*_workspace_size query; 256-byte aligned).  A workspace must not be shared by calls
 *     that may run concurrently.  Errors found by a kernel (an internal invariant broken, a
 *     bounded wait that ran out) are recorded in the workspace and reported by
 *     cicero_workspace_status.
 *   - Pixel p = j * width + i is the pixel of column i and row j; its centre is (i + 0.5, j + 0.5).
 *   - Camera poses c2w are row-major 3x4 camera-to-world matrices with OpenCV axes (x right,
 *     y down, z forward); f is the focal length in pixels and (cx, cy) the principal point, the
 *     intrinsics of Eq. 1 and Eq. 3.
 *   - On error the call returns a non-zero status and cicero_last_error() describes it.
 */
#ifndef CICERO_H
#define CICERO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CICERO_OK = 0,
    CICERO_ERR_INVALID_ARG = 1,        /* a NULL pointer, a bad size or an inconsistent descriptor */
    CICERO_ERR_UNSUPPORTED = 2,        /* a shape or option this build does not implement */
    CICERO_ERR_ALIGNMENT = 3,          /* a pointer or stride breaks the TMA 16-byte rules */
    CICERO_ERR_WORKSPACE_TOO_SMALL = 4,
    CICERO_ERR_CUDA = 5,               /* a CUDA runtime call failed (message in cicero_last_error) */
    CICERO_ERR_TIMEOUT = 6,            /* a kernel's bounded wait ran out (reported by cicero_workspace_status) */
    CICERO_ERR_INTERNAL = 7            /* a kernel found a broken invariant (reported by cicero_workspace_status) */
} cicero_status;

typedef enum { CICERO_F32 = 0, CICERO_F16 = 1 } cicero_dtype;

/* Arithmetic of Feature Computation (the MLP):
 * FP32: FP32 FFMA on CUDA cores.  BF16: tcgen05 tensor-core MMAs with BF16 operands (weights and
 * activations rounded to BF16) and FP32 accumulation in tensor memory.  FP32_SPLIT: FP32-class
 * accuracy on the tensor cores: every FP32 operand v of layers 1 and 2 is split into
 * hi = bf16(v) and lo = bf16(v - hi), each product taken as hi.hi + hi.lo + lo.hi (the method of
 * Henry, Tang and Heinecke, ARITH 2019) with FP32 accumulation in tensor memory, so a product keeps
 * ~16 of FP32's 24 significand bits; biases, layer 3 and the sigmoid in FP32.  It needs C <= 16
 * and is taken by cicero_render and cicero_render_rays only. */
typedef enum { CICERO_MLP_FP32 = 0, CICERO_MLP_BF16 = 1, CICERO_MLP_FP32_SPLIT = 2 } cicero_precision;

/* Dense voxel grid (Sec. II-B: a feature vector is stored at every vertex of the grid).
 * Vertices sit on the corners of the box [aabb_min, aabb_max]; n[a] vertices along axis a.
 *   density  [n2][n1][n0]       raw density, sigma = softplus(raw + act_shift)
 *   features [n2][n1][n0][C]    feature vectors
 *   occ      [R][R][R] uint8 or NULL: occupancy of R^3 equal cells over the box; samples in
 *            empty cells are skipped (alpha = 0, no gathering, no MLP).
 * Requirements: n[a] >= 2, 1 <= C <= 21 (the MLP input is C + 3 + 6 n_freq <= 48 for BF16),
 * features 16-byte aligned and n0 * C * sizeof(element) a multiple of 16 (TMA staging). */
typedef struct {
    int n[3];
    int C;
    float aabb_min[3], aabb_max[3];
    float act_shift;
    cicero_dtype dtype;
    const void *density;
    const void *features;
    const uint8_t *occ;
    int occ_res;
} cicero_grid;

/* Feature Computation MLP (Sec. II-B, a small MLP of unstated shape), FP32 weights, row-major [out][in]:
 *   x  = [features (C), d (3), sin(2^k d), cos(2^k d) for k = 0..n_freq-1 (6 n_freq)]
 *   h1 = relu(w1 x + b1)  (hidden), h2 = relu(w2 h1 + b2)  (hidden), c = sigmoid(w3 h2 + b3)  (3)
 * where d is the unit ray direction and each sin/cos block is (x, y, z) of sin then of cos.
 * This build supports hidden == 128 and in_dim == C + 3 + 6 n_freq <= 48. */
typedef struct {
    int in_dim, hidden, n_freq;
    const float *w1, *b1, *w2, *b2, *w3, *b3;
} cicero_mlp;

/* Sample placement and compositing (Sec. II-B Indexing and accumulation).
 *   step == 0: n_samples slots at near + (k + 1/2)(far - near)/n_samples, delta = (far-near)/n_samples
 *   step  > 0: slots at t_in + (k + 1/2) step, k < n_samples, while before the box exit t_out,
 *              where [t_in, t_out] is the ray's span inside the box clipped to [near, far]
 *   Before slot k the march stops if the transmittance T_k < t_stop (t_stop = 0: never).
 *   rgb = sum_k T_k alpha_k c_k + T_end bg,  acc = sum_k T_k alpha_k,
 *   depth = sum_k T_k alpha_k t_k / acc (ray distance), or +inf when acc < void_acc. */
typedef struct {
    float near_t, far_t;
    int n_samples;
    float step;
    float t_stop;
    float bg[3];
    float void_acc;
} cicero_sampling;

typedef struct {
    int width, height;
    float f, cx, cy;
    float c2w[12];
} cicero_camera;

/* Options of the rendering calls (NULL = defaults: FP32 MLP, bricks of 8^3 voxels, full capacity).
 * max_records caps the per-sample records the workspace holds (0 = n_rays * n_samples, which can
 * never overflow; 52 bytes per record).  Each ray reserves records for its active slots, the slots
 * inside the grid box and in an occupied cell, found exactly before its march (for slots past the
 * 256th, every slot before the box exit); the samples it composites are a subset of those (early
 * stop ends the rest).  If the reservations exceed max_records the rays that do not fit composite
 * nothing and cicero_workspace_status returns CICERO_ERR_WORKSPACE_TOO_SMALL. */
typedef struct {
    cicero_precision precision;
    int brick;          /* voxels per brick edge ("MVoxel", Sec. IV-A): 4, 8 or 16; 0 = 8 */
    long long max_records;
    int mlp_groups;     /* BF16 tensor-core MLP: 128-sample tiles in flight per SM (each tile runs its
                           own gather -> layer 1 -> 2 -> 3 chain), 1..4; 0 = as many as fit */
} cicero_options;

/* ---------------------------------------------------------------------------------------------
 * Rendering (Sec. II-B, run memory-centric as in Sec. IV-A).
 *
 * Every pixel of `cam` is rendered.  The samples that reach Feature Gathering are grouped by
 * brick (the Ray Index Table of Sec. IV-A, built by a counting sort on the brick id); each
 * brick is staged once into shared memory by TMA and all of its samples are interpolated from
 * there and passed through the MLP; per-ray colours are then composited in slot order.
 * Outputs (device): rgb [H*W][3], depth [H*W] (+inf = void), acc [H*W] or NULL,
 * n_steps [H*W] or NULL (slots visited before the early stop).
 */
cicero_status cicero_render(const cicero_grid *grid, const cicero_mlp *mlp, const cicero_camera *cam,
                            const cicero_sampling *sampling, const cicero_options *opt,
                            float *rgb, float *depth, float *acc, int32_t *n_steps,
                            void *workspace, size_t ws_bytes, void *stream);

/* Same as cicero_render for n_rays explicit rays: ray_o, ray_d [n_rays][3] (device, unit d). */
cicero_status cicero_render_rays(const cicero_grid *grid, const cicero_mlp *mlp,
                                 const float *ray_o, const float *ray_d, int n_rays,
                                 const cicero_sampling *sampling, const cicero_options *opt,
                                 float *rgb, float *depth, float *acc, int32_t *n_steps,
                                 void *workspace, size_t ws_bytes, void *stream);

/* Sparse NeRF rendering of the disoccluded pixels, Gamma_sp of Eq. 4, combined in place (the
 * circled-asterisk of Eq. 4): the pixels hole_idx[0 .. *n_holes) of `cam` are rendered and
 * written into rgb_inout [H*W][3] and depth_inout [H*W] (may be NULL); other pixels are left
 * untouched.  n_holes is a DEVICE scalar (as written by cicero_warp), so no host read-back is
 * needed; max_holes bounds it and sizes the workspace. */
cicero_status cicero_render_holes(const cicero_grid *grid, const cicero_mlp *mlp, const cicero_camera *cam,
                                  const cicero_sampling *sampling, const cicero_options *opt,
                                  const int32_t *hole_idx, const int32_t *n_holes, int max_holes,
                                  float *rgb_inout, float *depth_inout,
                                  void *workspace, size_t ws_bytes, void *stream);

/* Gamma_sp of Eq. 4 for several target frames in one pass: view v renders the pixels
 * hole_idx[v][0 .. n_holes[v]) of cams[v] into rgb_inout[v] / depth_inout[v].
 *   cams [n_views] (host), hole_idx / rgb_inout / depth_inout: host arrays of n_views device
 *   pointers (depth_inout, or any entry of it, may be NULL), n_holes: DEVICE array [n_views]
 *   (for example the n_holes scalars of n_views cicero_warp calls laid out contiguously),
 *   max_rays >= sum of n_holes bounds the rays and sizes the workspace (query it with
 *   n_rays = max_rays).  1 <= n_views <= 32.  The rays of all views share one march, one Ray
 *   Index Table and one tensor-core pass, so each brick is staged once for every view. */
cicero_status cicero_render_holes_batch(const cicero_grid *grid, const cicero_mlp *mlp, const cicero_camera *cams,
                                        int n_views, const cicero_sampling *sampling, const cicero_options *opt,
                                        const int32_t *const *hole_idx, const int32_t *n_holes, int max_rays,
                                        float *const *rgb_inout, float *const *depth_inout,
                                        void *workspace, size_t ws_bytes, void *stream);

/* Workspace bytes for cicero_render / cicero_render_rays / cicero_render_holes with n_rays rays
 * (H*W, n_rays or max_holes).  Host query, allocates nothing. */
size_t cicero_render_workspace_size(const cicero_grid *grid, int n_rays, const cicero_sampling *sampling,
                                    const cicero_options *opt);

/* Brick-size autotuner: renders `cam` once untimed and once timed with bricks of 4, 8 and 16
 * voxels (each size that fits `ws_bytes` and the kernels' shared memory) and returns the fastest in
 * *best_brick; ms[3] (may be NULL) receives the timed milliseconds (-1 = not tried).  rgb and depth
 * (device, [H*W][3] and [H*W]) are scratch.  Size the workspace with brick 4, the largest.
 * Synchronises `stream` (it times with CUDA events), unlike every other call. */
cicero_status cicero_autotune_brick(const cicero_grid *grid, const cicero_mlp *mlp, const cicero_camera *cam,
                                    const cicero_sampling *sampling, cicero_precision precision,
                                    float *rgb, float *depth, void *workspace, size_t ws_bytes, void *stream,
                                    int *best_brick, float *ms);

/* ---------------------------------------------------------------------------------------------
 * Batched rendering: many scene/view pairs of uneven size through one set of launches.
 *
 * The paper renders one frame at a time; it has no counterpart for this.  Each job is a full
 * cicero_render of its own grid, MLP, camera and sampling: the rays of all jobs share one march,
 * one Ray Index Table (brick ids numbered job after job) and one persistent tensor-core pass
 * whose CTAs each take a contiguous range of the brick-ordered work, loading a job's MLP weights
 * only where the range crosses into a job with other weights.  The BF16 tensor-core MLP only
 * (opt->precision must be CICERO_MLP_BF16); all jobs must share the grid dtype, the channel
 * count and the view encoding; at most 2048 jobs.  opt->brick applies to every job;
 * opt->max_records caps the records of the whole batch (0 = the sum of H*W*n_samples, which
 * must stay below 2^32).
 *
 * cicero_batch_create validates the jobs, encodes each grid's TMA descriptor and uploads the job
 * table into the workspace (a synchronous host-to-device copy; the host arrays, including the
 * grid/mlp/camera/sampling structs, may be freed afterwards, but the device buffers they point
 * to must outlive the handle).  cicero_batch_launch then issues kernels only (no host-device
 * copy, allocation or synchronisation), so it can be captured into a CUDA graph and replayed;
 * every launch renders every job again into its rgb [H*W][3] and depth [H*W] (or NULL) device
 * buffers.  Errors inside the kernels are read with cicero_workspace_status on
 * (char *)workspace + cicero_batch_table_bytes(n_jobs).  The handle is host memory owned by the
 * caller: cicero_batch_destroy frees it.  A workspace serves one handle at a time.
 */
typedef struct {
    const cicero_grid *grid;          /* the job's scene */
    const cicero_mlp *mlp;            /* its colour MLP */
    const cicero_camera *cam;         /* its view; every pixel is rendered */
    const cicero_sampling *sampling;
    float *rgb;                       /* device [H*W][3] */
    float *depth;                     /* device [H*W] (+inf = void) or NULL */
} cicero_job;

typedef struct cicero_batch cicero_batch;

size_t cicero_batch_workspace_size(const cicero_job *jobs, int n_jobs, const cicero_options *opt);
size_t cicero_batch_table_bytes(int n_jobs);
cicero_status cicero_batch_create(const cicero_job *jobs, int n_jobs, const cicero_options *opt,
                                  void *workspace, size_t ws_bytes, cicero_batch **out);
cicero_status cicero_batch_launch(const cicero_batch *batch, void *stream);
cicero_status cicero_batch_destroy(cicero_batch *batch);

/* Autotuner of a batch: creates the batch and launches it once untimed and once timed for every
 * brick of 4, 8 and 16 voxels and every count of MLP tiles in flight per SM (mlp_groups 1..4) that
 * fit ws_bytes and the kernels' shared memory, and writes the fastest into *best (a copy of opt with
 * brick and mlp_groups set).  ms [3][4] (may be NULL) receives the timed milliseconds, row = brick
 * 4 / 8 / 16, column = mlp_groups 1..4 (-1 = not tried).  Size the workspace with brick 4.
 * Synchronises `stream`; leaves no handle behind (create one with *best). */
cicero_status cicero_batch_autotune(const cicero_job *jobs, int n_jobs, const cicero_options *opt,
                                    void *workspace, size_t ws_bytes, void *stream, cicero_options *best,
                                    float *ms);

/* ---------------------------------------------------------------------------------------------
 * Hash-encoded rendering (the hierarchical-encoding workload of Sec. IV-A "Accommodating
 * Hierarchical Data Encodings"; Instant-NGP-like).  Density, occupancy and the box come from
 * `grid` (its `features` and `C` are ignored and may be NULL / 0); the colour features come from a
 * multiresolution hash encoding: level l divides the box into res[l] cells per axis; its
 * (res+1)^3 vertices are stored densely at x + (res+1)(y + (res+1) z) when they fit the level's
 * table of T = 2^log2_size entries, otherwise at the spatial hash (x * 1) xor (y * 2654435761) xor
 * (z * 805459861) mod T of 32-bit unsigned integers; each level's 2 features are the trilinear
 * interpolation of its 8 corner entries, and the levels are concatenated as the MLP's features
 * (mlp->in_dim = 2 levels + 3 + 6 n_freq <= 48).  Every level is gathered directly from the table
 * in global memory (the paper's non-streaming fallback; an Instant-NGP-sized table set fits in
 * GB300's L2), in the brick order of the density grid.  BF16 MLP only.  Workspace:
 * cicero_render_hash_workspace_size (rays = H*W). */
typedef struct {
    int levels;            /* 1..16 */
    int features;          /* per level: 2 */
    int log2_size;         /* entries per level T = 2^log2_size, 1..24 */
    int res[16];           /* cells per axis of each level */
    cicero_dtype dtype;    /* of the table: F16 or F32 */
    const void *table;     /* [levels][T][features], device */
} cicero_hash_grid;

cicero_status cicero_render_hash(const cicero_grid *grid, const cicero_hash_grid *hash, const cicero_mlp *mlp,
                                 const cicero_camera *cam, const cicero_sampling *sampling, const cicero_options *opt,
                                 float *rgb, float *depth, void *workspace, size_t ws_bytes, void *stream);
size_t cicero_render_hash_workspace_size(const cicero_grid *grid, const cicero_hash_grid *hash, int n_rays,
                                         const cicero_sampling *sampling, const cicero_options *opt);

/* ---------------------------------------------------------------------------------------------
 * Bilinear resampling, for the DS-2 comparator of the evaluation (render the frame at half
 * resolution, then upsample it to the original resolution by bilinear interpolation).  Pixel
 * centres align: output pixel (i, j) samples src at ((i + 1/2) w / W - 1/2, (j + 1/2) h / H - 1/2)
 * from the nearest two source pixel centres per axis, clamped to the image (a half-resolution
 * render is the frame rendered with f, cx, cy halved).  src [h][w][channels], dst [H][W][channels],
 * device FP32; 1 <= channels <= 16. */
cicero_status cicero_upsample_bilinear(const float *src, int w, int h, int channels, float *dst, int W, int H,
                                       void *stream);

/* ---------------------------------------------------------------------------------------------
 * Reference pose by extrapolation (Sec. III-C, Eq. 5-6): from the two latest camera poses `prev`
 * and `cur`, one frame interval apart, the velocity v = (cur - prev) / dt (Eq. 5) is applied for
 * t_r = lead * dt (Eq. 6, where the paper takes lead = N / 2 for N targets per reference):
 * position = p_cur + lead (p_cur - p_prev).  The paper states the velocity of the position only;
 * the orientation follows the same rule with the angular velocity: the rotation taken from prev to
 * cur is applied `lead` more times (shortest arc; FP64, rounded once to FP32).  Intrinsics are
 * copied from `cur`.  Host only. */
cicero_status cicero_extrapolate_pose(const cicero_camera *prev, const cicero_camera *cur, float lead,
                                      cicero_camera *out);

/* ---------------------------------------------------------------------------------------------
 * Reference poses of a trajectory (Sec. III-C, Eq. 5-6), for the overlapped pipeline below.
 * Frames are taken in windows of `window` targets; window w is warped from reference w.
 * Reference 0 is frame 0.  Reference w >= 1 is rendered while window w - 1 runs, so it can only
 * use the poses known when window w - 1 starts: it is extrapolated (cicero_extrapolate_pose) from
 * frames s - 1 and s, where s = max(1, (w - 1) window) is the first frame of window w - 1 (frame 1
 * for the first window, which needs two poses), with
 *   CICERO_LEAD_CENTRED: lead = w window + window / 2 - s, which carries the pose to the centre
 *                        of the window the reference serves (the paper's intent: the reference
 *                        sits in the middle of its targets);
 *   CICERO_LEAD_PAPER:   lead = window / 2, Eq. 6 read literally (t_r = N/2 frame intervals
 *                        after the latest pose).
 * targets [n_frames] and refs [ceil(n_frames / window)] are host arrays; every reference has the
 * intrinsics of its latest pose.  Host only, allocates nothing. */
typedef enum { CICERO_LEAD_CENTRED = 0, CICERO_LEAD_PAPER = 1 } cicero_lead;

cicero_status cicero_reference_poses(const cicero_camera *targets, int n_frames, int window, cicero_lead lead,
                                     cicero_camera *refs);

/* ---------------------------------------------------------------------------------------------
 * SpaRW over a trajectory with reference rendering overlapped (Sec. III-C, "Reference Frame
 * Rendering"): frames are taken in windows of `window` targets; window w is warped from
 * reference frame w (cicero_warp_batch) and its holes rendered (cicero_render_holes_batch),
 * while reference w + 1 is rendered on `stream_ref`.  The reference poses are derived from the
 * trajectory by cicero_reference_poses with the given lead.  Void holes are not tested
 * separately: their march in the hole render finds no occupied slot and writes the background
 * with depth +inf, the same frames as with the void depth test of cicero_warp_batch.  With
 * stream_ref == stream_tgt the same work runs serialised (same results).  Every frame, reference
 * or target, has the size and intrinsics of `cam`.
 *
 * The workspace holds two reference frames and their render workspaces (opt applies to them),
 * scratch for one window's hole masks and lists, and the hole-batch workspace of `hole_records`
 * records (opt's max_records for the hole batch).  The handle is host memory owned by the
 * caller; one run at a time per pipeline (the previous run's work is waited for on the streams,
 * not on the host).  targets [n_frames] is a host array; rgb / depth are host arrays of n_frames
 * device pointers ([H*W][3] / [H*W]; depth may be NULL).
 * cicero_pipeline_status reads the error bits of the kernels (synchronises `stream`). */
typedef struct cicero_pipeline cicero_pipeline;

size_t cicero_pipeline_workspace_size(const cicero_grid *grid, const cicero_camera *cam,
                                      const cicero_sampling *sampling, const cicero_options *opt, int window,
                                      long long hole_records);
cicero_status cicero_pipeline_create(const cicero_grid *grid, const cicero_mlp *mlp, const cicero_camera *cam,
                                     const cicero_sampling *sampling, const cicero_options *opt, int window,
                                     long long hole_records, float max_angle_deg, void *workspace, size_t ws_bytes,
                                     cicero_pipeline **out);
cicero_status cicero_pipeline_run(cicero_pipeline *pipeline, const cicero_camera *targets, int n_frames,
                                  cicero_lead lead, float *const *rgb, float *const *depth,
                                  void *stream_tgt, void *stream_ref);
cicero_status cicero_pipeline_status(const cicero_pipeline *pipeline, void *stream);
cicero_status cicero_pipeline_destroy(cicero_pipeline *pipeline);

/* ---------------------------------------------------------------------------------------------
 * SpaRW target frame, steps 1-3 (Eq. 1 point cloud, Eq. 2 transform, Eq. 3 re-projection) plus
 * the depth test, the void depth test and hole listing of step 4 (Sec. III-B).
 *
 *   ref_rgb [Hr*Wr][3], ref_depth [Hr*Wr] (ray distance; +inf = void) of the reference camera.
 *   Eq. 1: Z = D / |((u-cx)/f, (v-cy)/f, 1)|, P = Z ((u-cx)/f, (v-cy)/f, 1).
 *   Eq. 2: P' = R P + t with [R|t] = inverse(c2w_tgt) c2w_ref, formed in FP64 on the host and
 *          rounded once to FP32.
 *   Eq. 3: u' = f' X'/Z' + cx', v' = f' Y'/Z' + cy'; the point lands on pixel (floor u', floor v').
 *   Points with Z' <= 1e-6 or off the target image are dropped; void reference pixels are points
 *   at infinity (rotated direction, depth key +inf).  Depth test: a 64-bit atomicMin of
 *   (float bits of Z') << 32 | reference pixel index, so the nearest point wins and ties go to
 *   the lower index.  max_angle_deg < 180 enables the warp-angle heuristic phi (Sec. III-C): a
 *   point is kept only when the angle between its reference and target rays is below it.
 * Outputs: warped_rgb [Ht*Wt][3]; warped_depth [Ht*Wt] or NULL (distance |P'| of the winning
 * point, +inf for void, 0 for holes); hole_mask [Ht*Wt] (0 warped, 1 hole to render, 2 void);
 * hole_idx [Ht*Wt] (holes with mask 1 in ascending pixel order; also used as scratch during the call)
 * and *n_holes (device scalar).
 * void_grid (may be NULL) enables the void depth test: a hole whose target ray has no sample
 * inside the grid box (and in an occupied cell) gets void_sampling->bg, depth +inf, mask 2.
 * Decisions are taken in FP32 with round-to-nearest and no contraction, so the mask and the
 * list are reproducible bit for bit. */
cicero_status cicero_warp(const float *ref_rgb, const float *ref_depth,
                          const cicero_camera *ref_cam, const cicero_camera *tgt_cam,
                          float max_angle_deg, const cicero_grid *void_grid,
                          const cicero_sampling *void_sampling,
                          float *warped_rgb, float *warped_depth, uint8_t *hole_mask,
                          int32_t *hole_idx, int32_t *n_holes,
                          void *workspace, size_t ws_bytes, void *stream);

size_t cicero_warp_workspace_size(const cicero_camera *tgt_cam);

/* cicero_warp from one reference into n_views targets in one set of launches (the targets of a
 * SpaRW window, Sec. III-C).  tgt_cams [n_views] (host); warped_rgb, warped_depth (may be NULL, or
 * have NULL entries), hole_mask, hole_idx: host arrays of n_views device pointers; n_holes: DEVICE
 * array [n_views].  1 <= n_views <= 32.  Results are identical to n_views cicero_warp calls. */
cicero_status cicero_warp_batch(const float *ref_rgb, const float *ref_depth, const cicero_camera *ref_cam,
                                const cicero_camera *tgt_cams, int n_views, float max_angle_deg,
                                const cicero_grid *void_grid, const cicero_sampling *void_sampling,
                                float *const *warped_rgb, float *const *warped_depth, uint8_t *const *hole_mask,
                                int32_t *const *hole_idx, int32_t *n_holes,
                                void *workspace, size_t ws_bytes, void *stream);

size_t cicero_warp_batch_workspace_size(const cicero_camera *tgt_cams, int n_views);

/* cicero_warp without a workspace, for callers that cannot allocate device memory: real-time
 * loops that must not enter an allocator, host programs that link this library without a device
 * allocator of their own, plugins whose host framework owns all device memory.  The paper has no
 * counterpart: this is a packaging variant of the warp above, with the same arguments and outputs
 * minus the workspace.
 *   - Scratch (the depth buffer and scan sums, ~8 MiB) is a static array in the library's device
 *     image, present on every device that loads the library until the process exits.  The target
 *     image may have at most 1048576 pixels (width * height); larger targets return
 *     CICERO_ERR_UNSUPPORTED.  The call allocates and frees nothing.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *     that device current, and caches it for the life of the process.  After cudaDeviceReset on a
 *     device the cached address is stale: do not call this entry point on that device again.
 *   - Every call shares the one array: calls that may overlap on the GPU (different streams, or
 *     different host threads on one device) race and must be serialised by the caller.  The call
 *     clears what must start empty (the depth buffer) itself. */
cicero_status cicero_warp_noalloc(const float *ref_rgb, const float *ref_depth,
                                  const cicero_camera *ref_cam, const cicero_camera *tgt_cam,
                                  float max_angle_deg, const cicero_grid *void_grid,
                                  const cicero_sampling *void_sampling,
                                  float *warped_rgb, float *warped_depth, uint8_t *hole_mask,
                                  int32_t *hole_idx, int32_t *n_holes, void *stream);

/* ---------------------------------------------------------------------------------------------
 * Backward of cicero_render_rays with the FP32 MLP (not in the paper, whose models are trained
 * offline; the gradient of its rendering function).  Given d_rgb = dL/drgb [n_rays][3], the
 * gradient is ACCUMULATED into d_density [n2][n1][n0], d_features [n2][n1][n0][C] (both FP32;
 * zero them first) and, when d_mlp is not NULL, into the MLP gradient laid out as
 * [w1 [hidden][in_dim], b1 [hidden], w2 [hidden][hidden], b2 [hidden], w3 [3][hidden], b3 [3]]
 * (FP32, the layout of cicero_mlp's tensors back to back).  Gradients are summed with atomic adds,
 * so the order of the sums, and the last bits of the result, vary between calls.  Each ray's
 * forward pass is recomputed (nothing is stored by the forward).  Up to 16 feature channels the
 * recompute and the grid gradients run the MLP on the tensor cores with split-BF16 operands
 * (hi + lo, three products, FP32 accumulation), and the samples with a ReLU pre-activation within
 * an estimate of that precision's error of zero (~10 times the typical error) are recomputed in
 * FP32, so a mask differs from the FP32 MLP's only where the split products err by more than
 * that; wider grids recompute and differentiate in FP32 on the CUDA cores.  Early stop is a fixed
 * truncation.  For composited sample k:
 *   dL/dc_k = w_k g;  dL/dsigma_k = delta (T_{k+1} g.c_k - g.R_k), R_k = sum_{j>k} w_j c_j + T_end bg;
 *   dL/draw_k = dL/dsigma_k sigmoid(raw_k + shift); MLP chain rule; trilinear adjoint. */
cicero_status cicero_render_backward(const cicero_grid *grid, const cicero_mlp *mlp,
                                     const float *ray_o, const float *ray_d, int n_rays,
                                     const cicero_sampling *sampling, const float *d_rgb,
                                     float *d_density, float *d_features, float *d_mlp,
                                     void *workspace, size_t ws_bytes, void *stream);

size_t cicero_backward_workspace_size(const cicero_grid *grid, int n_rays, const cicero_sampling *sampling);

/* Workspace of cicero_render_backward with d_mlp on the tensor cores: the above plus each
 * composited sample's weight-gradient operands (x, h1, h2, dL/dh2, dL/dh1, dL/dz3, each value split
 * into two BF16 halves: 2,272 bytes per sample slot, n_rays * n_samples slots rounded up to 64).
 * Given a workspace at least this large (and a grid of at most 16 channels), the backward stages
 * those operands and forms dW1 | db1, dW2 | db2 and dW3 | db3 as split-BF16 tensor-core GEMMs over
 * the samples; with a smaller one (at least
 * cicero_backward_workspace_size) it takes the MLP weight gradients on the CUDA cores in FP32.
 * Both agree with the oracle's gradients to 1e-3 relative. */
size_t cicero_backward_mlp_workspace_size(const cicero_grid *grid, int n_rays, const cicero_sampling *sampling);

/* ---------------------------------------------------------------------------------------------
 * Pieces of the path, exposed for testing and for callers that drive the stages themselves.
 */

/* The Ray Index Table (Sec. IV-A) of a camera: the samples that reach Feature Gathering, grouped
 * by brick of opt->brick^3 voxels, brick id (bz * nby + by) * nbx + bx with nb = ceil((n-1)/brick).
 * brick_offsets [n_bricks + 1]: samples of brick b are samples[brick_offsets[b] .. brick_offsets[b+1]).
 * samples [H*W*n_samples]: sample id = ray * n_samples + slot.  Inside one brick the samples
 * are grouped by octant of the brick (x half, then y, then z as bits 0, 1, 2); their order inside
 * an octant is not specified.  n_bricks is returned through *n_bricks_out (host).  Size the workspace with
 * cicero_build_rit_workspace_size. */
cicero_status cicero_build_rit(const cicero_grid *grid, const cicero_camera *cam, const cicero_sampling *sampling,
                               const cicero_options *opt, int32_t *brick_offsets, int32_t *samples,
                               int *n_bricks_out, void *workspace, size_t ws_bytes, void *stream);

size_t cicero_build_rit_workspace_size(const cicero_grid *grid, const cicero_camera *cam,
                                       const cicero_sampling *sampling, const cicero_options *opt);

/* Feature Computation alone: c [M][3] = MLP(x [M][in_dim]) in the chosen precision. */
cicero_status cicero_mlp_eval(const cicero_mlp *mlp, const float *x, int M, cicero_precision precision,
                              float *c, void *workspace, size_t ws_bytes, void *stream);

size_t cicero_mlp_eval_workspace_size(int M);

/* Reads the error word of a workspace after the work queued on `stream` has finished (this call
 * synchronises `stream`).  Returns CICERO_OK, CICERO_ERR_TIMEOUT or CICERO_ERR_INTERNAL; the
 * word is cleared.  A rendering or backward call with no rays still clears the word (on its
 * stream), so the status after it is CICERO_OK whatever the workspace held. */
cicero_status cicero_workspace_status(void *workspace, void *stream);

/* Stage timing for measurement tools.  Between cicero_profile_begin and cicero_profile_end the
 * library records a pair of CUDA events on the caller's stream around each stage it launches;
 * cicero_profile_end synchronises on them and writes, per stage, the summed elapsed time in ms and
 * the number of timed launches.  Stages: 0 march (Indexing + density + transmittance),
 * 1 brick bucketing (Ray Index Table), 2 brick gather + MLP, 3 compositing, 4 warp splat
 * (Eq. 1-3 + depth test), 5 warp resolve + hole listing, 6 backward per ray, 7 backward per
 * brick (grid gradients; with the weight gradients on CUDA cores, those too), 8 MLP alone,
 * 9 MLP weight gradients from the staged operands.  Profiling state is process-wide; do not profile from several threads. */
cicero_status cicero_profile_begin(void);
cicero_status cicero_profile_end(double *total_ms, long long *launches, int n_stages);

/* Number of CUDA kernels this library has launched since it was loaded (all devices). */
long long cicero_launch_count(void);

/* Thread-local description of the last error returned on this thread. */
const char *cicero_last_error(void);

/* Library version string. */
const char *cicero_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CICERO_H */
