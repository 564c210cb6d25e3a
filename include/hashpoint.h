/*
 * hashpoint.h -- C-ABI of the B300 (sm_103a) HashPoint hot path.
 *
 * The per-frame path of "HashPoint: Accelerated Point Searching and Sampling
 * for Neural Rendering" (CVPR 2024):
 *   hp_build_table      Sec. 3.2 "Accelerated structure construction": project
 *                       the visible points, keep every point per pixel, reorder
 *                       the list so each pixel's points are contiguous, and
 *                       keep a pixel-keyed table of (start, count).
 *   hp_search_sample    Sec. 3.2 "Searching" (window walk, radius test with the
 *                       fixed radius or the cone radius of Eq. radius /
 *                       Eq. r_approx2) and Sec. 3.3 "Adaptive primary surface
 *                       sampling" (pseudo-UDF d_j, alpha_j, Eq. weight).
 *   hp_aggregate_render Sec. 3.4 integration: inverse-distance aggregation of
 *                       neighbour features, a radiance MLP, and the volume
 *                       rendering of Eq. 2.
 *
 * Conventions (all entry points):
 *   - Pointers named d_* are device pointers; they are owned by the caller and
 *     must stay valid until the work enqueued on `stream` has finished.
 *     Other pointers are host pointers, read during the call only.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call only enqueues work; nothing is synchronised except
 *     by hp_get_status.
 *   - Errors a host can see (bad sizes, NULL pointers, unbuilt table, missing
 *     workspace) are returned at once and nothing is enqueued.  Errors found on
 *     the device (sample capacity overflow, a bounded wait that gave up, a ray
 *     pixel out of range) are recorded in the context's device status word and
 *     reported by hp_get_status; the kernels still terminate.
 *   - A context is used by one host thread at a time (thread-compatible, not
 *     thread-safe).  Nothing is printed; no exception crosses the ABI.
 *   - Float inputs are IEEE binary32.  Every discrete decision (pixel keys,
 *     radius tests, orderings, neighbour sets, weights vs eps_w, clusters,
 *     sample counts) follows a written float32 arithmetic contract so that it
 *     is reproducible bit for bit by an independent CPU implementation.
 */
#ifndef HASHPOINT_H
#define HASHPOINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HP_OK = 0,
    HP_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of range */
    HP_ERR_CUDA = 2,          /* a CUDA runtime call failed (launch, memset, alloc) */
    HP_ERR_OVERFLOW = 3,      /* device: more samples than hp_samples.capacity */
    HP_ERR_TIMEOUT = 4,       /* device: a bounded inter-block wait gave up */
    HP_ERR_NOT_BUILT = 5,     /* search before build, or build parameters changed */
    HP_ERR_NO_MEMORY = 6,     /* workspace too small / allocation failed */
    HP_ERR_BAD_RAY = 7,       /* device: a ray pixel id outside [0, W*H) */
    HP_ERR_TOO_LARGE = 8,     /* a size above the fixed limit of an allocation-free entry point */
    HP_ERR_BOUNDS = 9         /* device, bounds-check build (libhashpoint_checks.so) only: an index
                                 outside its array (detail: the index); the access was skipped */
} hp_status;

typedef struct hp_ctx hp_ctx;

/* Pinhole camera.  World -> camera: X_cam = R X_world + t (R row-major),
 * camera axes x right, y down, z forward; pixel (u, v) has its centre at
 * (u + 0.5, v + 0.5).  Rays start at the camera centre through pixel centres;
 * points are searched for t (distance along the unit ray) in [t_near, t_far];
 * points with camera depth <= z_near are dropped. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float t_near, t_far, z_near;
} hp_camera;

enum {
    HP_RADIUS_FIXED = 0,        /* r(t) = r (Point-NeRF style fixed radius)            */
    HP_RADIUS_CONE = 1,         /* r(t) = Eq. radius (exact similar-triangle form)      */
    HP_RADIUS_CONE_APPROX = 2   /* r(t) = Eq. r_approx2 (small-angle form)              */
};

/* Method parameters (Sec. 3.2-3.3). */
typedef struct {
    int32_t radius_mode;  /* HP_RADIUS_* */
    float rho;            /* cone modes: r_ddot / r_dot (kernel size s = 2*ceil(rho)+1);
                             <= 0: chosen so that r(t_near) on the central ray equals r */
    float gamma;          /* alpha_j = gamma * exp(-d_j^2 / beta2); 0 < gamma <= 1 */
    float beta2;          /* beta^2 > 0 */
    float eps_w;          /* a candidate is kept when w_j > eps_w (>= 0) */
    float gap_k;          /* primary cluster: consecutive t-gap <= gap_k * r(t); 0 disables the
                             gate, so lowering gamma moves sampling from the primary surface
                             towards multi-surface sampling (Supplementary, noisy input) */
    float eps_d;          /* IDW distance floor (> 0) */
    int32_t cand_cap;     /* candidates kept per ray, 1..128 (the smallest (t, id)) */
    int32_t bg_mode;      /* 0 black background, 1 white */
    int32_t window_h;     /* 0: derive the window half-width; > 0: force it */
} hp_config;

/* Per-sample / per-ray outputs of hp_search_sample (caller-owned device
 * buffers).  R = number of rays; cap = capacity (rows of the per-sample
 * arrays, R * n_samples always suffices).  Samples are packed ray by ray in
 * ray order; the samples of ray i are rows sample_offset[i] ..
 * sample_offset[i+1]-1, in increasing depth. */
typedef struct {
    int32_t *n_s;            /* [R]   samples kept (0..n_samples) */
    int32_t *primary;        /* [R]   table key (padded pixel index) of the primary
                                      surface's first point, -1 when none */
    int32_t *cand_count;     /* [R]   points that passed the radius test, before cand_cap */
    int64_t *sample_offset;  /* [R+1] exclusive prefix sum of n_s; [R] = total S */
    float *t;                /* [cap] sample depth along the unit ray */
    int32_t *ray;            /* [cap] ray index of the sample */
    int32_t *src;            /* [cap] id of the point whose projection is the sample */
    float *delta;            /* [cap] interval to the next sample; 2 r(t) for the last (Eq. 2) */
    int32_t *nbr;            /* [cap*K] neighbour point ids, nearest first; -1 pads.  May be
                                NULL together with nbr_dist: the lists then stay in the
                                context's search workspace (not copied), where
                                hp_aggregate_render reads them; they are valid until the
                                next search on the context, and the backward needs them
                                packed */
    float *nbr_dist;         /* [cap*K] distances of those neighbours to the sample */
    int64_t capacity;        /* rows available in the per-sample arrays */
} hp_samples;

#define HP_MLP_MAX_LAYERS 8
#define HP_MLP_MAX_WIDTH 128

/* Decode arithmetic (hp_mlp.decode). */
enum {
    HP_DECODE_FP32 = 0,       /* FP32-accurate; tensor cores (tcgen05) with the error-corrected
                                 FP16 split when every hidden layer has fan-in a multiple of 16
                                 (<= 128) and width 16..128 step 16, else FP32 FMA cores */
    HP_DECODE_FP32_SIMT = 1,  /* FP32 FMA cores only */
    HP_DECODE_BF16 = 2        /* BF16 operands on the tensor cores, FP32 accumulation (hidden
                                 layers); output layer, activations and compositing stay FP32 */
};

/* Radiance MLP: n_layers linear layers with ReLU between them, input width
 * dims[0] = F, output dims[n_layers] = 4 (density logit, r, g, b logits).
 * params (device) packs W0 (dims[1] x dims[0], row-major), b0, W1, b1, ...
 * density = softplus(o0), colour = sigmoid(o1..3).  Hidden widths are 16, 32,
 * 64 or 128; the packed size is at most 40960 floats. */
typedef struct {
    int32_t n_layers;
    int32_t dims[HP_MLP_MAX_LAYERS + 1];
    const float *d_params;
    int32_t decode;          /* HP_DECODE_* */
} hp_mlp;

/* Read-only view of the table built by the last hp_build_table. */
typedef struct {
    int32_t h;               /* window half-width; table covers the image padded by h */
    int32_t padded_width;    /* W + 2h */
    int32_t padded_height;   /* H + 2h */
    int64_t n_buckets;       /* padded_width * padded_height */
    float r_ddot;            /* cone modes: r_ddot on the f = 1 image plane */
    const uint32_t *d_start; /* [n_buckets+1] first list position of each bucket */
    const float *d_points;   /* [N][4]: the reordered list, rows 0 .. d_start[n_buckets]-1:
                                camera-space x, y, z and the point id (int32 bits),
                                bucket by bucket; inside a bucket in the order the
                                build's atomics left them (hp_table_copy returns each
                                bucket ordered by (z, x, y, id)) */
} hp_table;

/* Create a context for `cfg` on the current CUDA device.  Allocates only the
 * 64-byte device status word.  Returns HP_ERR_INVALID_ARG for bad parameters. */
hp_status hp_create(hp_ctx **ctx, const hp_config *cfg);

/* Release the context and any workspace it allocated itself. */
hp_status hp_destroy(hp_ctx *ctx);

/* Bytes of device workspace one frame needs: the table for n_points points
 * seen by `cam` with radius r, plus scratch for n_rays rays of up to
 * n_samples samples with K neighbours each.  The result is a multiple of 256. */
hp_status hp_workspace_size(const hp_config *cfg, const hp_camera *cam, float r, int64_t n_points,
                            int64_t n_rays, int32_t K, int32_t n_samples, size_t *bytes);

/* Host-only: the search-window half-width h (kernel size s = 2h+1) and, in
 * the cone modes, r_ddot on the f = 1 image plane, for `cam`, `cfg` and
 * radius r.  The window is the smallest that provably contains every point
 * the radius test can accept (see the comment of derive_window in the
 * library source), or the paper's s when that is larger (cone modes, Sec. 3.2). */
hp_status hp_window(const hp_config *cfg, const hp_camera *cam, float r, int32_t *h, float *r_ddot);

/* Give the context a caller-owned device workspace (256-byte aligned).  Without
 * one the context allocates (and grows) its own with cudaMalloc. */
hp_status hp_set_workspace(hp_ctx *ctx, void *d_ptr, size_t bytes);

/* Sec. 3.2 table build for d_points (n_points x 3, world xyz) seen by `cam`.
 * Fixed mode: r is the search radius.  Cone modes: r is used only when
 * cfg.rho <= 0 (r_min at t_near).  n_points may be 0.  Kernels: projection +
 * atomic bucket counts, decoupled-lookback scan, scatter.  No result of the
 * search, the sampling or the proposal depends on the order of the points
 * inside a bucket; the per-bucket depth order is established when the table
 * is read out (hp_table_copy). */
hp_status hp_build_table(hp_ctx *ctx, const float *d_points, int64_t n_points, const hp_camera *cam,
                         float r, void *stream);

/* Describe the current table (valid after hp_build_table was enqueued). */
hp_status hp_table_info(const hp_ctx *ctx, hp_table *out);

/* Copy the current table into caller buffers (enqueued on `stream`):
 * d_start receives n_buckets+1 uint32 starts, d_points receives n_points x 4
 * floats: the reordered list of hp_table.d_points with every bucket sorted by
 * (camera depth z, x, y, id) -- the canonical, input-order-independent table
 * (Sec. 3.2, "Z-order manner": reading c1).  Rows past d_start[n_buckets],
 * the number of kept points, are unspecified.  The sort runs on the GPU and
 * uses the context's count array as scratch. */
hp_status hp_table_copy(const hp_ctx *ctx, uint32_t *d_start, float *d_points, void *stream);

/* Sec. 3.2 window search + Sec. 3.3 primary-surface sampling for n_rays rays.
 * d_ray_pixels: pixel ids v*W + u (device, n_rays), or NULL for all W*H
 * pixels in row-major order (then n_rays must be W*H).  K: neighbours per
 * candidate, 1..32; n_samples: 1..16.  Writes `out` (see hp_samples). */
hp_status hp_search_sample(hp_ctx *ctx, const int32_t *d_ray_pixels, int64_t n_rays, int32_t K,
                           int32_t n_samples, const hp_samples *out, void *stream);

/* Sec. 3.4 + Eq. 2 for the samples of the last hp_search_sample: features
 * d_feats (n_points x F, F in {4,8,16,32,64,128}) blended by inverse distance
 * (weights 1/max(dist, eps_d)), decoded by `mlp`, composited front to back.
 * Writes d_rgb (n_rays x 3) and d_wsum (n_rays, the sum of compositing
 * weights, <= 1).  `samples` must be the buffers given to hp_search_sample;
 * when their nbr/nbr_dist are NULL the neighbour lists are read from the
 * search's workspace (HP_ERR_INVALID_ARG if the last search on this context
 * packed them or if only one of the two is NULL). */
hp_status hp_aggregate_render(hp_ctx *ctx, const hp_samples *samples, int64_t n_rays, const float *d_feats,
                              int32_t F, const hp_mlp *mlp, float *d_rgb, float *d_wsum, void *stream);

/* ---- Learned depth-interval proposal (an extension beyond the paper, like
 * the learned samplers it cites as related work).  A 16 -> 32 -> 32 -> 2 MLP
 * (ReLU) reads a ray's depth histogram -- the camera depths of the points in
 * the 3 x 3 buckets around its pixel in 16 bins over [t_near, t_far], as
 * log(1 + n) -- and outputs (a, b): t0 = t_near + (t_far - t_near) sigmoid(a),
 * t1 = t0 + (t_far - t0) sigmoid(b).  Parameters (HP_PROP_PARAMS floats):
 * W0 [32][16], b0 [32], W1 [32][32], b1 [32], W2 [2][32], b2 [2]. */
#define HP_PROP_BINS 16
#define HP_PROP_PARAMS 1666

/* Interval [t0, t1] (d_interval, R x 2 floats) for every ray from the current
 * table, with BF16 weights (d_weights_bf16, HP_PROP_PARAMS) and FP32
 * accumulation; a ray whose 3 x 3 buckets are empty gets [t_near, t_far].
 * Rays: as hp_search_sample. */
hp_status hp_proposal_infer(hp_ctx *ctx, const int32_t *d_ray_pixels, int64_t n_rays, const uint16_t *d_weights_bf16,
                            float *d_interval, void *stream);

/* One Adam step of the proposal on a batch of rays of the current table,
 * against the first and last sample depths of a plain hp_search_sample of
 * those rays (`plain`).  The loss per ray is
 * softplus(k (t0n - s0n + m))/k + softplus(k (s1n - t1n + m))/k + l (t1n - t0n)
 * in units of t_far - t_near (k = 200, m = 0.01, l = 0.05), averaged over rays
 * with samples.  d_params (FP32 master), d_adam_m, d_adam_v and d_grad
 * (zero on the first call) hold HP_PROP_PARAMS floats each; d_weights_bf16
 * receives the updated BF16 copy; d_loss (2 floats, optional) receives the
 * summed loss and the number of rays used.  step counts from 1. */
hp_status hp_proposal_train_step(hp_ctx *ctx, const int32_t *d_ray_pixels, int64_t n_rays, const hp_samples *plain,
                                 float *d_params, float *d_adam_m, float *d_adam_v, float *d_grad,
                                 uint16_t *d_weights_bf16, int32_t step, float lr, float *d_loss, void *stream);

/* hp_search_sample restricted per ray to the depth interval d_interval
 * (R x 2, e.g. from hp_proposal_infer): only points with t in [t0, t1] are
 * candidates, and in the fixed-radius mode the window shrinks to the bound
 * that t0 allows.  Rays that keep no sample are searched again without the
 * restriction (plain-search fallback) unless their whole plain window holds
 * no point, or the restricted walk covered the plain window and the plain
 * radius test accepted none of its points, so a ray is empty only if the
 * plain search finds nothing either; also when the plain search accepts a
 * point in front of t0, or behind t1 while the selection ran out of
 * candidates (decision contract D12).
 * Outputs as hp_search_sample; d_fallback_count (device, optional) receives
 * the number of rays searched again. */
hp_status hp_search_sample_proposal(hp_ctx *ctx, const int32_t *d_ray_pixels, int64_t n_rays, int32_t K,
                                    int32_t n_samples, const float *d_interval, const hp_samples *out,
                                    uint32_t *d_fallback_count, void *stream);

/* hp_search_sample_proposal with the intervals inferred inside the search
 * (no interval buffer, no separate inference launch): each ray computes the
 * interval hp_proposal_infer would give it from d_weights_bf16 (the 1666
 * BF16 proposal weights, device) with the same arithmetic, so the results
 * equal hp_proposal_infer followed by hp_search_sample_proposal bit for bit.
 * The proposal is not part of the paper's method (see hp_proposal_infer).
 * Errors as hp_search_sample; HP_ERR_INVALID_ARG when d_weights_bf16 is NULL. */
hp_status hp_search_sample_learned(hp_ctx *ctx, const int32_t *d_ray_pixels, int64_t n_rays, int32_t K,
                                   int32_t n_samples, const uint16_t *d_weights_bf16, const hp_samples *out,
                                   uint32_t *d_fallback_count, void *stream);

/* Backward of hp_aggregate_render (Sec. 3.4 + Eq. 2) with respect to the point
 * features and the point positions, the discrete structure of the last
 * hp_search_sample (neighbour sets, samples) held fixed -- it is not
 * differentiable.  Sample depths move with their source point
 * (t_j = <P_src, d>, P = R p + t), so positions receive gradient through the
 * inverse-distance weights, the sample positions and the Delta's of Eq. 2.
 * Call it after hp_aggregate_render with the same `samples`, before the next
 * hp_aggregate_render on this context (it reuses the decoded samples that
 * call kept in the workspace), with the ray list of the last search still
 * valid.  d_points (N x 3 world) and d_feats (N x F) are the forward inputs;
 * d_grad_rgb (R x 3) and d_grad_wsum (R, or NULL) the output gradients.
 * Gradients are ADDED (atomically, FP32) into d_grad_feats (N x F) and
 * d_grad_points (N x 3, world space); either may be NULL.  The MLP weights
 * get no gradient.  The neighbour lists must be packed (samples.nbr and
 * samples.nbr_dist non-NULL: HP_ERR_INVALID_ARG otherwise). */
hp_status hp_aggregate_render_backward(hp_ctx *ctx, const hp_samples *samples, int64_t n_rays,
                                       const float *d_points, const float *d_feats, int32_t F, const hp_mlp *mlp,
                                       const float *d_grad_rgb, const float *d_grad_wsum, float *d_grad_feats,
                                       float *d_grad_points, void *stream);

/* Synchronise `stream`, then return the device status word recorded since the
 * last call (HP_OK if none) and its detail (e.g. the tile or ray index), and
 * clear it.  The return value is HP_ERR_CUDA if the synchronisation failed. */
hp_status hp_get_status(hp_ctx *ctx, void *stream, int32_t *dev_status, int64_t *detail);

/* Test hook for the bounded waits: the scan tile `skip_tile` (>= 0) does not
 * publish its prefix, and a waiting block gives up after `spin_limit`
 * iterations (0 = default).  skip_tile < 0 turns the hook off.  The waiter
 * records HP_ERR_TIMEOUT and finishes; nothing hangs. */
hp_status hp_debug_fault(hp_ctx *ctx, int32_t skip_tile, int32_t spin_limit);

/* Per-kernel device timing (CUDA events recorded on the launching stream
 * around every kernel the context launches, or around a kernel and the one
 * that prepares its input: the point-major pass and the selection of a
 * whole-frame search; the weight image and the tensor-core decode).
 * hp_profile_start(ctx, n) begins recording up to n timed launches (events
 * are created here, on the host); hp_profile_stop synchronises those events,
 * writes per kernel id the summed milliseconds, the timed launches and the
 * CUDA kernels those launches ran into ms[HP_PROF_KERNELS],
 * launches[HP_PROF_KERNELS] and kernels[HP_PROF_KERNELS] (any may be NULL),
 * and stops recording.  Kernel ids: see hp_profile_kernel_name. */
#define HP_PROF_KERNELS 15
hp_status hp_profile_start(hp_ctx *ctx, int32_t max_launches);
hp_status hp_profile_stop(hp_ctx *ctx, double *ms, int32_t *launches, int32_t *kernels);
const char *hp_profile_kernel_name(int32_t id);

/* Self-test of the tensor-core path: D = A B^T for A (128 x K) and B (N x K),
 * row-major 16-bit inputs, D (128 x N) FP32, all device pointers; K in
 * 16..128 and N in 16..256, multiples of 16.  flags bit 0: BF16 inputs (else
 * FP16); bit 1: A is placed in tensor memory (two elements per 32-bit column,
 * row m in lane m) instead of shared memory.  One block stages the operands,
 * issues K/16 tcgen05.mma and reads the TMEM accumulator back.  A device-side
 * timeout is reported by hp_get_status. */
hp_status hp_selftest_mma(hp_ctx *ctx, const uint16_t *d_a, const uint16_t *d_b, float *d_d, int32_t K, int32_t N,
                          int32_t flags, void *stream);

/* Allocation-free exclusive prefix sum -- not part of the paper's method (the
 * paper has no counterpart); it is the bucket-count scan of hp_build_table
 * offered on its own for callers that must not allocate device memory: code
 * hosted by an application that owns the whole device memory budget and
 * forbids libraries to call cudaMalloc, or a real-time loop where a
 * cudaMalloc, which can synchronise the device, would stall the frame.
 *
 * d_out[i] = d_in[0] + ... + d_in[i-1] for i < n (uint32, wrapping), d_in and
 * d_out device pointers, 16-byte aligned, n <= HP_SCAN_NOALLOC_MAX_N (larger
 * n returns HP_ERR_TOO_LARGE; n == 0 does nothing).  If d_status (device,
 * optional) is given, the call's device status (HP_OK or HP_ERR_TIMEOUT from
 * the bounded inter-block wait) is copied there on `stream`.
 *
 * Memory: the scratch (look-back words, ticket, status) lives in one
 * file-scope static device array of 65,568 bytes that every device which
 * loads the library holds until the process exits.  The call allocates and
 * frees nothing; it only clears the part of the array it uses.  The first
 * call on a device looks the array's device address up (cudaGetSymbolAddress,
 * with that device current) and caches it; make that first call before any
 * stream capture.  The cached address belongs to the device's primary
 * context: after cudaDeviceReset on that device it is stale, and the process
 * must not call hp_scan_noalloc on that device again.  All calls share the one array: calls whose GPU work
 * overlaps (different streams, or several host threads without ordering)
 * race and give wrong sums -- order them on one stream. */
#define HP_SCAN_NOALLOC_MAX_N 67108864
hp_status hp_scan_noalloc(const uint32_t *d_in, uint32_t *d_out, int64_t n, int32_t *d_status, void *stream);

/* Static string for a status code. */
const char *hp_status_string(hp_status s);

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t hp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HASHPOINT_H */
