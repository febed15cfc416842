/*
 * scalp.h -- C ABI of libscalp, a GB300 (sm_103a) implementation of the
 * iterative clustering of SCALP ("Superpixels with Contour Adherence using
 * Linear Path", Giraud, Ta, Papadakis, ICPR 2018).
 *
 * The problem (Algorithm 1): given an image, a number of superpixels k and a
 * soft contour prior C in [0,1], output a superpixel decomposition S.  Each
 * iteration assigns every pixel p to the cluster C_k = [l_k, a_k, b_k, X_k]
 * minimising D(p, C_k) of Eq. 3 over the clusters whose (2r+1)x(2r+1) window
 * (r = sqrt(N/k)) holds p, where D combines the CIELab colour distance along
 * the linear path from p to the barycenter X_k (Eq. 1), the contour prior
 * along the same path (Eq. 2) and the spatial distance; then it recomputes the
 * cluster means and projects each barycenter that falls outside its
 * superpixel onto the nearest pixel of that superpixel (Eq. 4).
 *
 * Conventions for every entry point:
 *   - Return value: SCALP_OK (0) or a negative SCALP_E_* code.  An argument
 *     error (SCALP_E_ARG) has no side effect.  scalp_last_error() gives text.
 *   - Device work is enqueued on params->stream (a cudaStream_t; NULL = the
 *     legacy default stream).  Errors of asynchronous work surface at the next
 *     call that synchronises (scalp_labels, scalp_clusters, scalp_get_state,
 *     scalp_debug_paths, scalp_sync).
 *   - The caller owns every input and output buffer.  Inputs are copied into
 *     the workspace by scalp_init and never referenced after it returns.
 *   - The library allocates no device memory: all device buffers are carved
 *     from params->workspace (caller-allocated, at least
 *     scalp_workspace_bytes() bytes, 256-byte aligned), which must stay valid
 *     until scalp_destroy().  The context itself is host memory.  A host
 *     thread that reads a context's status (scalp_labels and other calls that
 *     synchronise) keeps 64 bytes of pinned host memory until it exits; a
 *     batch holds about 110 bytes of pinned host memory per image
 *     (staging for its per-call pointer tables and its gathered status).
 *   - Images are row-major, pixel (x, y) at row y, column x, with integer
 *     coordinates at pixel centres.  Labels are int32, row-major H x W.
 *   - One context, or one batch, is used by one host thread at a time.
 */
#ifndef SCALP_H
#define SCALP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SCALP_OK 0
#define SCALP_E_ARG (-1)      /* invalid argument; nothing was done */
#define SCALP_E_NOMEM (-2)    /* workspace missing or smaller than required */
#define SCALP_E_CUDA (-3)     /* a CUDA runtime call failed */
#define SCALP_E_TIMEOUT (-4)  /* a bounded device-side wait gave up */
#define SCALP_E_STATE (-5)    /* call not valid in the context's state */
#define SCALP_E_INTERNAL (-6) /* a device-side consistency check failed */

#define SCALP_STORAGE_F32 0   /* Lab + contour planes stored as 4 x fp32 per pixel */
#define SCALP_STORAGE_F16 1   /* the same planes stored as 4 x fp16 per pixel */

#define SCALP_PRIOR_INPUT 0     /* the contour prior is the scalp_contour argument */
#define SCALP_PRIOR_GRADIENT 1  /* computed on the GPU from the image: scalp_gradient_prior */

/* Input image: 8-bit sRGB, interleaved R, G, B. */
typedef struct {
    int32_t H, W;          /* rows and columns, both >= 1 */
    const uint8_t *rgb;    /* H rows of W*3 bytes */
    int64_t rgb_stride;    /* bytes between rows; 0 means 3*W */
    int32_t on_device;     /* 1: rgb (and the contour) are device pointers */
} scalp_image;

/* Soft contour prior C (Sec. II-E): fp32 in [0,1], 1 on a contour. */
typedef struct {
    const float *data;     /* H rows of W floats; NULL means C = 0 everywhere */
    int64_t stride;        /* floats between rows; 0 means W */
} scalp_contour;

/* Parameters of Eq. 1-3; defaults of Sec. III-A3 via scalp_default_params(). */
typedef struct {
    float lambda;          /* Eq. 1 weight of the pixel's own colour, in [0,1]; 0.5 */
    float sigma;           /* Eq. 2 contour scale, > 0; 0.25 */
    float gamma;           /* Eq. 2 contour weight, >= 0; < 0 selects 2r */
    int32_t storage;       /* SCALP_STORAGE_F32 or SCALP_STORAGE_F16 */
    int32_t use_graph;     /* 1: replay each iteration as a CUDA graph (non-NULL stream) */
    int32_t global_walk;   /* bit 0: walk every path on the plane in global memory (no distance
                              maps); bit 1: evaluate every (pixel, candidate) pair, without the
                              lower bound that skips pairs which cannot win (the same labels and
                              state, slower: for tests) */
    int32_t prior;         /* SCALP_PRIOR_INPUT (default) or SCALP_PRIOR_GRADIENT; with the
                              latter the contour argument must be NULL or have NULL data */
    void *stream;          /* cudaStream_t for all device work */
    void *workspace;       /* device memory owned by the caller */
    size_t workspace_bytes;
} scalp_params;

/* Sizes fixed by scalp_init. */
typedef struct {
    int32_t H, W, K;       /* image size and requested number of superpixels */
    int32_t nx, ny, Keff;  /* regular grid, Keff = nx*ny clusters */
    double r;              /* sqrt(H*W/K), the grid step and window half-size */
    double gamma;          /* resolved Eq. 2 weight */
    int32_t map_pairs;     /* shared-memory distance-map capacity of an assignment CTA, in
                              (d_c, w) pairs (0: every path walks the plane) */
    int32_t iterations;    /* iterations run so far */
} scalp_info;

/* Host view of the solver state: the data one iteration reads.  Arrays are
 * caller-allocated host memory. */
typedef struct {
    int32_t *labels;       /* H*W current labels S */
    int64_t *n;            /* Keff: |S_k| */
    int64_t *sx, *sy;      /* Keff: sums of x and y over S_k; X_k = (sx/n, sy/n) */
    double *color;         /* Keff x 3: mean (l_k, a_k, b_k) */
    int32_t *endpoint;     /* Keff x 2: path end, X_k rounded half-up or X_k^* (Eq. 4) */
} scalp_state;

typedef struct scalp_ctx scalp_ctx;

/* Fills *p with lambda=0.5, sigma=0.25, gamma=2r, FP32 storage, graphs on. */
void scalp_default_params(scalp_params *p);

/* Workspace bytes scalp_init needs for an H x W image and K superpixels
 * (0 on invalid sizes).  Depends on p->storage only among the parameters. */
size_t scalp_workspace_bytes(int32_t H, int32_t W, int32_t K, const scalp_params *p);

/* Algorithm 1 initialisation.  Converts the image to CIELab (Sec. II-A),
 * precomputes the per-pixel contour factor 1 - exp(-C^2/sigma^2) of Eq. 2,
 * seeds Keff clusters on the regular grid of step r = sqrt(N/K) and labels
 * every pixel with its grid cell.  K in [1, H*W]; m > 0 is the compactness of
 * Eq. 3.  On success *out receives a context (free with scalp_destroy). */
int scalp_init(scalp_ctx **out, const scalp_image *image, const scalp_contour *contour,
               int32_t K, float m, const scalp_params *params);

/* Reloads a new image and contour of the same H x W into an existing context
 * and re-initialises the clusters, keeping K, m and the parameters. */
int scalp_reload(scalp_ctx *ctx, const scalp_image *image, const scalp_contour *contour);

/* Enqueues n >= 0 iterations of Algorithm 1: assignment by Eq. 3 over the
 * window of each cluster (strict '<' in ascending k, so ties go to the
 * smallest k; a pixel no window reaches keeps its label), cluster update, and
 * the projection of Eq. 4.  Asynchronous. */
int scalp_iterate(scalp_ctx *ctx, int32_t n);

/* Writes the decomposition to out (H*W int32, host or device memory per
 * out_on_device) and synchronises the stream.  enforce != 0 first applies
 * the connectivity enforcement (not part of the paper): 4-connected
 * components of equal label, each component of at most floor(N/(4K)) pixels
 * merged into the component left of (else above) its first pixel, and the
 * result numbered 0.. in raster order; *n_labels gets the count.  With
 * enforce == 0 the cluster labels are returned and *n_labels = Keff. */
int scalp_labels(scalp_ctx *ctx, int32_t *out, int32_t out_on_device, int32_t enforce,
                 int32_t *n_labels);

int scalp_get_info(const scalp_ctx *ctx, scalp_info *info);

/* Copies the state to host memory (synchronises). */
int scalp_get_state(scalp_ctx *ctx, const scalp_state *state);

/* The cluster descriptors C_k = [l_k, a_k, b_k, X_k] of Sec. II-A, as
 * Algorithm 1's last update left them: out (host memory, Keff x 5 floats,
 * caller-owned) receives per cluster k the mean CIELab colour (l_k, a_k, b_k)
 * and the barycenter X_k = (x_k, y_k) in pixel coordinates (the exact integer
 * coordinate sums divided by |S_k|, rounded once to float); *K_eff receives
 * Keff.  A cluster that has lost every pixel keeps its last descriptor.
 * Synchronises the stream; out must hold scalp_get_info()'s Keff x 5 floats. */
int scalp_clusters(scalp_ctx *ctx, float *out, int32_t *K_eff);

/* Replaces the state (checkpoint restore, or injecting a state to compute one
 * assignment from).  Labels must be in [0, Keff), n >= 1, 0 <= sx/n <= W-1,
 * 0 <= sy/n <= H-1 and endpoints inside the image; otherwise SCALP_E_ARG. */
int scalp_set_state(scalp_ctx *ctx, const scalp_state *state);

/* Linear paths (Sec. II-B) as the assignment kernel walks them, for checking:
 * pairs holds M rows (px, py, ex, ey) of host int32; out_len[i] receives
 * max(|ex-px|, |ey-py|) + 1 and out_xy[i*stride_xy .. ] the (x, y) pixels in
 * walking order (as many as stride_xy int32 per row hold; 2*out_len[i] for
 * the whole path).  The kernels step along a path in two equivalent forms (an
 * error term; a 32-bit fixed-point slope for paths of at most 512 steps): both
 * are walked, and out_len[i] = -1 reports a path on which they disagree.  All
 * host memory; coordinates must lie in the image. */
int scalp_debug_paths(scalp_ctx *ctx, const int32_t *pairs, int32_t M, int32_t *out_xy,
                      int32_t stride_xy, int32_t *out_len);

/* Per-kernel timing of the assignment kernel with CUDA events on the
 * context's stream.  enable != 0 starts counting (and resets the totals);
 * *ms and *launches receive the totals so far (synchronises). */
int scalp_profile(scalp_ctx *ctx, int32_t enable, double *ms, int64_t *launches);

/* Work of the last assignment, counted on the device while counting is
 * enabled (scalp_count_samples(ctx, 1, ...) resets and enables, 0 disables,
 * -1 only reads; a few atomics per tile; off by default):
 *   samples      sum of |P| over the evaluated (pixel, cluster) pairs
 *   pairs        evaluated (pixel, cluster) pairs
 *   map_rects    (tile, cluster) rectangles whose paths walked a shared-memory
 *                distance map
 *   plane_rects  (tile, cluster) rectangles whose paths walked the plane in
 *                global memory (map buffer full, global_walk, or a tile with
 *                more candidates than shared memory holds)
 * Any output pointer may be NULL.  Synchronises the stream. */
int scalp_count_samples(scalp_ctx *ctx, int32_t enable, int64_t *samples, int64_t *pairs,
                        int64_t *map_rects, int64_t *plane_rects);

/* Synchronises the context's stream and reports pending device errors. */
int scalp_sync(scalp_ctx *ctx);

const char *scalp_last_error(const scalp_ctx *ctx);
void scalp_destroy(scalp_ctx *ctx);

/* ---- Batches: many images of uneven size and K solved together ----------------
 *
 * The paper solves one image at a time; solving many at once is this library's
 * addition.  Every image gets its own solver state (as scalp_init would give
 * it) inside one caller-owned workspace of scalp_batch_workspace_bytes()
 * bytes; each iteration of Algorithm 1 then runs as one launch per kernel for
 * all images together, and n iterations replay as one CUDA graph (non-NULL
 * stream, params->use_graph), or all n iterations run as one persistent
 * launch (scalp_batch_set_launch).  Results are identical to solving each
 * image alone with the same parameters. */
typedef struct scalp_batch scalp_batch;

size_t scalp_batch_workspace_bytes(int32_t count, const int32_t *H, const int32_t *W,
                                   const int32_t *K, const scalp_params *params);

/* images[i], contours[i] (contours may be NULL: no prior), K[i], m[i] as for
 * scalp_init; params->workspace/stream/storage apply to the whole batch. */
int scalp_batch_init(scalp_batch **out, int32_t count, const scalp_image *images,
                     const scalp_contour *contours, const int32_t *K, const float *m,
                     const scalp_params *params);

/* New images and contours of the same sizes; clusters re-initialised
 * (asynchronous).  The set-up of all images runs as one launch (after one that
 * clears every image's sums and counters).  Device-side inputs are read in
 * place; host inputs are copied into the workspace first, so they must stay
 * valid until the call returns.  The input pointers are kept in device memory
 * and uploaded (from pinned staging the batch owns) only when they change. */
int scalp_batch_reload(scalp_batch *b, const scalp_image *images, const scalp_contour *contours);

/* n iterations for every image (asynchronous).  In the flat launch mode (the
 * default) each iteration is one launch per kernel for all images and the n
 * iterations replay as one CUDA graph; in a persistent mode all n iterations
 * are one cooperative launch (see scalp_batch_set_launch).  The results are
 * the same bits in every mode. */
int scalp_batch_iterate(scalp_batch *b, int32_t n);

/* Launch modes of scalp_batch_iterate (Algorithm 1's iteration loop for every
 * image of the batch):
 *   SCALP_BATCH_FLAT: per iteration one launch each for the assignment, the
 *     update, the projection and the candidate lists of all images;
 *   SCALP_BATCH_PERSISTENT: one cooperative launch of one CTA per resident
 *     slot (two per SM) for all n iterations; per iteration the CTAs take the
 *     tiles of all images from a queue in batch order, then update,
 *     project and rebuild the lists, with grid-wide barriers between the
 *     phases;
 *   SCALP_BATCH_PERSISTENT_COST: the same, the queue taking the images by
 *     descending grid step r (longest paths first; ties in batch order).
 * Every barrier wait of a persistent launch is bounded (scalp_batch_set_wait;
 * 2 s by default): a CTA that waits longer abandons the launch, every CTA
 * returns, and the next call that reads the status (scalp_batch_labels)
 * returns SCALP_E_TIMEOUT.  The images' state is then undefined until
 * scalp_batch_reload, after which the batch works as before.  A persistent
 * mode needs cooperative launch support, two resident CTAs per SM and a batch
 * of at most about 14,000 images:
 * otherwise SCALP_E_STATE (the mode is unchanged).  Synchronises the stream. */
#define SCALP_BATCH_FLAT 0
#define SCALP_BATCH_PERSISTENT 1
#define SCALP_BATCH_PERSISTENT_COST 2
int scalp_batch_set_launch(scalp_batch *b, int32_t mode);
/* The current mode and the persistent grid (CTAs; -1 until a persistent mode
 * was first asked for, 0 if none fits). */
int scalp_batch_get_launch(const scalp_batch *b, int32_t *mode, int32_t *grid);
/* Bound on each barrier wait of a persistent launch, 1 ms <= limit_ns <= 60 s.
 * hold > 0 is a fault-injection hook for tests: every barrier then waits for
 * `hold` arrivals that never come, so the first one runs out (no GPU fault is
 * made; the CTAs return).  Applies from the next scalp_batch_iterate. */
int scalp_batch_set_wait(scalp_batch *b, int64_t limit_ns, int32_t hold);
/* As scalp_count_samples, summed over the images: the path samples and the
 * (pixel, cluster) pairs the assignments evaluated since counting was
 * enabled (enable 1 resets and counts, 0 stops, -1 only reads).  Synchronises. */
int scalp_batch_count_samples(scalp_batch *b, int32_t enable, int64_t *samples, int64_t *pairs);
/* As scalp_profile, for the batched assignment (every tile of every image in
 * one launch per iteration, the inner loops of Algorithm 1 with Eq. 1-3):
 * enable != 0 starts timing each assignment launch with CUDA events on the
 * batch's stream (and resets the totals), 0 stops, -1 only reads; *ms and
 * *launches receive the totals so far (synchronises).  While timing, the
 * iteration's launches are not programmatically overlapped.  The persistent
 * launch modes run the assignment inside one launch: nothing is timed there
 * and *launches stays 0.  Errors: SCALP_E_ARG for a NULL batch, SCALP_E_CUDA
 * if an event cannot be made or read. */
int scalp_batch_profile(scalp_batch *b, int32_t enable, double *ms, int64_t *launches);
/* Autotuner (not part of the paper): times `iters` iterations of the batch in
 * each launch mode this device supports (the faster of two runs after a
 * warm-up, each from a fresh scalp_batch_reload of images/contours), keeps
 * the fastest and leaves the batch freshly reloaded in it.  *mode receives
 * the choice, trial_ms[3] (may be NULL) the time of each mode (-1: not run).
 * With cache_path (a JSON file, may be NULL) the choice is looked up first
 * under a key of the device's SM count, the storage and the batch's shape
 * class (images, total tiles to two significant digits, mean grid step); a
 * hit (*from_cache = 1) skips the trials; a new choice is written back.
 * Synchronises the stream. */
int scalp_batch_autotune(scalp_batch *b, const scalp_image *images, const scalp_contour *contours,
                         int32_t iters, const char *cache_path, int32_t *mode, float *trial_ms,
                         int32_t *from_cache);

/* Labels of every image into outs[i] (H_i*W_i int32, host or device memory per
 * out_on_device), connectivity enforced when enforce != 0; n_labels[i] gets
 * the count.  Synchronises the stream once.  With enforce, each connectivity
 * pass runs once for all images and writes device outputs directly (host
 * outputs are copied out afterwards, one copy per image on params->stream);
 * without it the label copies, and in scalp_batch_reload the gradient priors
 * and host-input copies, run on streams of the batch's own, forked from and
 * joined back to params->stream.  Host outputs should be pinned for their
 * copies to overlap. */
int scalp_batch_labels(scalp_batch *b, int32_t *const *outs, int32_t out_on_device,
                       int32_t enforce, int32_t *n_labels);

int scalp_batch_get_state(scalp_batch *b, int32_t index, const scalp_state *state);
int scalp_batch_get_info(const scalp_batch *b, int32_t index, scalp_info *info);
void scalp_batch_destroy(scalp_batch *b);

/* ---- Contour prior from the image ----------------------------------------
 * Sec. II-E lets SCALP take any soft contour prior with values in [0, 1] (or a
 * binary one) from any contour detector.  The detectors the paper uses need
 * trained models, so this library offers one computed from the image alone:
 * the magnitude of the CIELab gradient divided by its maximum over the image
 * (0 everywhere for a flat image).  Per channel and axis the derivative is
 * the central difference (f[i+1] - f[i-1]) / 2, the one-sided difference at
 * the first and last pixel, and 0 along an axis of length 1; the magnitude is
 * the Euclidean norm of the six derivatives (FP32).
 *
 * image: H x W sRGB (host or device, image->on_device).  out: H rows of
 * out_stride floats (0 means W), host or device memory (out_on_device).  The
 * work runs on `stream`; with host output the call synchronises it.  The
 * workspace (device memory, 256-byte aligned, owned by the caller) must hold
 * scalp_gradient_prior_workspace_bytes(...) bytes; it stages host data.
 * Errors: SCALP_E_ARG for NULL pointers or bad sizes and strides,
 * SCALP_E_NOMEM for a small workspace, SCALP_E_CUDA for a failed CUDA call.
 * The same prior is used inside scalp_init when params->prior is
 * SCALP_PRIOR_GRADIENT. */
size_t scalp_gradient_prior_workspace_bytes(int32_t H, int32_t W, int32_t image_on_device,
                                            int32_t out_on_device);
int scalp_gradient_prior(const scalp_image *image, float *out, int64_t out_stride,
                         int32_t out_on_device, void *stream, void *workspace,
                         size_t workspace_bytes);

/* ---- Supervoxels --------------------------------------------------------
 * SCALP on a video volume, the extension the paper's conclusion names as
 * future work.  Every rule is the 2-D one taken axis by axis: r = cbrt(N/K)
 * (N = T*H*W voxels) and a 3-D regular grid of step r; cluster k's candidates
 * are the voxels with |v - v_k| <= r on each axis (r the real cube root, so
 * K*|n*v - S_v|^3 <= N*n^3, decided exactly); the linear path is the
 * 3-D digital segment traced from the lexicographically smaller end
 * (x, then y, then t), the axis with the largest |delta| stepping by one and
 * each other axis by round-half-up(i*|delta_j|/|delta_major|); D is Eq. 3
 * with the squared 3-D distance; projection (Eq. 4) in exact integers, ties
 * to the smallest voxel index.  There is no connectivity step.  FP32 planes
 * and the input prior only (params->storage and params->prior otherwise give
 * SCALP_E_ARG); params->use_graph and global_walk are ignored.  Voxel
 * (x, y, t) is element (t*H + y)*W + x of every volume. */
typedef struct {
    int32_t T, H, W;          /* frames, rows, columns, each >= 1, T*H*W <= 2^30 */
    const uint8_t *rgb;       /* T*H*W*3 sRGB bytes, contiguous */
    const float *contour;     /* T*H*W prior values in [0, 1], or NULL for 0 */
    int32_t on_device;        /* 1 if rgb and contour are device pointers */
} scalp_volume;

typedef struct {
    int32_t T, H, W, K;
    int32_t nx, ny, nt, Keff; /* the 3-D grid, Keff = nx*ny*nt clusters */
    double r;                 /* cbrt(N/K) */
    double gamma;             /* resolved Eq. 2 weight */
    int32_t iterations;
} scalp_voxel_info;

typedef struct {
    int32_t *labels;          /* N */
    int64_t *n, *sx, *sy, *st;/* Keff: |S_k| and the coordinate sums */
    double *color;            /* Keff x 3 */
    int32_t *endpoint;        /* Keff x 3: (x, y, t) path end */
} scalp_voxel_state;

typedef struct scalp_vctx scalp_vctx;

size_t scalp_voxel_workspace_bytes(int32_t T, int32_t H, int32_t W, int32_t K,
                                   const scalp_params *params);
/* Set-up and grid initialisation (synchronises the stream). */
int scalp_voxel_init(scalp_vctx **out, const scalp_volume *volume, int32_t K, float m,
                     const scalp_params *params);
int scalp_voxel_iterate(scalp_vctx *ctx, int32_t n);
/* Labels (N int32) to host or device memory; synchronises and reports device
 * errors. */
int scalp_voxel_labels(scalp_vctx *ctx, int32_t *out, int32_t out_on_device);
int scalp_voxel_get_info(const scalp_vctx *ctx, scalp_voxel_info *info);
int scalp_voxel_get_state(scalp_vctx *ctx, const scalp_voxel_state *state);
/* Loads a state (synchronises).  Each cluster needs 1 <= n <= 2^30 (the
 * bound of the exact window arithmetic), a barycenter inside the volume
 * (0 <= S_v <= n*(dim - 1) on each axis) and an endpoint inside it; labels in
 * [0, Keff).  The sums need not be those of the labels (test states). */
int scalp_voxel_set_state(scalp_vctx *ctx, const scalp_voxel_state *state);
/* As scalp_count_samples, for the supervoxel assignment. */
int scalp_voxel_count_samples(scalp_vctx *ctx, int32_t enable, int64_t *samples, int64_t *pairs);
/* As scalp_profile, for the supervoxel assignment: with enable = 1 each
 * assignment launch of scalp_voxel_iterate is bracketed by CUDA events;
 * *ms and *launches receive the accumulated time and count (synchronises
 * when events are pending; 1 resets, 0 stops, -1 only reads). */
int scalp_voxel_profile(scalp_vctx *ctx, int32_t enable, double *ms, int64_t *launches);
void scalp_voxel_destroy(scalp_vctx *ctx);

/* ---- Serving: continuous batching of solves in flight ------------------------
 *
 * Not part of the paper.  A server owns a caller-allocated device memory pool
 * (pool_bytes, 256-byte aligned; the first scalp_server_reserve_bytes(max_slots)
 * bytes are its own).  scalp_server_submit() admits a request when its solver
 * state (scalp_workspace_bytes of the image) fits in the pool and fewer than
 * max_slots requests are in flight, and returns SCALP_E_NOMEM otherwise (nothing
 * done; retry after a step has freed memory).  Each scalp_server_step() runs one
 * iteration of Algorithm 1 for every admitted request that still has
 * iterations to do, all sizes together in one launch per kernel; requests that
 * finish are retired: connectivity enforcement (if asked) and the copy of their
 * labels to the caller's host buffer are enqueued.  scalp_server_poll() reports
 * whether a request's labels have arrived (and then releases its memory).  The
 * labels equal those of scalp_init + scalp_iterate + scalp_labels on the same
 * image.  labels_out should be pinned host memory: with pageable memory the copy
 * synchronises the stream.  No call waits for the stream to drain: a step waits
 * only for the step two launches back (so a request admitted between steps
 * joins within two steps) and for the step eight argument uploads back (the
 * argument blocks form a ring in the reserve); a request's status travels
 * with its labels.
 * scalp_server_destroy() synchronises the stream.  One server is driven by one
 * host thread. */
typedef struct scalp_server scalp_server;

size_t scalp_server_reserve_bytes(int32_t max_slots);
int scalp_server_create(scalp_server **out, void *pool, size_t pool_bytes, int32_t max_slots,
                        const scalp_params *params);
/* image/contour/K/m as scalp_init; iters >= 0; labels_out: H*W int32 host buffer
 * the caller keeps until poll reports done; *id receives the request id. */
int scalp_server_submit(scalp_server *s, const scalp_image *image, const scalp_contour *contour,
                        int32_t K, float m, int32_t iters, int32_t enforce, int32_t *labels_out,
                        uint64_t *id);
int scalp_server_step(scalp_server *s, int32_t *n_running);
/* Optional step budget: with max_pixels > 0 a step iterates only the requests
 * with the least remaining work (pixels x iterations left, ties to the
 * earlier request) whose pixels sum to at most max_pixels (always at least
 * one); the others wait for a later step.  Under a steady stream of smaller
 * requests a large one can wait indefinitely: route large requests to a
 * server of their own (e.g. on a lower-priority stream) where that matters.
 * 0 (the default) iterates every request in flight.  *n_running of
 * scalp_server_step counts those iterated. */
int scalp_server_set_step_budget(scalp_server *s, int64_t max_pixels);
/* *done = 1 once request id has been delivered or has failed; its memory is
 * then released and the id is forgotten.  A device-side check or bounded wait
 * that failed in the request's own work returns SCALP_E_INTERNAL or
 * SCALP_E_TIMEOUT with *done = 1 (its labels are not valid). */
int scalp_server_poll(scalp_server *s, uint64_t id, int32_t *done, int32_t *n_labels);
/* Fault injection for tests of the error path, on the host: when request id
 * completes, its status reads as if a device-side check had failed with
 * `error` (nonzero), or a bounded wait had given up (timeout nonzero).  No
 * GPU work is changed. */
int scalp_server_inject_status(scalp_server *s, uint64_t id, int32_t error, int32_t timeout);
int scalp_server_stats(const scalp_server *s, int32_t *in_flight, size_t *pool_free_bytes);
void scalp_server_destroy(scalp_server *s);

/* ---- Multi-scale boundary map (Sec. III-A2) -----------------------------------
 *
 * The precision-recall evaluation of the paper averages the boundary maps of
 * decompositions at several scales (12 scales from 6 to 600 superpixels) into
 * a boundary confidence map.  labels: host array of `count` device pointers
 * to H*W int32 label maps (1 <= count <= SCALP_MAX_MAPS); out: device H*W
 * float.  out[p] = (number of maps in which a 4-neighbour of p has another
 * label) / count.  Asynchronous on `stream`. */
#define SCALP_MAX_MAPS 64
int scalp_boundary_map(const int32_t *const *labels, int32_t count, int32_t H, int32_t W,
                       float *out, void *stream);

/* ---- Superpixel quality metrics (Sec. III-A2, Eq. 5-8) -------------------------
 *
 * Scores of a decomposition `labels` (values in [0, n_labels)) against a
 * ground-truth segmentation `gt` (values in [0, n_gt)), both device H*W int32.
 * Boundary pixels are pixels with a 4-neighbour of another label.
 *   br  Eq. 5, boundary recall: ground-truth boundary pixels with a superpixel
 *       boundary pixel at Euclidean distance < eps (the paper uses eps = 2)
 *   asa Eq. 6, achievable segmentation accuracy
 *   ue  Eq. 7, undersegmentation error, sum over segments and the superpixels
 *       meeting them of |S_k - G_i|, over the pixel count
 *   co  Eq. 8, compactness, the perimeter |P(S_k)| counted as pixel edges between
 *       S_k and the rest of the image (image border included)
 * The workspace (device, scalp_quality_workspace_bytes) is caller-owned; the
 * call synchronises `stream` and fills *out.  n_labels * n_gt <= 2^28. */
typedef struct {
    double br, asa, ue, co;
} scalp_quality;
size_t scalp_quality_workspace_bytes(int32_t H, int32_t W, int32_t n_labels, int32_t n_gt);
int scalp_quality_metrics(const int32_t *labels, int32_t n_labels, const int32_t *gt, int32_t n_gt,
                          int32_t H, int32_t W, double eps, void *workspace, size_t workspace_bytes,
                          scalp_quality *out, void *stream);

/* ---- An entry point that allocates nothing (no counterpart in the paper) ----
 *
 * For callers that cannot allocate device memory: code running while another
 * component owns the device memory budget, plugins handed only their input
 * and output buffers, or hosts where an allocation would synchronise the
 * device at the wrong moment.  It computes, for each label of a label map,
 * the mean CIELab colour and barycenter of its pixels (the means of the
 * cluster update, for a decomposition the caller holds), using no workspace:
 * its scratch is a fixed file-scope device array of SCALP_STATIC_MAX_LABELS
 * integer sums plus a 1 KB table, about 4 MB that every GPU loading this
 * library keeps until the process exits.  No cudaMalloc, cudaFree or other
 * allocating call is made.
 *
 *   rgb       device pointer, H rows of W*3 bytes of 8-bit sRGB
 *   rgb_stride bytes between rows; 0 means 3*W
 *   labels    device pointer, H*W int32; labels outside [0, n_labels) are skipped
 *   n_labels  1 <= n_labels <= SCALP_STATIC_MAX_LABELS, else SCALP_E_ARG
 *   out       device pointer, n_labels x 6 doubles per label:
 *             (pixel count, mean L, mean a, mean b, mean x, mean y); zeros if empty
 *   stream    cudaStream_t the work is enqueued on (asynchronous)
 *
 * The first call on each device sets up the scratch (looks up its device
 * address and fills the table, synchronising that stream once); make that
 * first call before any stream capture.  Every call shares the one scratch
 * array and clears the sums it uses, so calls that overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller.
 * Errors: SCALP_E_ARG / SCALP_E_CUDA, text via scalp_last_error(NULL). */
#define SCALP_STATIC_MAX_LABELS 65536
int scalp_label_means_static(const uint8_t *rgb, int64_t rgb_stride, const int32_t *labels,
                             int32_t H, int32_t W, int32_t n_labels, double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SCALP_H */
