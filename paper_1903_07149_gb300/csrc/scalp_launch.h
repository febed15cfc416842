// scalp_launch.h -- host-side launchers of the libscalp kernels (internal).
#pragma once

#include "scalp_internal.cuh"

typedef struct scalp_ctx scalp_ctx;

#include <utility>

namespace scalp {

// Launch with programmatic stream serialization (see pdl_wait/pdl_release):
// with pdl false it is an ordinary launch.
template <typename... Params, typename... Args>
cudaError_t pdl_launch(bool pdl, void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Sets the text scalp_last_error(NULL) returns on this thread.
void set_last_error(const char *msg);
// This thread's pinned buffer for reading device counters (NULL if pinned
// memory could not be had; the caller then copies to pageable memory).
DevCounters *pinned_status_buffer();

// Per-pixel set-up: CIELab (Sec. II-A), contour factor 1-exp(-C^2/sigma^2)
// of Eq. 2, grid label, and the grid clusters' integer sums of (1, x, y, L,
// a, b) into a.acc.  It first zeroes the sums, the counters, the tile counts
// and the list cursors.  rgb/contour are device pointers with row strides.
void launch_setup(const SolveArgs &a, const uint8_t *rgb, long long rgb_stride,
                  const float *contour, long long contour_stride, int storage,
                  void *plane, cudaStream_t st);
// The 256-entry inverse sRGB transfer function of the current device, built
// on the first request (which synchronises `st` once) in static device memory.
cudaError_t srgb_table(const float **table, cudaStream_t st);
// Contour prior from the image (CIELab gradient magnitude / its maximum) into
// out (H rows of out_stride floats); lut = the transfer-function table, gmax
// one word of scratch.  rgb and out are device pointers.
void launch_gradient_prior(const uint8_t *rgb, long long rgb_stride, int H, int W, const float *lut,
                           float *out, long long out_stride, unsigned *gmax, cudaStream_t st);
// Cluster update (Algorithm 1) from a.acc when from_acc (queueing projections,
// Eq. 4), then windows, the cluster records and the tile counts.  The tile
// counts and list cursors must be zero on entry.
void launch_update(const SolveArgs &a, int from_acc, cudaStream_t st, bool pdl = false);
// Eq. 4 for the queued clusters; whole_image=1 searches every pixel.
void launch_project(const SolveArgs &a, int whole_image, cudaStream_t st, bool pdl = false);
// Per-tile candidate lists from the tile counts (no other state is touched).
void launch_lists(const SolveArgs &a, cudaStream_t st, bool pdl = false);
// The projection and the candidate lists as one launch (when the lists'
// scan fits shared memory, project_lists_fused()).
bool project_lists_fused(const SolveArgs &a);
void launch_project_lists(const SolveArgs &a, cudaStream_t st, bool pdl = false);
// Batch: the assignment of every tile of every image in one launch, and one
// iteration's update, projection and candidate lists for every image.
void launch_assign_batch(const BatchArgs &b, int storage, int total_tiles, size_t smem_bytes,
                         cudaStream_t st, bool pdl = false);
cudaError_t assign_batch_configure(int storage);
// The persistent batched iterations (scalp_persistent.cu): the cooperative
// grid that fits (*grid = 0: not available on this device), and the launch.
cudaError_t batch_persistent_grid(int storage, size_t smem, int *grid);
cudaError_t launch_batch_persistent(const PersistArgs &q, int storage, size_t smem, int grid, cudaStream_t st);
void launch_batch_update(const BatchArgs &b, int total_clusters, int total_fill, cudaStream_t st,
                         bool pdl = false, cudaStream_t side = nullptr, cudaEvent_t fork = nullptr,
                         cudaEvent_t join = nullptr, int whole_image = 0);
// Assignment (Algorithm 1 inner loops, Eq. 1-3) with a.map_cap distance-map
// pairs per CTA; smem_bytes = assign_smem_bytes(a.map_cap).
void launch_assign(const SolveArgs &a, int storage, size_t smem_bytes, cudaStream_t st, bool pdl = false);
size_t assign_smem_bytes(int map_cap);
// Distance-map pairs that fit when ASSIGN_CTAS_PER_SM assignment CTAs share an SM.
int assign_map_capacity(int device);
cudaError_t assign_configure(int storage);
// Debug: record the pixels of M paths.
void launch_debug_paths(const int *pairs, int M, int *out_xy, int stride_xy, int *out_len,
                        int W, cudaStream_t st);

// Connectivity enforcement; returns the number of labels through *d_nlab.
struct CclBuffers {
    int *parent, *size, *link, *scan;
    int *scan_tmp;     // block sums for the multi-level scan
    long long scan_tmp_len;
};
long long ccl_scan_tmp_len(long long N);
void launch_ccl(const int *labels, int H, int W, int K, int *out, const CclBuffers &b,
                int *d_nlab, DevCounters *ctr, cudaStream_t st);

// Connectivity of a whole batch, one launch per pass.  Each pass gives every
// image a range of blocks; base[kind] (count+1 ints) is the prefix of the
// per-image block counts ccl_batch_blocks() returns.
enum { CCL_KIND_TILES, CCL_KIND_BORDER, CCL_KIND_PIXELS, CCL_KIND_QUADS, CCL_KIND_CHUNKS, CCL_KINDS };
struct CclImage {
    const int *labels;
    int *parent, *size, *link, *scan, *scan_tmp;  // the image's CclBuffers
    int *nlab;                 // receives the number of labels
    DevCounters *ctr;          // the image's counters (error flags are raised here)
    DevCounters *ctr_out;      // a copy of them once the connectivity has run
    long long N, T;            // pixels, small-component bound floor(N / (4K))
    int H, W, n_tx, n_ty;      // n_tx, n_ty: 32 x 32 tiles
};
struct CclBatch {
    const CclImage *img;
    int *const *out;           // per image: where its final labels go
    const int *base[CCL_KINDS];
    int count;
};
void ccl_batch_blocks(int H, int W, long long blocks[CCL_KINDS]);
void launch_ccl_batch(const CclBatch &cb, const int total[CCL_KINDS], cudaStream_t st);

// Set-up of a whole batch (device-side inputs of each image; contour NULL for
// none): the image's counters, cluster sums, tile counts and list cursors
// zeroed, then the per-pixel set-up of launch_setup, one launch each.
// setup_base (count+1 ints) is the prefix of setup_blocks() per image;
// zero_parts CTAs zero each image (the largest zero_blocks() of the batch).
struct SetupInput {
    const uint8_t *rgb;
    const float *contour;
    long long rgb_stride, contour_stride;
};
long long setup_blocks(int H, int W, int ny);
int zero_blocks(int Keff, int tiles);
void launch_setup_batch(const BatchArgs &b, const SetupInput *in, const int *setup_base, int total_blocks,
                        int zero_parts, int storage, cudaStream_t st);

// Per-context accessors used by the serving loop.
SolveArgs scalp_ctx_args(const scalp_ctx *c);
void scalp_ctx_set_stream(scalp_ctx *c, cudaStream_t st);  // where its own work goes
size_t scalp_ctx_smem(const scalp_ctx *c);
void scalp_ctx_count_iteration(scalp_ctx *c);
// status of a delivered solve, copied to pinned host memory behind its labels
struct CtxStatus {
    int error, timeout;  // the device-side flags (DevCounters order)
    int n_labels;
    int pad;
};
int scalp_ctx_enqueue_labels(scalp_ctx *c, int32_t *out, int enforce, CtxStatus *status);
int scalp_ctx_finish_labels(scalp_ctx *c, const CtxStatus *status, int32_t *n_labels);
void scalp_ctx_release(scalp_ctx *c);

}  // namespace scalp
