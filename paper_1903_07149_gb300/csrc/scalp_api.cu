// scalp_api.cu -- the C ABI of libscalp (declared in include/scalp.h):
// argument checks, workspace carving, kernel configuration, CUDA-graph replay
// of one iteration, state I/O.  All device work is in the kernel files.
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <new>
#include <map>
#include <string>
#include <vector>

#include "../../include/scalp.h"
#include "scalp_launch.h"

using namespace scalp;

namespace {

thread_local std::string g_last_error;

struct Layout {
    size_t rgb, contour, plane, labels, parent, size, link, scan, scan_tmp;
    size_t st_n, st_sx, st_sy, st_col, st_end, cdev, acc, proj, prev_win;
    size_t tile_count, tile_off, tile_cursor, tile_list, ctr, nlab, debug;
    size_t total;
    long long tile_cap, scan_tmp_len;
    int n_tx, n_ty, pitch;
};

constexpr size_t ALIGN = 256;
constexpr size_t DEBUG_BYTES = 1 << 20;

size_t carve(size_t &cur, size_t bytes)
{
    size_t off = (cur + ALIGN - 1) & ~(ALIGN - 1);
    cur = off + bytes;
    return off;
}

bool grid_dims(int H, int W, int K, int &nx, int &ny, double &r)
{
    double N = (double)H * (double)W;
    r = std::sqrt(N / (double)K);
    long long gx = (long long)std::floor((double)W / r + 0.5);
    long long gy = (long long)std::floor((double)H / r + 0.5);
    nx = (int)std::min<long long>(std::max<long long>(gx, 1), W);
    ny = (int)std::min<long long>(std::max<long long>(gy, 1), H);
    return true;
}

bool sizes_ok(int H, int W, int K)
{
    if (H < 1 || W < 1 || K < 1) return false;
    long long N = (long long)H * W;
    if (N > (1LL << 30)) return false;  // int32 pixel indices with headroom
    return K <= N;
}

Layout make_layout(int H, int W, int K, int storage)
{
    Layout L{};
    long long N = (long long)H * W;
    int nx, ny;
    double r;
    grid_dims(H, W, K, nx, ny, r);
    long long Keff = (long long)nx * ny;
    L.pitch = (W + 3) & ~3;
    L.n_tx = (int)ceil_div_ll(W, TILE_X);
    L.n_ty = (int)ceil_div_ll(H, TILE_Y);
    long long n_tiles = (long long)L.n_tx * L.n_ty;
    L.tile_cap = Keff * tiles_per_window(r, TILE_X) * tiles_per_window(r, TILE_Y);
    L.scan_tmp_len = ccl_scan_tmp_len(N);
    size_t elem = storage == 0 ? 16 : 8;
    size_t cur = 0;
    L.rgb = carve(cur, (size_t)N * 3);
    L.contour = carve(cur, (size_t)N * 4);
    L.plane = carve(cur, (size_t)L.pitch * H * elem);
    L.labels = carve(cur, (size_t)N * 4);
    L.parent = carve(cur, (size_t)N * 4);
    L.size = carve(cur, (size_t)N * 4);
    L.link = carve(cur, (size_t)N * 4);
    L.scan = carve(cur, (size_t)N * 4);
    L.scan_tmp = carve(cur, (size_t)L.scan_tmp_len * 4);
    L.st_n = carve(cur, Keff * 8);
    L.st_sx = carve(cur, Keff * 8);
    L.st_sy = carve(cur, Keff * 8);
    L.st_col = carve(cur, Keff * 16);
    L.st_end = carve(cur, Keff * 8);
    L.cdev = carve(cur, Keff * sizeof(ClusterDev));
    L.acc = carve(cur, Keff * sizeof(ClusterAcc));
    L.proj = carve(cur, Keff * 4);
    L.prev_win = carve(cur, Keff * 16);
    L.tile_count = carve(cur, n_tiles * 4);
    L.tile_off = carve(cur, (n_tiles + 1) * 4);
    L.tile_cursor = carve(cur, n_tiles * 4);
    L.tile_list = carve(cur, (size_t)L.tile_cap * 4);
    L.ctr = carve(cur, sizeof(DevCounters));
    L.nlab = carve(cur, 16);
    L.debug = carve(cur, DEBUG_BYTES);
    L.total = (cur + ALIGN - 1) & ~(ALIGN - 1);
    return L;
}

}  // namespace

namespace scalp {
// Sets the text scalp_last_error(NULL) returns on this thread.
void set_last_error(const char *msg) { g_last_error = msg; }

// One pinned buffer per host thread for status reads: a read is a copy and a
// synchronisation inside one call, and a context is used by one thread at a
// time.  Made on the thread's first read and freed when the thread exits, so
// that contexts made for one image each allocate nothing.
struct PinnedStatus {
    DevCounters *buf = nullptr;
    bool tried = false;
    ~PinnedStatus()
    {
        // at thread (or process) exit; a runtime already torn down is no error here
        if (buf) cudaFreeHost(buf);
    }
};

DevCounters *pinned_status_buffer()
{
    thread_local PinnedStatus t;
    if (!t.buf && !t.tried) {
        t.tried = true;
        const cudaError_t pending = cudaPeekAtLastError();
        if (cudaMallocHost(&t.buf, sizeof(DevCounters)) != cudaSuccess) {
            t.buf = nullptr;
            // clear only the error this allocation raised, not one pending before it
            if (pending == cudaSuccess) cudaGetLastError();
        }
    }
    return t.buf;
}
}  // namespace scalp

struct scalp_ctx {
    int H, W, K;
    long long N;
    float m;
    scalp_params p;
    int nx, ny, Keff;
    double r, gamma;
    cudaStream_t st;
    unsigned char *ws;
    Layout L;
    SolveArgs a;
    CclBuffers ccl;
    size_t smem;
    cudaGraphExec_t gexec;
    bool graph_valid;
    int graph_n;           // iterations in the captured graph
    bool graph_prof;       // graph records the profiling events
    bool profiling;
    std::vector<cudaEvent_t> ev_pool;  // pairs around each assignment launch
    cudaStream_t side;     // captured iterations: the lists beside the projection
    cudaEvent_t fork_ev, join_ev;
    int prof_pending;      // event pairs recorded and not yet read
    double prof_ms;
    long long prof_launches;
    int iterations;
    std::string err;
};

namespace {

int fail(scalp_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    g_last_error = buf;
    return code;
}

int cuda_check(scalp_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return SCALP_OK;
    return fail(c, SCALP_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int launch_check(scalp_ctx *c, const char *what) { return cuda_check(c, cudaGetLastError(), what); }

// Reads the device counters after a synchronisation; reports device-side failures.
// The counters go to the thread's pinned status buffer (a pageable copy when
// there is none): one asynchronous copy and one synchronisation, where a
// pageable destination would cost a round trip of its own.  n_labels (if not
// NULL) receives the label count the last connectivity enforcement wrote.
int device_status(scalp_ctx *c, int *n_labels = nullptr)
{
    DevCounters local;
    DevCounters *h = pinned_status_buffer();
    if (!h) h = &local;
    int rc = cuda_check(c, cudaMemcpyAsync(h, c->a.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->st),
                        "read device counters");
    if (rc) return rc;
    rc = cuda_check(c, cudaStreamSynchronize(c->st), "synchronise");
    if (rc) return rc;
    if (h->timeout) return fail(c, SCALP_E_TIMEOUT, "a bounded device-side wait gave up");
    if (h->error) return fail(c, SCALP_E_INTERNAL, "device-side check failed (code %d)", h->error);
    if (n_labels) *n_labels = h->n_labels;
    return SCALP_OK;
}

// Tile counts and list cursors start at zero before an update (the
// assignment kernel re-zeroes each tile's pair after reading its list).
// floor(v * cells / len) for 0 <= v < len equals the high word of
// (v * cells) * ceil(2^32 / len) when (len - 1) * cells * len < 2^32: with
// m = ceil(2^32 / len) = (2^32 + e) / len, 0 <= e < len, the product exceeds
// v * cells / len by (v * cells) * e / (len * 2^32) < 1 / len, less than the
// distance of v * cells / len to the next integer.  0 where that does not hold.
unsigned grid_reciprocal(long long len, long long cells)
{
    if (len < 2) return 0;
    const unsigned long long num = (unsigned long long)(len - 1) * (unsigned long long)cells;
    if (num > 0xffffffffULL / (unsigned long long)len) return 0;
    return (unsigned)((0x100000000ULL + (unsigned long long)len - 1) / (unsigned long long)len);
}

int zero_tile_counts(scalp_ctx *c)
{
    const size_t bytes = sizeof(int) * (size_t)c->L.n_tx * c->L.n_ty;
    int rc = cuda_check(c, cudaMemsetAsync(c->a.tile_count, 0, bytes, c->st), "memset");
    return rc ? rc : cuda_check(c, cudaMemsetAsync(c->a.tile_cursor, 0, bytes, c->st), "memset");
}

// The inputs of the set-up on the device: the image (and contour) copied into
// the workspace when they are on the host; the gradient prior computed from
// the image when the context uses it.
int stage_inputs(scalp_ctx *c, const scalp_image *img, const scalp_contour *con, SetupInput *in)
{
    const uint8_t *rgb = img->rgb;
    long long rs = img->rgb_stride ? img->rgb_stride : 3LL * c->W;
    const float *cp = con ? con->data : nullptr;
    long long cs = (con && con->stride) ? con->stride : c->W;
    int rc;
    if (!img->on_device) {
        uint8_t *d_rgb = c->ws + c->L.rgb;
        rc = cuda_check(c, cudaMemcpy2DAsync(d_rgb, 3 * (size_t)c->W, rgb, (size_t)rs, 3 * (size_t)c->W,
                                             c->H, cudaMemcpyHostToDevice, c->st),
                        "copy image to device");
        if (rc) return rc;
        rgb = d_rgb;
        rs = 3LL * c->W;
        if (cp) {
            float *d_c = reinterpret_cast<float *>(c->ws + c->L.contour);
            rc = cuda_check(c, cudaMemcpy2DAsync(d_c, 4 * (size_t)c->W, cp, 4 * (size_t)cs,
                                                 4 * (size_t)c->W, c->H, cudaMemcpyHostToDevice, c->st),
                            "copy contour to device");
            if (rc) return rc;
            cp = d_c;
            cs = c->W;
        }
    }
    if (c->p.prior == SCALP_PRIOR_GRADIENT) {
        // the prior computed from the image, into the contour staging area
        float *d_c = reinterpret_cast<float *>(c->ws + c->L.contour);
        launch_gradient_prior(rgb, rs, c->H, c->W, c->a.lut, d_c, c->W, &c->a.ctr->prior_max, c->st);
        rc = launch_check(c, "gradient prior");
        if (rc) return rc;
        cp = d_c;
        cs = c->W;
    }
    *in = SetupInput{rgb, cp, rs, cs};
    return SCALP_OK;
}

int load_inputs(scalp_ctx *c, const scalp_image *img, const scalp_contour *con)
{
    SetupInput in;
    int rc = stage_inputs(c, img, con, &in);
    if (rc) return rc;
    void *plane = c->ws + c->L.plane;
    // zeroing of the sums and counters, set-up (with the grid clusters'
    // sums), then the initial update, projection and lists, as programmatic
    // launches (each waits for its predecessor before its first read)
    launch_setup(c->a, in.rgb, in.rgb_stride, in.contour, in.contour_stride, c->p.storage, plane, c->st);
    launch_update(c->a, 1, c->st, true);
    launch_project(c->a, 1, c->st, true);
    launch_lists(c->a, c->st, true);
    c->iterations = 0;
    return launch_check(c, "initialisation kernels");
}

int validate_image(const scalp_image *img, const scalp_contour *con, const char **why)
{
    if (!img || !img->rgb) { *why = "image or image->rgb is NULL"; return 0; }
    if (img->H < 1 || img->W < 1) { *why = "image size must be at least 1 x 1"; return 0; }
    if (img->rgb_stride != 0 && img->rgb_stride < 3LL * img->W) { *why = "rgb_stride < 3*W"; return 0; }
    if (con && con->data && con->stride != 0 && con->stride < img->W) { *why = "contour stride < W"; return 0; }
    return 1;
}

// The checks of a reload: a valid image of the context's size, and no
// contour where the context computes its own prior.
int check_reload(scalp_ctx *c, const scalp_image *image, const scalp_contour *contour)
{
    const char *why = nullptr;
    if (!validate_image(image, contour, &why)) return fail(c, SCALP_E_ARG, "%s", why);
    if (c->p.prior == SCALP_PRIOR_GRADIENT && contour && contour->data)
        return fail(c, SCALP_E_ARG, "a contour was given with SCALP_PRIOR_GRADIENT");
    if (image->H != c->H || image->W != c->W)
        return fail(c, SCALP_E_ARG, "reload needs the same image size");
    return SCALP_OK;
}

int ensure_events(scalp_ctx *c, size_t pairs)
{
    while (c->ev_pool.size() < 2 * pairs) {
        cudaEvent_t e;
        int rc = cuda_check(c, cudaEventCreate(&e), "create event");
        if (rc) return rc;
        c->ev_pool.push_back(e);
    }
    return SCALP_OK;
}

// Adds the durations of the recorded assignment launches to the totals.
int harvest_profile(scalp_ctx *c)
{
    if (c->prof_pending == 0) return SCALP_OK;
    int rc = cuda_check(c, cudaStreamSynchronize(c->st), "synchronise");
    if (rc) return rc;
    for (int i = 0; i < c->prof_pending; ++i) {
        float t = 0.f;
        rc = cuda_check(c, cudaEventElapsedTime(&t, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]),
                        "event time");
        if (rc) return rc;
        c->prof_ms += t;
        c->prof_launches += 1;
    }
    c->prof_pending = 0;
    return SCALP_OK;
}

// One iteration of Algorithm 1; with profiling, event pair `slot` brackets
// the assignment kernel.  Under stream capture the records must be external
// so that they become event-record nodes of the graph.
void enqueue_iteration(scalp_ctx *c, int slot, bool capturing)
{
    const unsigned flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (c->profiling) cudaEventRecordWithFlags(c->ev_pool[2 * slot], c->st, flags);
    // programmatic launches overlap each kernel's placement with the drain of
    // the one before (not across the profiling event records)
    const bool pdl = !c->profiling;
    launch_assign(c->a, c->p.storage, c->smem, c->st, pdl);
    if (c->profiling) cudaEventRecordWithFlags(c->ev_pool[2 * slot + 1], c->st, flags);
    launch_update(c->a, 1, c->st, pdl);
    if (project_lists_fused(c->a)) {
        // the projection and the candidate lists in one launch
        launch_project_lists(c->a, c->st, pdl);
    } else if (capturing && c->side) {
        // the candidate lists need only the windows the update wrote, not the
        // projected endpoints: a second branch of the graph runs them beside
        // the projection, and the next assignment waits for both
        cudaEventRecord(c->fork_ev, c->st);
        cudaStreamWaitEvent(c->side, c->fork_ev, 0);
        launch_lists(c->a, c->side, false);
        cudaEventRecord(c->join_ev, c->side);
        launch_project(c->a, 0, c->st, pdl);
        cudaStreamWaitEvent(c->st, c->join_ev, 0);
    } else {
        launch_project(c->a, 0, c->st, pdl);
        launch_lists(c->a, c->st, pdl);
    }
}

// The second stream and the fork/join events of captured iterations, made
// before a capture begins (none: the iterations stay in one stream).
void ensure_side_stream(scalp_ctx *c)
{
    if (c->side) return;
    int prio = 0;
    cudaStream_t t = nullptr;
    cudaEvent_t f = nullptr, j = nullptr;
    if (cudaStreamGetPriority(c->st, &prio) == cudaSuccess &&
        cudaStreamCreateWithPriority(&t, cudaStreamNonBlocking, prio) == cudaSuccess &&
        cudaEventCreateWithFlags(&f, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&j, cudaEventDisableTiming) == cudaSuccess) {
        c->side = t;
        c->fork_ev = f;
        c->join_ev = j;
        return;
    }
    if (t) cudaStreamDestroy(t);
    if (f) cudaEventDestroy(f);
    if (j) cudaEventDestroy(j);
    cudaGetLastError();  // not sticky: the iterations run in one stream
}

// Host-side resources of a context (its enqueued work has completed).
void free_ctx(scalp_ctx *c)
{
    if (c->graph_valid) cudaGraphExecDestroy(c->gexec);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->side) {
        cudaStreamDestroy(c->side);
        cudaEventDestroy(c->fork_ev);
        cudaEventDestroy(c->join_ev);
    }
    delete c;
}

}  // namespace

extern "C" {

void scalp_default_params(scalp_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->lambda = 0.5f;
    p->sigma = 0.25f;
    p->gamma = -1.0f;
    p->storage = SCALP_STORAGE_F32;
    p->use_graph = 1;
    p->global_walk = 0;
}

size_t scalp_workspace_bytes(int32_t H, int32_t W, int32_t K, const scalp_params *p)
{
    if (!sizes_ok(H, W, K)) return 0;
    int storage = p ? p->storage : 0;
    if (storage != 0 && storage != 1) return 0;
    return make_layout(H, W, K, storage).total;
}

int scalp_init(scalp_ctx **out, const scalp_image *image, const scalp_contour *contour, int32_t K,
               float m, const scalp_params *params)
{
    const char *why = nullptr;
    if (!out) return fail(nullptr, SCALP_E_ARG, "out is NULL");
    *out = nullptr;
    if (!params) return fail(nullptr, SCALP_E_ARG, "params is NULL");
    if (!validate_image(image, contour, &why)) return fail(nullptr, SCALP_E_ARG, "%s", why);
    if (params->prior != SCALP_PRIOR_INPUT && params->prior != SCALP_PRIOR_GRADIENT)
        return fail(nullptr, SCALP_E_ARG, "params->prior must be SCALP_PRIOR_INPUT or SCALP_PRIOR_GRADIENT");
    if (params->prior == SCALP_PRIOR_GRADIENT && contour && contour->data)
        return fail(nullptr, SCALP_E_ARG, "a contour was given with SCALP_PRIOR_GRADIENT");
    if (!sizes_ok(image->H, image->W, K))
        return fail(nullptr, SCALP_E_ARG, "need H, W >= 1, H*W <= 2^30 and 1 <= K <= H*W");
    if (!(m > 0.0f) || !std::isfinite(m)) return fail(nullptr, SCALP_E_ARG, "m must be > 0");
    if (!(params->lambda >= 0.0f && params->lambda <= 1.0f))
        return fail(nullptr, SCALP_E_ARG, "lambda must be in [0, 1]");
    if (!(params->sigma > 0.0f) || !std::isfinite(params->sigma))
        return fail(nullptr, SCALP_E_ARG, "sigma must be > 0");
    if (!std::isfinite(params->gamma)) return fail(nullptr, SCALP_E_ARG, "gamma must be finite");
    if (params->storage != 0 && params->storage != 1)
        return fail(nullptr, SCALP_E_ARG, "storage must be SCALP_STORAGE_F32 or _F16");
    const int H = image->H, W = image->W;
    Layout L = make_layout(H, W, K, params->storage);
    if (!params->workspace || params->workspace_bytes < L.total)
        return fail(nullptr, SCALP_E_NOMEM, "workspace of %zu bytes needed, %zu given", L.total,
                    params->workspace ? params->workspace_bytes : (size_t)0);
    if (reinterpret_cast<uintptr_t>(params->workspace) % ALIGN)
        return fail(nullptr, SCALP_E_ARG, "workspace must be 256-byte aligned");

    scalp_ctx *c = new (std::nothrow) scalp_ctx();
    if (!c) return fail(nullptr, SCALP_E_NOMEM, "host allocation failed");
    c->H = H; c->W = W; c->K = K; c->N = (long long)H * W; c->m = m;
    c->p = *params;
    grid_dims(H, W, K, c->nx, c->ny, c->r);
    c->Keff = c->nx * c->ny;
    c->gamma = params->gamma < 0 ? 2.0 * c->r : (double)params->gamma;
    c->st = reinterpret_cast<cudaStream_t>(params->stream);
    c->ws = reinterpret_cast<unsigned char *>(params->workspace);
    c->L = L;

    SolveArgs &a = c->a;
    std::memset(&a, 0, sizeof a);
    a.H = H; a.W = W; a.K = K; a.Keff = c->Keff; a.nx = c->nx; a.ny = c->ny; a.N = c->N;
    a.r = c->r;
    a.lam = params->lambda;
    a.gamma = (float)c->gamma;
    a.sigma = params->sigma;
    a.ms2 = (float)((double)m * (double)m * (double)K / (double)c->N);  // m^2 / r^2
    a.n_tx = L.n_tx; a.n_ty = L.n_ty;
    a.pitch = L.pitch;
    a.grid_rcp_x = grid_reciprocal(W, c->nx);
    a.plane32 = params->storage == 0 ? reinterpret_cast<const float4 *>(c->ws + L.plane) : nullptr;
    a.plane16 = params->storage == 1 ? reinterpret_cast<const uint2 *>(c->ws + L.plane) : nullptr;
    a.labels = reinterpret_cast<int *>(c->ws + L.labels);
    a.st_n = reinterpret_cast<long long *>(c->ws + L.st_n);
    a.st_sx = reinterpret_cast<long long *>(c->ws + L.st_sx);
    a.st_sy = reinterpret_cast<long long *>(c->ws + L.st_sy);
    a.st_col = reinterpret_cast<float4 *>(c->ws + L.st_col);
    a.st_end = reinterpret_cast<int2 *>(c->ws + L.st_end);
    a.cdev = reinterpret_cast<ClusterDev *>(c->ws + L.cdev);
    a.acc = reinterpret_cast<ClusterAcc *>(c->ws + L.acc);
    a.proj_list = reinterpret_cast<int *>(c->ws + L.proj);
    a.tile_count = reinterpret_cast<int *>(c->ws + L.tile_count);
    a.tile_off = reinterpret_cast<int *>(c->ws + L.tile_off);
    a.tile_cursor = reinterpret_cast<int *>(c->ws + L.tile_cursor);
    a.tile_list = reinterpret_cast<int *>(c->ws + L.tile_list);
    a.tile_cap = L.tile_cap;
    a.tpw_x = tiles_per_window(c->r, TILE_X);
    a.tpw_y = tiles_per_window(c->r, TILE_Y);
    a.prev_win = reinterpret_cast<int4 *>(c->ws + L.prev_win);
    a.ctr = reinterpret_cast<DevCounters *>(c->ws + L.ctr);
    c->ccl.parent = reinterpret_cast<int *>(c->ws + L.parent);
    c->ccl.size = reinterpret_cast<int *>(c->ws + L.size);
    c->ccl.link = reinterpret_cast<int *>(c->ws + L.link);
    c->ccl.scan = reinterpret_cast<int *>(c->ws + L.scan);
    c->ccl.scan_tmp = reinterpret_cast<int *>(c->ws + L.scan_tmp);
    c->ccl.scan_tmp_len = L.scan_tmp_len;

    // distance maps of the assignment CTAs (none: every path walks the plane)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    a.map_cap = (params->global_walk & 1) ? 0 : assign_map_capacity(dev);
    a.prune = (params->global_walk & 2) ? 0 : 1;
    c->smem = assign_smem_bytes(a.map_cap);
    int rc = cuda_check(c, assign_configure(params->storage), "configure kernel");
    if (rc == SCALP_OK) rc = cuda_check(c, srgb_table(&a.lut, c->st), "transfer-function table");
    if (rc == SCALP_OK) rc = load_inputs(c, image, contour);
    if (rc != SCALP_OK) {
        delete c;
        return rc;
    }
    *out = c;
    return SCALP_OK;
}

int scalp_reload(scalp_ctx *c, const scalp_image *image, const scalp_contour *contour)
{
    if (!c) return fail(nullptr, SCALP_E_ARG, "ctx is NULL");
    const int rc = check_reload(c, image, contour);
    return rc ? rc : load_inputs(c, image, contour);
}

int scalp_iterate(scalp_ctx *c, int32_t n)
{
    if (!c) return fail(nullptr, SCALP_E_ARG, "ctx is NULL");
    if (n < 0) return fail(c, SCALP_E_ARG, "n must be >= 0");
    if (n == 0) return SCALP_OK;
    int rc;
    if (c->profiling) {
        rc = harvest_profile(c);  // the events are about to be re-recorded
        if (rc) return rc;
        rc = ensure_events(c, (size_t)n);
        if (rc) return rc;
    }
    const bool graphs = c->p.use_graph && c->st != nullptr;
    if (graphs && !(c->graph_valid && c->graph_n == n && c->graph_prof == c->profiling)) {
        if (c->graph_valid) {
            cudaGraphExecDestroy(c->gexec);
            c->graph_valid = false;
        }
        ensure_side_stream(c);
        cudaGraph_t g;
        rc = cuda_check(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal),
                        "begin capture");
        if (rc) return rc;
        for (int i = 0; i < n; ++i) enqueue_iteration(c, i, true);
        cudaError_t le = cudaGetLastError();
        rc = cuda_check(c, cudaStreamEndCapture(c->st, &g), "end capture");
        if (rc) return rc;
        if (le != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_check(c, le, "capture iterations");
        }
        rc = cuda_check(c, cudaGraphInstantiate(&c->gexec, g, 0), "instantiate graph");
        cudaGraphDestroy(g);
        if (rc) return rc;
        c->graph_valid = true;
        c->graph_n = n;
        c->graph_prof = c->profiling;
    }
    if (graphs) {
        rc = cuda_check(c, cudaGraphLaunch(c->gexec, c->st), "launch graph");
        if (rc) return rc;
    } else {
        for (int i = 0; i < n; ++i) enqueue_iteration(c, i, false);
        rc = launch_check(c, "iteration kernels");
        if (rc) return rc;
    }
    if (c->profiling) c->prof_pending = n;
    c->iterations += n;
    return SCALP_OK;
}

int scalp_labels(scalp_ctx *c, int32_t *out, int32_t out_on_device, int32_t enforce,
                 int32_t *n_labels)
{
    if (!c) return fail(nullptr, SCALP_E_ARG, "ctx is NULL");
    if (!out) return fail(c, SCALP_E_ARG, "out is NULL");
    int rc;
    int nlab = c->Keff;
    size_t bytes = sizeof(int) * (size_t)c->N;
    if (enforce) {
        // the final labels go straight to a device output (which must not alias
        // the workspace), else to the link buffer, free once the links are
        // resolved, and from there to the host
        int *dst = out_on_device ? out : c->ccl.link;
        int *d_nlab = &c->a.ctr->n_labels;  // read back with the counters
        launch_ccl(c->a.labels, c->H, c->W, c->K, dst, c->ccl, d_nlab, c->a.ctr, c->st);
        rc = launch_check(c, "connectivity kernels");
        if (rc) return rc;
        if (!out_on_device) {
            rc = cuda_check(c, cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, c->st),
                            "copy labels");
            if (rc) return rc;
        }
    } else {
        rc = cuda_check(c, cudaMemcpyAsync(out, c->a.labels, bytes,
                                           out_on_device ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyDeviceToHost,
                                           c->st),
                        "copy labels");
        if (rc) return rc;
    }
    rc = device_status(c, enforce ? &nlab : nullptr);
    if (rc) return rc;
    if (n_labels) *n_labels = nlab;
    return SCALP_OK;
}

int scalp_get_info(const scalp_ctx *c, scalp_info *info)
{
    if (!c || !info) return fail(nullptr, SCALP_E_ARG, "ctx or info is NULL");
    info->H = c->H; info->W = c->W; info->K = c->K;
    info->nx = c->nx; info->ny = c->ny; info->Keff = c->Keff;
    info->r = c->r; info->gamma = c->gamma;
    info->map_pairs = c->a.map_cap;
    info->iterations = c->iterations;
    return SCALP_OK;
}

int scalp_get_state(scalp_ctx *c, const scalp_state *s)
{
    if (!c || !s) return fail(nullptr, SCALP_E_ARG, "ctx or state is NULL");
    if (!s->labels || !s->n || !s->sx || !s->sy || !s->color || !s->endpoint)
        return fail(c, SCALP_E_ARG, "state arrays must all be given");
    const size_t K = c->Keff;
    std::vector<float4> col(K);
    std::vector<int2> end(K);
    int rc = 0;
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(s->labels, c->a.labels, 4 * (size_t)c->N,
                                                 cudaMemcpyDeviceToHost, c->st), "copy state");
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(s->n, c->a.st_n, 8 * K, cudaMemcpyDeviceToHost, c->st), "copy state");
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(s->sx, c->a.st_sx, 8 * K, cudaMemcpyDeviceToHost, c->st), "copy state");
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(s->sy, c->a.st_sy, 8 * K, cudaMemcpyDeviceToHost, c->st), "copy state");
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(col.data(), c->a.st_col, 16 * K, cudaMemcpyDeviceToHost, c->st), "copy state");
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(end.data(), c->a.st_end, 8 * K, cudaMemcpyDeviceToHost, c->st), "copy state");
    if (rc) return rc;
    rc = device_status(c);
    if (rc) return rc;
    for (size_t k = 0; k < K; ++k) {
        s->color[3 * k] = col[k].x;
        s->color[3 * k + 1] = col[k].y;
        s->color[3 * k + 2] = col[k].z;
        s->endpoint[2 * k] = end[k].x;
        s->endpoint[2 * k + 1] = end[k].y;
    }
    return SCALP_OK;
}

int scalp_clusters(scalp_ctx *c, float *out, int32_t *K_eff)
{
    if (!c || !out || !K_eff) return fail(c, SCALP_E_ARG, "ctx, out and K_eff are required");
    const size_t K = c->Keff;
    std::vector<float4> col(K);
    std::vector<long long> n(K), sx(K), sy(K);
    int rc = 0;
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(col.data(), c->a.st_col, 16 * K, cudaMemcpyDeviceToHost, c->st), "copy clusters");
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(n.data(), c->a.st_n, 8 * K, cudaMemcpyDeviceToHost, c->st), "copy clusters");
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(sx.data(), c->a.st_sx, 8 * K, cudaMemcpyDeviceToHost, c->st), "copy clusters");
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(sy.data(), c->a.st_sy, 8 * K, cudaMemcpyDeviceToHost, c->st), "copy clusters");
    if (rc) return rc;
    rc = device_status(c);
    if (rc) return rc;
    for (size_t k = 0; k < K; ++k) {
        float *o = out + 5 * k;
        o[0] = col[k].x;
        o[1] = col[k].y;
        o[2] = col[k].z;
        // X_k = (Sx/n, Sy/n) from the exact integer sums, rounded once
        o[3] = (float)((double)sx[k] / (double)n[k]);
        o[4] = (float)((double)sy[k] / (double)n[k]);
    }
    *K_eff = c->Keff;
    return SCALP_OK;
}

int scalp_set_state(scalp_ctx *c, const scalp_state *s)
{
    if (!c || !s) return fail(nullptr, SCALP_E_ARG, "ctx or state is NULL");
    if (!s->labels || !s->n || !s->sx || !s->sy || !s->color || !s->endpoint)
        return fail(c, SCALP_E_ARG, "state arrays must all be given");
    const size_t K = c->Keff;
    for (long long p = 0; p < c->N; ++p)
        if (s->labels[p] < 0 || s->labels[p] >= c->Keff)
            return fail(c, SCALP_E_ARG, "label %d at pixel %lld out of range", s->labels[p], p);
    std::vector<float4> col(K);
    std::vector<int2> end(K);
    for (size_t k = 0; k < K; ++k) {
        long long n = s->n[k];
        if (n < 1 || n > c->N || s->sx[k] < 0 || s->sy[k] < 0 || s->sx[k] > (long long)(c->W - 1) * n ||
            s->sy[k] > (long long)(c->H - 1) * n)
            return fail(c, SCALP_E_ARG, "cluster %zu: bad n / coordinate sums", k);
        int ex = s->endpoint[2 * k], ey = s->endpoint[2 * k + 1];
        if (ex < 0 || ex >= c->W || ey < 0 || ey >= c->H)
            return fail(c, SCALP_E_ARG, "cluster %zu: endpoint outside the image", k);
        double L = s->color[3 * k], A = s->color[3 * k + 1], B = s->color[3 * k + 2];
        if (!std::isfinite(L) || !std::isfinite(A) || !std::isfinite(B))
            return fail(c, SCALP_E_ARG, "cluster %zu: colour not finite", k);
        col[k] = make_float4((float)L, (float)A, (float)B, 0.f);
        end[k] = make_int2(ex, ey);
    }
    int rc = 0;
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(c->a.labels, s->labels, 4 * (size_t)c->N,
                                                 cudaMemcpyHostToDevice, c->st), "copy state");
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(c->a.st_n, s->n, 8 * K, cudaMemcpyHostToDevice, c->st), "copy state");
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(c->a.st_sx, s->sx, 8 * K, cudaMemcpyHostToDevice, c->st), "copy state");
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(c->a.st_sy, s->sy, 8 * K, cudaMemcpyHostToDevice, c->st), "copy state");
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(c->a.st_col, col.data(), 16 * K, cudaMemcpyHostToDevice, c->st), "copy state");
    rc = rc ? rc : cuda_check(c, cudaMemcpyAsync(c->a.st_end, end.data(), 8 * K, cudaMemcpyHostToDevice, c->st), "copy state");
    rc = rc ? rc : cuda_check(c, cudaMemsetAsync(c->a.acc, 0, sizeof(ClusterAcc) * K, c->st), "memset");
    rc = rc ? rc : zero_tile_counts(c);
    if (rc) return rc;
    launch_update(c->a, 0, c->st);
    launch_lists(c->a, c->st);
    rc = launch_check(c, "derive kernels");
    if (rc) return rc;
    // the host vectors must outlive the copies
    return device_status(c);
}

int scalp_debug_paths(scalp_ctx *c, const int32_t *pairs, int32_t M, int32_t *out_xy,
                      int32_t stride_xy, int32_t *out_len)
{
    if (!c) return fail(nullptr, SCALP_E_ARG, "ctx is NULL");
    if (M < 0 || (M > 0 && (!pairs || !out_xy || !out_len)) || stride_xy < 2)
        return fail(c, SCALP_E_ARG, "bad debug_paths arguments");
    for (int i = 0; i < M; ++i) {
        const int32_t *q = pairs + 4 * (size_t)i;
        if (q[0] < 0 || q[0] >= c->W || q[2] < 0 || q[2] >= c->W || q[1] < 0 || q[1] >= c->H ||
            q[3] < 0 || q[3] >= c->H)
            return fail(c, SCALP_E_ARG, "pair %d outside the image", i);
    }
    const size_t per = (size_t)(4 + stride_xy + 1) * 4;
    const int chunk = (int)std::max<size_t>(1, DEBUG_BYTES / per);
    if ((size_t)chunk * per > DEBUG_BYTES) return fail(c, SCALP_E_ARG, "stride_xy too large");
    int *d_pairs = reinterpret_cast<int *>(c->ws + c->L.debug);
    int *d_xy = d_pairs + 4 * (size_t)chunk;
    int *d_len = d_xy + (size_t)chunk * stride_xy;
    for (int b = 0; b < M; b += chunk) {
        int m = std::min(chunk, M - b);
        int rc = cuda_check(c, cudaMemcpyAsync(d_pairs, pairs + 4 * (size_t)b, 16 * (size_t)m,
                                               cudaMemcpyHostToDevice, c->st), "copy pairs");
        if (rc) return rc;
        launch_debug_paths(d_pairs, m, d_xy, stride_xy, d_len, c->W, c->st);
        rc = launch_check(c, "debug kernel");
        if (rc) return rc;
        rc = cuda_check(c, cudaMemcpyAsync(out_xy + (size_t)b * stride_xy, d_xy,
                                           4 * (size_t)m * stride_xy, cudaMemcpyDeviceToHost, c->st),
                        "copy paths");
        if (rc) return rc;
        rc = cuda_check(c, cudaMemcpyAsync(out_len + b, d_len, 4 * (size_t)m, cudaMemcpyDeviceToHost,
                                           c->st), "copy lengths");
        if (rc) return rc;
        rc = cuda_check(c, cudaStreamSynchronize(c->st), "synchronise");
        if (rc) return rc;
    }
    return SCALP_OK;
}

int scalp_profile(scalp_ctx *c, int32_t enable, double *ms, int64_t *launches)
{
    if (!c) return fail(nullptr, SCALP_E_ARG, "ctx is NULL");
    int rc = harvest_profile(c);
    if (rc) return rc;
    if (ms) *ms = c->prof_ms;
    if (launches) *launches = c->prof_launches;
    if (enable >= 0) {
        bool on = enable != 0;
        if (on) {
            c->prof_ms = 0;
            c->prof_launches = 0;
        }
        c->profiling = on;
    }
    return SCALP_OK;
}

int scalp_count_samples(scalp_ctx *c, int32_t enable, int64_t *samples, int64_t *pairs,
                        int64_t *map_rects, int64_t *plane_rects)
{
    if (!c) return fail(nullptr, SCALP_E_ARG, "ctx is NULL");
    DevCounters h;
    int rc = cuda_check(c, cudaMemcpyAsync(&h, c->a.ctr, sizeof h, cudaMemcpyDeviceToHost, c->st),
                        "read counters");
    if (rc) return rc;
    rc = cuda_check(c, cudaStreamSynchronize(c->st), "synchronise");
    if (rc) return rc;
    if (samples) *samples = (int64_t)h.samples;
    if (pairs) *pairs = (int64_t)h.pairs;
    if (map_rects) *map_rects = (int64_t)h.map_rects;
    if (plane_rects) *plane_rects = (int64_t)h.plane_rects;
    if (enable >= 0) {
        int on = enable != 0;
        if (on) {
            // samples, pairs, map_rects, plane_rects are consecutive
            unsigned long long z[4] = {0, 0, 0, 0};
            rc = cuda_check(c, cudaMemcpyAsync(&c->a.ctr->samples, z, sizeof z, cudaMemcpyHostToDevice,
                                               c->st), "reset counters");
            if (rc) return rc;
            rc = cuda_check(c, cudaStreamSynchronize(c->st), "synchronise");
            if (rc) return rc;
        }
        if (c->a.count_samples != on) {
            c->a.count_samples = on;
            if (c->graph_valid) {
                cudaGraphExecDestroy(c->gexec);
                c->graph_valid = false;
            }
        }
    }
    return SCALP_OK;
}

int scalp_sync(scalp_ctx *c)
{
    if (!c) return fail(nullptr, SCALP_E_ARG, "ctx is NULL");
    int rc = launch_check(c, "pending launch");
    if (rc) return rc;
    return device_status(c);
}

const char *scalp_last_error(const scalp_ctx *c)
{
    if (c) return c->err.c_str();
    return g_last_error.c_str();
}

void scalp_destroy(scalp_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->st);  // a side branch joins back into this stream
    free_ctx(c);
}


size_t scalp_gradient_prior_workspace_bytes(int32_t H, int32_t W, int32_t image_on_device,
                                            int32_t out_on_device)
{
    if (H < 1 || W < 1 || (long long)H * W > (1LL << 30)) return 0;
    const size_t N = (size_t)H * W;
    size_t cur = 0;
    carve(cur, 16);  // the running maximum
    if (!image_on_device) carve(cur, 3 * N);
    if (!out_on_device) carve(cur, 4 * N);
    return (cur + ALIGN - 1) & ~(ALIGN - 1);
}

int scalp_gradient_prior(const scalp_image *image, float *out, int64_t out_stride,
                         int32_t out_on_device, void *stream, void *workspace,
                         size_t workspace_bytes)
{
    const char *why = nullptr;
    if (!validate_image(image, nullptr, &why)) return fail(nullptr, SCALP_E_ARG, "%s", why);
    if (!out) return fail(nullptr, SCALP_E_ARG, "out is NULL");
    const int H = image->H, W = image->W;
    if (out_stride == 0) out_stride = W;
    if (out_stride < W) return fail(nullptr, SCALP_E_ARG, "out_stride < W");
    const size_t need = scalp_gradient_prior_workspace_bytes(H, W, image->on_device, out_on_device);
    if (need == 0) return fail(nullptr, SCALP_E_ARG, "invalid image size");
    if (!workspace || workspace_bytes < need)
        return fail(nullptr, SCALP_E_NOMEM, "gradient prior workspace of %zu bytes needed", need);
    if (reinterpret_cast<uintptr_t>(workspace) % ALIGN)
        return fail(nullptr, SCALP_E_ARG, "workspace must be 256-byte aligned");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *ws = reinterpret_cast<unsigned char *>(workspace);
    const size_t N = (size_t)H * W;
    size_t cur = 0;
    const size_t o_max = carve(cur, 16);
    const size_t o_rgb = image->on_device ? 0 : carve(cur, 3 * N);
    const size_t o_out = out_on_device ? 0 : carve(cur, 4 * N);
    unsigned *gmax = reinterpret_cast<unsigned *>(ws + o_max);
    const float *lut = nullptr;
    const uint8_t *rgb = image->rgb;
    long long rs = image->rgb_stride ? image->rgb_stride : 3LL * W;
    cudaError_t e = srgb_table(&lut, st);
    if (e == cudaSuccess && !image->on_device) {
        e = cudaMemcpy2DAsync(ws + o_rgb, 3 * (size_t)W, rgb, (size_t)rs, 3 * (size_t)W, H,
                              cudaMemcpyHostToDevice, st);
        rgb = ws + o_rgb;
        rs = 3LL * W;
    }
    float *d_out = out_on_device ? out : reinterpret_cast<float *>(ws + o_out);
    const long long d_stride = out_on_device ? out_stride : W;
    if (e == cudaSuccess) {
        launch_gradient_prior(rgb, rs, H, W, lut, d_out, d_stride, gmax, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !out_on_device) {
        e = cudaMemcpy2DAsync(out, (size_t)out_stride * 4, d_out, 4 * (size_t)W, 4 * (size_t)W, H,
                              cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return fail(nullptr, SCALP_E_CUDA, "gradient prior: %s", cudaGetErrorString(e));
    return SCALP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Accessors for the serving loop (scalp_server.cu), which keeps one context
// per request in flight.
// ---------------------------------------------------------------------------
namespace scalp {

SolveArgs scalp_ctx_args(const scalp_ctx *c) { return c->a; }
void scalp_ctx_set_stream(scalp_ctx *c, cudaStream_t st) { c->st = st; }
size_t scalp_ctx_smem(const scalp_ctx *c) { return c->smem; }
void scalp_ctx_count_iteration(scalp_ctx *c) { c->iterations += 1; }

// Enqueues the connectivity enforcement (if enforce), the copy of the labels
// to host memory `out` and the copy of the solve's status (label count and the
// device-side error flags) to pinned host memory `status`; no synchronisation.
int scalp_ctx_enqueue_labels(scalp_ctx *c, int32_t *out, int enforce, CtxStatus *status)
{
    const size_t bytes = sizeof(int) * (size_t)c->N;
    const int *src = c->a.labels;
    const int *d_nlab = reinterpret_cast<const int *>(c->ws + c->L.nlab);
    if (enforce) {
        launch_ccl(c->a.labels, c->H, c->W, c->K, c->ccl.link, c->ccl, const_cast<int *>(d_nlab),
                   c->a.ctr, c->st);
        src = c->ccl.link;
    }
    int rc = launch_check(c, "connectivity kernels");
    if (rc) return rc;
    rc = cuda_check(c, cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, c->st), "copy labels");
    if (rc) return rc;
    status->n_labels = c->Keff;
    if (enforce) {
        rc = cuda_check(c, cudaMemcpyAsync(&status->n_labels, d_nlab, sizeof(int), cudaMemcpyDeviceToHost, c->st),
                        "copy label count");
        if (rc) return rc;
    }
    return cuda_check(c, cudaMemcpyAsync(&status->error, &c->a.ctr->error, 2 * sizeof(int),
                                         cudaMemcpyDeviceToHost, c->st),
                      "copy status");
}

static_assert(offsetof(DevCounters, timeout) == offsetof(DevCounters, error) + sizeof(int) &&
                  offsetof(CtxStatus, timeout) == offsetof(CtxStatus, error) + sizeof(int),
              "the two flags are copied as one block");

// After the enqueued work has completed: the label count and device status.
int scalp_ctx_finish_labels(scalp_ctx *c, const CtxStatus *status, int32_t *n_labels)
{
    if (status->timeout) return fail(c, SCALP_E_TIMEOUT, "a bounded device-side wait gave up");
    if (status->error) return fail(c, SCALP_E_INTERNAL, "device-side check failed (code %d)", status->error);
    *n_labels = status->n_labels;
    return SCALP_OK;
}

// Frees a context's host state without synchronising: the caller has seen
// every piece of enqueued work that uses it complete (no graph, no events).
void scalp_ctx_release(scalp_ctx *c)
{
    if (!c) return;
    free_ctx(c);
}

}  // namespace scalp

// ---------------------------------------------------------------------------
// Batches: many images of uneven size and K solved together.  Each image is an
// ordinary context carved from the batch workspace; the set-up, the iteration
// and the connectivity kernels of all images run as one launch each (tiles,
// clusters, pixels and list slots of all images in one flat index space), and
// n iterations replay as one CUDA graph.
// ---------------------------------------------------------------------------

// A small per-image table in device memory that the host rewrites between
// calls (input or output pointers): uploaded through pinned staging, and only
// when its contents changed.
struct PinnedTable {
    void *host = nullptr;  // pinned staging
    void *dev = nullptr;
    size_t bytes = 0;
    cudaEvent_t ev = nullptr;  // the last upload has left the staging buffer
    std::vector<unsigned char> last;
    bool valid = false;

    cudaError_t init(void *d, size_t n)
    {
        dev = d;
        bytes = n;
        cudaError_t e = cudaMallocHost(&host, n);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        return e;
    }
    cudaError_t upload(const void *src, cudaStream_t st)
    {
        if (valid && std::memcmp(last.data(), src, bytes) == 0) return cudaSuccess;
        valid = false;
        cudaError_t e = cudaEventSynchronize(ev);
        if (e != cudaSuccess) return e;
        std::memcpy(host, src, bytes);
        e = cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev, st);
        if (e != cudaSuccess) return e;
        last.assign(static_cast<const unsigned char *>(src), static_cast<const unsigned char *>(src) + bytes);
        valid = true;
        return cudaSuccess;
    }
    void release()
    {
        if (ev) {
            cudaEventSynchronize(ev);
            cudaEventDestroy(ev);
        }
        if (host) cudaFreeHost(host);
        host = nullptr;
        ev = nullptr;
    }
};

struct scalp_batch {
    int count = 0;
    std::vector<scalp_ctx *> ctx;
    cudaStream_t st = nullptr;
    int storage = 0;
    int use_graph = 1;
    unsigned char *ws = nullptr;
    BatchArgs bargs{};
    int *d_nlab = nullptr;          // per image: labels after the connectivity
    DevCounters *d_ctr = nullptr;   // per image: counters, gathered for one read
    int total_tiles = 0, total_clusters = 0, total_fill = 0;
    size_t smem = 0;
    cudaGraphExec_t gexec{};
    bool graph_valid = false;
    int graph_n = 0;
    // flat set-up and connectivity
    const int *setup_base = nullptr;
    int setup_total = 0, zero_parts = 1;
    CclBatch cb{};
    int ccl_total[CCL_KINDS] = {};
    PinnedTable in_table;   // SetupInput per image
    PinnedTable out_table;  // int* per image
    DevCounters *pin_ctr = nullptr;  // pinned: the gathered counters, then the label counts
    int *pin_nlab = nullptr;
    // the per-image copies of a reload or of the labels fan out over
    // BATCH_STREAMS streams, and so does the gradient prior
    static constexpr int BATCH_STREAMS = 8;
    cudaStream_t sub[BATCH_STREAMS] = {};
    cudaEvent_t fork = nullptr, join[BATCH_STREAMS] = {};
    // captured iterations: the candidate lists on a second branch
    cudaStream_t it_side = nullptr;
    cudaEvent_t it_fork = nullptr, it_join = nullptr;
    // persistent launches (scalp_batch_set_launch): the queue orders, the
    // cooperative grid (-1: not asked yet) and the bounded-wait settings
    int launch_mode = SCALP_BATCH_FLAT;
    int persist_grid = -1;
    PersistSync *d_sync = nullptr;
    int *d_order = nullptr, *d_order_base = nullptr;
    std::vector<int> tiles;       // per image
    std::vector<double> r;        // per image: the grid step
    long long wait_ns = 2000000000LL;
    int hold = 0;
    // per-launch timing of the batched assignment (scalp_batch_profile):
    // event pair i brackets iteration i's assignment launch
    bool profiling = false, graph_prof = false;
    std::vector<cudaEvent_t> ev;
    int prof_pending = 0;
    double prof_ms = 0.0;
    long long prof_launches = 0;
};

namespace {

// Runs per_image(i) for every image with the image's context bound to one of
// the batch's streams; the batch stream forks to them and joins them after.
template <typename F>
cudaError_t batch_fan_out(scalp_batch *b, F &&per_image)
{
    cudaError_t e = cudaSuccess;
    if (!b->fork) {
        e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (int s = 0; s < scalp_batch::BATCH_STREAMS && e == cudaSuccess; ++s) {
            e = cudaStreamCreateWithFlags(&b->sub[s], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[s], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return e;
    }
    const int n_sub = std::min(b->count, scalp_batch::BATCH_STREAMS);
    e = cudaEventRecord(b->fork, b->st);
    for (int s = 0; s < n_sub && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(b->sub[s], b->fork, 0);
    int rc = SCALP_OK;
    for (int i = 0; i < b->count && e == cudaSuccess && rc == SCALP_OK; ++i) {
        scalp_ctx *c = b->ctx[i];
        c->st = b->sub[i % n_sub];
        rc = per_image(i);
        c->st = b->st;
    }
    // join whatever was enqueued, also after a failure
    for (int s = 0; s < n_sub; ++s) {
        const cudaError_t r = cudaEventRecord(b->join[s], b->sub[s]);
        const cudaError_t w = r == cudaSuccess ? cudaStreamWaitEvent(b->st, b->join[s], 0) : r;
        if (e == cudaSuccess) e = w;
    }
    if (e == cudaSuccess && rc != SCALP_OK) e = cudaErrorUnknown;
    return e;
}

// The batch's own head of the workspace, in carve order.
struct BatchHead {
    size_t args, tile, clus, fill, nlab, ctr, ccl_img, ccl_base[CCL_KINDS], setup_base, in, out, sync, order,
        order_base, bytes;
};

BatchHead batch_head(int count)
{
    BatchHead h;
    size_t cur = 0;
    const size_t prefix = (size_t)(count + 1) * sizeof(int);
    h.args = carve(cur, (size_t)count * sizeof(SolveArgs));
    h.tile = carve(cur, prefix);
    h.clus = carve(cur, prefix);
    h.fill = carve(cur, prefix);
    h.nlab = carve(cur, (size_t)count * sizeof(int));
    h.ctr = carve(cur, (size_t)count * sizeof(DevCounters));
    h.ccl_img = carve(cur, (size_t)count * sizeof(CclImage));
    for (int k = 0; k < CCL_KINDS; ++k) h.ccl_base[k] = carve(cur, prefix);
    h.setup_base = carve(cur, prefix);
    h.in = carve(cur, (size_t)count * sizeof(SetupInput));
    h.out = carve(cur, (size_t)count * sizeof(int *));
    h.sync = carve(cur, sizeof(PersistSync));
    h.order = carve(cur, (size_t)count * sizeof(int));
    h.order_base = carve(cur, prefix);
    h.bytes = (cur + ALIGN - 1) & ~(ALIGN - 1);
    return h;
}

size_t batch_head_bytes(int count) { return batch_head(count).bytes; }

int batch_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int batch_ensure_events(scalp_batch *b, size_t pairs)
{
    while (b->ev.size() < 2 * pairs) {
        cudaEvent_t e;
        const cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return batch_fail(SCALP_E_CUDA, "create event: %s", cudaGetErrorString(r));
        b->ev.push_back(e);
    }
    return SCALP_OK;
}

// Adds the durations of the recorded assignment launches to the totals.
int batch_harvest_profile(scalp_batch *b)
{
    if (b->prof_pending == 0) return SCALP_OK;
    cudaError_t e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "synchronise: %s", cudaGetErrorString(e));
    for (int i = 0; i < b->prof_pending; ++i) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, b->ev[2 * i], b->ev[2 * i + 1]);
        if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "event time: %s", cudaGetErrorString(e));
        b->prof_ms += t;
        b->prof_launches += 1;
    }
    b->prof_pending = 0;
    return SCALP_OK;
}

}  // namespace

extern "C" {

size_t scalp_batch_workspace_bytes(int32_t count, const int32_t *H, const int32_t *W,
                                   const int32_t *K, const scalp_params *p)
{
    if (count < 1 || !H || !W || !K) return 0;
    size_t total = batch_head_bytes(count);
    for (int i = 0; i < count; ++i) {
        const size_t b = scalp_workspace_bytes(H[i], W[i], K[i], p);
        if (b == 0) return 0;
        total += (b + ALIGN - 1) & ~(ALIGN - 1);
    }
    return total;
}

void scalp_batch_destroy(scalp_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->st);
    for (int s = 0; s < scalp_batch::BATCH_STREAMS; ++s) {
        if (b->sub[s]) {
            cudaStreamSynchronize(b->sub[s]);
            cudaStreamDestroy(b->sub[s]);
        }
        if (b->join[s]) cudaEventDestroy(b->join[s]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->it_side) {
        cudaStreamSynchronize(b->it_side);
        cudaStreamDestroy(b->it_side);
        cudaEventDestroy(b->it_fork);
        cudaEventDestroy(b->it_join);
    }
    if (b->graph_valid) cudaGraphExecDestroy(b->gexec);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    b->in_table.release();
    b->out_table.release();
    if (b->pin_ctr) cudaFreeHost(b->pin_ctr);
    for (scalp_ctx *c : b->ctx) scalp_destroy(c);
    delete b;
}

int scalp_batch_init(scalp_batch **out, int32_t count, const scalp_image *images,
                     const scalp_contour *contours, const int32_t *K, const float *m,
                     const scalp_params *params)
{
    if (!out) return batch_fail(SCALP_E_ARG, "out is NULL");
    *out = nullptr;
    if (count < 1 || !images || !K || !m || !params)
        return batch_fail(SCALP_E_ARG, "need count >= 1 and images, K, m, params");
    std::vector<int32_t> Hs(count), Ws(count);
    for (int i = 0; i < count; ++i) {
        Hs[i] = images[i].H;
        Ws[i] = images[i].W;
    }
    const size_t need = scalp_batch_workspace_bytes(count, Hs.data(), Ws.data(), K, params);
    if (need == 0) return batch_fail(SCALP_E_ARG, "invalid image size or K in the batch");
    if (!params->workspace || params->workspace_bytes < need)
        return batch_fail(SCALP_E_NOMEM, "batch workspace of %zu bytes needed, %zu given", need,
                          params->workspace ? params->workspace_bytes : (size_t)0);
    if (reinterpret_cast<uintptr_t>(params->workspace) % ALIGN)
        return batch_fail(SCALP_E_ARG, "workspace must be 256-byte aligned");
    scalp_batch *b = new (std::nothrow) scalp_batch();
    if (!b) return batch_fail(SCALP_E_NOMEM, "host allocation failed");
    b->count = count;
    b->st = reinterpret_cast<cudaStream_t>(params->stream);
    b->storage = params->storage;
    b->use_graph = params->use_graph;
    b->ws = reinterpret_cast<unsigned char *>(params->workspace);
    const BatchHead h = batch_head(count);
    size_t off = h.bytes;
    std::vector<SolveArgs> args(count);
    std::vector<int> tile_base(count + 1, 0), clus_base(count + 1, 0), fill_base(count + 1, 0);
    std::vector<int> setup_base(count + 1, 0);
    std::vector<std::vector<int>> ccl_base(CCL_KINDS, std::vector<int>(count + 1, 0));
    std::vector<CclImage> ccl_img(count);
    b->d_nlab = reinterpret_cast<int *>(b->ws + h.nlab);
    b->d_ctr = reinterpret_cast<DevCounters *>(b->ws + h.ctr);
    bool too_large = false;
    auto add = [&](std::vector<int> &base, int i, long long n) {
        const long long v = base[i] + n;
        too_large |= v > INT_MAX;
        base[i + 1] = (int)std::min<long long>(v, INT_MAX);
    };
    for (int i = 0; i < count; ++i) {
        scalp_params p = *params;
        p.use_graph = 0;
        p.workspace = b->ws + off;
        p.workspace_bytes = scalp_workspace_bytes(Hs[i], Ws[i], K[i], params);
        off += (p.workspace_bytes + ALIGN - 1) & ~(ALIGN - 1);
        scalp_ctx *c = nullptr;
        const int rc = scalp_init(&c, &images[i], contours ? &contours[i] : nullptr, K[i], m[i], &p);
        if (rc != SCALP_OK) {
            char msg[512];
            snprintf(msg, sizeof msg, "image %d: %s", i, g_last_error.c_str());
            scalp_batch_destroy(b);
            return batch_fail(rc, "%s", msg);
        }
        b->ctx.push_back(c);
        args[i] = c->a;
        add(tile_base, i, (long long)c->a.n_tx * c->a.n_ty);
        add(clus_base, i, c->Keff);
        add(fill_base, i, (long long)c->Keff * c->a.tpw_x * c->a.tpw_y);
        add(setup_base, i, setup_blocks(c->H, c->W, c->ny));
        b->zero_parts = std::max(b->zero_parts, zero_blocks(c->Keff, c->a.n_tx * c->a.n_ty));
        long long blocks[CCL_KINDS];
        ccl_batch_blocks(c->H, c->W, blocks);
        for (int k = 0; k < CCL_KINDS; ++k) add(ccl_base[k], i, blocks[k]);
        CclImage &m = ccl_img[i];
        m.labels = c->a.labels;
        m.parent = c->ccl.parent;
        m.size = c->ccl.size;
        m.link = c->ccl.link;
        m.scan = c->ccl.scan;
        m.scan_tmp = c->ccl.scan_tmp;
        m.nlab = b->d_nlab + i;
        m.ctr = c->a.ctr;
        m.ctr_out = b->d_ctr + i;
        m.N = c->N;
        m.T = c->N / (4LL * c->K);
        m.H = c->H;
        m.W = c->W;
        m.n_tx = (c->W + 31) / 32;
        m.n_ty = (c->H + 31) / 32;
        b->smem = std::max(b->smem, c->smem);
        b->tiles.push_back(c->a.n_tx * c->a.n_ty);
        b->r.push_back(c->r);
    }
    if (too_large) {
        scalp_batch_destroy(b);
        return batch_fail(SCALP_E_ARG, "the batch has more than 2^31-1 blocks in one launch");
    }
    b->total_tiles = tile_base[count];
    b->total_clusters = clus_base[count];
    b->total_fill = fill_base[count];
    b->setup_total = setup_base[count];
    b->bargs.args = reinterpret_cast<const SolveArgs *>(b->ws + h.args);
    b->bargs.tile_base = reinterpret_cast<const int *>(b->ws + h.tile);
    b->bargs.clus_base = reinterpret_cast<const int *>(b->ws + h.clus);
    b->bargs.fill_base = reinterpret_cast<const int *>(b->ws + h.fill);
    b->bargs.count = count;
    b->setup_base = reinterpret_cast<const int *>(b->ws + h.setup_base);
    b->cb.img = reinterpret_cast<const CclImage *>(b->ws + h.ccl_img);
    b->cb.out = reinterpret_cast<int *const *>(b->ws + h.out);
    for (int k = 0; k < CCL_KINDS; ++k) {
        b->cb.base[k] = reinterpret_cast<const int *>(b->ws + h.ccl_base[k]);
        b->ccl_total[k] = ccl_base[k][count];
    }
    b->cb.count = count;
    b->d_sync = reinterpret_cast<PersistSync *>(b->ws + h.sync);
    b->d_order = reinterpret_cast<int *>(b->ws + h.order);
    b->d_order_base = reinterpret_cast<int *>(b->ws + h.order_base);
    const size_t prefix = (count + 1) * sizeof(int);
    std::vector<std::pair<size_t, std::pair<const void *, size_t>>> copies = {
        {h.args, {args.data(), count * sizeof(SolveArgs)}},
        {h.tile, {tile_base.data(), prefix}},
        {h.clus, {clus_base.data(), prefix}},
        {h.fill, {fill_base.data(), prefix}},
        {h.setup_base, {setup_base.data(), prefix}},
        {h.ccl_img, {ccl_img.data(), count * sizeof(CclImage)}}};
    for (int k = 0; k < CCL_KINDS; ++k) copies.push_back({h.ccl_base[k], {ccl_base[k].data(), prefix}});
    cudaError_t e = cudaSuccess;
    for (const auto &cp : copies)
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->ws + cp.first, cp.second.first, cp.second.second, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);  // host vectors go out of scope
    if (e == cudaSuccess) e = b->in_table.init(b->ws + h.in, count * sizeof(SetupInput));
    if (e == cudaSuccess) e = b->out_table.init(b->ws + h.out, count * sizeof(int *));
    if (e == cudaSuccess) {
        void *pin = nullptr;
        e = cudaMallocHost(&pin, count * (sizeof(DevCounters) + sizeof(int)));
        if (e == cudaSuccess) {
            b->pin_ctr = static_cast<DevCounters *>(pin);
            b->pin_nlab = reinterpret_cast<int *>(b->pin_ctr + count);
        }
    }
    if (e == cudaSuccess) e = assign_batch_configure(b->storage);
    if (e != cudaSuccess) {
        scalp_batch_destroy(b);
        return batch_fail(SCALP_E_CUDA, "batch set-up: %s", cudaGetErrorString(e));
    }
    *out = b;
    return SCALP_OK;
}

int scalp_batch_reload(scalp_batch *b, const scalp_image *images, const scalp_contour *contours)
{
    if (!b || !images) return batch_fail(SCALP_E_ARG, "batch or images is NULL");
    for (int i = 0; i < b->count; ++i) {
        const int rc = check_reload(b->ctx[i], &images[i], contours ? &contours[i] : nullptr);
        if (rc != SCALP_OK) return batch_fail(rc, "image %d: %s", i, b->ctx[i]->err.c_str());
    }
    // the inputs on the device (copies, gradient priors), per image
    std::vector<SetupInput> in(b->count);
    int bad = -1, bad_rc = SCALP_OK;
    auto stage = [&](int i) {
        const int rc = stage_inputs(b->ctx[i], &images[i], contours ? &contours[i] : nullptr, &in[i]);
        if (rc != SCALP_OK) {
            bad = i;
            bad_rc = rc;
        }
        return rc;
    };
    cudaError_t e = cudaSuccess;
    if (b->ctx[0]->p.prior == SCALP_PRIOR_GRADIENT) {
        e = batch_fan_out(b, stage);
    } else {
        for (int i = 0; i < b->count && bad < 0; ++i) stage(i);
    }
    if (bad >= 0) return batch_fail(bad_rc, "image %d: %s", bad, b->ctx[bad]->err.c_str());
    // then the set-up and the first update, projection and lists of all images
    if (e == cudaSuccess) e = b->in_table.upload(in.data(), b->st);
    if (e == cudaSuccess) {
        launch_setup_batch(b->bargs, static_cast<const SetupInput *>(b->in_table.dev), b->setup_base,
                           b->setup_total, b->zero_parts, b->storage, b->st);
        launch_batch_update(b->bargs, b->total_clusters, b->total_fill, b->st, true, nullptr, nullptr, nullptr, 1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "batch reload: %s", cudaGetErrorString(e));
    for (scalp_ctx *c : b->ctx) c->iterations = 0;
    return SCALP_OK;
}

int scalp_batch_iterate(scalp_batch *b, int32_t n)
{
    if (!b) return batch_fail(SCALP_E_ARG, "batch is NULL");
    if (n < 0) return batch_fail(SCALP_E_ARG, "n must be >= 0");
    if (n == 0) return SCALP_OK;
    if (b->launch_mode != SCALP_BATCH_FLAT) {
        // all n iterations in one cooperative launch; its barrier words start at zero
        PersistArgs q{};
        q.b = b->bargs;
        q.order = b->d_order;
        q.order_base = b->d_order_base;
        q.sync = b->d_sync;
        q.total_tiles = b->total_tiles;
        q.total_clusters = b->total_clusters;
        q.total_fill = b->total_fill;
        q.iters = n;
        q.wait_ns = b->wait_ns;
        q.hold = b->hold;
        cudaError_t e = cudaMemsetAsync(b->d_sync, 0, sizeof(PersistSync), b->st);
        if (e == cudaSuccess) e = launch_batch_persistent(q, b->storage, b->smem, b->persist_grid, b->st);
        if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "persistent batch launch: %s", cudaGetErrorString(e));
        for (scalp_ctx *c : b->ctx) c->iterations += n;
        return SCALP_OK;
    }
    if (b->profiling) {
        int rc = batch_harvest_profile(b);  // the events are about to be re-recorded
        if (rc) return rc;
        rc = batch_ensure_events(b, (size_t)n);
        if (rc) return rc;
    }
    bool capturing = false;
    // programmatic launches overlap each kernel's placement with the drain of
    // the one before (not across the profiling event records)
    const bool pdl = !b->profiling;
    auto enqueue = [&](int iters) {
        // under stream capture the records become event-record nodes
        const unsigned flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
        for (int i = 0; i < iters; ++i) {
            if (b->profiling) cudaEventRecordWithFlags(b->ev[2 * i], b->st, flags);
            launch_assign_batch(b->bargs, b->storage, b->total_tiles, b->smem, b->st, pdl);
            if (b->profiling) cudaEventRecordWithFlags(b->ev[2 * i + 1], b->st, flags);
            launch_batch_update(b->bargs, b->total_clusters, b->total_fill, b->st, pdl,
                                capturing ? b->it_side : nullptr, b->it_fork, b->it_join);
        }
    };
    const bool graphs = b->use_graph && b->st != nullptr;
    cudaError_t e = cudaSuccess;
    if (graphs && !(b->graph_valid && b->graph_n == n && b->graph_prof == b->profiling)) {
        if (b->graph_valid) {
            cudaGraphExecDestroy(b->gexec);
            b->graph_valid = false;
        }
        if (!b->it_side) {  // made before the capture; without it, one stream
            int prio = 0;
            cudaStream_t t = nullptr;
            cudaEvent_t f = nullptr, j = nullptr;
            if (cudaStreamGetPriority(b->st, &prio) == cudaSuccess &&
                cudaStreamCreateWithPriority(&t, cudaStreamNonBlocking, prio) == cudaSuccess &&
                cudaEventCreateWithFlags(&f, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&j, cudaEventDisableTiming) == cudaSuccess) {
                b->it_side = t;
                b->it_fork = f;
                b->it_join = j;
            } else {
                if (t) cudaStreamDestroy(t);
                if (f) cudaEventDestroy(f);
                if (j) cudaEventDestroy(j);
                cudaGetLastError();
            }
        }
        cudaGraph_t g;
        e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "begin capture: %s", cudaGetErrorString(e));
        capturing = true;
        enqueue(n);
        capturing = false;
        const cudaError_t le = cudaGetLastError();
        e = cudaStreamEndCapture(b->st, &g);
        if (e == cudaSuccess && le != cudaSuccess) {
            cudaGraphDestroy(g);
            e = le;
        }
        if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "instantiate: %s", cudaGetErrorString(e));
        b->graph_valid = true;
        b->graph_n = n;
        b->graph_prof = b->profiling;
    }
    if (graphs) {
        e = cudaGraphLaunch(b->gexec, b->st);
    } else {
        enqueue(n);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "batch iteration: %s", cudaGetErrorString(e));
    if (b->profiling) b->prof_pending = n;
    for (scalp_ctx *c : b->ctx) c->iterations += n;
    return SCALP_OK;
}

int scalp_batch_labels(scalp_batch *b, int32_t *const *outs, int32_t out_on_device, int32_t enforce,
                       int32_t *n_labels)
{
    if (!b || !outs) return batch_fail(SCALP_E_ARG, "batch or outs is NULL");
    for (int i = 0; i < b->count; ++i)
        if (!outs[i]) return batch_fail(SCALP_E_ARG, "outs[%d] is NULL", i);
    int *d_nlab = b->d_nlab;
    DevCounters *d_ctr = b->d_ctr;
    cudaError_t e = cudaSuccess;
    if (enforce) {
        // the connectivity of all images, one launch per pass, into the
        // caller's buffers or the images' staging; the passes also gather
        // the label counts and the counters
        std::vector<int *> dst(b->count);
        for (int i = 0; i < b->count; ++i) dst[i] = out_on_device ? outs[i] : b->ctx[i]->ccl.link;
        e = b->out_table.upload(dst.data(), b->st);
        if (e == cudaSuccess) {
            launch_ccl_batch(b->cb, b->ccl_total, b->st);
            e = cudaGetLastError();
        }
        for (int i = 0; i < b->count && e == cudaSuccess && !out_on_device; ++i)
            e = cudaMemcpyAsync(outs[i], dst[i], sizeof(int) * (size_t)b->ctx[i]->N, cudaMemcpyDeviceToHost, b->st);
    } else {
        cudaError_t ce = cudaSuccess;
        e = batch_fan_out(b, [&](int i) {
            scalp_ctx *c = b->ctx[i];
            cudaError_t r = cudaMemcpyAsync(outs[i], c->a.labels, sizeof(int) * (size_t)c->N,
                                            out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st);
            if (r == cudaSuccess)
                r = cudaMemcpyAsync(d_ctr + i, c->a.ctr, sizeof(DevCounters), cudaMemcpyDeviceToDevice, c->st);
            ce = r;
            return r == cudaSuccess ? SCALP_OK : SCALP_E_CUDA;
        });
        if (ce != cudaSuccess) e = ce;
    }
    if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "batch labels: %s", cudaGetErrorString(e));
    // both gathers into pinned memory: two asynchronous copies, one synchronisation
    const int *nlab = b->pin_nlab;
    const DevCounters *ctr = b->pin_ctr;
    e = cudaMemcpyAsync(b->pin_nlab, d_nlab, sizeof(int) * b->count, cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->pin_ctr, d_ctr, sizeof(DevCounters) * b->count, cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "batch labels: %s", cudaGetErrorString(e));
    for (int i = 0; i < b->count; ++i) {
        if (ctr[i].timeout) return batch_fail(SCALP_E_TIMEOUT, "image %d: a bounded wait gave up", i);
        if (ctr[i].error) return batch_fail(SCALP_E_INTERNAL, "image %d: device check failed (%d)", i, ctr[i].error);
        if (n_labels) n_labels[i] = enforce ? nlab[i] : b->ctx[i]->Keff;
    }
    return SCALP_OK;
}

int scalp_batch_get_state(scalp_batch *b, int32_t index, const scalp_state *state)
{
    if (!b || index < 0 || index >= b->count) return batch_fail(SCALP_E_ARG, "bad batch or index");
    return scalp_get_state(b->ctx[index], state);
}

int scalp_batch_get_info(const scalp_batch *b, int32_t index, scalp_info *info)
{
    if (!b || index < 0 || index >= b->count) return batch_fail(SCALP_E_ARG, "bad batch or index");
    return scalp_get_info(b->ctx[index], info);
}

int scalp_batch_set_launch(scalp_batch *b, int32_t mode)
{
    if (!b) return batch_fail(SCALP_E_ARG, "batch is NULL");
    if (mode != SCALP_BATCH_FLAT && mode != SCALP_BATCH_PERSISTENT && mode != SCALP_BATCH_PERSISTENT_COST)
        return batch_fail(SCALP_E_ARG, "unknown launch mode %d", mode);
    if (mode == SCALP_BATCH_FLAT) {
        b->launch_mode = mode;
        return SCALP_OK;
    }
    if (b->persist_grid < 0) {
        int grid = 0;
        const cudaError_t e = batch_persistent_grid(b->storage, b->smem, &grid);
        if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "persistent launch set-up: %s", cudaGetErrorString(e));
        b->persist_grid = grid;
    }
    if (b->persist_grid <= 0)
        return batch_fail(SCALP_E_STATE, "no cooperative persistent launch fits this device");
    // the projection phase lays out the images' queue lengths and their
    // prefix in the dynamic shared memory
    if ((size_t)(2 * b->count + 1) * sizeof(int) > b->smem)
        return batch_fail(SCALP_E_STATE, "too many images (%d) for the persistent launch's work list", b->count);
    // the queue's image order: batch order, or by descending grid step r
    // (the images whose tiles walk the longest paths first; ties in batch order)
    std::vector<int> order(b->count), base(b->count + 1, 0);
    for (int i = 0; i < b->count; ++i) order[i] = i;
    if (mode == SCALP_BATCH_PERSISTENT_COST)
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->r[x] > b->r[y]; });
    for (int j = 0; j < b->count; ++j) base[j + 1] = base[j] + b->tiles[order[j]];
    cudaError_t e = cudaMemcpyAsync(b->d_order, order.data(), b->count * sizeof(int), cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_order_base, base.data(), (b->count + 1) * sizeof(int), cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);  // the host vectors go out of scope
    if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "queue order: %s", cudaGetErrorString(e));
    b->launch_mode = mode;
    return SCALP_OK;
}

int scalp_batch_get_launch(const scalp_batch *b, int32_t *mode, int32_t *grid)
{
    if (!b) return batch_fail(SCALP_E_ARG, "batch is NULL");
    if (mode) *mode = b->launch_mode;
    if (grid) *grid = b->persist_grid;
    return SCALP_OK;
}

int scalp_batch_set_wait(scalp_batch *b, int64_t limit_ns, int32_t hold)
{
    if (!b) return batch_fail(SCALP_E_ARG, "batch is NULL");
    if (limit_ns < 1000000LL || limit_ns > 60000000000LL || hold < 0 || hold > 1024)
        return batch_fail(SCALP_E_ARG, "need 1 ms <= limit_ns <= 60 s and 0 <= hold <= 1024");
    b->wait_ns = limit_ns;
    b->hold = hold;
    return SCALP_OK;
}

}  // extern "C"

namespace {

// The autotuner's key: the device (SM count), the storage and the batch's
// shape class (images, total tiles to two significant digits, mean grid step).
std::string autotune_key(const scalp_batch *b)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double rsum = 0.0;
    for (double r : b->r) rsum += r;
    long long t = b->total_tiles, scale = 1;
    while (t >= 100) {
        t = (t + 5) / 10;
        scale *= 10;
    }
    char key[160];
    snprintf(key, sizeof key, "scalp-batch/sm%d/%s/n%d/tiles%lld/r%d", sms, b->storage ? "f16" : "f32", b->count,
             t * scale, (int)std::lround(rsum / b->count));
    return key;
}

// The cache: a JSON object, one entry per line, "key": {"mode": M, "ms": [...]}.
std::map<std::string, std::string> read_cache(const char *path)
{
    std::map<std::string, std::string> out;
    FILE *f = path ? fopen(path, "r") : nullptr;
    if (!f) return out;
    char line[1024];
    while (fgets(line, sizeof line, f)) {
        const char *q0 = strchr(line, '"');
        const char *q1 = q0 ? strchr(q0 + 1, '"') : nullptr;
        const char *brace = q1 ? strchr(q1, '{') : nullptr;
        const char *end = brace ? strrchr(brace, '}') : nullptr;
        if (!end) continue;
        out[std::string(q0 + 1, q1)] = std::string(brace, end + 1);
    }
    fclose(f);
    return out;
}

int cached_mode(const std::map<std::string, std::string> &cache, const std::string &key)
{
    const auto it = cache.find(key);
    int mode = -1;
    if (it != cache.end() && sscanf(it->second.c_str(), "{\"mode\": %d", &mode) != 1) mode = -1;
    return mode;
}

bool write_cache(const char *path, const std::map<std::string, std::string> &cache)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fprintf(f, "{\n");
    size_t i = 0;
    for (const auto &kv : cache)
        fprintf(f, "  \"%s\": %s%s\n", kv.first.c_str(), kv.second.c_str(), ++i < cache.size() ? "," : "");
    fprintf(f, "}\n");
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path) == 0;
}

}  // namespace

extern "C" {

int scalp_batch_autotune(scalp_batch *b, const scalp_image *images, const scalp_contour *contours, int32_t iters,
                         const char *cache_path, int32_t *mode, float *trial_ms, int32_t *from_cache)
{
    if (!b || !images || iters < 1) return batch_fail(SCALP_E_ARG, "need a batch, its images and iters >= 1");
    const std::string key = autotune_key(b);
    std::map<std::string, std::string> cache = read_cache(cache_path);
    if (trial_ms)
        for (int m = 0; m < 3; ++m) trial_ms[m] = -1.f;
    if (from_cache) *from_cache = 0;
    int best = cached_mode(cache, key);
    if (best >= SCALP_BATCH_FLAT && best <= SCALP_BATCH_PERSISTENT_COST) {
        int rc = scalp_batch_set_launch(b, best);
        if (rc == SCALP_OK) {
            if (from_cache) *from_cache = 1;
            if (mode) *mode = best;
            return scalp_batch_reload(b, images, contours);
        }
    }
    // trials: each mode once to warm up (graph capture, module load), then
    // the faster of two timed runs of `iters` iterations from a fresh reload
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return batch_fail(SCALP_E_CUDA, "autotune events");
    }
    float ms[3] = {-1.f, -1.f, -1.f};
    int rc = SCALP_OK;
    for (int m = SCALP_BATCH_FLAT; m <= SCALP_BATCH_PERSISTENT_COST && rc == SCALP_OK; ++m) {
        if (scalp_batch_set_launch(b, m) != SCALP_OK) continue;  // not available here
        for (int rep = 0; rep < 3 && rc == SCALP_OK; ++rep) {
            rc = scalp_batch_reload(b, images, contours);
            if (rc == SCALP_OK && rep > 0 && cudaEventRecord(e0, b->st) != cudaSuccess) rc = SCALP_E_CUDA;
            if (rc == SCALP_OK) rc = scalp_batch_iterate(b, iters);
            if (rc == SCALP_OK && rep > 0) {
                float t = 0.f;
                if (cudaEventRecord(e1, b->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                    rc = batch_fail(SCALP_E_CUDA, "autotune timing");
                else if (ms[m] < 0.f || t < ms[m])
                    ms[m] = t;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SCALP_OK) return rc;
    best = SCALP_BATCH_FLAT;
    for (int m = 0; m < 3; ++m)
        if (ms[m] >= 0.f && ms[m] < ms[best]) best = m;
    if (trial_ms)
        for (int m = 0; m < 3; ++m) trial_ms[m] = ms[m];
    rc = scalp_batch_set_launch(b, best);
    if (rc == SCALP_OK) rc = scalp_batch_reload(b, images, contours);
    if (rc != SCALP_OK) return rc;
    if (mode) *mode = best;
    if (cache_path) {
        char entry[256];
        snprintf(entry, sizeof entry, "{\"mode\": %d, \"iters\": %d, \"ms\": [%.4f, %.4f, %.4f]}", best, iters,
                 ms[0], ms[1], ms[2]);
        cache[key] = entry;
        if (!write_cache(cache_path, cache)) return batch_fail(SCALP_E_ARG, "cannot write the cache %s", cache_path);
    }
    return SCALP_OK;
}

int scalp_batch_profile(scalp_batch *b, int32_t enable, double *ms, int64_t *launches)
{
    if (!b) return batch_fail(SCALP_E_ARG, "batch is NULL");
    const int rc = batch_harvest_profile(b);
    if (rc) return rc;
    if (ms) *ms = b->prof_ms;
    if (launches) *launches = b->prof_launches;
    if (enable >= 0) {
        const bool on = enable != 0;
        if (on) {
            b->prof_ms = 0.0;
            b->prof_launches = 0;
        }
        b->profiling = on;
    }
    return SCALP_OK;
}

int scalp_batch_count_samples(scalp_batch *b, int32_t enable, int64_t *samples, int64_t *pairs)
{
    if (!b) return batch_fail(SCALP_E_ARG, "batch is NULL");
    std::vector<DevCounters> h(b->count);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < b->count && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(&h[i], b->ctx[i]->a.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "read counters: %s", cudaGetErrorString(e));
    long long ns = 0, np = 0;
    for (const DevCounters &c : h) {
        ns += (long long)c.samples;
        np += (long long)c.pairs;
    }
    if (samples) *samples = ns;
    if (pairs) *pairs = np;
    if (enable < 0) return SCALP_OK;
    const int on = enable != 0;
    std::vector<SolveArgs> args(b->count);
    for (int i = 0; i < b->count && e == cudaSuccess; ++i) {
        scalp_ctx *c = b->ctx[i];
        c->a.count_samples = on;
        args[i] = c->a;
        if (on) e = cudaMemsetAsync(&c->a.ctr->samples, 0, 4 * sizeof(unsigned long long), b->st);
    }
    // the argument blocks the kernels read, then the replayed graph, change
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(const_cast<SolveArgs *>(b->bargs.args), args.data(), b->count * sizeof(SolveArgs),
                            cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return batch_fail(SCALP_E_CUDA, "count samples: %s", cudaGetErrorString(e));
    if (b->graph_valid) {
        cudaGraphExecDestroy(b->gexec);
        b->graph_valid = false;
    }
    return SCALP_OK;
}

}  // extern "C"
