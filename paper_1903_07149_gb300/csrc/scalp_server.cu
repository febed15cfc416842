// scalp_server.cu -- continuous batching of many SCALP solves (serving).
//
// A server owns a caller-allocated device memory pool.  A request is admitted
// when its workspace fits in the pool and a slot is free; its state then stays
// resident until its labels have been delivered.  Each scalp_server_step()
// runs one iteration of Algorithm 1 for every solve in flight, whatever its
// size, as one launch per kernel (the batched kernels), so requests admitted
// while others are running share the device with them.  A solve that has done
// its iterations is retired: connectivity enforcement and the copy of its
// labels to the caller's buffer are enqueued, followed by an event that
// scalp_server_poll() checks.
//
// The host never drains the stream while serving: the per-step argument
// blocks live in a ring of ARG_RING device blocks, each staged from pinned
// host memory and reused only after the event behind the last step that read
// it; a delivered solve's status arrives in pinned memory with its labels.
// A request's own work runs beside the steps, on SIDE_STREAMS streams of the
// server: its set-up (the step that first includes it waits for its `ready`
// event) and its retirement (forked from the step stream after its last step;
// later steps do not read it, so they need not wait).
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/scalp.h"
#include "scalp_launch.h"

using namespace scalp;

namespace {

constexpr size_t SALIGN = 256;
constexpr int ARG_RING = 8;      // argument blocks in flight
constexpr int SIDE_STREAMS = 4;  // for the requests' set-up and retirement
constexpr int STEPS_AHEAD = 2;   // steps enqueued beyond the one the GPU runs

size_t salign(size_t x) { return (x + SALIGN - 1) & ~(SALIGN - 1); }

struct Solve {
    uint64_t id = 0;
    scalp_ctx *ctx = nullptr;
    size_t off = 0, bytes = 0;  // its part of the pool
    int iters_left = 0;
    long long pixels = 0;  // H * W
    int enforce = 1;
    int32_t *labels_out = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t ready = nullptr;  // its set-up has run
    int status_slot = -1;         // its entry in the pinned status array
    bool joined = false;          // the step stream has waited for `ready`
    bool retired = false;
    int32_t inject_error = 0, inject_timeout = 0;  // host-side fault injection (tests)
};

int server_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    scalp::set_last_error(buf);
    return code;
}

// one argument block: the solves' SolveArgs, then their tile, cluster and
// list-slot prefix sums
size_t block_bytes(int slots)
{
    return salign((size_t)slots * sizeof(SolveArgs)) + 3 * salign((size_t)(slots + 1) * sizeof(int));
}

size_t head_bytes(int slots) { return ARG_RING * block_bytes(slots); }

}  // namespace

struct scalp_server {
    cudaStream_t st = nullptr;
    unsigned char *pool = nullptr;
    size_t pool_bytes = 0;
    scalp_params params{};
    int max_slots = 0;
    std::map<size_t, size_t> free_list;  // offset -> size, coalesced
    std::vector<Solve *> active;          // admitted, iterating or retired-but-not-polled
    std::map<uint64_t, Solve *> by_id;
    uint64_t next_id = 1;
    bool args_dirty = true;
    BatchArgs bargs{};
    int total_tiles = 0, total_clusters = 0, total_fill = 0;
    size_t smem = 0;
    std::vector<cudaEvent_t> spare_events;
    unsigned char *stage = nullptr;  // pinned: ARG_RING argument blocks
    CtxStatus *status = nullptr;     // pinned: max_slots status entries
    std::vector<int> free_status;
    cudaEvent_t ring_ev[ARG_RING] = {};
    bool ring_live[ARG_RING] = {};
    int ring_next = 0, ring_cur = 0;
    cudaStream_t side[SIDE_STREAMS] = {};
    cudaEvent_t step_ev = nullptr;  // the step stream's position, for forks
    int side_next = 0;
    long long step_pixels = 0;      // 0: every request iterates each step
    std::vector<uint64_t> arg_ids;  // the requests of the current argument block
    cudaEvent_t step_done[STEPS_AHEAD] = {};
    bool step_live[STEPS_AHEAD] = {};
    int step_next = 0;
};

namespace {

bool pool_alloc(scalp_server *s, size_t bytes, size_t &off)
{
    bytes = salign(bytes);
    for (auto it = s->free_list.begin(); it != s->free_list.end(); ++it) {
        if (it->second >= bytes) {
            off = it->first;
            const size_t rest = it->second - bytes;
            s->free_list.erase(it);
            if (rest) s->free_list[off + bytes] = rest;
            return true;
        }
    }
    return false;
}

void pool_free(scalp_server *s, size_t off, size_t bytes)
{
    bytes = salign(bytes);
    auto it = s->free_list.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != s->free_list.end() && it->first + it->second == next->first) {
        it->second += next->second;
        s->free_list.erase(next);
    }
    if (it != s->free_list.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second == it->first) {
            prev->second += it->second;
            s->free_list.erase(it);
        }
    }
}

// Uploads the argument block of the solves still iterating into the next ring
// slot (compact: offsets follow the count n).
int rebuild_args(scalp_server *s, std::vector<Solve *> &running)
{
    const int n = (int)running.size();
    const int slot = s->ring_next;
    s->ring_next = (slot + 1) % ARG_RING;
    if (s->ring_live[slot]) {  // a step in flight may still read this slot
        const cudaError_t w = cudaEventSynchronize(s->ring_ev[slot]);
        if (w != cudaSuccess) return server_fail(SCALP_E_CUDA, "argument ring: %s", cudaGetErrorString(w));
        s->ring_live[slot] = false;
    }
    const size_t blk = block_bytes(s->max_slots);
    unsigned char *h = s->stage + slot * blk;
    unsigned char *d = s->pool + slot * blk;
    const size_t o_tile = salign((size_t)n * sizeof(SolveArgs));
    const size_t o_clus = o_tile + salign((size_t)(n + 1) * sizeof(int));
    const size_t o_fill = o_clus + salign((size_t)(n + 1) * sizeof(int));
    SolveArgs *args = reinterpret_cast<SolveArgs *>(h);
    int *tile = reinterpret_cast<int *>(h + o_tile);
    int *clus = reinterpret_cast<int *>(h + o_clus);
    int *fill = reinterpret_cast<int *>(h + o_fill);
    tile[0] = clus[0] = fill[0] = 0;
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
        const scalp_ctx *c = running[i]->ctx;
        args[i] = scalp_ctx_args(c);
        tile[i + 1] = tile[i] + args[i].n_tx * args[i].n_ty;
        clus[i + 1] = clus[i] + args[i].Keff;
        fill[i + 1] = fill[i] + args[i].Keff * args[i].tpw_x * args[i].tpw_y;
        smem = std::max(smem, scalp_ctx_smem(c));
    }
    cudaError_t e = cudaMemcpyAsync(d, h, o_fill + (size_t)(n + 1) * sizeof(int), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaEventRecord(s->ring_ev[slot], s->st);
    if (e != cudaSuccess) return server_fail(SCALP_E_CUDA, "server arguments: %s", cudaGetErrorString(e));
    s->ring_live[slot] = true;
    s->ring_cur = slot;
    s->bargs.args = reinterpret_cast<const SolveArgs *>(d);
    s->bargs.tile_base = reinterpret_cast<const int *>(d + o_tile);
    s->bargs.clus_base = reinterpret_cast<const int *>(d + o_clus);
    s->bargs.fill_base = reinterpret_cast<const int *>(d + o_fill);
    s->bargs.count = n;
    s->total_tiles = tile[n];
    s->total_clusters = clus[n];
    s->total_fill = fill[n];
    s->smem = smem;
    s->args_dirty = false;
    return SCALP_OK;
}

cudaError_t spare_event(scalp_server *s, cudaEvent_t &ev)
{
    if (s->spare_events.empty()) {
        cudaEvent_t e;
        const cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (r != cudaSuccess) return r;
        s->spare_events.push_back(e);
    }
    ev = s->spare_events.back();
    s->spare_events.pop_back();
    return cudaSuccess;
}

void free_host(scalp_server *s)
{
    for (cudaStream_t t : s->side)
        if (t) {
            cudaStreamSynchronize(t);
            cudaStreamDestroy(t);
        }
    if (s->step_ev) cudaEventDestroy(s->step_ev);
    for (cudaEvent_t e : s->step_done)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : s->ring_ev)
        if (e) cudaEventDestroy(e);
    if (s->stage) cudaFreeHost(s->stage);
    delete s;
}

}  // namespace

extern "C" {

size_t scalp_server_reserve_bytes(int32_t max_slots)
{
    return max_slots < 1 ? 0 : head_bytes(max_slots);
}

int scalp_server_create(scalp_server **out, void *pool, size_t pool_bytes, int32_t max_slots,
                        const scalp_params *params)
{
    if (!out) return server_fail(SCALP_E_ARG, "out is NULL");
    *out = nullptr;
    if (!params || !pool || max_slots < 1) return server_fail(SCALP_E_ARG, "need params, pool, max_slots >= 1");
    if (reinterpret_cast<uintptr_t>(pool) % SALIGN) return server_fail(SCALP_E_ARG, "pool must be 256-byte aligned");
    const size_t head = head_bytes(max_slots);
    if (pool_bytes <= head) return server_fail(SCALP_E_NOMEM, "pool smaller than the %zu-byte reserve", head);
    if (params->storage != 0 && params->storage != 1) return server_fail(SCALP_E_ARG, "bad storage");
    scalp_server *s = new (std::nothrow) scalp_server();
    if (!s) return server_fail(SCALP_E_NOMEM, "host allocation failed");
    s->st = reinterpret_cast<cudaStream_t>(params->stream);
    s->pool = reinterpret_cast<unsigned char *>(pool);
    s->pool_bytes = pool_bytes;
    s->params = *params;
    s->params.use_graph = 0;
    s->max_slots = max_slots;
    s->free_list[head] = (pool_bytes - head) & ~(SALIGN - 1);
    // the batched assignment may need up to the full shared memory of an SM
    cudaError_t e = assign_batch_configure(params->storage);
    const size_t ring = ARG_RING * block_bytes(max_slots);
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void **>(&s->stage), ring + (size_t)max_slots * sizeof(CtxStatus),
                          cudaHostAllocDefault);
    for (int i = 0; i < ARG_RING && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&s->ring_ev[i], cudaEventDisableTiming);
    // side streams share the priority of the server's stream
    int prio = 0;
    if (e == cudaSuccess && s->st) e = cudaStreamGetPriority(s->st, &prio);
    for (int i = 0; i < SIDE_STREAMS && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithPriority(&s->side[i], cudaStreamNonBlocking, prio);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->step_ev, cudaEventDisableTiming);
    for (int i = 0; i < STEPS_AHEAD && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&s->step_done[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_host(s);
        return server_fail(SCALP_E_CUDA, "server setup: %s", cudaGetErrorString(e));
    }
    s->status = reinterpret_cast<CtxStatus *>(s->stage + ring);
    for (int i = max_slots - 1; i >= 0; --i) s->free_status.push_back(i);
    *out = s;
    return SCALP_OK;
}

int scalp_server_submit(scalp_server *s, const scalp_image *image, const scalp_contour *contour,
                        int32_t K, float m, int32_t iters, int32_t enforce, int32_t *labels_out,
                        uint64_t *id)
{
    if (!s || !image || !labels_out || !id) return server_fail(SCALP_E_ARG, "null argument");
    if (iters < 0) return server_fail(SCALP_E_ARG, "iters must be >= 0");
    if ((int)s->active.size() >= s->max_slots) return server_fail(SCALP_E_NOMEM, "no free slot");
    const size_t bytes = scalp_workspace_bytes(image->H, image->W, K, &s->params);
    if (bytes == 0) return server_fail(SCALP_E_ARG, "invalid image size or K");
    size_t off;
    if (!pool_alloc(s, bytes, off)) return server_fail(SCALP_E_NOMEM, "pool full");
    Solve *v = new (std::nothrow) Solve();
    if (!v) {
        pool_free(s, off, bytes);
        return server_fail(SCALP_E_NOMEM, "host allocation failed");
    }
    // the region's previous owner was delivered, so no enqueued work uses it:
    // the set-up runs on a side stream right away
    scalp_params p = s->params;
    p.workspace = s->pool + off;
    p.workspace_bytes = bytes;
    cudaStream_t side = s->side[s->side_next++ % SIDE_STREAMS];
    p.stream = side;
    int rc = scalp_init(&v->ctx, image, contour, K, m, &p);
    if (rc != SCALP_OK) {
        pool_free(s, off, bytes);
        delete v;
        return rc;
    }
    cudaError_t e = spare_event(s, v->done);
    if (e == cudaSuccess) e = spare_event(s, v->ready);
    if (e == cudaSuccess) e = cudaEventRecord(v->ready, side);
    if (e != cudaSuccess) {
        scalp_destroy(v->ctx);
        if (v->done) s->spare_events.push_back(v->done);
        if (v->ready) s->spare_events.push_back(v->ready);
        pool_free(s, off, bytes);
        delete v;
        return server_fail(SCALP_E_CUDA, "request set-up: %s", cudaGetErrorString(e));
    }
    v->status_slot = s->free_status.back();
    s->free_status.pop_back();
    v->id = s->next_id++;
    v->off = off;
    v->bytes = bytes;
    v->iters_left = iters;
    v->pixels = (long long)image->H * image->W;
    v->enforce = enforce;
    v->labels_out = labels_out;
    s->active.push_back(v);
    s->by_id[v->id] = v;
    s->args_dirty = true;
    *id = v->id;
    return SCALP_OK;
}

int scalp_server_step(scalp_server *s, int32_t *n_running)
{
    if (!s) return server_fail(SCALP_E_ARG, "server is NULL");
    std::vector<Solve *> running;  // admission (id) order
    for (Solve *v : s->active)
        if (!v->retired && v->iters_left > 0) running.push_back(v);
    if (s->step_pixels > 0 && running.size() > 1) {
        // least remaining work first (pixels x iterations left, then id), as
        // many as the budget holds, at least one; back in id order after
        std::stable_sort(running.begin(), running.end(), [](const Solve *u, const Solve *v) {
            return u->pixels * u->iters_left < v->pixels * v->iters_left;
        });
        size_t take = 1;
        long long sum = running[0]->pixels;
        while (take < running.size() && sum + running[take]->pixels <= s->step_pixels)
            sum += running[take++]->pixels;
        running.resize(take);
        std::sort(running.begin(), running.end(), [](const Solve *u, const Solve *v) { return u->id < v->id; });
    }
    if (!running.empty()) {
        // bounded run-ahead: wait for the step STEPS_AHEAD launches back, so a
        // request admitted now joins within that many steps instead of
        // queueing behind every step the host could enqueue
        const int slot = s->step_next;
        if (s->step_live[slot]) {
            const cudaError_t w = cudaEventSynchronize(s->step_done[slot]);
            if (w != cudaSuccess) return server_fail(SCALP_E_CUDA, "step wait: %s", cudaGetErrorString(w));
            s->step_live[slot] = false;
        }
        std::vector<uint64_t> ids(running.size());
        for (size_t i = 0; i < running.size(); ++i) ids[i] = running[i]->id;
        if (s->args_dirty || ids != s->arg_ids) {
            const int rc = rebuild_args(s, running);
            if (rc) return rc;
            s->arg_ids.swap(ids);
        }
        for (Solve *v : running) {  // new requests: their set-up first
            if (v->joined) continue;
            const cudaError_t w = cudaStreamWaitEvent(s->st, v->ready, 0);
            if (w != cudaSuccess) return server_fail(SCALP_E_CUDA, "join: %s", cudaGetErrorString(w));
            v->joined = true;
        }
        launch_assign_batch(s->bargs, s->params.storage, s->total_tiles, s->smem, s->st, true);
        launch_batch_update(s->bargs, s->total_clusters, s->total_fill, s->st, true);
        cudaError_t e = cudaGetLastError();
        // the argument slot stays live until this step has run
        if (e == cudaSuccess) e = cudaEventRecord(s->ring_ev[s->ring_cur], s->st);
        if (e == cudaSuccess) e = cudaEventRecord(s->step_done[slot], s->st);
        if (e == cudaSuccess) {
            s->step_live[slot] = true;
            s->step_next = (slot + 1) % STEPS_AHEAD;
        }
        if (e != cudaSuccess) return server_fail(SCALP_E_CUDA, "server step: %s", cudaGetErrorString(e));
        for (Solve *v : running) {
            --v->iters_left;
            scalp_ctx_count_iteration(v->ctx);
        }
    }
    // retire the solves whose iterations are done: connectivity and copies on
    // a side stream, after the steps so far (and the set-up, for a request
    // that never ran one)
    bool forked = false;
    for (Solve *v : s->active) {
        if (v->retired || v->iters_left > 0) continue;
        cudaError_t e = cudaSuccess;
        if (!forked) {
            e = cudaEventRecord(s->step_ev, s->st);
            forked = true;
        }
        cudaStream_t side = s->side[s->side_next++ % SIDE_STREAMS];
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, s->step_ev, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, v->ready, 0);
        if (e != cudaSuccess) return server_fail(SCALP_E_CUDA, "retire: %s", cudaGetErrorString(e));
        scalp_ctx_set_stream(v->ctx, side);
        const int rc = scalp_ctx_enqueue_labels(v->ctx, v->labels_out, v->enforce, &s->status[v->status_slot]);
        if (rc) return rc;
        e = cudaEventRecord(v->done, side);
        if (e != cudaSuccess) return server_fail(SCALP_E_CUDA, "record: %s", cudaGetErrorString(e));
        v->retired = true;
        s->args_dirty = true;
    }
    if (n_running) *n_running = (int32_t)running.size();
    return SCALP_OK;
}

int scalp_server_set_step_budget(scalp_server *s, int64_t max_pixels)
{
    if (!s || max_pixels < 0) return server_fail(SCALP_E_ARG, "need a server and max_pixels >= 0");
    s->step_pixels = max_pixels;
    return SCALP_OK;
}

int scalp_server_poll(scalp_server *s, uint64_t id, int32_t *done, int32_t *n_labels)
{
    if (!s || !done) return server_fail(SCALP_E_ARG, "null argument");
    *done = 0;
    auto it = s->by_id.find(id);
    if (it == s->by_id.end()) return server_fail(SCALP_E_ARG, "unknown or already delivered request");
    Solve *v = it->second;
    if (!v->retired) return SCALP_OK;
    const cudaError_t q = cudaEventQuery(v->done);
    if (q == cudaErrorNotReady) return SCALP_OK;
    if (q != cudaSuccess) return server_fail(SCALP_E_CUDA, "request %llu: %s", (unsigned long long)id, cudaGetErrorString(q));
    int32_t nl = 0;
    CtxStatus &status = s->status[v->status_slot];
    if (v->inject_error) status.error = v->inject_error;
    if (v->inject_timeout) status.timeout = v->inject_timeout;
    // the request's work is complete either way: a failed request is released
    // too, so that it neither holds its pool region nor counts against
    // max_slots
    const int rc = scalp_ctx_finish_labels(v->ctx, &status, &nl);
    *done = 1;
    if (n_labels) *n_labels = rc ? 0 : nl;
    // release: the state leaves the pool.  Its done event covers every step
    // that read it (later argument blocks leave it out), so no stream wait.
    scalp_ctx_release(v->ctx);
    pool_free(s, v->off, v->bytes);
    s->free_status.push_back(v->status_slot);
    s->spare_events.push_back(v->ready);
    s->spare_events.push_back(v->done);
    s->active.erase(std::find(s->active.begin(), s->active.end(), v));
    s->by_id.erase(it);
    delete v;
    return rc;
}

int scalp_server_inject_status(scalp_server *s, uint64_t id, int32_t error, int32_t timeout)
{
    if (!s) return server_fail(SCALP_E_ARG, "server is NULL");
    auto it = s->by_id.find(id);
    if (it == s->by_id.end()) return server_fail(SCALP_E_ARG, "unknown or already delivered request");
    it->second->inject_error = error;
    it->second->inject_timeout = timeout;
    return SCALP_OK;
}

int scalp_server_stats(const scalp_server *s, int32_t *in_flight, size_t *pool_free_bytes)
{
    if (!s) return server_fail(SCALP_E_ARG, "server is NULL");
    if (in_flight) *in_flight = (int32_t)s->active.size();
    if (pool_free_bytes) {
        size_t f = 0;
        for (const auto &kv : s->free_list) f += kv.second;
        *pool_free_bytes = f;
    }
    return SCALP_OK;
}

void scalp_server_destroy(scalp_server *s)
{
    if (!s) return;
    cudaStreamSynchronize(s->st);
    for (cudaStream_t t : s->side)  // retirements still in flight
        if (t) cudaStreamSynchronize(t);
    for (Solve *v : s->active) {
        scalp_ctx_release(v->ctx);
        cudaEventDestroy(v->done);
        cudaEventDestroy(v->ready);
        delete v;
    }
    for (cudaEvent_t e : s->spare_events) cudaEventDestroy(e);
    free_host(s);
}

}  // extern "C"
