// scalp_persistent.cu -- the iterations of a whole batch as one persistent
// launch.
//
// n iterations of Algorithm 1 for every image of a batch run in one
// cooperative launch with one CTA per resident slot (two per SM).  Each
// iteration is four phases separated by grid-wide barriers:
//   1. assignment: the CTAs take tiles from a queue over every tile of every
//      image and label each (the body of the per-iteration kernels,
//      scalp_assign_tile.cuh), with the update's fused partial sums;
//   2. update of every cluster of every image, one thread each;
//   3. the scan of each image's tile counts (one CTA per image) and the
//      projection (Eq. 4) of each image's queued clusters (one CTA per queued
//      cluster, spread over the grid);
//   4. the candidate lists: every (cluster, tile) slot of every image.
// The phases run the same device bodies in the same order of effects as the
// per-kernel launches (the sums are integers, so the order in which tiles
// add to them does not matter), so the results are bit-identical to those.
//
// The queue takes the images in a host-chosen order: in batch order, or by
// descending grid step r, so that the tiles with the longest paths start
// first and the cheap ones fill the tail of the phase.
//
// Every barrier wait is bounded.  A CTA that has waited longer than the
// batch's wait limit raises the timeout flag in every image's counters and an
// abort word, and returns; the other CTAs find the abort word at their next
// wait and return too.  The host reads SCALP_E_TIMEOUT at its next status
// read, and the batch stays usable after a reload.  A cooperative launch
// places every CTA at once (or fails to launch), so no CTA waits on one that
// has not started.
#include <algorithm>

#include "scalp_launch.h"
#include "scalp_assign_tile.cuh"
#include "scalp_phases.cuh"

namespace scalp {

namespace {

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with a bounded wait (target arrivals, wait_ns at most);
// false: the launch is being abandoned (this CTA or another gave up), and
// the caller returns at once.
__device__ __noinline__ bool grid_wait(PersistSync *y, unsigned target, long long wait_ns,
                                       const SolveArgs *args, int count)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = ld_acquire(&y->abort) == 0;
        if (ok) {
            const unsigned gen = ld_acquire(&y->gen);
            __threadfence();  // this CTA's writes before its arrival
            if (atomicAdd(&y->arrive, 1u) + 1u == target) {
                atomicExch(&y->arrive, 0u);
                __threadfence();
                atomicAdd(&y->gen, 1u);
            } else {
                const unsigned long long t0 = global_ns();
                // a cap on the polls as well, in case the timer stalls: each
                // poll is an L2 round trip plus a sleep of at least 64 ns
                const unsigned long long max_polls = (unsigned long long)wait_ns / 64 + 4096;
                unsigned long long polls = 0;
                unsigned sleep_ns = 64;
                while (ld_acquire(&y->gen) == gen) {
                    if (ld_acquire(&y->abort)) {
                        ok = 0;
                        break;
                    }
                    if (global_ns() - t0 > (unsigned long long)wait_ns || ++polls > max_polls) {
                        ok = 0;
                        atomicExch(&y->abort, 1u);
                        for (int i = 0; i < count; ++i) atomicExch(&args[i].ctr->timeout, 1);
                        break;
                    }
                    __nanosleep(sleep_ns);
                    if (sleep_ns < 2048) sleep_ns <<= 1;
                }
            }
            __threadfence();  // the other CTAs' writes after the barrier
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Phases 2-4 out of line: their registers (128-bit projection arithmetic)
// stay out of the assignment's allocation.
//
// The update of one cluster is a chain of dependent loads and 128-bit window
// arithmetic: every CTA takes an equal run of consecutive clusters, so that
// the chains spread over all SMs (a grid-stride loop would leave most CTAs
// idle: a batch has far fewer clusters than the grid has threads).
__device__ __noinline__ void phase_update(const BatchArgs &b, int total_clusters)
{
    const int chunk = (total_clusters + gridDim.x - 1) / gridDim.x;
    const int end = min(total_clusters, (int)(blockIdx.x + 1) * chunk);
    for (int g = blockIdx.x * chunk + threadIdx.x; g < end; g += blockDim.x) {
        const int i = batch_find(b.clus_base, b.count, g);
        update_cluster(b.args[i], g - b.clus_base[i], 1);
    }
}


// The whole-image searches (an image whose last assignment left pixels with
// no candidate), one CTA per queued cluster: out of line, so that their
// registers stay out of the other phases' allocation.
__device__ __noinline__ void project_whole_image(const SolveArgs &a, int j)
{
    project_cta(a, 0, j, INT_MAX);
}

// Tile-count scans (one CTA per image), then the projections: every CTA
// lays out the same list of all queued clusters of all images (a prefix over
// the images' queue lengths, in the dynamic shared memory the assignment
// phase has finished with) and its warps take entries in turn, a warp per
// cluster; the clusters of images that need a whole-image search are taken
// by whole CTAs afterwards.  Needs 2 * count + 1 ints of shared memory
// (checked on the host).
__device__ __noinline__ void phase_project(const BatchArgs &b, unsigned char *smem)
{
    __shared__ int s_warp[32];
    const int G = gridDim.x, count = b.count;
    for (int i = blockIdx.x; i < count; i += G) scan_tiles_cta<ASSIGN_THREADS>(b.args[i]);
    int *s_cnt = reinterpret_cast<int *>(smem);  // per image: queue length, 0 for whole-image
    int *s_pref = s_cnt + count;                 // count + 1: its prefix
    for (int i = threadIdx.x; i < count; i += blockDim.x)
        s_cnt[i] = b.args[i].ctr->proj_all ? 0 : b.args[i].ctr->nproj;
    __syncthreads();
    cta_scan(s_cnt, s_pref, count, ASSIGN_THREADS, s_warp);
    const int total = s_pref[count];
    const int warps = blockDim.x / 32;
    for (int t = blockIdx.x * warps + (int)(threadIdx.x >> 5); t < total; t += G * warps) {
        const int i = batch_find(s_pref, count, t);
        project_warp(b.args[i], t - s_pref[i]);
    }
    // whole-image searches: image by image, entry j on CTA (j mod G)
    for (int i = 0; i < count; ++i) {
        if (s_cnt[i] != 0 || !b.args[i].ctr->proj_all) continue;
        const int nproj = b.args[i].ctr->nproj;
        for (int j = blockIdx.x; j < nproj; j += G) project_whole_image(b.args[i], j);
    }
}

__device__ __noinline__ void phase_lists(const BatchArgs &b, int total_fill)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total_fill; g += stride) {
        const int i = batch_find(b.fill_base, b.count, (int)g);
        fill_slot(b.args[i], g - b.fill_base[i]);
    }
}

// The assignment phase: tiles from the queue until it runs dry.  The next
// tile's index is fetched while the current tile is labelled, so the queue's
// round trip is off the critical path.
template <typename T>
__device__ __forceinline__ void phase_assign(const BatchArgs &b, const int *order, const int *order_base,
                                             unsigned *queue, int total_tiles, unsigned char *smem)
{
    __shared__ int s_tile[2];
    if (threadIdx.x == 0) s_tile[0] = (int)atomicAdd(queue, 1u);
    __syncthreads();
    int slot = 0;
    for (int g = s_tile[0]; g < total_tiles; g = s_tile[slot]) {
        if (threadIdx.x == 0) s_tile[slot ^ 1] = (int)atomicAdd(queue, 1u);
        const int j = batch_find(order_base, b.count, g);
        assign_tile<T>(b.args[order[j]], g - order_base[j], smem);
        __syncthreads();  // the tile's shared memory is reused; the next index is visible
        slot ^= 1;
    }
}

template <typename T>
__global__ void __launch_bounds__(ASSIGN_THREADS, ASSIGN_CTAS_PER_SM) k_batch_persistent(PersistArgs q)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // the barrier target: every CTA, plus the test hold (never reached when > 0)
#define SCALP_GRID_WAIT() grid_wait(q.sync, (unsigned)gridDim.x + (unsigned)q.hold, q.wait_ns, q.b.args, q.b.count)
    for (int it = 0; it < q.iters; ++it) {
        // 1. assignment
        phase_assign<T>(q.b, q.order, q.order_base, &q.sync->queue, q.total_tiles, smem);
        if (!SCALP_GRID_WAIT()) return;
        // 2. update; the queue restarts for the next assignment (every CTA
        // has left it, and none reads it before two more barriers)
        if (blockIdx.x == 0 && threadIdx.x == 0) q.sync->queue = 0u;
        phase_update(q.b, q.total_clusters);
        if (!SCALP_GRID_WAIT()) return;
        // 3. scans and projections
        phase_project(q.b, smem);
        if (!SCALP_GRID_WAIT()) return;
        // 4. candidate lists
        phase_lists(q.b, q.total_fill);
        if (it + 1 < q.iters && !SCALP_GRID_WAIT()) return;
    }
#undef SCALP_GRID_WAIT
}

template <typename T>
cudaError_t persistent_query(size_t smem, int *grid)
{
    *grid = 0;
    const void *f = reinterpret_cast<const void *>(k_batch_persistent<T>);
    int dev = 0, coop = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persistent<T>, ASSIGN_THREADS, smem);
    if (e != cudaSuccess) return e;
    // the map capacity leaves PERSIST_STATIC_SMEM beside the dynamic buffer
    if (!coop || fa.sharedSizeBytes > (size_t)PERSIST_STATIC_SMEM) return cudaSuccess;
    *grid = per_sm * sms;
    return cudaSuccess;
}

}  // namespace

cudaError_t batch_persistent_grid(int storage, size_t smem, int *grid)
{
    return storage == 0 ? persistent_query<float4>(smem, grid) : persistent_query<uint2>(smem, grid);
}

cudaError_t launch_batch_persistent(const PersistArgs &q, int storage, size_t smem, int grid, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(ASSIGN_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (storage == 0) return cudaLaunchKernelEx(&cfg, k_batch_persistent<float4>, q);
    return cudaLaunchKernelEx(&cfg, k_batch_persistent<uint2>, q);
}

}  // namespace scalp
