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
__device__ __noinline__ void phase_update(const BatchArgs &b, int total_clusters)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total_clusters; g += stride) {
        const int i = batch_find(b.clus_base, b.count, (int)g);
        update_cluster(b.args[i], (int)g - b.clus_base[i], 1);
    }
}

// Tile-count scans, then the projections: image i's queue entries start at
// a CTA that moves with i, so the first entries of the images do not all
// fall on the same CTAs.
__device__ __noinline__ void phase_project(const BatchArgs &b)
{
    const int G = gridDim.x;
    for (int i = blockIdx.x; i < b.count; i += G) scan_tiles_cta<ASSIGN_THREADS>(b.args[i]);
    for (int i = 0; i < b.count; ++i) {
        const int j0 = (int)((blockIdx.x + (long long)i * (G - 97 % G)) % G);
        project_cta(b.args[i], 0, j0, G);
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

// The assignment phase: tiles from the queue until it runs dry.
template <typename T>
__device__ __noinline__ void phase_assign(const BatchArgs &b, const int *order, const int *order_base,
                                          unsigned *queue, int total_tiles, unsigned char *smem)
{
    __shared__ int s_tile;
    while (true) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int g = s_tile;
        if (g >= total_tiles) break;
        const int j = batch_find(order_base, b.count, g);
        assign_tile<T>(b.args[order[j]], g - order_base[j], smem);
        __syncthreads();  // the tile's shared memory and s_tile are reused
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
        phase_project(q.b);
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
