// scalp_assign.cu -- the assignment step of SCALP (Algorithm 1, inner loops)
// restated per tile of pixels, plus the fused partial sums of the update.
//
// Algorithm 1 loops over clusters and, for each pixel of a cluster's
// (2r+1)x(2r+1) window, keeps the cluster with the smallest D(p, C_k) (Eq. 3)
// under a strict '<' in ascending k.  Here each pixel evaluates the same set of
// clusters (those whose window holds it, from its tile's candidate list) and
// keeps the smallest (D, k) pair: the same result, in any evaluation order.
//
// One CTA of 512 threads (two per SM) labels a 32 x 32 tile:
//   1. The tile's candidate clusters are copied to shared memory, sorted by
//      cluster index.
//   2. Distance maps.  For a candidate k, every path from a tile pixel in its
//      window to its endpoint e_k lies in the bounding box of those pixels and
//      e_k.  Over that box the CTA computes once the colour distance
//      d_c(q, C_k) of Eq. 1 and the contour factor w(q) of Eq. 2 (an FP32
//      pair per pixel, read from the (L, a, b, w) plane in global memory).
//      The boxes of the candidates are packed in candidate order into the map
//      buffer; a candidate whose box no longer fits walks the plane in global
//      memory instead, with the same per-sample arithmetic and order.
//   3. Pass 1: each warp evaluates its own 64 pixels' previous labels (when
//      they are candidates of the pixel); the previous label usually wins
//      again, and its D stays in the thread's registers.
//   4. Pass 2: each warp checks its pixels against the other candidates
//      whose rectangle (the tile's pixels inside the window) holds them.  A
//      pair whose lower bound fl(fl(lam*d_c(p)) + fl(m^2/r^2*d_s)) exceeds
//      the pixel's pass-1 D cannot win or tie (its computed D is never below
//      the bound) and is not walked; the others are queued per warp and
//      walked 32 at a time by that warp.
//   5. Each walk follows the pixel's path to the candidate's endpoint (one
//      8-byte map load and one packed two-float add per sample), forms D
//      (Eq. 1-3) and takes a 64-bit shared-memory atomicMin of (D bits,
//      candidate slot) for its pixel; slots are in cluster order, so ties go
//      to the smallest k.  The argmin is that of evaluating every pair.
//   6. Each thread writes its pixels' labels; warp-aggregated integer sums of
//      (1, x, y, L, a, b) per label go to the global cluster sums as
//      fire-and-forget reductions.
// The tile body is in scalp_assign_tile.cuh (shared with the persistent
// batched kernel).
// A tile with more candidates than shared memory holds evaluates its pixels
// one by one from the global candidate list instead.
#include <algorithm>
#include <cfloat>
#include <climits>

#include "scalp_launch.h"
#include "scalp_assign_tile.cuh"

namespace scalp {

size_t assign_smem_bytes(int map_cap)
{
    return tile_layout(MAX_TILE_CANDIDATES).maps + (size_t)map_cap * sizeof(float2);
}

// Map capacity (pairs) when ASSIGN_CTAS_PER_SM CTAs share an SM's shared memory.
int assign_map_capacity(int device)
{
    int per_sm = 0, per_cta_max = 0, reserved = 0;
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&per_cta_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device) !=
            cudaSuccess)
        return 0;
    // PERSIST_STATIC_SMEM stays free for the persistent batched kernel's own
    // static shared memory (the same capacity serves every assignment kernel)
    long long per_cta = std::min((long long)per_cta_max,
                                 (long long)per_sm / ASSIGN_CTAS_PER_SM - reserved) - PERSIST_STATIC_SMEM;
    per_cta &= ~15LL;
    const long long cap = (per_cta - (long long)tile_layout(MAX_TILE_CANDIDATES).maps) / (long long)sizeof(float2);
    return cap > 0 ? (int)cap : 0;
}

template <typename T>
__global__ void __launch_bounds__(ASSIGN_THREADS, ASSIGN_CTAS_PER_SM) k_assign(SolveArgs a)
{
    pdl_wait();
    pdl_release();
    extern __shared__ __align__(16) unsigned char smem[];
    assign_tile<T>(a, blockIdx.x, smem);
}

// All tiles of all images of a batch in one launch: block g is tile
// g - tile_base[i] of image i, tile_base being the prefix of tile counts.
template <typename T>
__global__ void __launch_bounds__(ASSIGN_THREADS, ASSIGN_CTAS_PER_SM) k_assign_batch(BatchArgs b)
{
    pdl_wait();
    pdl_release();
    extern __shared__ __align__(16) unsigned char smem[];
    const int g = blockIdx.x;
    const int i = batch_find(b.tile_base, b.count, g);
    assign_tile<T, true>(b.args[i], g - b.tile_base[i], smem);
}

void launch_assign(const SolveArgs &a, int storage, size_t smem_bytes, cudaStream_t st, bool pdl)
{
    const dim3 grid(a.n_tx * a.n_ty), block(ASSIGN_THREADS);
    if (storage == 0) pdl_launch(pdl, k_assign<float4>, grid, block, smem_bytes, st, a);
    else pdl_launch(pdl, k_assign<uint2>, grid, block, smem_bytes, st, a);
}

void launch_assign_batch(const BatchArgs &b, int storage, int total_tiles, size_t smem_bytes,
                         cudaStream_t st, bool pdl)
{
    if (total_tiles <= 0) return;
    const dim3 grid(total_tiles), block(ASSIGN_THREADS);
    if (storage == 0) pdl_launch(pdl, k_assign_batch<float4>, grid, block, smem_bytes, st, b);
    else pdl_launch(pdl, k_assign_batch<uint2>, grid, block, smem_bytes, st, b);
}

// The limit is a property of the kernel, shared by every context on the
// device: it is always set to the full map buffer, which covers any launch.
static cudaError_t configure(const void *f)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)assign_smem_bytes(assign_map_capacity(dev)));
}

cudaError_t assign_batch_configure(int storage)
{
    return configure(storage == 0 ? (const void *)k_assign_batch<float4> : (const void *)k_assign_batch<uint2>);
}

cudaError_t assign_configure(int storage)
{
    return configure(storage == 0 ? (const void *)k_assign<float4> : (const void *)k_assign<uint2>);
}

}  // namespace scalp
