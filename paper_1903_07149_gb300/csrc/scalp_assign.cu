// scalp_assign.cu -- the assignment step of SCALP (Algorithm 1, inner loops)
// restated per pixel, plus the fused partial sums of the cluster update.
//
// Algorithm 1 loops over clusters and, for each pixel of a cluster's
// (2r+1)x(2r+1) window, keeps the cluster with the smallest D(p, C_k) (Eq. 3)
// under a strict '<' in ascending k.  Here each pixel evaluates the same set
// of clusters (those whose window holds it, taken from its tile's candidate
// list) and keeps the lexicographically smallest (D, k): the same result,
// independent of the visiting order.
//
// One CTA labels a 32 x 16 tile; each warp an 8 x 4 block, one pixel per lane.
// Staged variant: the (L, a, b, w) plane of the tile plus a halo of
// round(r) + 2 pixels is copied into shared memory by one TMA bulk-tensor load
// (tile mode, zero fill outside the image), so every path to an endpoint
// within the halo is walked on-chip; a path to a farther endpoint (a
// projected barycenter, Eq. 4) is walked in global memory with the same code.
// Unstaged variant (halo does not fit): every path is walked in global memory.
#include <cfloat>
#include <climits>

#include "scalp_launch.h"

namespace scalp {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Waits on phase `parity` of an mbarrier for at most `max_polls` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int max_polls)
{
    for (int i = 0; i < max_polls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <typename T>
__device__ __forceinline__ void tma_load_region(const CUtensorMap *tmap, uint32_t dst, uint32_t bar,
                                                int rx0, int ry0);

// FP32 planes: 3-D map {4 channels, W, H} of fp32, box {4, BX, BY}.
template <>
__device__ __forceinline__ void tma_load_region<float4>(const CUtensorMap *tmap, uint32_t dst,
                                                        uint32_t bar, int rx0, int ry0)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];"
        :
        : "r"(dst), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(0), "r"(rx0), "r"(ry0), "r"(bar)
        : "memory");
}

// FP16 planes: 2-D map {W, H} of 8-byte pixels, box {BX, BY}; rx0 is even.
template <>
__device__ __forceinline__ void tma_load_region<uint2>(const CUtensorMap *tmap, uint32_t dst,
                                                       uint32_t bar, int rx0, int ry0)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];"
        :
        : "r"(dst), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(rx0), "r"(ry0), "r"(bar)
        : "memory");
}

__host__ __device__ inline size_t region_bytes(int halo, int elem)
{
    size_t bx = TILE_X + 2 * halo, by = TILE_Y + 2 * halo;
    return (bx * by * elem + 127) & ~(size_t)127;
}

size_t assign_smem_bytes(int halo, int storage)
{
    size_t elem = storage == 0 ? 16 : 8;
    size_t r = halo > 0 ? region_bytes(halo, (int)elem) : 0;
    return r + MAX_TILE_CANDIDATES * sizeof(ClusterDev) + MAX_TILE_CANDIDATES * sizeof(ClusterAcc) +
           16;
}

constexpr int MBAR_MAX_POLLS = 1 << 22;

template <typename T, bool STAGED>
__global__ void __launch_bounds__(ASSIGN_THREADS, 1)
    k_assign(SolveArgs a, const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const T *__restrict__ plane = reinterpret_cast<const T *>(
        sizeof(T) == 16 ? (const void *)a.plane32 : (const void *)a.plane16);
    const int tile = blockIdx.x;
    const int tx = tile % a.n_tx, ty = tile / a.n_tx;
    const int x0 = tx * TILE_X, y0 = ty * TILE_Y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px = x0 + (warp % (TILE_X / WARP_BLOCK_X)) * WARP_BLOCK_X + (lane % WARP_BLOCK_X);
    const int py = y0 + (warp / (TILE_X / WARP_BLOCK_X)) * WARP_BLOCK_Y + (lane / WARP_BLOCK_X);
    const bool valid = px < a.W && py < a.H;
    const long long p = (long long)py * a.W + px;

    const int halo = STAGED ? a.halo : 0;
    const int BX = TILE_X + 2 * halo, BY = TILE_Y + 2 * halo;
    const int rx0 = x0 - halo, ry0 = y0 - halo;
    const size_t rbytes = STAGED ? region_bytes(halo, sizeof(T)) : 0;
    T *region = reinterpret_cast<T *>(smem);
    ClusterDev *cand = reinterpret_cast<ClusterDev *>(smem + rbytes);
    ClusterAcc *sacc = reinterpret_cast<ClusterAcc *>(cand + MAX_TILE_CANDIDATES);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sacc + MAX_TILE_CANDIDATES);

    if (STAGED && threadIdx.x == 0) {
        uint32_t bar = smem_u32(mbar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        uint32_t bytes = (uint32_t)(BX * BY * sizeof(T));
        asm volatile(
            "{\n\t.reg .b64 st;\n\t"
            "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
            "r"(bytes)
            : "memory");
        tma_load_region<T>(&tmap, smem_u32(region), bar, rx0, ry0);
    }

    const int off = a.tile_off[tile];
    // the list capacity is a proven bound; the clamp only guards memory if the
    // device-side overflow check (reported as an error) ever fired
    const int cnt = (int)max(0LL, min((long long)a.tile_off[tile + 1], a.tile_cap) - off);
    for (int i = threadIdx.x; i < MAX_TILE_CANDIDATES * 8; i += ASSIGN_THREADS)
        reinterpret_cast<unsigned long long *>(sacc)[i] = 0ull;

    bool staged_ok = true;
    if (STAGED) {
        __syncthreads();  // barrier initialised before anyone polls it
        staged_ok = mbar_wait_bounded(smem_u32(mbar), 0, MBAR_MAX_POLLS);
        if (!staged_ok) {
            if (threadIdx.x == 0) atomicExch(&a.ctr->timeout, 1);
            // let the copy land (bounded) before the CTA releases its memory
            mbar_wait_bounded(smem_u32(mbar), 0, MBAR_MAX_POLLS);
        }
    }
    if (!__syncthreads_and(staged_ok)) return;

    float4 own = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        own = STAGED ? fetch_sample<T>(region + (py - ry0) * BX + (px - rx0))
                     : fetch_sample<T>(plane + (long long)py * a.pitch + px);
    }
    float best = FLT_MAX;
    int bestk = INT_MAX, bestslot = -1;
    unsigned long long my_samples = 0, my_pairs = 0;

    for (int base = 0; base < cnt; base += MAX_TILE_CANDIDATES) {
        const int nb = min(MAX_TILE_CANDIDATES, cnt - base);
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += ASSIGN_THREADS)
            cand[i] = a.cdev[a.tile_list[off + base + i]];
        __syncthreads();
        if (!valid) continue;
        for (int c = 0; c < nb; ++c) {
            const ClusterDev cd = cand[c];
            if (px < cd.xlo || px > cd.xhi || py < cd.ylo || py > cd.yhi) continue;
            const PathSetup s = path_setup(px, py, cd.ex, cd.ey);
            float sdc, sw;
            int len;
            bool inside = STAGED && cd.ex >= rx0 && cd.ex < rx0 + BX && cd.ey >= ry0 &&
                          cd.ey < ry0 + BY;
            if (inside) len = path_sums<T>(region, BX, rx0, ry0, s, cd.L, cd.a, cd.b, sdc, sw);
            else len = path_sums<T>(plane, a.pitch, 0, 0, s, cd.L, cd.a, cd.b, sdc, sw);
            float dl = own.x - cd.L, da = own.y - cd.a, db = own.z - cd.b;
            float dcp = fmaf(dl, dl, fmaf(da, da, db * db));
            float ddx = (float)px - cd.xk, ddy = (float)py - cd.yk;
            float ds = fmaf(ddx, ddx, ddy * ddy);
            float D = scalp_distance(dcp, sdc, sw, len, a.lam, a.gamma, a.ms2, ds);
            const int k = cd.pad;
            if (D < best || (D == best && k < bestk)) {
                best = D;
                bestk = k;
                bestslot = base + c;
            }
            my_samples += len;
            my_pairs += 1;
        }
    }

    int lab = 0;
    if (valid) {
        if (bestk != INT_MAX) {
            lab = bestk;
            a.labels[p] = lab;
        } else {
            lab = a.labels[p];  // no window reaches p: keep its label
            atomicAdd(&a.ctr->orphans, 1);
        }
    }
    const bool in_slot = valid && bestslot >= 0 && bestslot < MAX_TILE_CANDIDATES;
    warp_aggregate_tile(in_slot, bestslot, px, py, own, sacc);
    const bool direct = valid && !in_slot;
    if (__any_sync(0xffffffffu, direct)) warp_aggregate_global(direct, lab, px, py, own, a.acc);
    if (a.count_samples) {
        for (int o = 16; o > 0; o >>= 1) {
            my_samples += __shfl_down_sync(0xffffffffu, my_samples, o);
            my_pairs += __shfl_down_sync(0xffffffffu, my_pairs, o);
        }
        if (lane == 0) {
            atomicAdd(&a.ctr->samples, my_samples);
            atomicAdd(&a.ctr->pairs, my_pairs);
        }
    }
    __syncthreads();
    const int nslots = min(cnt, MAX_TILE_CANDIDATES);
    for (int s = threadIdx.x; s < nslots; s += ASSIGN_THREADS) {
        const ClusterAcc c = sacc[s];
        if (c.n == 0) continue;
        ClusterAcc *g = &a.acc[a.tile_list[off + s]];
        atomicAdd(&g->n, c.n);
        atomicAdd(&g->sx, c.sx);
        atomicAdd(&g->sy, c.sy);
        atomicAdd(&g->sL, c.sL);
        atomicAdd(&g->sa, c.sa);
        atomicAdd(&g->sb, c.sb);
    }
}

template <typename T, bool STAGED>
static void launch_one(const SolveArgs &a, const CUtensorMap &tmap, size_t smem, cudaStream_t st)
{
    k_assign<T, STAGED><<<a.n_tx * a.n_ty, ASSIGN_THREADS, smem, st>>>(a, tmap);
}

void launch_assign(const SolveArgs &a, int storage, bool staged, const CUtensorMap &tmap,
                   size_t smem_bytes, cudaStream_t st)
{
    if (storage == 0) {
        if (staged) launch_one<float4, true>(a, tmap, smem_bytes, st);
        else launch_one<float4, false>(a, tmap, smem_bytes, st);
    } else {
        if (staged) launch_one<uint2, true>(a, tmap, smem_bytes, st);
        else launch_one<uint2, false>(a, tmap, smem_bytes, st);
    }
}

cudaError_t assign_configure(int storage, bool staged, size_t smem_bytes)
{
    const void *f;
    if (storage == 0) f = staged ? (const void *)k_assign<float4, true> : (const void *)k_assign<float4, false>;
    else f = staged ? (const void *)k_assign<uint2, true> : (const void *)k_assign<uint2, false>;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

}  // namespace scalp
