// scalp_assign.cu -- the assignment step of SCALP (Algorithm 1, inner loops)
// restated per tile of pixels, plus the fused partial sums of the update.
//
// Algorithm 1 loops over clusters and, for each pixel of a cluster's
// (2r+1)x(2r+1) window, keeps the cluster with the smallest D(p, C_k) (Eq. 3)
// under a strict '<' in ascending k.  Here each pixel evaluates the same set of
// clusters (those whose window holds it, from its tile's candidate list) and
// keeps the smallest (D, k) pair: the same result, in any evaluation order.
//
// One CTA (1024 threads for FP32 planes, 512 for FP16) labels a 32 x 32 tile:
//   1. One thread issues a TMA bulk-tensor load of the (L, a, b, w) plane of
//      the tile plus a halo of round(r) + 2 pixels into shared memory (zero
//      fill outside the image).  Every path to an endpoint inside that region
//      is walked on-chip; a farther endpoint (a projected barycenter, Eq. 4)
//      is walked in global memory with the same stepping rule.
//   2. Meanwhile the tile's candidate clusters are copied to shared memory,
//      sorted by cluster index.
//   3. The pixels of the tile inside a candidate's window form a rectangle,
//      cut into 8 x 4 blocks; each (candidate, block) is one work item, and
//      warps take items from a shared-memory counter until none are left (no
//      per-pixel scan of the candidate list, no idle warps at a barrier).
//   4. Each lane walks its pixel's path to the candidate's endpoint, forms D
//      (Eq. 1-3) and takes a 64-bit shared-memory atomicMin of (D bits,
//      candidate slot) for its pixel; slots are in cluster order, so ties go
//      to the smallest k.
//   5. Each thread writes its pixel's label; warp-aggregated integer sums of
//      (1, x, y, L, a, b) per label go to the global cluster sums as
//      fire-and-forget reductions.
// A tile with more candidates or pairs than shared memory holds evaluates
// its pixels one by one from the global candidate list instead.
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

// FP32 planes: 2-D map {2W, H} of 8-byte elements (half a pixel each), box
// {2BX, BY}: long contiguous rows per request; x = 2*rx0 is 16-byte aligned.
template <>
__device__ __forceinline__ void tma_load_region<float4>(const CUtensorMap *tmap, uint32_t dst,
                                                        uint32_t bar, int rx0, int ry0)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];"
        :
        : "r"(dst), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(2 * rx0), "r"(ry0), "r"(bar)
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

// One sample of the staged plane, by 32-bit shared-memory byte address.
template <typename T>
__device__ __forceinline__ float4 lds_sample(uint32_t addr);
template <>
__device__ __forceinline__ float4 lds_sample<float4>(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}
template <>
__device__ __forceinline__ float4 lds_sample<uint2>(uint32_t addr)
{
    uint2 u;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(u.x), "=r"(u.y) : "r"(addr));
    __half2 lo = *reinterpret_cast<__half2 *>(&u.x);
    __half2 hi = *reinterpret_cast<__half2 *>(&u.y);
    float2 a = __half22float2(lo), b = __half22float2(hi);
    return make_float4(a.x, a.y, b.x, b.y);
}

// Path sums of Eq. 1 and Eq. 2 over the staged region (row pitch BX elements,
// element (0,0) = image pixel (rx0, ry0)).
template <typename T>
__device__ __forceinline__ int path_sums_smem(uint32_t region, int BX, int rx0, int ry0,
                                              const PathSetup &s, float cL, float ca, float cb,
                                              float &sum_dc, float &sum_w)
{
    int smaj, smin;
    path_strides(s, BX, smaj, smin);
    const uint32_t q0 = region + (uint32_t)(((s.ay - ry0) * BX + (s.ax - rx0)) * (int)sizeof(T));
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, bw = 0.f;
    int len = walk_steps(q0, smaj * (int)sizeof(T), smin * (int)sizeof(T), s, [&](uint32_t q) {
        float4 v = lds_sample<T>(q);
        float dl = v.x - cL, da = v.y - ca, db = v.z - cb;
        a0 = fmaf(dl, dl, a0);
        a1 = fmaf(da, da, a1);
        a2 = fmaf(db, db, a2);
        bw += v.w;
    });
    sum_dc = (a0 + a1) + a2;
    sum_w = bw;
    return len;
}

__host__ __device__ inline size_t region_bytes(int halo, int elem)
{
    size_t bx = TILE_X + 2 * halo, by = TILE_Y + 2 * halo;
    return (bx * by * elem + 127) & ~(size_t)127;
}

// Shared-memory layout after the staged region; every section starts on a
// 16-byte boundary (int4 loads, 8-byte atomics and the mbarrier need it).
constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
constexpr int STRIP = 4;  // items run along strips STRIP pixels wide
constexpr int MAX_ITEMS = MAX_TILE_CANDIDATES * (TILE_PIXELS / 32);
constexpr int STRIP_RCP_BITS = 20;
// the strip index j / (STRIP * len) by a STRIP_RCP_BITS-bit reciprocal is exact
// when the rounding error j / 2^STRIP_RCP_BITS stays below 1 / (STRIP * len)
static_assert((long long)TILE_PIXELS * STRIP * (TILE_X > TILE_Y ? TILE_X : TILE_Y) <
                  (1LL << STRIP_RCP_BITS),
              "exact strip index");
struct AssignSmem {
    static constexpr size_t cand = 0;
    static constexpr size_t cid = align16(cand + MAX_TILE_CANDIDATES * sizeof(ClusterDev));
    static constexpr size_t rect = align16(cid + MAX_TILE_CANDIDATES * sizeof(int));
    static constexpr size_t meta = align16(rect + MAX_TILE_CANDIDATES * sizeof(int4));
    static constexpr size_t nit = align16(meta + MAX_TILE_CANDIDATES * sizeof(int2));
    static constexpr size_t best = align16(nit + MAX_TILE_CANDIDATES * sizeof(int));
    static constexpr size_t first = align16(best + TILE_PIXELS * sizeof(unsigned long long));
    static constexpr size_t owner = align16(first + (MAX_TILE_CANDIDATES + 1) * sizeof(int));
    static constexpr size_t misc = align16(owner + MAX_ITEMS);
    static constexpr size_t total = align16(misc + 64);
};
static_assert(AssignSmem::cid % 16 == 0 && AssignSmem::rect % 16 == 0 && AssignSmem::meta % 16 == 0 &&
                  AssignSmem::nit % 16 == 0 &&
                  AssignSmem::best % 16 == 0 && AssignSmem::first % 16 == 0 &&
                  AssignSmem::owner % 16 == 0 && AssignSmem::misc % 16 == 0 &&
                  (AssignSmem::misc + 32) % 8 == 0,
              "shared-memory sections aligned");
static_assert(MAX_TILE_CANDIDATES <= 256, "item owners are bytes");
static_assert(MAX_TILE_CANDIDATES % 32 == 0, "the item scan gives each lane whole candidates");

size_t assign_smem_bytes(int halo, int storage)
{
    size_t elem = storage == 0 ? 16 : 8;
    size_t r = halo > 0 ? region_bytes(halo, (int)elem) : 0;
    return r + AssignSmem::total;
}

// Threads per CTA: FP32 tiles use one 1024-thread CTA per SM (the staged
// region fills shared memory); FP16 tiles use 512-thread CTAs, two per SM, so
// one CTA's set-up and tail overlap the other's walks.
int assign_threads(int storage) { return storage == 0 ? 1024 : 512; }

constexpr int MBAR_MAX_POLLS = 1 << 22;

__device__ __forceinline__ unsigned long long pack_best(float D, int slot)
{
    // D >= 0, so its IEEE bits order like the value; ties fall to the slot
    return ((unsigned long long)__float_as_uint(D) << 32) | (unsigned)slot;
}

// Items: the pixels of a candidate's window that lie in the tile form a
// rectangle.  When the rectangle lies mostly left or right of the path
// endpoint (paths mostly along x, |P| set by the column) it is cut into
// vertical strips STRIP columns wide, otherwise into horizontal strips STRIP
// rows high.  The strips are read one after the other, each across its width
// first, and every 32 consecutive pixels of that order form one warp's item.
// So a warp's pixels lie in a few neighbouring columns (rows), where the path
// lengths differ little, and only the last item of a rectangle has idle lanes.
// One tile of one image (the body shared by the single-image and the batched
// kernels).  `tmap` is the image's tensor map (kernel parameter or global).
template <typename T, bool STAGED, int THREADS>
__device__ __forceinline__ void assign_tile(const SolveArgs &a, const CUtensorMap *tmap, int tile,
                                            unsigned char *smem)
{
    constexpr int PIX_PER_THREAD = TILE_PIXELS / THREADS;
    constexpr int WARPS = THREADS / 32;
    const T *__restrict__ plane = reinterpret_cast<const T *>(
        sizeof(T) == 16 ? (const void *)a.plane32 : (const void *)a.plane16);
    const int tx = tile % a.n_tx, ty = tile / a.n_tx;
    const int x0 = tx * TILE_X, y0 = ty * TILE_Y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int halo = STAGED ? a.halo : 0;
    const int BX = TILE_X + 2 * halo, BY = TILE_Y + 2 * halo;
    const int rx0 = x0 - halo, ry0 = y0 - halo;
    const size_t rbytes = STAGED ? region_bytes(halo, sizeof(T)) : 0;
    unsigned char *sm = smem + rbytes;
    const uint32_t region = smem_u32(smem);
    ClusterDev *cand = reinterpret_cast<ClusterDev *>(sm + AssignSmem::cand);
    int *cid = reinterpret_cast<int *>(sm + AssignSmem::cid);
    int4 *rect = reinterpret_cast<int4 *>(sm + AssignSmem::rect);
    int2 *meta = reinterpret_cast<int2 *>(sm + AssignSmem::meta);
    int *nit = reinterpret_cast<int *>(sm + AssignSmem::nit);
    unsigned long long *best = reinterpret_cast<unsigned long long *>(sm + AssignSmem::best);
    int *first = reinterpret_cast<int *>(sm + AssignSmem::first);
    unsigned char *owner = sm + AssignSmem::owner;
    int *misc = reinterpret_cast<int *>(sm + AssignSmem::misc);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + AssignSmem::misc + 32);

    if (STAGED && tid == 0) {
        uint32_t bar = smem_u32(mbar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        uint32_t bytes = (uint32_t)(BX * BY * sizeof(T));
        asm volatile(
            "{\n\t.reg .b64 st;\n\t"
            "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
            "r"(bytes)
            : "memory");
        tma_load_region<T>(tmap, region, bar, rx0, ry0);
    }

    const int off = a.tile_off[tile];
    // the list capacity is a proven bound; the clamp only guards memory if the
    // device-side overflow check (reported as an error) ever fired
    const int cnt = (int)max(0LL, min((long long)a.tile_off[tile + 1], a.tile_cap) - off);
    const bool fast = cnt <= MAX_TILE_CANDIDATES;

    // candidates sorted by cluster index (ranks of distinct ids); the id
    // staging reuses the `best` words before they are initialised
    int *ids = reinterpret_cast<int *>(best);
    int myid = INT_MAX;
    if (fast && tid < cnt) {
        myid = a.tile_list[off + tid];
        ids[tid] = myid;
    }
    if (tid == 0) misc[1] = 0;  // work counter
    __syncthreads();
    if (fast && tid < cnt) {
        int rank = 0;
        for (int j = 0; j < cnt; ++j) rank += ids[j] < myid;
        const ClusterDev cd = a.cdev[myid];
        cid[rank] = myid;
        cand[rank] = cd;
        // window x tile (clipped to the image), cut into strips
        const int xa = max(cd.xlo, x0), xb = min(min(cd.xhi, x0 + TILE_X - 1), a.W - 1);
        const int ya = max(cd.ylo, y0), yb = min(min(cd.yhi, y0 + TILE_Y - 1), a.H - 1);
        const int w = max(xb - xa + 1, 0), h = max(yb - ya + 1, 0);
        const bool vert = abs(xa + xb - 2 * cd.ex) >= abs(ya + yb - 2 * cd.ey);
        const int slen = max(vert ? h : w, 1);  // pixels along one strip
        const bool inside = STAGED && cd.ex >= rx0 && cd.ex < rx0 + BX && cd.ey >= ry0 &&
                            cd.ey < ry0 + BY;
        rect[rank] = make_int4(xa, ya, w, h);
        // strip direction and endpoint-in-region flags, reciprocal of the
        // pixels per full strip
        meta[rank] = make_int2((int)vert | ((int)inside << 1),
                               ((1 << STRIP_RCP_BITS) + STRIP * slen - 1) / (STRIP * slen));
        nit[rank] = (w * h + 31) >> 5;
    }
    __syncthreads();
    for (int i = tid; i < TILE_PIXELS; i += THREADS) best[i] = ~0ull;
    if (warp == 0 && fast) {
        // exclusive prefix of the per-candidate block counts (4 per lane)
        constexpr int PER = MAX_TILE_CANDIDATES / 32;
        int v[PER], sum = 0;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int c = lane * PER + i;
            v[i] = c < cnt ? nit[c] : 0;
            sum += v[i];
        }
        int incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int run = incl - sum;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int c = lane * PER + i;
            if (c < cnt) first[c] = run;
            run += v[i];
        }
        if (lane == 31) first[cnt] = incl;
    }
    __syncthreads();
    if (fast && tid < cnt) {
        const int f = first[tid], n = nit[tid];
        for (int j = 0; j < n; ++j) owner[f + j] = (unsigned char)tid;
    }

    bool staged_ok = true;
    if (STAGED) {
        staged_ok = mbar_wait_bounded(smem_u32(mbar), 0, MBAR_MAX_POLLS);
        if (!staged_ok) {
            if (tid == 0) atomicExch(&a.ctr->timeout, 1);
            // let the copy land (bounded) before the CTA releases its memory
            mbar_wait_bounded(smem_u32(mbar), 0, MBAR_MAX_POLLS);
        }
    }
    if (!__syncthreads_and(staged_ok)) return;

    unsigned long long my_samples = 0, my_pairs = 0;
    int bestk[PIX_PER_THREAD];  // per-pixel path only
#pragma unroll
    for (int j = 0; j < PIX_PER_THREAD; ++j) bestk[j] = INT_MAX;

    // this thread's pixels: block (warp + j*WARPS) of the tile, lane within it
    auto my_pixel = [&](int j, int &qx, int &qy) {
        const int blk = warp + j * WARPS;
        qx = x0 + (blk % (TILE_X / WARP_BLOCK_X)) * WARP_BLOCK_X + (lane % WARP_BLOCK_X);
        qy = y0 + (blk / (TILE_X / WARP_BLOCK_X)) * WARP_BLOCK_Y + (lane / WARP_BLOCK_X);
    };

    if (fast) {
        const int n_items = first[cnt];
        while (true) {
            int item = 0;
            if (lane == 0) item = atomicAdd(&misc[1], 1);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item >= n_items) break;
            const int c = owner[item];
            const int4 rc = rect[c];
            const int2 mt = meta[c];
            const int j = ((item - first[c]) << 5) + lane;  // pixel of the rectangle
            if (j >= rc.z * rc.w) continue;
            const bool vert = (mt.x & 1) != 0;
            const int slen = vert ? rc.w : rc.z, across = vert ? rc.z : rc.w;
            const int strip = (j * mt.y) >> STRIP_RCP_BITS;
            const int t = j - strip * STRIP * slen;
            // t / width for a strip 1..4 wide: exact 16-bit reciprocals
            const int width = min(STRIP, across - strip * STRIP);
            const int along = (t * (width == 3 ? 21846 : 65536 >> (width >> 1))) >> 16;
            const int off = strip * STRIP + (t - along * width);
            const int qx = rc.x + (vert ? off : along);
            const int qy = rc.y + (vert ? along : off);
            const ClusterDev cd = cand[c];
            const PathSetup s = path_setup(qx, qy, cd.ex, cd.ey);
            const bool inside = (mt.x >> 1) != 0;
            float sdc, sw;
            int len;
            float4 v;
            if (inside) {
                len = path_sums_smem<T>(region, BX, rx0, ry0, s, cd.L, cd.a, cd.b, sdc, sw);
                v = lds_sample<T>(region + (uint32_t)(((qy - ry0) * BX + (qx - rx0)) * (int)sizeof(T)));
            } else {
                len = path_sums<T>(plane, a.pitch, 0, 0, s, cd.L, cd.a, cd.b, sdc, sw);
                v = fetch_sample<T>(plane + (long long)qy * a.pitch + qx);
            }
            const float dl = v.x - cd.L, da = v.y - cd.a, db = v.z - cd.b;
            const float dcp = fmaf(dl, dl, fmaf(da, da, db * db));
            const float ddx = (float)qx - cd.xk, ddy = (float)qy - cd.yk;
            const float ds = fmaf(ddx, ddx, ddy * ddy);
            const float D = scalp_distance(dcp, sdc, sw, len, a.lam, a.gamma, a.ms2, ds);
            atomicMin(&best[(qy - y0) * TILE_X + (qx - x0)], pack_best(D, c));
            my_samples += len;
            my_pairs += 1;
        }
    } else {
        // per-pixel path: every candidate straight from the global list
#pragma unroll 1
        for (int j = 0; j < PIX_PER_THREAD; ++j) {
            int px, py;
            my_pixel(j, px, py);
            if (px >= a.W || py >= a.H) continue;
            const float4 own = STAGED ? lds_sample<T>(region + (uint32_t)(((py - ry0) * BX + (px - rx0)) * (int)sizeof(T)))
                                      : fetch_sample<T>(plane + (long long)py * a.pitch + px);
            float bestD = FLT_MAX;
            for (int i = 0; i < cnt; ++i) {
                const int k = a.tile_list[off + i];
                const ClusterDev cd = a.cdev[k];
                if (px < cd.xlo || px > cd.xhi || py < cd.ylo || py > cd.yhi) continue;
                const PathSetup s = path_setup(px, py, cd.ex, cd.ey);
                const bool inside = STAGED && cd.ex >= rx0 && cd.ex < rx0 + BX && cd.ey >= ry0 &&
                                    cd.ey < ry0 + BY;
                float sdc, sw;
                const int len = inside ? path_sums_smem<T>(region, BX, rx0, ry0, s, cd.L, cd.a, cd.b, sdc, sw)
                                       : path_sums<T>(plane, a.pitch, 0, 0, s, cd.L, cd.a, cd.b, sdc, sw);
                const float dl = own.x - cd.L, da = own.y - cd.a, db = own.z - cd.b;
                const float dcp = fmaf(dl, dl, fmaf(da, da, db * db));
                const float ddx = (float)px - cd.xk, ddy = (float)py - cd.yk;
                const float ds = fmaf(ddx, ddx, ddy * ddy);
                const float D = scalp_distance(dcp, sdc, sw, len, a.lam, a.gamma, a.ms2, ds);
                if (D < bestD || (D == bestD && k < bestk[j])) {
                    bestD = D;
                    bestk[j] = k;
                }
                my_samples += len;
                my_pairs += 1;
            }
        }
    }
    __syncthreads();

    // labels and the warp-aggregated integer sums of the update
#pragma unroll 1
    for (int j = 0; j < PIX_PER_THREAD; ++j) {
        int px, py;
        my_pixel(j, px, py);
        const bool valid = px < a.W && py < a.H;
        const long long p = (long long)py * a.W + px;
        float4 own = make_float4(0.f, 0.f, 0.f, 0.f);
        int lab = -1;
        if (valid) {
            own = STAGED ? lds_sample<T>(region + (uint32_t)(((py - ry0) * BX + (px - rx0)) * (int)sizeof(T)))
                         : fetch_sample<T>(plane + (long long)py * a.pitch + px);
            if (fast) {
                const unsigned long long b = best[(py - y0) * TILE_X + (px - x0)];
                if (b != ~0ull) lab = cid[(int)(b & 0xffffffffu)];
            } else if (bestk[j] != INT_MAX) {
                lab = bestk[j];
            }
            if (lab >= 0) {
                a.labels[p] = lab;
            } else {
                lab = a.labels[p];  // no window reaches p: keep its label
                atomicAdd(&a.ctr->orphans, 1);
            }
        }
        // fire-and-forget reductions into the global cluster sums, one set
        // per label group of the warp (offsets within the tile)
        warp_aggregate_global(valid, lab, x0, y0, px - x0, py - y0, own, a.acc);
    }
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
}

template <typename T, bool STAGED, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
    k_assign(SolveArgs a, const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    assign_tile<T, STAGED, THREADS>(a, &tmap, blockIdx.x, smem);
}

// All tiles of all images of a batch in one launch: block g is tile
// g - tile_base[i] of image i, tile_base being the prefix of tile counts.
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_assign_batch(BatchArgs b)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int g = blockIdx.x;
    const int i = batch_find(b.tile_base, b.count, g);
    const SolveArgs &a = b.args[i];
    if (a.halo > 0) assign_tile<T, true, THREADS>(a, &b.tmaps[i], g - b.tile_base[i], smem);
    else assign_tile<T, false, THREADS>(a, &b.tmaps[i], g - b.tile_base[i], smem);
}

template <typename T, bool STAGED, int THREADS>
static void launch_one(const SolveArgs &a, const CUtensorMap &tmap, size_t smem, cudaStream_t st)
{
    k_assign<T, STAGED, THREADS><<<a.n_tx * a.n_ty, THREADS, smem, st>>>(a, tmap);
}

void launch_assign(const SolveArgs &a, int storage, bool staged, const CUtensorMap &tmap,
                   size_t smem_bytes, cudaStream_t st)
{
    if (storage == 0) {
        if (staged) launch_one<float4, true, 1024>(a, tmap, smem_bytes, st);
        else launch_one<float4, false, 1024>(a, tmap, smem_bytes, st);
    } else {
        if (staged) launch_one<uint2, true, 512>(a, tmap, smem_bytes, st);
        else launch_one<uint2, false, 512>(a, tmap, smem_bytes, st);
    }
}

void launch_assign_batch(const BatchArgs &b, int storage, int total_tiles, size_t smem_bytes,
                         cudaStream_t st)
{
    if (total_tiles <= 0) return;
    if (storage == 0) k_assign_batch<float4, 1024><<<total_tiles, 1024, smem_bytes, st>>>(b);
    else k_assign_batch<uint2, 512><<<total_tiles, 512, smem_bytes, st>>>(b);
}

cudaError_t assign_batch_configure(int storage, size_t smem_bytes)
{
    const void *f = storage == 0 ? (const void *)k_assign_batch<float4, 1024>
                                 : (const void *)k_assign_batch<uint2, 512>;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

cudaError_t assign_configure(int storage, bool staged, size_t smem_bytes)
{
    const void *f;
    if (storage == 0)
        f = staged ? (const void *)k_assign<float4, true, 1024> : (const void *)k_assign<float4, false, 1024>;
    else
        f = staged ? (const void *)k_assign<uint2, true, 512> : (const void *)k_assign<uint2, false, 512>;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

}  // namespace scalp
