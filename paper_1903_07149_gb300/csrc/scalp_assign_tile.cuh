// scalp_assign_tile.cuh -- the assignment of one 32 x 32 tile (Algorithm 1's
// inner loops restated per tile, with the fused partial sums of the update):
// the body shared by the per-iteration assignment kernels (scalp_assign.cu)
// and the persistent batched kernel (scalp_persistent.cu).
#pragma once

#include <cfloat>
#include <climits>

#include "scalp_internal.cuh"

namespace scalp {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// One FP32 pair of a distance map, by 32-bit shared-memory byte address.
__device__ __forceinline__ float2 lds_pair(uint32_t addr)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

// The same pair as the two floats' bits in one 64-bit word (d_c low).
__device__ __forceinline__ unsigned long long lds_pair_bits(uint32_t addr)
{
    unsigned long long v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}

// Both running sums of a walk advanced at once: (d_c, w) += pair, each half
// an FP32 addition rounded to nearest (the same result as two scalar adds).
__device__ __forceinline__ void add_pair(unsigned long long &acc, unsigned long long v)
{
    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc) : "l"(v));
}

// Path sums of Eq. 1 and Eq. 2 over a distance map (row pitch `bw` pairs,
// pair (0,0) = image pixel (bx0, by0)).  The same samples, in the same order
// and with the same FP32 additions, as path_sums over the plane.
__device__ __forceinline__ int path_sums_map(uint32_t map, int bw, int bx0, int by0,
                                             const PathSetup &s, float &sum_dc, float &sum_w)
{
    int smaj, smin;
    path_strides(s, bw, smaj, smin);
    const uint32_t q0 = map + (uint32_t)(((s.ay - by0) * bw + (s.ax - bx0)) * 8);
    unsigned long long acc = 0;  // (+0.0f, +0.0f)
    const auto visit = [&](uint32_t q) { add_pair(acc, lds_pair_bits(q)); };
    // the fixed-point forms of the steps (fewer instructions per sample)
    // cover every path of up to FIXED_STEP_MAX_NS steps
    const int len = s.ns <= FIXED_STEP_MAX_NS ? walk_grouped<4>(q0, smaj * 8, smin * 8, s, visit)
                                              : walk_with<ErrorTermStep>(q0, smaj * 8, smin * 8, s, visit);
    sum_dc = __uint_as_float((unsigned)acc);
    sum_w = __uint_as_float((unsigned)(acc >> 32));
    return len;
}

// Shared-memory layout; every section starts on a 16-byte boundary (int4
// loads and 8-byte atomics need it).  The fixed sections come first; the
// per-candidate records follow, sized for the tile's own candidate count, and
// the distance maps fill the rest (a tile with few candidates has more room).
__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
struct AssignSmem {
    static constexpr size_t best = 0;
    static constexpr size_t prev = align16(best + TILE_PIXELS * sizeof(unsigned long long));
    static constexpr size_t queue = align16(prev + TILE_PIXELS);
    static constexpr size_t misc = align16(queue + (ASSIGN_THREADS / 32) * 64 * sizeof(uint32_t));
    static constexpr size_t records = align16(misc + 64);
};
static_assert(AssignSmem::prev % 16 == 0 && AssignSmem::queue % 16 == 0 &&
                  AssignSmem::misc % 16 == 0 && AssignSmem::records % 16 == 0,
              "shared-memory sections aligned");
// Per candidate (rank c): three 16-byte records the walk reads,
//   rec0 = (xa, ya, w | h << 8, 0)                   its rectangle
//   rec1 = (ex, ey, xk bits, yk bits)                endpoint, X_k
//   rec2 = (bx0, by0, pitch, map byte offset, or -1: walk the plane)
// the map box for the build, box = (bx0, by0, pitch, 32-bit reciprocal of
// the pitch), the colour C_k, col = (l_k, a_k, b_k, 0), the cluster index
// cid, the box area and the prefixes mfirst and cfirst of the map layout.
struct TileLayout {
    uint32_t rec0, rec1, rec2, box, col, cid, area, mfirst, cfirst, maps;
};
__host__ __device__ constexpr TileLayout tile_layout(int n)
{
    TileLayout t{};
    t.rec0 = (uint32_t)AssignSmem::records;
    t.rec1 = t.rec0 + (uint32_t)n * 16u;
    t.rec2 = t.rec1 + (uint32_t)n * 16u;
    t.box = t.rec2 + (uint32_t)n * 16u;
    t.col = t.box + (uint32_t)n * 16u;
    t.cid = t.col + (uint32_t)n * 16u;
    t.area = (uint32_t)align16(t.cid + (size_t)n * 4);
    t.mfirst = (uint32_t)align16(t.area + (size_t)n * 4);
    t.cfirst = (uint32_t)align16(t.mfirst + (size_t)(n + 1) * 4);
    t.maps = (uint32_t)align16(t.cfirst + (size_t)(n + 1) * 4);
    return t;
}
// The map pairs a tile of n candidates has beyond the capacity sized for
// MAX_TILE_CANDIDATES.
__host__ __device__ constexpr int extra_map_pairs(int n)
{
    return (int)((tile_layout(MAX_TILE_CANDIDATES).maps - tile_layout(n).maps) / 8u);
}
static_assert(MAX_TILE_CANDIDATES < 255, "slots are bytes; 0xff is none");
static_assert(TILE_PIXELS <= 1024 && MAX_TILE_CANDIDATES < (1 << 21), "queued pairs pack into 32 bits");
static_assert(MAX_TILE_CANDIDATES % 32 == 0, "the scans give each lane whole candidates");

// Rank of cluster k among the tile's candidates (cid sorted ascending), or -1.
__device__ __forceinline__ int find_slot(const int *cid, int cnt, int k)
{
    int lo = 0, hi = cnt;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cid[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return lo < cnt && cid[lo] == k ? lo : -1;
}

// A lower bound of D (Eq. 3) from the pixel's own colour distance and the
// spatial term, in FP32 such that it never exceeds the D scalp_distance()
// computes from the same dcp and ds: there dcol = lam*dcp + (1-lam)*avg is a
// rounded sum of non-negative terms, so dcol >= fl(lam*dcp); dcon =
// 1 + gamma*avg_w >= 1; D = fl(dcol*dcon + fl(ms2*ds)) >= fl(fl(lam*dcp) +
// fl(ms2*ds)), rounding being monotone.  (lam in [0, 1], gamma >= 0.)
__device__ __forceinline__ float distance_lower_bound(float dcp, float lam, float ms2, float ds)
{
    return __fadd_rn(__fmul_rn(lam, dcp), __fmul_rn(ms2, ds));
}

__device__ __forceinline__ unsigned long long pack_best(float D, int slot)
{
    // D >= 0, so its IEEE bits order like the value; ties fall to the slot
    return ((unsigned long long)__float_as_uint(D) << 32) | (unsigned)slot;
}

// The map layout by one warp: mfirst = exclusive prefix of the box areas
// (cnt + 1 entries); the leading candidates whose boxes end within cap get a
// map, of CHUNK-entry chunks whose prefix goes to cfirst (cnt + 1 entries;
// none for the others).  Returns the map entries used.
template <int CHUNK>
__device__ __forceinline__ int warp_scan_maps(const int *area, int *mfirst, int *cfirst, int cnt, int cap,
                                              int lane)
{
    constexpr int PER = MAX_TILE_CANDIDATES / 32;
    int v[PER], ch[PER], sum = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int c = lane * PER + i;
        v[i] = c < cnt ? area[c] : 0;
        sum += v[i];
    }
    int incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    // a box fits when its prefix end is within cap (the ends only grow)
    int run = incl - sum, fit = 0, csum = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int c = lane * PER + i;
        if (c < cnt) mfirst[c] = run;
        run += v[i];
        const bool mapped = c < cnt && v[i] > 0 && run <= cap;
        if (c < cnt && run <= cap) fit = run;
        ch[i] = mapped ? (v[i] + CHUNK - 1) / CHUNK : 0;
        csum += ch[i];
    }
    if (lane == 31) mfirst[cnt] = incl;
    int cincl = csum;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, cincl, o);
        if (lane >= o) cincl += t;
    }
    int crun = cincl - csum;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int c = lane * PER + i;
        if (c < cnt) cfirst[c] = crun;
        crun += ch[i];
    }
    if (lane == 31) cfirst[cnt] = cincl;
    return (int)__reduce_max_sync(0xffffffffu, (unsigned)fit);
}

// One tile of one image (the body shared by the single-image and the batched
// kernels).  The pixels of a candidate's window that lie in the tile form a
// rectangle; each warp owns 64 pixels of the tile (two blocks of 8 x 4).
// PREFETCH_TILE: the tile's plane rows are first asked into L2 (for batches,
// whose planes outgrow L2; an image whose plane stays in L2 only pays for it).
template <typename T, bool PREFETCH_TILE = false>
__device__ __forceinline__ void assign_tile(const SolveArgs &a, int tile, unsigned char *smem)
{
    constexpr int THREADS = ASSIGN_THREADS;
    constexpr int PIX_PER_THREAD = TILE_PIXELS / THREADS;
    constexpr int WARPS = THREADS / 32;
    constexpr int BUILD_UNROLL = 4;
    constexpr int BUILD_CHUNK = BUILD_UNROLL * 32;  // map entries per warp task
    const T *__restrict__ plane = reinterpret_cast<const T *>(
        sizeof(T) == 16 ? (const void *)a.plane32 : (const void *)a.plane16);
    const int tx = tile % a.n_tx, ty = tile / a.n_tx;
    const int x0 = tx * TILE_X, y0 = ty * TILE_Y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    unsigned long long *best = reinterpret_cast<unsigned long long *>(smem + AssignSmem::best);
    unsigned char *prev_slot = smem + AssignSmem::prev;
    int *misc = reinterpret_cast<int *>(smem + AssignSmem::misc);

    // this thread's pixels: block (warp * PIX_PER_THREAD + j) of the tile
    // (a warp's blocks lie side by side), lane within it
    auto my_pixel = [&](int j, int &qx, int &qy) {
        const int blk = warp + j * WARPS;
        qx = x0 + (blk % (TILE_X / WARP_BLOCK_X)) * WARP_BLOCK_X + (lane % WARP_BLOCK_X);
        qy = y0 + (blk / (TILE_X / WARP_BLOCK_X)) * WARP_BLOCK_Y + (lane / WARP_BLOCK_X);
    };

    const int off = a.tile_off[tile];
    // the list capacity is a proven bound; the clamp only guards memory if the
    // device-side overflow check (reported as an error) ever fired
    const int cnt = (int)max(0LL, min((long long)a.tile_off[tile + 1], a.tile_cap) - off);
    const bool fast = cnt <= MAX_TILE_CANDIDATES;
    // the records for this tile's candidates, then its maps
    const TileLayout lay = tile_layout(fast ? cnt : 0);
    int4 *rec0 = reinterpret_cast<int4 *>(smem + lay.rec0);
    int4 *rec1 = reinterpret_cast<int4 *>(smem + lay.rec1);
    int4 *rec2 = reinterpret_cast<int4 *>(smem + lay.rec2);
    int4 *box = reinterpret_cast<int4 *>(smem + lay.box);
    float4 *col = reinterpret_cast<float4 *>(smem + lay.col);
    int *cid = reinterpret_cast<int *>(smem + lay.cid);
    int *area = reinterpret_cast<int *>(smem + lay.area);
    int *mfirst = reinterpret_cast<int *>(smem + lay.mfirst);
    int *cfirst = reinterpret_cast<int *>(smem + lay.cfirst);
    const uint32_t maps_u32 = smem_u32(smem + lay.maps);
    float2 *maps = reinterpret_cast<float2 *>(smem + lay.maps);
    const int map_cap = a.map_cap > 0 ? a.map_cap + extra_map_pairs(fast ? cnt : 0) : 0;
    if (tid == 0) {  // this tile's list is read: ready the counts for the next update
        a.tile_count[tile] = 0;
        a.tile_cursor[tile] = 0;
        // the last projection (and lists) completed before this launch: its
        // queue starts again for the next update
        if (tile == 0) a.ctr->nproj = 0;
    }

    // the tile's plane rows into L2 while the set-up runs, so that the map
    // build finds them there (x0 * sizeof(T) and the row pitch are multiples
    // of 16 bytes, and so is every row's length: the bulk prefetch's rules)
    static_assert(TILE_Y <= 32, "one row per lane");
    if (PREFETCH_TILE && warp == WARPS - 1) {
        const int rows = min(a.H - y0, TILE_Y);
        const uint32_t bytes = (uint32_t)(min(TILE_X, a.pitch - x0) * (int)sizeof(T));
        if (lane < rows) {
            const T *p = plane + (long long)(y0 + lane) * a.pitch + x0;
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
        }
    }

    // this thread's pixels' previous labels (their loads overlap the set-up)
    int prev_lab[PIX_PER_THREAD];
#pragma unroll
    for (int j = 0; j < PIX_PER_THREAD; ++j) {
        int px, py;
        my_pixel(j, px, py);
        prev_lab[j] = fast && px < a.W && py < a.H ? a.labels[(long long)py * a.W + px] : -1;
    }
    if (tid == 0) {
        misc[4] = 0;  // path samples and pairs (counting on)
        misc[5] = 0;
    }
    // the records of candidate id (rank among the tile's sorted ids)
    const auto write_records = [&](int rank, int id, const ClusterDev &cd) {
        cid[rank] = id;
        // window x tile (clipped to the image)
        const int xa = max(cd.xlo, x0), xb = min(min(cd.xhi, x0 + TILE_X - 1), a.W - 1);
        const int ya = max(cd.ylo, y0), yb = min(min(cd.yhi, y0 + TILE_Y - 1), a.H - 1);
        const int w = max(xb - xa + 1, 0), h = max(yb - ya + 1, 0);
        rec0[rank] = make_int4(xa, ya, w | (h << 8), 0);
        rec1[rank] = make_int4(cd.ex, cd.ey, __float_as_int(cd.xk), __float_as_int(cd.yk));
        col[rank] = make_float4(cd.L, cd.a, cd.b, 0.f);
        // map box: the rectangle and the endpoint (both inside the image).
        // Rows are padded to a pitch = 4 (mod 8) pairs: the walks of a warp
        // then spread over the shared-memory banks (neighbouring rows start
        // 8 banks apart); 32-bit reciprocal of the pitch for the build.
        int bx0 = 0, by0 = 0, pitch = 1;
        long long n = 0;
        if (w > 0 && h > 0) {
            bx0 = min(xa, cd.ex);
            by0 = min(ya, cd.ey);
            const int bw = max(xb, cd.ex) - bx0 + 1;
            pitch = bw + ((4 - bw) & 7);
            n = (long long)pitch * (max(yb, cd.ey) - by0 + 1);
        }
        // ceil(2^32 / pitch) = floor((2^32 - 1) / pitch) + 1 for pitch >= 2
        // (an empty box has pitch 1 and no map)
        const unsigned rcp = pitch > 1 ? 0xffffffffu / (unsigned)pitch + 1u : 0u;
        box[rank] = make_int4(bx0, by0, pitch, (int)rcp);
        // a box larger than the whole buffer never fits: clamp it so that the
        // prefix sums stay small
        area[rank] = map_cap > 0 ? (int)min(n, (long long)map_cap + 1) : 0;
    };
    // the candidates sorted by cluster index (ranks of distinct ids), their
    // records and the map layout; each warp readies its own pixels' best words
    if (fast && cnt <= 32) {
        // one warp: ranks by shuffles, no block barrier until the layout is done
        if (warp == 0) {
            int myid = INT_MAX;
            ClusterDev cd;
            if (lane < cnt) {
                myid = a.tile_list[off + lane];
                cd = a.cdev[myid];
            }
            int rank = 0;
            for (int j = 0; j < 32; ++j) rank += __shfl_sync(0xffffffffu, myid, j) < myid;
            if (lane < cnt) write_records(rank, myid, cd);
            __syncwarp();
            const int used = warp_scan_maps<BUILD_CHUNK>(area, mfirst, cfirst, cnt, map_cap, lane);
            if (lane == 0) misc[2] = used;
        }
#pragma unroll
        for (int j = 0; j < PIX_PER_THREAD; ++j) {
            int px, py;
            my_pixel(j, px, py);
            best[(py - y0) * TILE_X + (px - x0)] = ~0ull;
        }
    } else {
        // the id staging reuses the `best` words before they are initialised
        int *ids = reinterpret_cast<int *>(best);
        int myid = INT_MAX;
        ClusterDev cd;  // this thread's candidate: its load overlaps the barrier
        if (fast && tid < cnt) {
            myid = a.tile_list[off + tid];
            ids[tid] = myid;
            cd = a.cdev[myid];
        }
        __syncthreads();
        if (fast && tid < cnt) {
            int rank = 0;
            for (int j = 0; j < cnt; ++j) rank += ids[j] < myid;
            write_records(rank, myid, cd);
        }
        __syncthreads();
        for (int i = tid; i < TILE_PIXELS; i += THREADS) best[i] = ~0ull;
        if (warp == 0 && fast) {
            const int used = warp_scan_maps<BUILD_CHUNK>(area, mfirst, cfirst, cnt, map_cap, lane);
            if (lane == 0) misc[2] = used;
        }
    }
    __syncthreads();

    // each pixel's previous label, as a candidate slot when the pixel lies in
    // that candidate's rectangle (0xff otherwise): pass 1 below evaluates it
    // first, pass 2 skips it
    if (fast) {
#pragma unroll
        for (int j = 0; j < PIX_PER_THREAD; ++j) {
            int px, py;
            my_pixel(j, px, py);
            int c = prev_lab[j] >= 0 ? find_slot(cid, cnt, prev_lab[j]) : -1;
            if (c >= 0) {
                const int4 r0 = rec0[c];
                if (px < r0.x || px >= r0.x + (r0.z & 0xff) || py < r0.y || py >= r0.y + ((r0.z >> 8) & 0xff))
                    c = -1;
            }
            prev_slot[(py - y0) * TILE_X + (px - x0)] = (unsigned char)(c >= 0 ? c : 0xff);
        }
    }

    // the distance maps of the candidates whose boxes fit: entries [0, used)
    // hold the leading candidates' boxes back to back, row-major; the
    // padding columns of a row are left unwritten (no walk reads them)
    const int used = fast ? misc[2] : 0;
    if (fast) {
        if (tid < cnt) {
            const int4 b = box[tid];
            const bool mapped = area[tid] > 0 && mfirst[tid + 1] <= used;
            rec2[tid] = make_int4(b.x, b.y, b.z, mapped ? mfirst[tid] * (int)sizeof(float2) : -1);
        }
        // warps take the chunks in turn; within one the candidate is uniform
        // and the lanes read consecutive entries (coalesced plane rows)
        const int n_chunks = cfirst[cnt];
        int c = 0;
        for (int g = warp; g < n_chunks; g += WARPS) {
            while (g >= cfirst[c + 1]) ++c;
            const int4 b = box[c];
            // unpadded width: from the rectangle's right edge and e_k
            const int4 r0 = rec0[c];
            const int bw = max(r0.x + (r0.z & 0xff) - 1, rec1[c].x) - b.x + 1;
            const float4 ck = col[c];
            const int m0 = mfirst[c];
            const int n_le = mfirst[c + 1] - m0;
            const int le0 = (g - cfirst[c]) * BUILD_CHUNK + lane;
            // the box's first pixel; offsets within the box fit 32 bits: a
            // box of at most map_cap pairs has row < min(H, map_cap / 4) and
            // the plane pitch is at most W + 3, so row * pitch + column < 2^31
            const T *__restrict__ pbox = plane + (long long)b.y * a.pitch + b.x;
            float2 *mrow = maps + (m0 + le0);
            T v[BUILD_UNROLL];  // raw samples: all loads issue before any use
            bool ok[BUILD_UNROLL];
#pragma unroll
            for (int u = 0; u < BUILD_UNROLL; ++u) {
                const int le = le0 + u * 32;
                // a mapped box has pitch >= 4 and le * pitch < 2^32, so the
                // 32-bit reciprocal gives the exact row
                const int row = (int)__umulhi((unsigned)le, (unsigned)b.w);
                const int cx = le - row * b.z;
                ok[u] = le < n_le && cx < bw;
                if (ok[u]) v[u] = __ldg(pbox + (row * a.pitch + cx));
            }
#pragma unroll
            for (int u = 0; u < BUILD_UNROLL; ++u) {
                if (ok[u]) {
                    const float4 q = sample_value(v[u]);
                    mrow[u * 32] = make_float2(colour_dist(q, ck.x, ck.y, ck.z), q.w);
                }
            }
        }
    }
    __syncthreads();

    // with counting on, the tile's path samples and pairs are summed in
    // misc[4], misc[5] (zeroed at the start; far below 2^32 per tile)
    unsigned *tile_samples = reinterpret_cast<unsigned *>(misc + 4);
    int bestk[PIX_PER_THREAD];  // per-pixel path only
#pragma unroll
    for (int j = 0; j < PIX_PER_THREAD; ++j) bestk[j] = INT_MAX;

    // D of pixel (qx, qy) for candidate slot c (Eq. 1-3), its path length in
    // *len; on a map when the candidate has one, else on the plane
    auto pair_distance = [&](int qx, int qy, int c, int4 r1, int4 r2, float dcp, float ds, int *len) {
        const PathSetup s = path_setup(qx, qy, r1.x, r1.y);
        float sdc, sw;
        if (r2.w >= 0) {
            *len = path_sums_map(maps_u32 + (uint32_t)r2.w, r2.z, r2.x, r2.y, s, sdc, sw);
        } else {
            const float4 ck = col[c];
            *len = path_sums<T>(plane, a.pitch, 0, 0, s, ck.x, ck.y, ck.z, sdc, sw);
        }
        return scalp_distance(dcp, sdc, sw, *len, a.lam, a.gamma, a.ms2, ds);
    };
    // the pixel's own colour distance d_c(p, C_c) (map entry, else the plane)
    auto own_distance = [&](int qx, int qy, int c, int4 r2) {
        if (r2.w >= 0)
            return lds_pair(maps_u32 + (uint32_t)r2.w + (uint32_t)(((qy - r2.y) * r2.z + (qx - r2.x)) * 8)).x;
        const float4 ck = col[c];
        return colour_dist(fetch_sample<T>(plane + (long long)qy * a.pitch + qx), ck.x, ck.y, ck.z);
    };
    auto spatial = [&](int qx, int qy, int4 r1) {
        const float ddx = (float)qx - __int_as_float(r1.z), ddy = (float)qy - __int_as_float(r1.w);
        return fmaf(ddx, ddx, ddy * ddy);
    };
    auto count_pair = [&](int len) {
        if (a.count_samples) {
            atomicAdd(tile_samples, (unsigned)len);
            atomicAdd(tile_samples + 1, 1u);
        }
    };

    if (fast) {
        // Pass 1: each pixel's previous label first, when it is a candidate
        // of the pixel (it usually wins again).  Its D bounds the minimum, so
        // pass 2 can skip every candidate whose lower bound exceeds it: such
        // a candidate's D is larger than the minimum and cannot win or tie.
        // The argmin is unchanged.  Each warp walks its own pixels here.
        float dprev[PIX_PER_THREAD];  // D of the previous label; NaN: none
#pragma unroll
        for (int j = 0; j < PIX_PER_THREAD; ++j) dprev[j] = __int_as_float(0x7fffffff);
#pragma unroll 1
        for (int j = 0; j < PIX_PER_THREAD; ++j) {
            int px, py;
            my_pixel(j, px, py);
            const int pix = (py - y0) * TILE_X + (px - x0);
            const int c = prev_slot[pix];
            if (c != 0xff) {
                const int4 r1 = rec1[c], r2 = rec2[c];
                int len;
                const float D = pair_distance(px, py, c, r1, r2, own_distance(px, py, c, r2), spatial(px, py, r1),
                                              &len);
                atomicMin(&best[pix], pack_best(D, c));
#pragma unroll
                for (int i = 0; i < PIX_PER_THREAD; ++i)  // (registers: constant indices)
                    if (i == j) dprev[i] = D;
                count_pair(len);
            }
        }

        // Pass 2: each warp checks its own pixels against every other
        // candidate whose rectangle holds them.  A surviving pair goes to the
        // warp's queue (slot << 10 | tile pixel); each time 32 are queued the
        // warp walks them, one per lane, and the last few at the end.  (A
        // barrier before the walks, to share them among the warps, cost more
        // than the uneven loads it evens out.)
        const auto walk_queued = [&](uint32_t e) {
            const int pix = (int)(e & 1023u), c = (int)(e >> 10);
            const int qx = x0 + (pix & (TILE_X - 1)), qy = y0 + (pix / TILE_X);
            const int4 r1 = rec1[c], r2 = rec2[c];
            int len;
            const float D = pair_distance(qx, qy, c, r1, r2, own_distance(qx, qy, c, r2), spatial(qx, qy, r1), &len);
            atomicMin(&best[pix], pack_best(D, c));
            count_pair(len);
        };
        uint32_t *wq = reinterpret_cast<uint32_t *>(smem + AssignSmem::queue) + warp * 64;
        const unsigned lanes_below = (1u << lane) - 1u;
        int queued = 0;  // warp-uniform
        for (int c = 0; c < cnt; ++c) {
            const int4 r0 = rec0[c];
            const unsigned rw = (unsigned)(r0.z & 0xff), rh = (unsigned)((r0.z >> 8) & 0xff);
            bool in[PIX_PER_THREAD];
            bool any = false;
#pragma unroll
            for (int j = 0; j < PIX_PER_THREAD; ++j) {
                int px, py;
                my_pixel(j, px, py);
                // (a pixel of the rectangle lies in the image)
                in[j] = (unsigned)(px - r0.x) < rw && (unsigned)(py - r0.y) < rh &&
                        prev_slot[(py - y0) * TILE_X + (px - x0)] != c;
                any = any || in[j];
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            const int4 r1 = rec1[c], r2 = rec2[c];
#pragma unroll
            for (int j = 0; j < PIX_PER_THREAD; ++j) {
                int px, py;
                my_pixel(j, px, py);
                bool keep = false;
                if (in[j]) {
                    const float dcp = own_distance(px, py, c, r2);
                    keep = !a.prune || !(distance_lower_bound(dcp, a.lam, a.ms2, spatial(px, py, r1)) > dprev[j]);
                    // a pair that cannot win is not walked (counted as the method's work)
                    if (!keep) count_pair(max(abs(px - r1.x), abs(py - r1.y)) + 1);
                }
                const unsigned kept = __ballot_sync(0xffffffffu, keep);
                if (keep)
                    wq[queued + __popc(kept & lanes_below)] =
                        ((uint32_t)c << 10) | (uint32_t)((py - y0) * TILE_X + (px - x0));
                queued += __popc(kept);
                __syncwarp();
                if (queued >= 32) {
                    const uint32_t e = wq[lane];
                    __syncwarp();
                    if (lane < queued - 32) wq[lane] = wq[32 + lane];
                    queued -= 32;
                    __syncwarp();
                    walk_queued(e);
                }
            }
        }
        if (lane < queued) walk_queued(wq[lane]);
    } else {
        // per-pixel path: every candidate straight from the global list
#pragma unroll 1
        for (int j = 0; j < PIX_PER_THREAD; ++j) {
            int px, py;
            my_pixel(j, px, py);
            if (px >= a.W || py >= a.H) continue;
            const float4 own = fetch_sample<T>(plane + (long long)py * a.pitch + px);
            float bestD = FLT_MAX;
            for (int i = 0; i < cnt; ++i) {
                const int k = a.tile_list[off + i];
                const ClusterDev cd = a.cdev[k];
                if (px < cd.xlo || px > cd.xhi || py < cd.ylo || py > cd.yhi) continue;
                const PathSetup s = path_setup(px, py, cd.ex, cd.ey);
                float sdc, sw;
                const int len = path_sums<T>(plane, a.pitch, 0, 0, s, cd.L, cd.a, cd.b, sdc, sw);
                const float dcp = colour_dist(own, cd.L, cd.a, cd.b);
                const float ddx = (float)px - cd.xk, ddy = (float)py - cd.yk;
                const float ds = fmaf(ddx, ddx, ddy * ddy);
                const float D = scalp_distance(dcp, sdc, sw, len, a.lam, a.gamma, a.ms2, ds);
                if (D < bestD || (D == bestD && k < bestk[j])) {
                    bestD = D;
                    bestk[j] = k;
                }
                if (a.count_samples) {
                    atomicAdd(tile_samples, (unsigned)len);
                    atomicAdd(tile_samples + 1, 1u);
                }
            }
        }
    }
    // a warp's pixels were walked by that warp alone (both passes, or the
    // per-pixel path), so its lanes' writes to them need only a warp barrier
    __syncwarp();

    // labels and the warp-aggregated integer sums of the update; the
    // pixels' own samples are all requested first
    float4 owns[PIX_PER_THREAD];
#pragma unroll
    for (int j = 0; j < PIX_PER_THREAD; ++j) {
        int px, py;
        my_pixel(j, px, py);
        owns[j] = px < a.W && py < a.H ? fetch_sample<T>(plane + (long long)py * a.pitch + px)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < PIX_PER_THREAD; ++j) {
        int px, py;
        my_pixel(j, px, py);
        const bool valid = px < a.W && py < a.H;
        const long long p = (long long)py * a.W + px;
        const float4 own = owns[j];
        int lab = -1;
        if (valid) {
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
        __syncthreads();  // every warp's counts are in (a CTA-uniform branch)
        if (tid == 0) {
            atomicAdd(&a.ctr->samples, (unsigned long long)tile_samples[0]);
            atomicAdd(&a.ctr->pairs, (unsigned long long)tile_samples[1]);
        }
        // (candidate, tile) rectangles walked on a map and on the plane
        if (tid == 0) {
            unsigned long long on_map = 0, on_plane = 0;
            for (int c = 0; c < cnt; ++c) {
                if (fast && (rec0[c].z & 0xff) * ((rec0[c].z >> 8) & 0xff) == 0) continue;  // no pixel
                if (fast && rec2[c].w >= 0) ++on_map;
                else ++on_plane;
            }
            atomicAdd(&a.ctr->map_rects, on_map);
            atomicAdd(&a.ctr->plane_rects, on_plane);
        }
    }
}

}  // namespace scalp
