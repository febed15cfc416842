// scalp_ccl.cu -- connectivity enforcement of the final decomposition.
//
// The paper does not describe this step.  The rule implemented (bit-exact,
// independent of thread scheduling):
//   1. 4-connected components of equal label; a component's seed is its
//      smallest raster index (the root of a union-find forest whose links
//      always point to smaller indices), built inside 32 x 32 tiles in shared
//      memory first and then joined across tile borders.
//   2. A component is small iff it has at most floor(N / (4K)) pixels.
//   3. A small component whose seed s is not pixel 0 is absorbed by the
//      component holding s-1 (if s is not in column 0) or s-W; that component
//      has a smaller seed, so the absorption links form a forest.  A small
//      component takes the identity of its first non-small ancestor (or the
//      component of pixel 0).
//   4. The surviving components are numbered 0.. in raster order of seeds
//      (per 4096-pixel chunk: a count, a scan of the counts, the ranks).
#include <algorithm>
#include <cstdint>

#include "scalp_launch.h"

namespace scalp {

constexpr int CCL_THREADS = 256;

__device__ __forceinline__ int find_root(const volatile int *parent, int x)
{
    int p = parent[x];
    while (p != x) {
        x = p;
        p = parent[x];
    }
    return x;
}

// Union of the trees of a and b: the larger root is linked under the smaller
// one with atomicMin.  If the root changed meanwhile the attempt is repeated
// from the value found, so no link is lost.
__device__ __forceinline__ void unite(int *parent, int a, int b)
{
    bool done;
    do {
        a = find_root(parent, a);
        b = find_root(parent, b);
        if (b < a) {
            int old = atomicMin(&parent[a], b);
            done = old == a;
            a = old;
        } else if (a < b) {
            int old = atomicMin(&parent[b], a);
            done = old == b;
            b = old;
        } else {
            done = true;
        }
    } while (!done);
}

// Pass 1: union-find inside each 32 x 32 tile in shared memory.  Tile-local
// raster order is global raster order, so the local root (smallest local
// index of a tile-local component) is also its smallest global index; each
// pixel gets that root's global index as parent.  size[] is cleared.
constexpr int CCL_TILE = 32;

// The root of x, halving the path on the way with atomicMin: links always
// point to smaller indices and a root is the least index of its tree, so a
// pointer only ever moves toward the root and concurrent finds, unions and
// the heads' final root writes cannot undo one another.
__device__ __forceinline__ int find_local(int *sp, int x)
{
    volatile int *v = sp;
    int p = v[x];
    while (p != x) {
        const int gp = v[p];
        if (gp != p) atomicMin(&sp[x], gp);
        x = p;
        p = gp;
    }
    return x;
}

__device__ __forceinline__ void unite_local(int *sp, int a, int b)
{
    bool done;
    do {
        a = find_local(sp, a);
        b = find_local(sp, b);
        if (b < a) {
            int old = atomicMin(&sp[a], b);
            done = old == a;
            a = old;
        } else if (a < b) {
            int old = atomicMin(&sp[b], a);
            done = old == b;
            b = old;
        } else {
            done = true;
        }
    } while (!done);
}

// 256 threads: each warp takes four rows of the tile (all loads first), so
// eight tiles of an SM are in flight.  size[] is cleared at local roots only:
// a component's seed is the local root of its tile part, and no other entry
// of size[] is read.
constexpr int CCL_LOCAL_THREADS = 256;
constexpr int CCL_ROWS = CCL_TILE / (CCL_LOCAL_THREADS / 32);  // rows per warp

__device__ __forceinline__ void ccl_local(const int *__restrict__ labels, int *parent, int *size, int H, int W,
                                          int n_tx, int tile)
{
    __shared__ int sp[CCL_TILE * CCL_TILE];
    __shared__ int sl[CCL_TILE * CCL_TILE];
    __shared__ unsigned srun[CCL_TILE];  // per row: bit x set where a run starts
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = (tile % n_tx) * CCL_TILE, y0 = (tile / n_tx) * CCL_TILE;
    const int x = x0 + lane;
    int lab[CCL_ROWS];
    bool valid[CCL_ROWS];
#pragma unroll
    for (int r = 0; r < CCL_ROWS; ++r) {
        const int y = y0 + warp + r * (CCL_LOCAL_THREADS / 32);
        valid[r] = x < W && y < H;
        lab[r] = valid[r] ? labels[(long long)y * W + x] : 0;
    }
    // runs of equal label along each row: a pixel's head is the last run
    // start at or before it
    bool is_head[CCL_ROWS];
#pragma unroll
    for (int r = 0; r < CCL_ROWS; ++r) {
        const int ly = warp + r * (CCL_LOCAL_THREADS / 32), t = ly * CCL_TILE + lane;
        sl[t] = lab[r];
        const int left = __shfl_up_sync(0xffffffffu, lab[r], 1);
        const unsigned starts = __ballot_sync(0xffffffffu, lane == 0 || !valid[r] || left != lab[r]);
        const int head = 31 - __clz(starts & (0xffffffffu >> (31 - lane)));
        sp[t] = ly * CCL_TILE + head;
        is_head[r] = head == lane;
        if (lane == 0) srun[ly] = starts;
    }
    __syncthreads();
    // one union per pair of vertically touching runs: at the first pixel of
    // their overlap, where this pixel or the one above starts a run
#pragma unroll
    for (int r = 0; r < CCL_ROWS; ++r) {
        const int ly = warp + r * (CCL_LOCAL_THREADS / 32), t = ly * CCL_TILE + lane;
        if (valid[r] && ly > 0 && sl[t - CCL_TILE] == lab[r] &&
            (((srun[ly] >> lane) & 1u) || ((srun[ly - 1] >> lane) & 1u)))
            unite_local(sp, t, t - CCL_TILE);
    }
    __syncthreads();
    // each run head finds its root once and stores it (finds passing through
    // it meanwhile still reach the same root); a pixel is then two lookups
    // from its root: pixel -> head -> root
#pragma unroll
    for (int r = 0; r < CCL_ROWS; ++r) {
        const int t = (warp + r * (CCL_LOCAL_THREADS / 32)) * CCL_TILE + lane;
        if (valid[r] && is_head[r]) sp[t] = find_local(sp, t);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < CCL_ROWS; ++r) {
        const int ly = warp + r * (CCL_LOCAL_THREADS / 32), t = ly * CCL_TILE + lane;
        if (!valid[r]) continue;
        const long long p = (long long)(y0 + ly) * W + x;
        const int root = sp[sp[t]];
        parent[p] = (int)((long long)(y0 + root / CCL_TILE) * W + x0 + root % CCL_TILE);
        if (root == t) size[p] = 0;
    }
}

// Pass 2: unions across tile borders (left edge and top edge of each tile).
// The passes from here on take their block index and block count as blk and
// nblk (a batch gives each image its own range of blocks).
__device__ __forceinline__ void ccl_border(const int *__restrict__ labels, int *parent, int H, int W, int n_tx,
                                           int n_ty, unsigned blk, unsigned nblk)
{
    const long long nv = (long long)(n_tx - 1) * H;  // vertical border pixels
    const long long nh = (long long)(n_ty - 1) * W;  // horizontal border pixels
    for (long long i = blk * (long long)blockDim.x + threadIdx.x; i < nv + nh; i += (long long)nblk * blockDim.x) {
        long long p, q;
        if (i < nv) {
            const int y = (int)(i / (n_tx - 1)), bx = (int)(i % (n_tx - 1)) + 1;
            p = (long long)y * W + bx * CCL_TILE;
            q = p - 1;
        } else {
            const long long j = i - nv;
            const int by = (int)(j / W) + 1, x = (int)(j % W);
            p = (long long)by * CCL_TILE * W + x;
            q = p - W;
        }
        if (labels[p] == labels[q]) unite(parent, (int)p, (int)q);
    }
}

// Roots and component sizes; the lanes of a warp (32 consecutive pixels, most
// of them in one component) add their counts once per distinct root.  A warp
// takes CCL_FLAT_RUNS runs of 32 pixels at once and follows their parent
// pointers in lockstep, so that many loads are in flight.  No union happens
// any more: the forest is fixed and the writes here only shorten paths, so
// any pointer value read leads to the same root.
constexpr int CCL_FLAT_RUNS = 4;

__device__ __forceinline__ void ccl_flatten_count(int *parent, int *size, long long N, unsigned blk, unsigned nblk)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)nblk * (blockDim.x / 32);
    for (long long w0 = blk * (long long)(blockDim.x / 32) + (threadIdx.x >> 5); w0 * 32 < N;
         w0 += warps * CCL_FLAT_RUNS) {
        int x[CCL_FLAT_RUNS];
#pragma unroll
        for (int u = 0; u < CCL_FLAT_RUNS; ++u) {
            const long long p = (w0 + u * warps) * 32 + lane;
            x[u] = p < N ? parent[p] : -1;
        }
        bool more = true;
        while (more) {
            int nx[CCL_FLAT_RUNS];
#pragma unroll
            for (int u = 0; u < CCL_FLAT_RUNS; ++u) nx[u] = x[u] >= 0 ? parent[x[u]] : -1;
            more = false;
#pragma unroll
            for (int u = 0; u < CCL_FLAT_RUNS; ++u) {
                more |= nx[u] != x[u];
                x[u] = nx[u];
            }
        }
#pragma unroll
        for (int u = 0; u < CCL_FLAT_RUNS; ++u) {
            const long long p = (w0 + u * warps) * 32 + lane;
            const bool valid = p < N;
            if (valid) parent[p] = x[u];
            const unsigned act = __ballot_sync(0xffffffffu, valid);
            if (valid) {
                const unsigned grp = __match_any_sync(act, x[u]);
                if (lane == __ffs(grp) - 1) atomicAdd(&size[x[u]], __popc(grp));
            }
        }
    }
}

// Four consecutive pixels per thread (one 16-byte load of their parents; the
// buffers are 256-byte aligned).
// The four parents from quad g (16-byte aligned buffers); -1 past N.
__device__ __forceinline__ int4 load_quad(const int *__restrict__ a, long long g, long long N)
{
    const long long s0 = 4 * g;
    if (s0 + 4 <= N) return reinterpret_cast<const int4 *>(a)[g];
    return make_int4(s0 < N ? a[s0] : -1, s0 + 1 < N ? a[s0 + 1] : -1, s0 + 2 < N ? a[s0 + 2] : -1,
                     s0 + 3 < N ? a[s0 + 3] : -1);
}

// Quads per thread and round in the passes below: their loads are issued
// together before any is used.
constexpr int CCL_QUAD_ROUND = 4;

__device__ __forceinline__ void ccl_link(const int *__restrict__ parent, const int *__restrict__ size, int *link,
                                         int W, long long N, long long T, unsigned blk, unsigned nblk)
{
    const long long quads = (N + 3) / 4, stride = (long long)nblk * blockDim.x;
    for (long long g0 = blk * (long long)blockDim.x + threadIdx.x; g0 < quads; g0 += stride * CCL_QUAD_ROUND) {
        int4 q[CCL_QUAD_ROUND];
#pragma unroll
        for (int u = 0; u < CCL_QUAD_ROUND; ++u) {
            const long long g = g0 + u * stride;
            q[u] = g < quads ? load_quad(parent, g, N) : make_int4(-1, -1, -1, -1);
        }
        // the sizes of the same quads, streamed alike (only seeds' entries
        // are meaningful)
        int4 z[CCL_QUAD_ROUND];
#pragma unroll
        for (int u = 0; u < CCL_QUAD_ROUND; ++u) {
            const long long g = g0 + u * stride;
            z[u] = g < quads ? load_quad(size, g, N) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < CCL_QUAD_ROUND; ++u) {
            const long long s0 = 4 * (g0 + u * stride);
            const int pv[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
            const int zv[4] = {z[u].x, z[u].y, z[u].z, z[u].w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const long long s = s0 + i;
                if (pv[i] != s) continue;
                const bool small = zv[i] <= T && s != 0;
                int to = (int)s;
                if (small) {
                    // the pixel before s (in this quad unless i = 0), else
                    // the one above for column 0; N <= 2^30
                    if (((int)s % W) > 0) to = i > 0 ? pv[i - 1] : parent[s - 1];
                    else to = parent[s - W];
                }
                link[s] = to;
            }
        }
    }
}

// Numbering works on chunks of CCL_CHUNK pixels, one CTA each.
constexpr int CCL_CHUNK = 4096;
constexpr int CCL_CHUNK_THREADS = 256;
constexpr int CCL_PER = CCL_CHUNK / CCL_CHUNK_THREADS;  // consecutive pixels per thread
static_assert(CCL_PER % 4 == 0, "runs are read as int4");

// The CCL_PER values of a thread's run from `base` (a multiple of CCL_PER; the
// buffers are 256-byte aligned) as 16-byte loads; -1 past N.
__device__ __forceinline__ void load_run(const int *__restrict__ a, long long base, long long N, int (&v)[CCL_PER])
{
    if (base + CCL_PER <= N) {
        const int4 *a4 = reinterpret_cast<const int4 *>(a + base);
#pragma unroll
        for (int i = 0; i < CCL_PER / 4; ++i) {
            const int4 q = a4[i];
            v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < CCL_PER; ++i) v[i] = base + i < N ? a[base + i] : -1;
    }
}

// Sum of v over the CTA (all threads receive it); s_warp holds 32 ints.
__device__ __forceinline__ int cta_sum(int v, int *s_warp)
{
    v = __reduce_add_sync(0xffffffffu, (unsigned)v);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
    __syncthreads();
    int t = (int)(threadIdx.x & 31) < (int)(blockDim.x >> 5) ? s_warp[threadIdx.x & 31] : 0;
    t = __reduce_add_sync(0xffffffffu, (unsigned)t);
    __syncthreads();
    return t;
}

// final[s] = first non-small ancestor of seed s (written over size[]), and
// per chunk the number of surviving components (seeds with final[s] == s).
__device__ __forceinline__ void ccl_resolve_count(const int *__restrict__ parent, const int *__restrict__ link,
                                                  int *final_id, long long N, DevCounters *ctr, int *chunk_count,
                                                  unsigned chunk)
{
    __shared__ int s_warp[32];
    // CCL_PER consecutive pixels per thread, their parents and links loaded
    // first (a seed's link sits at its own index; other entries are unused)
    const long long base = chunk * (long long)CCL_CHUNK + (long long)threadIdx.x * CCL_PER;
    int par[CCL_PER], lk[CCL_PER];
    load_run(parent, base, N, par);
    load_run(link, base, N, lk);
    int cnt = 0;
#pragma unroll
    for (int i = 0; i < CCL_PER; ++i) {
        const long long s = base + i;
        if (par[i] != s) continue;
        int f = (int)s, nf = lk[i];
        long long guard = 0;
        while (nf != f) {
            f = nf;
            if (++guard > N) {
                atomicExch(&ctr->error, ERR_CCL_CHAIN);
                break;
            }
            nf = link[f];
        }
        final_id[s] = f;
        cnt += f == s;
    }
    cnt = cta_sum(cnt, s_warp);
    if (threadIdx.x == 0) chunk_count[chunk] = cnt;
}

// Exclusive scan of the chunk counts by one CTA (each thread a contiguous
// run); *total receives the number of labels.
constexpr int CCL_SCAN_THREADS = 1024;

__device__ __forceinline__ void ccl_chunk_scan(int *counts, long long n, int *total)
{
    __shared__ int s_warp[32];
    const long long per = (n + CCL_SCAN_THREADS - 1) / CCL_SCAN_THREADS;
    const long long b = threadIdx.x * per, e = min(n, b + per);
    int tsum = 0;
    for (long long i = b; i < e; ++i) tsum += counts[i];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = tsum;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    int run = (wid ? s_warp[wid - 1] : 0) + incl - tsum;
    for (long long i = b; i < e; ++i) {
        const int v = counts[i];
        counts[i] = run;
        run += v;
    }
    if (threadIdx.x == CCL_SCAN_THREADS - 1) *total = s_warp[31];
}

// number[s] for each surviving seed s: its rank in raster order (the chunk's
// offset plus the rank inside the chunk); only seeds are written.
__device__ __forceinline__ void ccl_number(const int *__restrict__ parent, const int *__restrict__ final_id,
                                           const int *__restrict__ chunk_off, int *number, long long N,
                                           unsigned chunk)
{
    __shared__ int s_warp[32];
    const long long base = chunk * (long long)CCL_CHUNK + (long long)threadIdx.x * CCL_PER;
    int par[CCL_PER];
    load_run(parent, base, N, par);
    unsigned flags = 0;
#pragma unroll
    for (int i = 0; i < CCL_PER; ++i) {
        const long long s = base + i;
        if (par[i] == s && final_id[s] == s) flags |= 1u << i;
    }
    const int mine = __popc(flags);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = lane < CCL_CHUNK_THREADS / 32 ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    int rank = chunk_off[chunk] + (wid ? s_warp[wid - 1] : 0) + incl - mine;
    while (flags) {
        const int i = __ffs(flags) - 1;
        number[base + i] = rank++;
        flags &= flags - 1;
    }
}

// Four consecutive pixels per thread; the output is written as one 16-byte
// store when the caller's buffer is 16-byte aligned.
__device__ __forceinline__ void ccl_out(const int *__restrict__ parent, const int *__restrict__ final_id,
                                        const int *__restrict__ number, int *out, long long N, unsigned blk,
                                        unsigned nblk)
{
    const bool vec_out = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    const long long quads = (N + 3) / 4;
    for (long long g = blk * (long long)blockDim.x + threadIdx.x; g < quads; g += (long long)nblk * blockDim.x) {
        const long long s0 = 4 * g;
        if (s0 + 4 <= N) {
            const int4 q = reinterpret_cast<const int4 *>(parent)[g];
            const int4 o = make_int4(number[final_id[q.x]], number[final_id[q.y]], number[final_id[q.z]],
                                     number[final_id[q.w]]);
            if (vec_out) {
                reinterpret_cast<int4 *>(out)[g] = o;
            } else {
                out[s0] = o.x; out[s0 + 1] = o.y; out[s0 + 2] = o.z; out[s0 + 3] = o.w;
            }
        } else {
            for (long long p = s0; p < N; ++p) out[p] = number[final_id[parent[p]]];
        }
    }
}

// ---------------------------------------------------------------------------
// Kernels: one image (block index and grid as above), or a batch, where each
// pass gives every image its own range of blocks and a block finds its image
// in the prefix of the per-image block counts.  Every pass is a programmatic
// launch: its CTAs are placed while the previous pass drains and wait for it
// before their first read.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CCL_LOCAL_THREADS)
    k_ccl_local(const int *__restrict__ labels, int *parent, int *size, int H, int W, int n_tx)
{
    pdl_wait();
    pdl_release();
    ccl_local(labels, parent, size, H, W, n_tx, blockIdx.x);
}

__global__ void k_ccl_border(const int *__restrict__ labels, int *parent, int H, int W, int n_tx, int n_ty)
{
    pdl_wait();
    pdl_release();
    ccl_border(labels, parent, H, W, n_tx, n_ty, blockIdx.x, gridDim.x);
}

__global__ void k_ccl_flatten_count(int *parent, int *size, long long N)
{
    pdl_wait();
    pdl_release();
    ccl_flatten_count(parent, size, N, blockIdx.x, gridDim.x);
}

__global__ void k_ccl_link(const int *__restrict__ parent, const int *__restrict__ size, int *link, int W,
                           long long N, long long T)
{
    pdl_wait();
    pdl_release();
    ccl_link(parent, size, link, W, N, T, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(CCL_CHUNK_THREADS)
    k_ccl_resolve_count(const int *__restrict__ parent, const int *__restrict__ link, int *final_id,
                        long long N, DevCounters *ctr, int *chunk_count)
{
    pdl_wait();
    pdl_release();
    ccl_resolve_count(parent, link, final_id, N, ctr, chunk_count, blockIdx.x);
}

__global__ void __launch_bounds__(CCL_SCAN_THREADS) k_ccl_chunk_scan(int *counts, long long n, int *total)
{
    pdl_wait();
    pdl_release();
    ccl_chunk_scan(counts, n, total);
}

__global__ void __launch_bounds__(CCL_CHUNK_THREADS)
    k_ccl_number(const int *__restrict__ parent, const int *__restrict__ final_id,
                 const int *__restrict__ chunk_off, int *number, long long N)
{
    pdl_wait();
    pdl_release();
    ccl_number(parent, final_id, chunk_off, number, N, blockIdx.x);
}

__global__ void k_ccl_out(const int *__restrict__ parent, const int *__restrict__ final_id,
                          const int *__restrict__ number, int *out, long long N)
{
    pdl_wait();
    pdl_release();
    ccl_out(parent, final_id, number, out, N, blockIdx.x, gridDim.x);
}

// The image of this block in pass `kind`, and the block's place in its range.
struct CclBlock {
    int i;
    unsigned blk, nblk;
};

__device__ __forceinline__ CclBlock ccl_block(const CclBatch &cb, int kind)
{
    const int *base = cb.base[kind];
    const int g = (int)blockIdx.x;
    const int i = batch_find(base, cb.count, g);
    return {i, (unsigned)(g - base[i]), (unsigned)(base[i + 1] - base[i])};
}

__global__ void __launch_bounds__(CCL_LOCAL_THREADS) k_ccl_local_batch(CclBatch cb)
{
    pdl_wait();
    pdl_release();
    const CclBlock b = ccl_block(cb, CCL_KIND_TILES);
    const CclImage &m = cb.img[b.i];
    const unsigned tiles = (unsigned)(m.n_tx * m.n_ty);
    for (unsigned t = b.blk; t < tiles; t += b.nblk) {
        ccl_local(m.labels, m.parent, m.size, m.H, m.W, m.n_tx, (int)t);
        __syncthreads();  // the shared arrays are reused by the next tile
    }
}

__global__ void k_ccl_border_batch(CclBatch cb)
{
    pdl_wait();
    pdl_release();
    const CclBlock b = ccl_block(cb, CCL_KIND_BORDER);
    const CclImage &m = cb.img[b.i];
    ccl_border(m.labels, m.parent, m.H, m.W, m.n_tx, m.n_ty, b.blk, b.nblk);
}

__global__ void k_ccl_flatten_count_batch(CclBatch cb)
{
    pdl_wait();
    pdl_release();
    const CclBlock b = ccl_block(cb, CCL_KIND_PIXELS);
    const CclImage &m = cb.img[b.i];
    ccl_flatten_count(m.parent, m.size, m.N, b.blk, b.nblk);
}

__global__ void k_ccl_link_batch(CclBatch cb)
{
    pdl_wait();
    pdl_release();
    const CclBlock b = ccl_block(cb, CCL_KIND_QUADS);
    const CclImage &m = cb.img[b.i];
    ccl_link(m.parent, m.size, m.link, m.W, m.N, m.T, b.blk, b.nblk);
}

__global__ void __launch_bounds__(CCL_CHUNK_THREADS) k_ccl_resolve_count_batch(CclBatch cb)
{
    pdl_wait();
    pdl_release();
    const CclBlock b = ccl_block(cb, CCL_KIND_CHUNKS);
    const CclImage &m = cb.img[b.i];
    ccl_resolve_count(m.parent, m.link, m.size, m.N, m.ctr, m.scan_tmp, b.blk);
}

// One CTA per image; it also copies the image's counters (no later pass
// writes them) to where the host gathers them.
__global__ void __launch_bounds__(CCL_SCAN_THREADS) k_ccl_chunk_scan_batch(CclBatch cb)
{
    pdl_wait();
    pdl_release();
    const int i = blockIdx.x;
    const CclImage &m = cb.img[i];
    ccl_chunk_scan(m.scan_tmp, ceil_div_ll(m.N, CCL_CHUNK), m.nlab);
    if (threadIdx.x == 0) *m.ctr_out = *m.ctr;
}

__global__ void __launch_bounds__(CCL_CHUNK_THREADS) k_ccl_number_batch(CclBatch cb)
{
    pdl_wait();
    pdl_release();
    const CclBlock b = ccl_block(cb, CCL_KIND_CHUNKS);
    const CclImage &m = cb.img[b.i];
    ccl_number(m.parent, m.size, m.scan_tmp, m.scan, m.N, b.blk);
}

__global__ void k_ccl_out_batch(CclBatch cb)
{
    pdl_wait();
    pdl_release();
    const CclBlock b = ccl_block(cb, CCL_KIND_QUADS);
    const CclImage &m = cb.img[b.i];
    ccl_out(m.parent, m.size, m.scan, cb.out[b.i], m.N, b.blk, b.nblk);
}

long long ccl_scan_tmp_len(long long N) { return ceil_div_ll(N, CCL_CHUNK) + 64; }

void launch_ccl(const int *labels, int H, int W, int K, int *out, const CclBuffers &b, int *d_nlab,
                DevCounters *ctr, cudaStream_t st)
{
    const long long N = (long long)H * W;
    const long long T = N / (4LL * K);
    const int blocks = (int)std::min<long long>(ceil_div_ll(N, CCL_THREADS), 152 * 16);
    const int qblocks = (int)std::min<long long>(ceil_div_ll((N + 3) / 4, CCL_THREADS), 152 * 16);
    const int n_tx = (W + CCL_TILE - 1) / CCL_TILE, n_ty = (H + CCL_TILE - 1) / CCL_TILE;
    pdl_launch(true, k_ccl_local, dim3(n_tx * n_ty), dim3(CCL_LOCAL_THREADS), 0, st, labels, b.parent, b.size,
               H, W, n_tx);
    const long long nb = (long long)(n_tx - 1) * H + (long long)(n_ty - 1) * W;
    if (nb > 0)
        pdl_launch(true, k_ccl_border, dim3((unsigned)std::min<long long>(ceil_div_ll(nb, CCL_THREADS), 152 * 16)),
                   dim3(CCL_THREADS), 0, st, labels, b.parent, H, W, n_tx, n_ty);
    pdl_launch(true, k_ccl_flatten_count, dim3(blocks), dim3(CCL_THREADS), 0, st, b.parent, b.size, N);
    pdl_launch(true, k_ccl_link, dim3(qblocks), dim3(CCL_THREADS), 0, st, (const int *)b.parent,
               (const int *)b.size, b.link, W, N, T);
    const long long chunks = ceil_div_ll(N, CCL_CHUNK);
    pdl_launch(true, k_ccl_resolve_count, dim3((unsigned)chunks), dim3(CCL_CHUNK_THREADS), 0, st,
               (const int *)b.parent, (const int *)b.link, b.size, N, ctr, b.scan_tmp);
    pdl_launch(true, k_ccl_chunk_scan, dim3(1), dim3(CCL_SCAN_THREADS), 0, st, b.scan_tmp, chunks, d_nlab);
    pdl_launch(true, k_ccl_number, dim3((unsigned)chunks), dim3(CCL_CHUNK_THREADS), 0, st, (const int *)b.parent,
               (const int *)b.size, (const int *)b.scan_tmp, b.scan, N);
    pdl_launch(true, k_ccl_out, dim3(qblocks), dim3(CCL_THREADS), 0, st, (const int *)b.parent,
               (const int *)b.size, (const int *)b.scan, out, N);
}

// Blocks of one image per pass in a batch.  A block first finds its image, so
// each takes several units (tiles, border pixels, 32-pixel runs, quads) to
// pay for that lookup; chunks are large enough alone.
constexpr int CCL_BATCH_TILES = 4, CCL_BATCH_BORDER = 1, CCL_BATCH_RUNS = 8, CCL_BATCH_QUADS = 8;

void ccl_batch_blocks(int H, int W, long long blocks[CCL_KINDS])
{
    const long long N = (long long)H * W;
    const long long n_tx = (W + CCL_TILE - 1) / CCL_TILE, n_ty = (H + CCL_TILE - 1) / CCL_TILE;
    blocks[CCL_KIND_TILES] = ceil_div_ll(n_tx * n_ty, CCL_BATCH_TILES);
    blocks[CCL_KIND_BORDER] = ceil_div_ll((n_tx - 1) * H + (n_ty - 1) * W, (long long)CCL_THREADS * CCL_BATCH_BORDER);
    blocks[CCL_KIND_PIXELS] = ceil_div_ll(N, (long long)CCL_THREADS * CCL_BATCH_RUNS);  // warps of 32 pixels
    blocks[CCL_KIND_QUADS] = ceil_div_ll((N + 3) / 4, (long long)CCL_THREADS * CCL_BATCH_QUADS);
    blocks[CCL_KIND_CHUNKS] = ceil_div_ll(N, CCL_CHUNK);
}

void launch_ccl_batch(const CclBatch &cb, const int total[CCL_KINDS], cudaStream_t st)
{
    if (cb.count <= 0) return;
    pdl_launch(true, k_ccl_local_batch, dim3(total[CCL_KIND_TILES]), dim3(CCL_LOCAL_THREADS), 0, st, cb);
    if (total[CCL_KIND_BORDER] > 0)
        pdl_launch(true, k_ccl_border_batch, dim3(total[CCL_KIND_BORDER]), dim3(CCL_THREADS), 0, st, cb);
    pdl_launch(true, k_ccl_flatten_count_batch, dim3(total[CCL_KIND_PIXELS]), dim3(CCL_THREADS), 0, st, cb);
    pdl_launch(true, k_ccl_link_batch, dim3(total[CCL_KIND_QUADS]), dim3(CCL_THREADS), 0, st, cb);
    pdl_launch(true, k_ccl_resolve_count_batch, dim3(total[CCL_KIND_CHUNKS]), dim3(CCL_CHUNK_THREADS), 0, st, cb);
    pdl_launch(true, k_ccl_chunk_scan_batch, dim3(cb.count), dim3(CCL_SCAN_THREADS), 0, st, cb);
    pdl_launch(true, k_ccl_number_batch, dim3(total[CCL_KIND_CHUNKS]), dim3(CCL_CHUNK_THREADS), 0, st, cb);
    pdl_launch(true, k_ccl_out_batch, dim3(total[CCL_KIND_QUADS]), dim3(CCL_THREADS), 0, st, cb);
}

}  // namespace scalp
