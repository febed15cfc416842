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
//   4. The surviving components are numbered 0.. in raster order of seeds.
#include <algorithm>

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

__device__ __forceinline__ int find_local(const volatile int *sp, int x)
{
    int p = sp[x];
    while (p != x) {
        x = p;
        p = sp[x];
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

__global__ void __launch_bounds__(CCL_TILE * CCL_TILE)
    k_ccl_local(const int *__restrict__ labels, int *parent, int *size, int H, int W, int n_tx)
{
    __shared__ int sp[CCL_TILE * CCL_TILE];
    __shared__ int sl[CCL_TILE * CCL_TILE];
    __shared__ unsigned srun[CCL_TILE];  // per row: bit x set where a run starts
    const int t = threadIdx.x;
    const int lx = t % CCL_TILE, ly = t / CCL_TILE;  // one warp per tile row
    const int x0 = (blockIdx.x % n_tx) * CCL_TILE, y0 = (blockIdx.x / n_tx) * CCL_TILE;
    const int x = x0 + lx, y = y0 + ly;
    const bool valid = x < W && y < H;
    const long long p = (long long)y * W + x;
    const int lab = valid ? labels[p] : 0;
    sl[t] = lab;
    // runs of equal label along the row: each pixel's head is the last run
    // start at or before it
    const int left = __shfl_up_sync(0xffffffffu, lab, 1);
    const unsigned starts = __ballot_sync(0xffffffffu, lx == 0 || !valid || left != lab);
    const int head = 31 - __clz(starts & (0xffffffffu >> (31 - lx)));
    sp[t] = ly * CCL_TILE + head;
    if (lx == 0) srun[ly] = starts;
    __syncthreads();
    // one union per pair of vertically touching runs: at the first pixel of
    // their overlap, where this pixel or the one above starts a run
    if (valid && ly > 0 && sl[t - CCL_TILE] == lab &&
        (((starts >> lx) & 1u) || ((srun[ly - 1] >> lx) & 1u)))
        unite_local(sp, t, t - CCL_TILE);
    __syncthreads();
    if (valid) {
        const int r = find_local(sp, t);
        parent[p] = (int)((long long)(y0 + r / CCL_TILE) * W + x0 + r % CCL_TILE);
        size[p] = 0;
    }
}

// Pass 2: unions across tile borders (left edge and top edge of each tile).
__global__ void k_ccl_border(const int *__restrict__ labels, int *parent, int H, int W, int n_tx,
                             int n_ty)
{
    const long long nv = (long long)(n_tx - 1) * H;  // vertical border pixels
    const long long nh = (long long)(n_ty - 1) * W;  // horizontal border pixels
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv + nh;
         i += (long long)gridDim.x * blockDim.x) {
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

__global__ void k_ccl_flatten_count(int *parent, int *size, long long N)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        int r = find_root(parent, (int)p);
        parent[p] = r;
        atomicAdd(&size[r], 1);
    }
}

__global__ void k_ccl_link(const int *__restrict__ parent, const int *__restrict__ size, int *link,
                           int W, long long N, long long T)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        if (parent[s] != s) continue;
        bool small = size[s] <= T && s != 0;
        long long nb = (s % W) > 0 ? s - 1 : s - W;
        link[s] = small ? parent[nb] : (int)s;
    }
}

// final[s] = first non-small ancestor of seed s; written over size[].
__global__ void k_ccl_resolve(const int *__restrict__ parent, const int *__restrict__ link,
                              int *final_id, long long N, DevCounters *ctr)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        if (parent[s] != s) continue;
        int f = (int)s;
        long long guard = 0;
        while (true) {
            int nf = link[f];
            if (nf == f) break;
            f = nf;
            if (++guard > N) {
                atomicExch(&ctr->error, ERR_CCL_CHAIN);
                break;
            }
        }
        final_id[s] = f;
    }
}

__global__ void k_ccl_flag(const int *__restrict__ parent, const int *__restrict__ final_id,
                           int *flag, long long N)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x)
        flag[p] = (parent[p] == p && final_id[p] == p) ? 1 : 0;
}

__global__ void k_ccl_out(const int *__restrict__ parent, const int *__restrict__ final_id,
                          const int *__restrict__ number, int *out, long long N)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x)
        out[p] = number[final_id[parent[p]]];
}

// ---------------------------------------------------------------------------
// Exclusive scan of int32 in place: blocks of 4096, then the block sums.
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_block(int *data, long long n, int *sums)
{
    __shared__ int s_warp[32];
    const long long base = blockIdx.x * (long long)SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int tsum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < n ? data[base + i] : 0;
        tsum += v[i];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = tsum;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    int run = (wid ? s_warp[wid - 1] : 0) + incl - tsum;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) data[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == SCAN_THREADS - 1) sums[blockIdx.x] = run;
}

__global__ void k_scan_add(int *data, long long n, const int *__restrict__ sums)
{
    const long long base = blockIdx.x * (long long)SCAN_CHUNK;
    const int add = sums[blockIdx.x];
    for (int i = threadIdx.x; i < SCAN_CHUNK; i += blockDim.x)
        if (base + i < n) data[base + i] += add;
}

long long ccl_scan_tmp_len(long long N)
{
    long long len = 0, n = N;
    do {
        n = ceil_div_ll(n, SCAN_CHUNK);
        len += n + 64;
    } while (n > 1);
    return len + 64;
}

// After the call, *total holds the sum of the n inputs.
static void scan_exclusive(int *data, long long n, int *tmp, int *total, cudaStream_t st)
{
    long long nb = ceil_div_ll(n, SCAN_CHUNK);
    k_scan_block<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(data, n, tmp);
    if (nb == 1) {
        cudaMemcpyAsync(total, tmp, sizeof(int), cudaMemcpyDeviceToDevice, st);
        return;
    }
    scan_exclusive(tmp, nb, tmp + nb + 64, total, st);
    k_scan_add<<<(unsigned)nb, 256, 0, st>>>(data, n, tmp);
}

void launch_ccl(const int *labels, int H, int W, int K, int *out, const CclBuffers &b, int *d_nlab,
                DevCounters *ctr, cudaStream_t st)
{
    const long long N = (long long)H * W;
    const long long T = N / (4LL * K);
    const int blocks = (int)std::min<long long>(ceil_div_ll(N, CCL_THREADS), 152 * 16);
    const int n_tx = (W + CCL_TILE - 1) / CCL_TILE, n_ty = (H + CCL_TILE - 1) / CCL_TILE;
    k_ccl_local<<<n_tx * n_ty, CCL_TILE * CCL_TILE, 0, st>>>(labels, b.parent, b.size, H, W, n_tx);
    const long long nb = (long long)(n_tx - 1) * H + (long long)(n_ty - 1) * W;
    if (nb > 0)
        k_ccl_border<<<(int)std::min<long long>(ceil_div_ll(nb, CCL_THREADS), 152 * 16), CCL_THREADS, 0,
                       st>>>(labels, b.parent, H, W, n_tx, n_ty);
    k_ccl_flatten_count<<<blocks, CCL_THREADS, 0, st>>>(b.parent, b.size, N);
    k_ccl_link<<<blocks, CCL_THREADS, 0, st>>>(b.parent, b.size, b.link, W, N, T);
    k_ccl_resolve<<<blocks, CCL_THREADS, 0, st>>>(b.parent, b.link, b.size, N, ctr);
    k_ccl_flag<<<blocks, CCL_THREADS, 0, st>>>(b.parent, b.size, b.scan, N);
    scan_exclusive(b.scan, N, b.scan_tmp, d_nlab, st);
    k_ccl_out<<<blocks, CCL_THREADS, 0, st>>>(b.parent, b.size, b.scan, out, N);
}

}  // namespace scalp
