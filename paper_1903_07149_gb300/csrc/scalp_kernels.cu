// scalp_kernels.cu -- set-up, cluster update, projection and candidate-list
// kernels of libscalp.  The assignment kernel is in scalp_assign.cu and the
// connectivity enforcement in scalp_ccl.cu.
#include <cfloat>
#include <climits>

#include <algorithm>
#include <mutex>

#include "scalp_launch.h"
#include "scalp_phases.cuh"

namespace scalp {

// ---------------------------------------------------------------------------
// Set-up (once per solve): sRGB -> CIELab, contour factor, grid label.
// CIELab follows the sRGB standard: inverse transfer function, the D65
// sRGB->XYZ matrix, normalisation by the XYZ of sRGB white (the matrix row
// sums), then the CIE 1976 L*a*b* companding with the linear segment below
// (6/29)^3.
// ---------------------------------------------------------------------------
// Inverse sRGB transfer function for the 256 byte values, in double.  It is
// a constant of the method: built once per device into static device memory
// (spread over SRGB_TABLE_CTAS CTAs, FP64 being slow on one SM).
constexpr int SRGB_TABLE_CTAS = 8;
static __device__ float g_srgb_lut[256];

__global__ void k_srgb_table(float *lut)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 256) {
        const double c = i / 255.0;
        lut[i] = (float)(c <= 0.04045 ? c / 12.92 : pow((c + 0.055) / 1.055, 2.4));
    }
}

cudaError_t srgb_table(const float **table, cudaStream_t st)
{
    constexpr int MAX_DEVICES = 64;
    static std::mutex mu;
    static const float *ready[MAX_DEVICES] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!ready[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_srgb_lut);
        if (e == cudaSuccess) {
            k_srgb_table<<<SRGB_TABLE_CTAS, 256 / SRGB_TABLE_CTAS, 0, st>>>(static_cast<float *>(p));
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        ready[dev] = static_cast<const float *>(p);
    }
    *table = ready[dev];
    return cudaSuccess;
}

// The set-up in warp tasks.  A task is a strip of 32 columns over at most
// SETUP_ROWS rows of one row of grid cells; along those rows the strip's
// pixels keep their grid cells (Algorithm 1 initialisation: the label of a
// pixel is its cell of the regular grid).  Per pixel: CIELab, contour factor,
// plane sample and label; each lane sums the colour of its pixels (fixed
// point, from the values as stored: FP16-rounded in that format).  Once per
// task the lanes of each cell add the integer sums of (1, x, y, L, a, b) of
// their pixels to the cell, counts and coordinates in closed form.  With
// wait_sums the warp waits for its predecessor launch (which zeroes the sums)
// only before that addition.
constexpr int SETUP_THREADS = 256;
constexpr int SETUP_ROWS = 8;

// Warp tasks of one image: strips x cell rows x chunks of SETUP_ROWS rows (a
// cell row is at most ceil(H/ny) rows high; shorter ones leave tasks empty).
__host__ __device__ inline long long setup_task_count(int H, int W, int ny, int &strips, int &chunks)
{
    strips = (W + 31) / 32;
    chunks = ((H + ny - 1) / ny + SETUP_ROWS - 1) / SETUP_ROWS;
    return (long long)strips * ny * chunks;
}

// Exact sum over the warp of per-lane values below 2^31 in magnitude: the
// high and low 16-bit halves are reduced apart (neither sum can overflow).
__device__ __forceinline__ long long warp_sum_wide(int v)
{
    const int hi = __reduce_add_sync(0xffffffffu, v >> 16);
    const unsigned lo = __reduce_add_sync(0xffffffffu, (unsigned)v & 0xffffu);
    return (long long)hi * 65536 + (long long)lo;
}

__device__ __forceinline__ void setup_task(const SolveArgs &a, const float *lin, const uint8_t *__restrict__ rgb,
                                           long long rgb_stride, const float *__restrict__ contour,
                                           long long contour_stride, int storage, void *plane, long long task,
                                           bool wait_sums)
{
    int strips, chunks;
    setup_task_count(a.H, a.W, a.ny, strips, chunks);
    const int strip = (int)(task % strips);
    const long long rest = task / strips;
    const int chunk = (int)(rest % chunks), cy = (int)(rest / chunks);
    // the rows of cell row cy are those with floor(y * ny / H) = cy
    const int ylo = (int)(((long long)cy * a.H + a.ny - 1) / a.ny);
    const int yend = (int)(((long long)(cy + 1) * a.H + a.ny - 1) / a.ny);
    const int y0 = ylo + chunk * SETUP_ROWS, y1 = min(y0 + SETUP_ROWS, yend);
    if (y0 >= y1) return;  // warp-uniform
    const int lane = threadIdx.x & 31, bx = strip * 32, x = bx + lane;
    const bool valid = x < a.W;
    const int cx = a.grid_rcp_x ? (int)__umulhi((unsigned)x * (unsigned)a.nx, a.grid_rcp_x)
                                : (int)((long long)x * a.nx / a.W);
    const int key = cy * a.nx + cx;
    const float inv_s2 = 1.0f / (a.sigma * a.sigma);
    const float scale = (float)(1 << COLOR_FRAC_BITS);
    // per lane: SETUP_ROWS * 108 * 2^COLOR_FRAC_BITS < 2^31
    static_assert((long long)SETUP_ROWS * 108 * (1LL << COLOR_FRAC_BITS) < (1LL << 31), "lane colour sums");
    int sL = 0, sa = 0, sb = 0;
    if (valid) {
#pragma unroll 4
        for (int y = y0; y < y1; ++y) {
            const float3 c3 = srgb_to_lab(lin, rgb + y * rgb_stride + 3 * (long long)x);
            const float c = contour ? contour[y * contour_stride + x] : 0.0f;
            const float w = -expm1f(-(c * c) * inv_s2);  // 1 - exp(-C^2/sigma^2), Eq. 2
            const long long q = (long long)y * a.pitch + x;
            float4 v;
            if (storage == 0) {
                v = make_float4(c3.x, c3.y, c3.z, w);
                reinterpret_cast<float4 *>(plane)[q] = v;
            } else {
                const __half2 lo = __floats2half2_rn(c3.x, c3.y), hi = __floats2half2_rn(c3.z, w);
                uint2 u;
                u.x = *reinterpret_cast<const unsigned *>(&lo);
                u.y = *reinterpret_cast<const unsigned *>(&hi);
                reinterpret_cast<uint2 *>(plane)[q] = u;
                v = sample_value(u);
            }
            a.labels[(long long)y * a.W + x] = key;
            sL += __float2int_rn(v.x * scale);
            sa += __float2int_rn(v.y * scale);
            sb += __float2int_rn(v.z * scale);
        }
    }
    if (wait_sums) pdl_wait();
    const long long rows = y1 - y0, row_sum = (long long)(y0 + y1 - 1) * rows / 2;
    unsigned pending = __ballot_sync(0xffffffffu, valid);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int k = __shfl_sync(0xffffffffu, key, leader);
        const bool mine = valid && key == k;
        const unsigned grp = __ballot_sync(0xffffffffu, mine);
        const long long n = __popc(grp);
        const unsigned lanes = __reduce_add_sync(0xffffffffu, mine ? (unsigned)lane : 0u);
        const long long tL = warp_sum_wide(mine ? sL : 0), ta = warp_sum_wide(mine ? sa : 0),
                        tb = warp_sum_wide(mine ? sb : 0);
        if (lane == leader) acc_add(&a.acc[k], n * rows, rows * (n * bx + lanes), n * row_sum, tL, ta, tb);
        pending &= ~grp;
    }
}

// The block's warps take tasks task0, task0 + 1, ...; lin is loaded first.
__device__ __forceinline__ void setup_block(const SolveArgs &a, const uint8_t *__restrict__ rgb, long long rgb_stride,
                                            const float *__restrict__ contour, long long contour_stride, int storage,
                                            void *plane, long long task0, bool wait_sums)
{
    __shared__ float lin[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) lin[i] = a.lut[i];
    __syncthreads();
    int strips, chunks;
    const long long tasks = setup_task_count(a.H, a.W, a.ny, strips, chunks);
    const long long task = task0 + (threadIdx.x >> 5);
    if (task < tasks)
        setup_task(a, lin, rgb, rgb_stride, contour, contour_stride, storage, plane, task, wait_sums);
}

// First the counters, cluster sums, tile counts and list cursors are zeroed
// (zero_blocks() CTAs per image), then the set-up runs as a programmatic launch:
// it is placed once the zeroing has waited for the work before it (the zeroing
// waits before it releases), converts its pixels meanwhile and waits for the
// zeroing before its first addition.  A batch gives each image its own range
// of set-up blocks.
constexpr int ZERO_THREADS = 256, ZERO_PER_THREAD = 8;

int zero_blocks(int Keff, int tiles)
{
    const long long words = std::max<long long>((long long)Keff * (long long)(sizeof(ClusterAcc) / sizeof(int4)), tiles);
    return (int)std::max<long long>(1, ceil_div_ll(words, (long long)ZERO_THREADS * ZERO_PER_THREAD));
}

__device__ __forceinline__ void zero_solver(const SolveArgs &a, int part, int parts)
{
    const int t0 = part * blockDim.x + threadIdx.x;
    const int step = parts * blockDim.x;
    static_assert(sizeof(ClusterAcc) % sizeof(int4) == 0, "cluster sums are cleared as int4");
    const int acc4 = a.Keff * (int)(sizeof(ClusterAcc) / sizeof(int4));
    for (int j = t0; j < acc4; j += step) reinterpret_cast<int4 *>(a.acc)[j] = make_int4(0, 0, 0, 0);
    const int tiles = a.n_tx * a.n_ty;
    for (int j = t0; j < tiles; j += step) {
        a.tile_count[j] = 0;
        a.tile_cursor[j] = 0;
    }
    for (int j = t0; j < (int)(sizeof(DevCounters) / sizeof(int)); j += step) reinterpret_cast<int *>(a.ctr)[j] = 0;
}

__global__ void k_zero(SolveArgs a)
{
    pdl_wait();
    pdl_release();
    zero_solver(a, blockIdx.x, gridDim.x);
}

__global__ void k_zero_batch(BatchArgs b, int parts)
{
    pdl_wait();
    pdl_release();
    const SolveArgs a = b.args[blockIdx.x / parts];
    zero_solver(a, blockIdx.x % parts, parts);
}

__global__ void __launch_bounds__(SETUP_THREADS)
    k_setup(SolveArgs a, const uint8_t *__restrict__ rgb, long long rgb_stride,
            const float *__restrict__ contour, long long contour_stride, int storage, void *plane)
{
    pdl_release();
    setup_block(a, rgb, rgb_stride, contour, contour_stride, storage, plane,
                (long long)blockIdx.x * (SETUP_THREADS / 32), true);
}

__global__ void __launch_bounds__(SETUP_THREADS)
    k_setup_batch(BatchArgs b, const SetupInput *__restrict__ in, const int *__restrict__ setup_base, int storage)
{
    pdl_release();
    const int g = (int)blockIdx.x;
    const int i = batch_find(setup_base, b.count, g);
    const SolveArgs a = b.args[i];
    const SetupInput u = in[i];
    void *plane = storage == 0 ? (void *)a.plane32 : (void *)a.plane16;
    setup_block(a, u.rgb, u.rgb_stride, u.contour, u.contour_stride, storage, plane,
                (long long)(g - setup_base[i]) * (SETUP_THREADS / 32), true);
}


// ---------------------------------------------------------------------------
// Contour prior from the image (Sec. II-E takes any soft prior in [0, 1]):
// the CIELab gradient magnitude over its maximum.  Per channel and axis the
// derivative is the central difference / 2 inside, one-sided at the ends, 0
// along an axis of length 1; the magnitude is the norm of the six.  A CTA
// converts its tile plus a one-pixel ring (coordinates clamped; the ring is
// only read where the derivative uses it) into shared memory, writes the
// magnitudes and raises the global maximum (float bits order like the
// values for g >= 0); a second pass divides by it.
// ---------------------------------------------------------------------------
constexpr int PRIOR_TX = 32, PRIOR_TY = 32;  // pixels per CTA
constexpr int PRIOR_THREADS = 256;            // PRIOR_TX x 8: four rows per thread

__device__ __forceinline__ float axis_derivative(float fm, float f0, float fp, int i, int n)
{
    if (n < 2) return 0.0f;
    if (i == 0) return fp - f0;
    if (i == n - 1) return f0 - fm;
    return (fp - fm) * 0.5f;
}

__global__ void __launch_bounds__(PRIOR_THREADS)
    k_prior_gradient(const uint8_t *__restrict__ rgb, long long rgb_stride, int H, int W,
                     const float *__restrict__ lut, float *out, long long out_stride, unsigned *gmax)
{
    pdl_wait();  // the table and the cleared maximum
    pdl_release();
    __shared__ float lin[256];
    __shared__ float s_lab[3][PRIOR_TY + 2][PRIOR_TX + 2];
    __shared__ unsigned s_max;
    const int tid = threadIdx.x;
    for (int i = tid; i < 256; i += PRIOR_THREADS) lin[i] = lut[i];
    if (tid == 0) s_max = 0u;
    __syncthreads();
    const int x0 = blockIdx.x * PRIOR_TX, y0 = blockIdx.y * PRIOR_TY;
    for (int i = tid; i < (PRIOR_TX + 2) * (PRIOR_TY + 2); i += PRIOR_THREADS) {
        const int hx = i % (PRIOR_TX + 2), hy = i / (PRIOR_TX + 2);
        const int x = min(max(x0 - 1 + hx, 0), W - 1), y = min(max(y0 - 1 + hy, 0), H - 1);
        const float3 lab = srgb_to_lab(lin, rgb + y * rgb_stride + 3 * (long long)x);
        s_lab[0][hy][hx] = lab.x;
        s_lab[1][hy][hx] = lab.y;
        s_lab[2][hy][hx] = lab.z;
    }
    __syncthreads();
    const int tx = tid % PRIOR_TX;
    float gm = 0.0f;
#pragma unroll
    for (int ty = tid / PRIOR_TX; ty < PRIOR_TY; ty += PRIOR_THREADS / PRIOR_TX) {
        const int x = x0 + tx, y = y0 + ty;
        if (x < W && y < H) {
            float s2 = 0.0f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float gx = axis_derivative(s_lab[c][ty + 1][tx], s_lab[c][ty + 1][tx + 1],
                                                 s_lab[c][ty + 1][tx + 2], x, W);
                const float gy = axis_derivative(s_lab[c][ty][tx + 1], s_lab[c][ty + 1][tx + 1],
                                                 s_lab[c][ty + 2][tx + 1], y, H);
                s2 += gx * gx + gy * gy;
            }
            const float g = sqrtf(s2);
            out[y * out_stride + x] = g;
            gm = fmaxf(gm, g);
        }
    }
    const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(gm));
    if ((tid & 31) == 0) atomicMax(&s_max, m);
    __syncthreads();
    if (tid == 0) atomicMax(gmax, s_max);
}

// The same tiles, four rows per thread.
__global__ void __launch_bounds__(PRIOR_THREADS)
    k_prior_normalise(float *out, long long out_stride, int H, int W, const unsigned *gmax)
{
    pdl_wait();  // every magnitude and the final maximum
    const float m = __uint_as_float(*gmax);
    const int x = blockIdx.x * PRIOR_TX + threadIdx.x % PRIOR_TX;
#pragma unroll
    for (int ty = threadIdx.x / PRIOR_TX; ty < PRIOR_TY; ty += PRIOR_THREADS / PRIOR_TX) {
        const int y = blockIdx.y * PRIOR_TY + ty;
        if (x < W && y < H) {
            float &v = out[y * out_stride + x];
            v = m > 0.0f ? v / m : 0.0f;
        }
    }
}

// The normalisation is a programmatic launch (it waits for the gradient pass
// before its first read).
void launch_gradient_prior(const uint8_t *rgb, long long rgb_stride, int H, int W, const float *lut,
                           float *out, long long out_stride, unsigned *gmax, cudaStream_t st)
{
    cudaMemsetAsync(gmax, 0, sizeof(unsigned), st);
    const dim3 grid((unsigned)ceil_div_ll(W, PRIOR_TX), (unsigned)ceil_div_ll(H, PRIOR_TY));
    pdl_launch(false, k_prior_gradient, grid, dim3(PRIOR_THREADS), 0, st, rgb, rgb_stride, H, W, lut,
               out, out_stride, gmax);
    pdl_launch(true, k_prior_normalise, grid, dim3(PRIOR_THREADS), 0, st, out, out_stride, H, W,
               (const unsigned *)gmax);
}

void launch_setup(const SolveArgs &a, const uint8_t *rgb, long long rgb_stride,
                  const float *contour, long long contour_stride, int storage, void *plane,
                  cudaStream_t st)
{
    const long long blocks = setup_blocks(a.H, a.W, a.ny);
    pdl_launch(false, k_zero, dim3(zero_blocks(a.Keff, a.n_tx * a.n_ty)), dim3(ZERO_THREADS), 0, st, a);
    pdl_launch(true, k_setup, dim3((unsigned)blocks), dim3(SETUP_THREADS), 0, st, a, rgb, rgb_stride, contour,
               contour_stride, storage, plane);
}

long long setup_blocks(int H, int W, int ny)
{
    int strips, chunks;
    return ceil_div_ll(setup_task_count(H, W, ny, strips, chunks), SETUP_THREADS / 32);
}

void launch_setup_batch(const BatchArgs &b, const SetupInput *in, const int *setup_base, int total_blocks,
                        int zero_parts, int storage, cudaStream_t st)
{
    if (b.count <= 0) return;
    pdl_launch(true, k_zero_batch, dim3((unsigned)(b.count * zero_parts)), dim3(ZERO_THREADS), 0, st, b,
               zero_parts);
    pdl_launch(true, k_setup_batch, dim3((unsigned)total_blocks), dim3(SETUP_THREADS), 0, st, b, in, setup_base,
               storage);
}


__global__ void k_update(SolveArgs a, int from_acc)
{
    pdl_wait();
    pdl_release();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < a.Keff) update_cluster(a, k, from_acc);
}

__global__ void k_update_batch(BatchArgs b, int from_acc)
{
    pdl_wait();
    pdl_release();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= b.clus_base[b.count]) return;
    const int i = batch_find(b.clus_base, b.count, g);
    update_cluster(b.args[i], g - b.clus_base[i], from_acc);
}

void launch_update(const SolveArgs &a, int from_acc, cudaStream_t st, bool pdl)
{
    // small blocks: one thread per cluster is latency-bound, so spread them
    pdl_launch(pdl, k_update, dim3((a.Keff + 63) / 64), dim3(64), 0, st, a, from_acc);
}

__global__ void __launch_bounds__(PROJ_THREADS) k_project(SolveArgs a, int whole_image)
{
    pdl_wait();
    pdl_release();
    project_cta(a, whole_image, blockIdx.x, gridDim.x);
}

// Batch of few images, or of more than the work lists' shared memory holds:
// PROJ_CTAS_PER_IMAGE CTAs per image, each cluster searched by a whole CTA.
constexpr int PROJ_CTAS_PER_IMAGE = 16;
constexpr int PROJ_LIST_MIN_IMAGES = 32;
constexpr int PROJ_LIST_MAX_IMAGES = 3071;  // (4 * count + 2) ints <= 48 KB

__global__ void __launch_bounds__(PROJ_THREADS) k_project_batch_images(BatchArgs b, int whole_image)
{
    pdl_wait();
    pdl_release();
    const int i = blockIdx.x / PROJ_CTAS_PER_IMAGE;
    project_cta(b.args[i], whole_image, blockIdx.x % PROJ_CTAS_PER_IMAGE, PROJ_CTAS_PER_IMAGE);
}

// Batch: the queued clusters of every image as work lists over the grid, each
// with the prefix of its images' queue lengths in shared memory.  A warp
// searches a window alone, so warps pay only when the clusters outnumber the
// CTAs several times (more than four per CTA): then one
// warp per cluster for the images whose windows have at most
// PROJ_WARP_MAX_AREA pixels, and one CTA per cluster for those with larger
// windows and for those whose projection searches the whole image (at
// set-up, or after orphans); with fewer clusters, one CTA per cluster for
// all.  Dynamic shared memory: 4 * count + 2 ints.
constexpr float PROJ_WARP_MAX_AREA = 4096.0f;

__global__ void __launch_bounds__(PROJ_THREADS) k_project_batch(BatchArgs b, int whole_image)
{
    pdl_wait();
    pdl_release();
    extern __shared__ int s_mem[];
    __shared__ int s_warp[32];
    const int count = b.count;
    int *s_nw = s_mem, *s_pw = s_nw + count;          // warp list: lengths, prefix
    int *s_nc = s_pw + count + 1, *s_pc = s_nc + count;  // CTA list: lengths, prefix
    const int G = gridDim.x;
    constexpr int warps = PROJ_THREADS / 32;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        s_nw[i] = 0;
        s_nc[i] = b.args[i].ctr->nproj;
    }
    __syncthreads();
    cta_scan(s_nc, s_pc, count, PROJ_THREADS, s_warp);
    if (s_pc[count] > 4 * G) {  // (the same decision in every CTA)
        for (int i = threadIdx.x; i < count; i += blockDim.x) {
            const SolveArgs &a = b.args[i];
            const float side = 2.0f * (float)a.r + 1.0f;  // window side
            const bool cta = whole_image || a.ctr->proj_all || side * side > PROJ_WARP_MAX_AREA;
            s_nw[i] = cta ? 0 : s_nc[i];
            s_nc[i] = cta ? s_nc[i] : 0;
        }
        __syncthreads();
        cta_scan(s_nc, s_pc, count, PROJ_THREADS, s_warp);
    }
    cta_scan(s_nw, s_pw, count, PROJ_THREADS, s_warp);
    const int total_w = s_pw[count], total_c = s_pc[count];
    for (int t = blockIdx.x * warps + (int)(threadIdx.x >> 5); t < total_w; t += G * warps) {
        const int i = batch_find(s_pw, count, t);
        project_warp(b.args[i], t - s_pw[i]);
    }
    // (t is CTA-uniform: the barriers inside project_cta are safe; it searches
    // the whole image only at set-up or after orphans)
    for (int t = blockIdx.x; t < total_c; t += G) {
        const int i = batch_find(s_pc, count, t);
        project_cta(b.args[i], whole_image, t - s_pc[i], INT_MAX);
    }
}

void launch_project(const SolveArgs &a, int whole_image, cudaStream_t st, bool pdl)
{
    pdl_launch(pdl, k_project, dim3(std::min(a.Keff, 2 * 152)), dim3(PROJ_THREADS), 0, st, a, whole_image);
}

__global__ void __launch_bounds__(SCAN1_THREADS) k_scan_tiles(SolveArgs a) { scan_tiles_cta(a); }

__global__ void __launch_bounds__(SCAN1_THREADS) k_scan_tiles_batch(BatchArgs b)
{
    pdl_wait();
    pdl_release();
    scan_tiles_cta(b.args[blockIdx.x]);
}

// Scan and fill in one launch: every CTA scans the counts into shared memory
// (LISTS_MAX_TILES bounds them), CTA 0 publishes the offsets, and the CTAs
// fill the slots grid-stride with offsets from their own copy.
constexpr int LISTS_THREADS = 256;
constexpr int LISTS_MAX_TILES = 12287;  // (n + 1) ints of shared memory <= 48 KB

// The scan and fill by CTA blk of nblk (blockDim.x threads); s_off holds
// n + 1 ints of dynamic shared memory.
__device__ __forceinline__ void lists_cta(const SolveArgs &a, int blk, int nblk, int *s_off, int *s_warp)
{
    const int n = a.n_tx * a.n_ty;
    cta_scan(a.tile_count, s_off, n, blockDim.x, s_warp);
    if (blk == 0) publish_offsets(a, s_off);
    const long long slots = (long long)a.Keff * a.tpw_x * a.tpw_y;
    const int tpw = a.tpw_x * a.tpw_y;
    for (long long i = blk * (long long)blockDim.x + threadIdx.x; i < slots; i += (long long)nblk * blockDim.x) {
        const int k = slots < (1LL << 32) ? (int)((unsigned)i / (unsigned)tpw) : (int)(i / tpw);
        const int j = (int)(i - (long long)k * tpw);
        const ClusterDev cd = a.cdev[k];
        if (cd.xlo > cd.xhi) continue;
        const int tx = cd.xlo / TILE_X + j % a.tpw_x, ty = cd.ylo / TILE_Y + j / a.tpw_x;
        if (tx > cd.xhi / TILE_X || ty > cd.yhi / TILE_Y) continue;
        const int t = ty * a.n_tx + tx;
        const int pos = s_off[t] + atomicAdd(&a.tile_cursor[t], 1);
        if (pos < a.tile_cap) a.tile_list[pos] = k;
    }
}

__global__ void __launch_bounds__(LISTS_THREADS) k_lists(SolveArgs a)
{
    pdl_wait();
    pdl_release();
    extern __shared__ int s_off[];
    __shared__ int s_warp[32];
    lists_cta(a, blockIdx.x, gridDim.x, s_off, s_warp);
}

// The candidate lists (CTAs [0, n_lists), placed first) and the projection
// (the others) in one launch: both need only the update's output, so the
// iteration stays one chain of programmatic launches.
__global__ void __launch_bounds__(PROJ_THREADS) k_project_lists(SolveArgs a, int n_lists)
{
    pdl_wait();
    pdl_release();
    extern __shared__ int s_off[];
    __shared__ int s_warp[32];
    if ((int)blockIdx.x < n_lists) lists_cta(a, blockIdx.x, n_lists, s_off, s_warp);
    else project_cta(a, 0, blockIdx.x - n_lists, gridDim.x - n_lists);
}

__global__ void k_fill_tiles(SolveArgs a)
{
    fill_slot(a, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

__global__ void k_fill_tiles_batch(BatchArgs b)
{
    pdl_wait();
    pdl_release();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= b.fill_base[b.count]) return;
    const int i = batch_find(b.fill_base, b.count, g);
    fill_slot(b.args[i], g - b.fill_base[i]);
}

// One iteration's update, projection and list kernels for a whole batch.
static void launch_project_batch(const BatchArgs &b, cudaStream_t st, bool pdl, int whole_image)
{
    // the work lists for batches of many images (measured: 64 images 33.26
    // -> 32.69 ms per 10 iterations); a few images keep the per-image CTAs
    // (12 scales of one image: 3.05 against 3.33 ms per map with the lists)
    if (b.count >= PROJ_LIST_MIN_IMAGES && b.count <= PROJ_LIST_MAX_IMAGES)
        pdl_launch(pdl, k_project_batch, dim3(2 * 152), dim3(PROJ_THREADS), (size_t)(4 * b.count + 2) * sizeof(int),
                   st, b, whole_image);
    else
        pdl_launch(pdl, k_project_batch_images, dim3(b.count * PROJ_CTAS_PER_IMAGE), dim3(PROJ_THREADS), 0, st, b,
                   whole_image);
}

void launch_batch_update(const BatchArgs &b, int total_clusters, int total_fill, cudaStream_t st, bool pdl,
                         cudaStream_t side, cudaEvent_t fork, cudaEvent_t join, int whole_image)
{
    if (b.count <= 0) return;
    pdl_launch(pdl, k_update_batch, dim3((total_clusters + 63) / 64), dim3(64), 0, st, b, 1);
    if (side) {  // the lists on a second branch, beside the projection
        cudaEventRecord(fork, st);
        cudaStreamWaitEvent(side, fork, 0);
        pdl_launch(false, k_scan_tiles_batch, dim3(b.count), dim3(SCAN1_THREADS), 0, side, b);
        pdl_launch(true, k_fill_tiles_batch, dim3((total_fill + 255) / 256), dim3(256), 0, side, b);
        cudaEventRecord(join, side);
        launch_project_batch(b, st, pdl, whole_image);
        cudaStreamWaitEvent(st, join, 0);
        return;
    }
    launch_project_batch(b, st, pdl, whole_image);
    pdl_launch(pdl, k_scan_tiles_batch, dim3(b.count), dim3(SCAN1_THREADS), 0, st, b);
    pdl_launch(pdl, k_fill_tiles_batch, dim3((total_fill + 255) / 256), dim3(256), 0, st, b);
}

bool project_lists_fused(const SolveArgs &a) { return a.n_tx * a.n_ty <= LISTS_MAX_TILES; }

void launch_project_lists(const SolveArgs &a, cudaStream_t st, bool pdl)
{
    const int n = a.n_tx * a.n_ty;
    const long long slots = (long long)a.Keff * a.tpw_x * a.tpw_y;
    // one resident wave (two 512-thread CTAs per SM): a few list CTAs, four
    // slots per thread, and the projection in the rest
    const int slots_per_cta = 4 * PROJ_THREADS;
    const int n_lists = (int)std::max(std::min(ceil_div_ll(slots, slots_per_cta), 64LL), 1LL);
    const int n_proj = std::max(std::min(a.Keff, 2 * 152 - n_lists), 1);
    pdl_launch(pdl, k_project_lists, dim3((unsigned)(n_lists + n_proj)), dim3(PROJ_THREADS),
               (size_t)(n + 1) * sizeof(int), st, a, n_lists);
}

void launch_lists(const SolveArgs &a, cudaStream_t st, bool pdl)
{
    const int n = a.n_tx * a.n_ty;
    const long long slots = (long long)a.Keff * a.tpw_x * a.tpw_y;
    if (n <= LISTS_MAX_TILES) {
        const long long blocks = std::min(ceil_div_ll(slots, LISTS_THREADS), 2LL * 152);
        pdl_launch(pdl, k_lists, dim3((unsigned)std::max(blocks, 1LL)), dim3(LISTS_THREADS),
                   (size_t)(n + 1) * sizeof(int), st, a);
    } else {
        k_scan_tiles<<<1, SCAN1_THREADS, 0, st>>>(a);
        k_fill_tiles<<<(unsigned)ceil_div_ll(slots, 256), 256, 0, st>>>(a);
    }
}

// ---------------------------------------------------------------------------
// Debug: the path pixels exactly as the assignment kernel steps through them.
// ---------------------------------------------------------------------------
// One path per thread, pixels in walking order.  The error-term steps give
// the pixels; paths short enough for the fixed-point forms are walked with
// the step form in lockstep and with the grouped closed form after it, and a
// disagreement on any sample reports length -1.
__global__ void k_debug_paths(const int *pairs, int M, int *out_xy, int stride_xy, int *out_len,
                              int W)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const PathSetup s = path_setup(pairs[4 * i], pairs[4 * i + 1], pairs[4 * i + 2], pairs[4 * i + 3]);
    int smaj, smin;
    path_strides(s, W, smaj, smin);
    // offsets in the image, row pitch W (nothing is dereferenced)
    const long long start = (long long)s.ay * W + s.ax;
    long long qe = start, qf = start;
    ErrorTermStep e(s, smaj, smin);
    FixedPointStep f(s, smaj, smin);
    const bool check = s.ns <= FIXED_STEP_MAX_NS;
    bool same = true;
    int *o = out_xy + (long long)i * stride_xy;
    for (int k = 0; k <= s.ns; ++k) {
        if (2 * k + 1 < stride_xy) {
            const int y = (int)(qe / W);
            o[2 * k] = (int)(qe - (long long)y * W);
            o[2 * k + 1] = y;
        }
        same = same && (!check || qf == qe);
        qe += e.next();
        if (check) qf += f.next();
    }
    if (check) {  // the grouped closed form, sample by sample against the error term
        long long qg = start;
        ErrorTermStep g(s, smaj, smin);
        walk_grouped<4>(start, smaj, smin, s, [&](long long q) {
            same = same && q == qg;
            qg += g.next();
        });
    }
    out_len[i] = same ? s.ns + 1 : -1;
}

void launch_debug_paths(const int *pairs, int M, int *out_xy, int stride_xy, int *out_len, int W,
                        cudaStream_t st)
{
    if (M <= 0) return;
    k_debug_paths<<<(M + 127) / 128, 128, 0, st>>>(pairs, M, out_xy, stride_xy, out_len, W);
}

}  // namespace scalp
