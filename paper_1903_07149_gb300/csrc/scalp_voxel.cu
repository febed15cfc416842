// scalp_voxel.cu -- supervoxels: SCALP on a video volume (T frames x H x W),
// the extension the paper's conclusion names as future work.  Each rule is the
// 2-D one taken axis by axis:
//   * r = cbrt(N/K) (computed on the host); a 3-D regular grid of step r;
//   * candidates of cluster k: |v - s_v/n| <= r on each axis, r the real
//     cube root of N/K, i.e. K*|n*v - s_v|^3 <= N*n^3 decided exactly, kept
//     as integer bounds per axis;
//   * the linear path is a 3-D digital segment traced from the
//     lexicographically smaller end (x, then y, then t); the axis with the
//     largest |delta| (ties: x, y, t) steps by one, each other axis by
//     round-half-up(i*|delta_j|/ns);
//   * D is Eq. 3 with the squared 3-D distance, the colour and contour terms of
//     Eq. 1-2 along the path;
//   * update and projection (Eq. 4) as in 2-D, with the voxel index as the
//     tie-break; there is no connectivity step.
//
// One iteration is four kernels: assignment (one 512-thread CTA per 16x8x4
// tile, one voxel per thread, paths walked in global memory, warp-aggregated
// integer sums), update (one thread per cluster), projection (one CTA per
// queued cluster), candidate lists (count scan, then slot fill).
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "scalp_launch.h"
#include "../../include/scalp.h"

namespace scalp {
namespace {

constexpr int VTX = 16, VTY = 8, VTT = 4;  // voxel tile
constexpr int VTILE = VTX * VTY * VTT;     // 512 voxels, one per thread
constexpr int VPROJ_THREADS = 512;

struct VoxCluster {  // 64 bytes: what the assignment reads about cluster k
    float L, a, b;
    float xk, yk, tk;
    int ex, ey, et;
    int xlo, xhi, ylo, yhi, tlo, thi;
    int pad;
};
static_assert(sizeof(VoxCluster) == 64, "VoxCluster layout");

struct VoxAcc {  // 64 bytes: integer sums of one assignment
    unsigned long long n, sx, sy, st, sL, sa, sb, pad;
};

struct VoxArgs {
    int T, H, W, K, Keff, nx, ny, nt;
    long long N, HW;
    double r;
    float lam, gamma, ms2;
    int n_tx, n_ty, n_tt;
    int tpw_x, tpw_y, tpw_t;  // bound on the tiles one window spans, per axis
    long long tile_cap;
    int count_samples;
    const float4 *plane;      // (L, a, b, w) per voxel
    int *labels;
    long long *st_n, *st_sx, *st_sy, *st_st;
    float4 *st_col;
    int4 *st_end;             // (ex, ey, et, 0)
    VoxCluster *cdev;
    VoxAcc *acc;
    int *prev_win;            // 6 ints per cluster: the window the last assignment used
    int *proj_list;
    int *tile_count, *tile_off, *tile_cursor, *tile_list;
    DevCounters *ctr;
    const float *lut;
};

// ---------------------------------------------------------------------------
// Windows: |v - s/n| <= r with r^3 = N/K, i.e. K*q^3 <= N*n^3 for
// q = |n*v - s|.  An FP32 comparison of q/n with r (each within 4e-7
// relative of exact) decides every value farther than 1e-5 relative from the
// edge; the rest are decided in 128-bit integers.  There q <= (1 + 1e-5) n r,
// and a volume holds at most 2^30 voxels (n, N <= 2^30), so K*q^3 and N*n^3
// both stay below 2^121.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool vin_window(long long v, long long n, long long s, long long N, long long K,
                                           double r)
{
    const long long d = n * v - s;
    const unsigned long long q = (unsigned long long)(d < 0 ? -d : d);
    // FP32 filter: q/n and r each within 4e-7 relative of exact, so outside
    // a 1e-5 band the FP32 comparison is the exact one
    const float x = __fdividef((float)q, (float)n), rf = (float)r;
    if (x < rf * (1.0f - 1e-5f)) return true;
    if (x > rf * (1.0f + 1e-5f)) return false;
    const unsigned __int128 lhs = (unsigned __int128)q * q * q * (unsigned long long)K;
    const unsigned __int128 rhs =
        (unsigned __int128)((unsigned long long)N * (unsigned long long)n) * ((unsigned long long)n * (unsigned long long)n);
    return lhs <= rhs;
}

__device__ __forceinline__ void vwindow(long long n, long long s, long long N, long long K, double r, int lim,
                                        int &lo, int &hi)
{
    long long a0, b0;
    window_start(s, n, r, lim, a0, b0);
    int a = (int)max(a0, 0LL), b = (int)min(b0, (long long)lim - 1);
    while (a <= b && !vin_window(a, n, s, N, K, r)) ++a;
    while (b >= a && !vin_window(b, n, s, N, K, r)) --b;
    lo = a;
    hi = b;
}

// ---------------------------------------------------------------------------
// Integer sums of (1, x, y, t, L, a, b) per label; colour fixed point
// 2^COLOR_FRAC_BITS.  A warp's 32 voxels share a frame and lie within 32
// columns and 2 rows of a base, so the three offsets pack into one 32-bit
// warp sum (10 bits each).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void vaggregate(const VoxArgs &a, bool valid, int lab, int bx, int by, int bt,
                                           int dx, int dy, int dt, float4 v)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const float scale = (float)(1 << COLOR_FRAC_BITS);
    const int qL = valid ? __float2int_rn(v.x * scale) : 0;
    const int qa = valid ? __float2int_rn(v.y * scale) : 0;
    const int qb = valid ? __float2int_rn(v.z * scale) : 0;
    const unsigned qc = valid ? (unsigned)dx | ((unsigned)dy << 10) | ((unsigned)dt << 20) : 0u;
    unsigned pending = __ballot_sync(FULL, valid);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int k = __shfl_sync(FULL, lab, leader);
        const bool mine = valid && lab == k;
        const unsigned grp = __ballot_sync(FULL, mine);
        const long long cnt = __popc(grp);
        const unsigned sc = __reduce_add_sync(FULL, mine ? qc : 0u);
        const long long sL = (int)__reduce_add_sync(FULL, mine ? (unsigned)qL : 0u);
        const long long sa = (int)__reduce_add_sync(FULL, mine ? (unsigned)qa : 0u);
        const long long sb = (int)__reduce_add_sync(FULL, mine ? (unsigned)qb : 0u);
        if (lane == leader) {
            VoxAcc *c = &a.acc[k];
            atomicAdd(&c->n, (unsigned long long)cnt);
            atomicAdd(&c->sx, (unsigned long long)(cnt * bx + (long long)(sc & 0x3ffu)));
            atomicAdd(&c->sy, (unsigned long long)(cnt * by + (long long)((sc >> 10) & 0x3ffu)));
            atomicAdd(&c->st, (unsigned long long)(cnt * bt + (long long)(sc >> 20)));
            atomicAdd(&c->sL, (unsigned long long)sL);
            atomicAdd(&c->sa, (unsigned long long)sa);
            atomicAdd(&c->sb, (unsigned long long)sb);
        }
        pending &= ~grp;
    }
}

// ---------------------------------------------------------------------------
// Set-up: CIELab, contour factor, grid label, initial sums.
// ---------------------------------------------------------------------------
// One warp per 32-voxel row segment: CIELab, contour factor, plane sample
// and grid label of each voxel, then the warp-aggregated integer sums of the
// initial clusters from the values just stored (the sums start at zero).
// The frame and row come once per segment; the cell column by a 32-bit
// division when W * nx < 2^32.
__global__ void __launch_bounds__(256) k_vsetup(VoxArgs a, const uint8_t *__restrict__ rgb,
                                               const float *__restrict__ contour, float sigma, float4 *plane)
{
    __shared__ float lin[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) lin[i] = a.lut[i];
    __syncthreads();
    const float inv_s2 = 1.0f / (sigma * sigma);
    const long long segs_per_row = (a.W + 31) / 32;
    const long long n_segs = segs_per_row * a.H * a.T;
    const long long warps = (long long)gridDim.x * (blockDim.x / 32);
    const int lane = threadIdx.x & 31;
    const bool narrow = (unsigned long long)a.W * (unsigned long long)a.nx < (1ULL << 32);
    for (long long s = blockIdx.x * (long long)(blockDim.x / 32) + (threadIdx.x >> 5); s < n_segs; s += warps) {
        const long long row = s / segs_per_row;
        const int x0 = (int)(s - row * segs_per_row) * 32;
        const int t = (int)(row / a.H), y = (int)(row - (long long)t * a.H);
        const int x = x0 + lane;
        const bool valid = x < a.W;
        const long long p = ((long long)t * a.H + y) * a.W + x;
        const int cy = (int)((long long)y * a.ny / a.H), ct = (int)((long long)t * a.nt / a.T);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        int lab = -1;
        if (valid) {
            const float3 c3 = srgb_to_lab(lin, rgb + 3 * p);
            const float c = contour ? contour[p] : 0.0f;
            v = make_float4(c3.x, c3.y, c3.z, -expm1f(-(c * c) * inv_s2));
            plane[p] = v;
            const int cx = narrow ? (int)((unsigned)x * (unsigned)a.nx / (unsigned)a.W)
                                  : (int)((long long)x * a.nx / a.W);
            lab = (ct * a.ny + cy) * a.nx + cx;
            a.labels[p] = lab;
        }
        vaggregate(a, valid, lab, x0, y, t, lane, 0, 0, v);
    }
}

// ---------------------------------------------------------------------------
// Update: means, endpoint, projection request, window, record, tile counts.
// ---------------------------------------------------------------------------
__global__ void k_vupdate(VoxArgs a, int from_acc)
{
    pdl_wait();
    pdl_release();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.Keff) return;
    if (from_acc) {
        const VoxAcc c = a.acc[k];
        a.acc[k] = VoxAcc{};
        const long long n = (long long)c.n;
        if (n > 0) {
            const long long sx = (long long)c.sx, sy = (long long)c.sy, st = (long long)c.st;
            a.st_n[k] = n;
            a.st_sx[k] = sx;
            a.st_sy[k] = sy;
            a.st_st[k] = st;
            const double den = (double)n * (double)(1 << COLOR_FRAC_BITS);
            a.st_col[k] = make_float4((float)((double)(long long)c.sL / den),
                                      (float)((double)(long long)c.sa / den),
                                      (float)((double)(long long)c.sb / den), 0.f);
            const int ex = (int)((2 * sx + n) / (2 * n));
            const int ey = (int)((2 * sy + n) / (2 * n));
            const int et = (int)((2 * st + n) / (2 * n));
            a.st_end[k] = make_int4(ex, ey, et, 0);
            if (a.labels[((long long)et * a.H + ey) * a.W + ex] != k)
                a.proj_list[atomicAdd(&a.ctr->nproj, 1)] = k;
        }
    }
    const long long n = a.st_n[k], sx = a.st_sx[k], sy = a.st_sy[k], st = a.st_st[k];
    const VoxCluster old = a.cdev[k];
    int *pw = a.prev_win + 6 * (long long)k;
    pw[0] = old.xlo; pw[1] = old.xhi; pw[2] = old.ylo; pw[3] = old.yhi; pw[4] = old.tlo; pw[5] = old.thi;
    VoxCluster cd;
    const float4 col = a.st_col[k];
    const int4 e = a.st_end[k];
    cd.L = col.x; cd.a = col.y; cd.b = col.z;
    cd.xk = (float)((double)sx / (double)n);
    cd.yk = (float)((double)sy / (double)n);
    cd.tk = (float)((double)st / (double)n);
    cd.ex = e.x; cd.ey = e.y; cd.et = e.z;
    cd.pad = k;
    vwindow(n, sx, a.N, a.K, a.r, a.W, cd.xlo, cd.xhi);
    vwindow(n, sy, a.N, a.K, a.r, a.H, cd.ylo, cd.yhi);
    vwindow(n, st, a.N, a.K, a.r, a.T, cd.tlo, cd.thi);
    a.cdev[k] = cd;
    if (cd.xlo > cd.xhi || cd.ylo > cd.yhi || cd.tlo > cd.thi) return;
    for (int tt = cd.tlo / VTT; tt <= cd.thi / VTT; ++tt)
        for (int ty = cd.ylo / VTY; ty <= cd.yhi / VTY; ++ty)
            for (int tx = cd.xlo / VTX; tx <= cd.xhi / VTX; ++tx)
                atomicAdd(&a.tile_count[(tt * a.n_ty + ty) * a.n_tx + tx], 1);
}

// ---------------------------------------------------------------------------
// Projection (Eq. 4) of the queued clusters: argmin over the voxels labelled
// k of (n*x - Sx)^2 + (n*y - Sy)^2 + (n*t - St)^2 in 128-bit integers, ties
// to the smallest voxel index; searched over the window the last assignment
// used (it holds S_k) unless some voxel kept its label for lack of a
// candidate, or at set-up: then over the whole volume.
// ---------------------------------------------------------------------------
struct VBest {
    unsigned long long hi, lo;
    long long p;
};

__device__ __forceinline__ bool vless(const VBest &u, const VBest &v)
{
    return u.hi < v.hi || (u.hi == v.hi && (u.lo < v.lo || (u.lo == v.lo && u.p < v.p)));
}

__device__ __forceinline__ void vshfl_min(VBest &b)
{
    for (int o = 16; o > 0; o >>= 1) {
        VBest c;
        c.hi = __shfl_xor_sync(0xffffffffu, b.hi, o);
        c.lo = __shfl_xor_sync(0xffffffffu, b.lo, o);
        c.p = __shfl_xor_sync(0xffffffffu, b.p, o);
        if (vless(c, b)) b = c;
    }
}

__global__ void __launch_bounds__(VPROJ_THREADS) k_vproject(VoxArgs a, int whole)
{
    pdl_wait();
    pdl_release();
    __shared__ VBest s_best[VPROJ_THREADS / 32];
    const int nproj = a.ctr->nproj;
    const bool all = whole || a.ctr->orphans > 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = blockIdx.x; j < nproj; j += gridDim.x) {
        const int k = a.proj_list[j];
        const long long n = a.st_n[k], sx = a.st_sx[k], sy = a.st_sy[k], st = a.st_st[k];
        int xlo = 0, xhi = a.W - 1, ylo = 0, yhi = a.H - 1, tlo = 0, thi = a.T - 1;
        if (!all) {
            const int *pw = a.prev_win + 6 * (long long)k;
            xlo = pw[0]; xhi = pw[1]; ylo = pw[2]; yhi = pw[3]; tlo = pw[4]; thi = pw[5];
        }
        const long long w = xhi - xlo + 1, h = yhi - ylo + 1;
        const long long vol = max(0LL, w) * max(0LL, h) * max(0LL, (long long)(thi - tlo + 1));
        // voxel i of the box: row i / w, frame row / h, by reciprocals
        const RowDiv div_w(w, vol), div_h(h, w > 0 ? vol / w : 0);
        // 64-bit squared distances when 3 (n * largest dimension)^2 < 2^62
        const double bound = (double)max(a.W, max(a.H, a.T));
        const bool small = 3.0 * ((double)n * bound) * ((double)n * bound) < 4.0e18;
        VBest b = {~0ull, ~0ull, LLONG_MAX};
        constexpr int VB = 8;  // label loads issued before any comparison
        for (long long base = 0; base < vol; base += (long long)VPROJ_THREADS * VB) {
            int lab[VB];
#pragma unroll
            for (int u = 0; u < VB; ++u) {
                const long long i = base + (long long)u * VPROJ_THREADS + tid;
                lab[u] = -1;
                if (i < vol) {
                    const long long row = div_w.row(i), fr = div_h.row(row);
                    const int x = xlo + (int)(i - row * w), y = ylo + (int)(row - fr * h), t = tlo + (int)fr;
                    lab[u] = a.labels[((long long)t * a.H + y) * a.W + x];
                }
            }
#pragma unroll
            for (int u = 0; u < VB; ++u) {
                if (lab[u] != k) continue;
                const long long i = base + (long long)u * VPROJ_THREADS + tid;
                const long long row = div_w.row(i), fr = div_h.row(row);
                const int x = xlo + (int)(i - row * w), y = ylo + (int)(row - fr * h), t = tlo + (int)fr;
                const long long p = ((long long)t * a.H + y) * a.W + x;
                VBest c;
                c.p = p;
                if (small) {
                    const long long dx = n * x - sx, dy = n * y - sy, dt = n * t - st;
                    c.hi = 0;
                    c.lo = (unsigned long long)(dx * dx) + (unsigned long long)(dy * dy) +
                           (unsigned long long)(dt * dt);
                } else {
                    const __int128 dx = (__int128)n * x - sx, dy = (__int128)n * y - sy, dt = (__int128)n * t - st;
                    const unsigned __int128 d2 = (unsigned __int128)(dx * dx) + (unsigned __int128)(dy * dy) +
                                                 (unsigned __int128)(dt * dt);
                    c.hi = (unsigned long long)(d2 >> 64);
                    c.lo = (unsigned long long)d2;
                }
                if (vless(c, b)) b = c;
            }
        }
        vshfl_min(b);
        if (lane == 0) s_best[warp] = b;
        __syncthreads();
        if (warp == 0) {
            b = lane < VPROJ_THREADS / 32 ? s_best[lane] : VBest{~0ull, ~0ull, LLONG_MAX};
            vshfl_min(b);
            if (lane == 0) {
                if (b.p == LLONG_MAX) {
                    atomicExch(&a.ctr->error, ERR_BAD_LABEL);
                } else {
                    const int t = (int)(b.p / a.HW);
                    const long long q = b.p - (long long)t * a.HW;
                    const int y = (int)(q / a.W), x = (int)(q - (long long)y * a.W);
                    a.st_end[k] = make_int4(x, y, t, 0);
                    a.cdev[k].ex = x;
                    a.cdev[k].ey = y;
                    a.cdev[k].et = t;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Candidate lists: exclusive scan of the tile counts (one CTA), then one
// thread per (cluster, tile slot).
// ---------------------------------------------------------------------------
constexpr int VSCAN_THREADS = 1024;

__global__ void __launch_bounds__(VSCAN_THREADS) k_vscan(VoxArgs a)
{
    pdl_wait();
    pdl_release();
    __shared__ int s_warp[32];
    const int n = a.n_tx * a.n_ty * a.n_tt;
    cta_scan(a.tile_count, a.tile_off, n, VSCAN_THREADS, s_warp);  // (ends with a barrier)
    for (int i = threadIdx.x; i < n; i += VSCAN_THREADS) {
        a.tile_cursor[i] = 0;
        a.tile_count[i] = 0;
    }
    if (threadIdx.x == 0) {  // (tile_off[n] is this thread's own write)
        if (a.tile_off[n] > a.tile_cap) atomicExch(&a.ctr->error, ERR_TILE_LIST_OVERFLOW);
        a.ctr->nproj = 0;
        a.ctr->orphans = 0;
    }
}

__global__ void k_vfill(VoxArgs a)
{
    pdl_wait();
    pdl_release();
    const long long slots = (long long)a.tpw_x * a.tpw_y * a.tpw_t;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)a.Keff * slots) return;
    const int k = (int)(i / slots);
    int j = (int)(i - (long long)k * slots);
    const VoxCluster cd = a.cdev[k];
    if (cd.xlo > cd.xhi || cd.ylo > cd.yhi || cd.tlo > cd.thi) return;
    const int jx = j % a.tpw_x;
    j /= a.tpw_x;
    const int jy = j % a.tpw_y, jt = j / a.tpw_y;
    const int tx = cd.xlo / VTX + jx, ty = cd.ylo / VTY + jy, tt = cd.tlo / VTT + jt;
    if (tx > cd.xhi / VTX || ty > cd.yhi / VTY || tt > cd.thi / VTT) return;
    const int tile = (tt * a.n_ty + ty) * a.n_tx + tx;
    const int pos = a.tile_off[tile] + atomicAdd(&a.tile_cursor[tile], 1);
    if (pos < a.tile_cap) a.tile_list[pos] = k;
}

// ---------------------------------------------------------------------------
// Assignment: one voxel per thread, every candidate of the tile whose window
// holds it, the smallest (D, k).  The path sums follow the 3-D stepping rule
// in walk order, FP32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int vpath_sums(const float4 *__restrict__ plane, int W, long long HW, int px,
                                          int py, int pt, int ex, int ey, int et, float cL, float ca,
                                          float cb, float &sum_dc, float &sum_w)
{
    const bool p_first = px < ex || (px == ex && (py < ey || (py == ey && pt <= et)));
    const int ax = p_first ? px : ex, ay = p_first ? py : ey, at = p_first ? pt : et;
    const int dx = (p_first ? ex : px) - ax, dy = (p_first ? ey : py) - ay, dt = (p_first ? et : pt) - at;
    const int adx = abs(dx), ady = abs(dy), adt = abs(dt);
    // strides (elements) of the three axes with their signs; the major axis
    // is the first largest |delta|.  A volume holds at most 2^30 voxels, so
    // offsets and strides are 32-bit.
    const int hw = (int)HW;
    const int sxs = dx < 0 ? -1 : 1, sys = dy < 0 ? -W : W, sts = dt < 0 ? -hw : hw;
    int ns, d1, d2, smaj, s1, s2;
    if (adx >= ady && adx >= adt) { ns = adx; smaj = sxs; d1 = ady; s1 = sys; d2 = adt; s2 = sts; }
    else if (ady >= adt) { ns = ady; smaj = sys; d1 = adx; s1 = sxs; d2 = adt; s2 = sts; }
    else { ns = adt; smaj = sts; d1 = adx; s1 = sxs; d2 = ady; s2 = sys; }
    int q = at * hw + ay * W + ax;
    float dc = 0.f, w = 0.f;
    if (ns <= FIXED_STEP_MAX_NS) {
        // the fixed-point rule in closed form per minor axis: sample i lies at
        // q + i smaj + m1_i s1 + m2_i s2 with m_i the high word of
        // 2^31 + i S; four samples per group from the group's accumulators
        const uint32_t S1 = fixed_step_slope(d1, ns), S2 = fixed_step_slope(d2, ns);
        uint32_t a1 = 0x80000000u, a2 = 0x80000000u;
        const int n = ns + 1;
        const auto at = [&](int k) {
            const int m1 = k == 0 ? 0 : (int)(((unsigned long long)S1 * (unsigned)k + a1) >> 32);
            const int m2 = k == 0 ? 0 : (int)(((unsigned long long)S2 * (unsigned)k + a2) >> 32);
            return q + k * smaj + m1 * s1 + m2 * s2;
        };
        int i = 0;
#pragma unroll 1
        for (; i + 4 <= n; i += 4) {
            float4 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = __ldg(plane + at(k));
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                dc += colour_dist(v[k], cL, ca, cb);
                w += v[k].w;
            }
            const unsigned long long t1 = (unsigned long long)S1 * 4u + a1, t2 = (unsigned long long)S2 * 4u + a2;
            a1 = (uint32_t)t1;
            a2 = (uint32_t)t2;
            q += 4 * smaj + (int)(t1 >> 32) * s1 + (int)(t2 >> 32) * s2;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (i + k < n) {
                const float4 v = __ldg(plane + at(k));
                dc += colour_dist(v, cL, ca, cb);
                w += v.w;
            }
        sum_dc = dc;
        sum_w = w;
        return n;
    }
    const int two_ns = 2 * ns, two_d1 = 2 * d1, two_d2 = 2 * d2;
    int e1 = ns, e2 = ns;
#pragma unroll 4
    for (int i = 0; i <= ns; ++i) {
        const float4 v = __ldg(plane + q);
        dc += colour_dist(v, cL, ca, cb);
        w += v.w;
        e1 += two_d1;
        e2 += two_d2;
        int step = smaj;
        if (e1 >= two_ns) { e1 -= two_ns; step += s1; }
        if (e2 >= two_ns) { e2 -= two_ns; step += s2; }
        q += step;
    }
    sum_dc = dc;
    sum_w = w;
    return ns + 1;
}

// Work items: the voxels of the tile inside candidate c's window form a box
// (x fastest, then y, then t: a warp's paths then start in neighbouring
// columns, so their global-memory samples share cache lines; ordering by the
// paths' dominant axis instead was measured slower); every 32 consecutive
// voxels of it are one warp's item.  Lanes walk their voxel's path and take a 64-bit shared-memory
// atomicMin of (D bits, candidate slot); slots follow the cluster index, so
// ties go to the smallest k.  A tile with more than VITEM_CAND candidates
// evaluates voxel by voxel over the global list instead.
constexpr int VITEM_CAND = 128;
constexpr int VMAX_ITEMS = VITEM_CAND * (VTILE / 32);

__device__ __forceinline__ unsigned long long vpack_best(float D, int slot)
{
    return ((unsigned long long)__float_as_uint(D) << 32) | (unsigned)slot;  // D >= 0
}

// Rank of cluster k among the sorted candidate ids, or -1.
__device__ __forceinline__ int vfind_slot(const int *ids, int cnt, int k)
{
    int lo = 0, hi = cnt;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ids[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return lo < cnt && ids[lo] == k ? lo : -1;
}

// The pruning of the 2-D assignment, in 3-D.  Pass 1 evaluates each voxel's
// previous label (when it is a candidate of the voxel); pass 2 skips every
// other candidate whose FP32 lower bound fl(fl(lam*d_c(p)) + fl(m^2/r^2*d_s))
// exceeds the voxel's best D so far (the computed D is never below that
// bound: dcol >= fl(lam*dcp), dcon >= 1, and rounding is monotone), so the
// argmin is unchanged; the surviving pairs are queued per warp and walked 32
// at a time.
__global__ void __launch_bounds__(VTILE) k_vassign(VoxArgs a)
{
    __shared__ VoxCluster cand[VITEM_CAND];
    __shared__ int s_sorted[VITEM_CAND];   // candidate ids in slot order
    __shared__ unsigned char s_prev[VTILE];  // each voxel's previous label as a slot, 0xff if none
    __shared__ unsigned s_queue[VTILE / 32][64];
    __shared__ int4 s_box[VITEM_CAND];     // (xa, ya, ta, w | h << 8 | d << 16)
    __shared__ int2 s_rcp[VITEM_CAND];     // 16-bit reciprocals of w and h
    __shared__ int s_ids[VITEM_CAND];
    __shared__ int s_nit[VITEM_CAND];
    __shared__ int s_first[VITEM_CAND + 1];
    __shared__ unsigned char s_owner[VMAX_ITEMS];
    __shared__ unsigned long long s_best[VTILE];
    __shared__ int s_counter;
    pdl_wait();
    pdl_release();
    const int tile = blockIdx.x;
    const int tx = tile % a.n_tx, ty = (tile / a.n_tx) % a.n_ty, tt = tile / (a.n_tx * a.n_ty);
    const int x0 = tx * VTX, y0 = ty * VTY, t0 = tt * VTT;
    const int tid = threadIdx.x, lane = tid & 31;
    const int lx = tid % VTX, ly = (tid / VTX) % VTY, lt = tid / (VTX * VTY);
    const int x = x0 + lx, y = y0 + ly, t = t0 + lt;
    const bool valid = x < a.W && y < a.H && t < a.T;
    const int off = a.tile_off[tile];
    const int cnt = (int)max(0LL, min((long long)a.tile_off[tile + 1], a.tile_cap) - off);
    const bool fast = cnt <= VITEM_CAND;
    const long long p = ((long long)t * a.H + y) * a.W + x;
    unsigned my_samples = 0, my_pairs = 0;
    int lab = -1;
    const int prev = fast && valid ? a.labels[p] : -1;  // overlaps the set-up

    if (fast) {
        // candidates sorted by cluster index (ranks of distinct ids)
        int myid = INT_MAX;
        if (tid < cnt) {
            myid = a.tile_list[off + tid];
            s_ids[tid] = myid;
        }
        s_best[tid] = ~0ull;
        if (tid == 0) s_counter = 0;
        __syncthreads();
        if (tid < cnt) {
            int rank = 0;
            for (int j = 0; j < cnt; ++j) rank += s_ids[j] < myid;
            const VoxCluster cd = a.cdev[myid];
            cand[rank] = cd;
            s_sorted[rank] = myid;
            const int xa = max(cd.xlo, x0), xb = min(min(cd.xhi, x0 + VTX - 1), a.W - 1);
            const int ya = max(cd.ylo, y0), yb = min(min(cd.yhi, y0 + VTY - 1), a.H - 1);
            const int ta = max(cd.tlo, t0), tb = min(min(cd.thi, t0 + VTT - 1), a.T - 1);
            const int w = max(xb - xa + 1, 0), h = max(yb - ya + 1, 0), d = max(tb - ta + 1, 0);
            s_box[rank] = make_int4(xa, ya, ta, w | (h << 8) | (d << 16));
            s_rcp[rank] = make_int2((65536 + max(w, 1) - 1) / max(w, 1), (65536 + max(h, 1) - 1) / max(h, 1));
            s_nit[rank] = (w * h * d + 31) >> 5;
        }
        __syncthreads();
        if (tid < 32) {  // exclusive prefix of the item counts
            constexpr int PER = VITEM_CAND / 32;
            int v[PER], sum = 0;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int c = lane * PER + i;
                v[i] = c < cnt ? s_nit[c] : 0;
                sum += v[i];
            }
            int incl = sum;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            int run = incl - sum;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int c = lane * PER + i;
                if (c < cnt) s_first[c] = run;
                run += v[i];
            }
            if (lane == 31) s_first[cnt] = incl;
        }
        __syncthreads();
        if (tid < cnt) {
            const int f = s_first[tid], n = s_nit[tid];
            for (int j = 0; j < n; ++j) s_owner[f + j] = (unsigned char)tid;
        }
        // this voxel's previous label as a slot when the voxel is in that box
        int pslot = prev >= 0 ? vfind_slot(s_sorted, cnt, prev) : -1;
        if (pslot >= 0) {
            const int4 b = s_box[pslot];
            if (x < b.x || x >= b.x + (b.w & 0xff) || y < b.y || y >= b.y + ((b.w >> 8) & 0xff) || t < b.z ||
                t >= b.z + (b.w >> 16))
                pslot = -1;
        }
        s_prev[tid] = (unsigned char)(pslot >= 0 ? pslot : 0xff);
        __syncthreads();
        // D of voxel (qx, qy, qt) for candidate slot c, from its own sample
        auto own_dc = [&](int qx, int qy, int qt, const VoxCluster &cd) {
            return colour_dist(__ldg(a.plane + ((long long)qt * a.H + qy) * a.W + qx), cd.L, cd.a, cd.b);
        };
        auto vspatial = [&](int qx, int qy, int qt, const VoxCluster &cd) {
            const float ddx = (float)qx - cd.xk, ddy = (float)qy - cd.yk, ddt = (float)qt - cd.tk;
            return fmaf(ddx, ddx, fmaf(ddy, ddy, ddt * ddt));
        };
        auto evaluate = [&](int qx, int qy, int qt, int c) {
            const VoxCluster &cd = cand[c];
            float sdc, sw;
            const int len = vpath_sums(a.plane, a.W, a.HW, qx, qy, qt, cd.ex, cd.ey, cd.et, cd.L, cd.a, cd.b,
                                       sdc, sw);
            const float D = scalp_distance(own_dc(qx, qy, qt, cd), sdc, sw, len, a.lam, a.gamma, a.ms2,
                                           vspatial(qx, qy, qt, cd));
            atomicMin(&s_best[((qt - t0) * VTY + (qy - y0)) * VTX + (qx - x0)], vpack_best(D, c));
            my_samples += len;
            my_pairs += 1;
        };
        // pass 1: the previous label (no barrier before pass 2: a voxel whose
        // pass 1 is still running elsewhere is simply not pruned yet)
        if (pslot >= 0) evaluate(x, y, t, pslot);
        // pass 2: the candidates' boxes, cut into items; survivors queued
        unsigned *wq = s_queue[tid >> 5];
        const unsigned lanes_below = (1u << lane) - 1u;
        int queued = 0;
        auto walk_queued = [&](unsigned e) {
            const int v = (int)(e & (VTILE - 1)), c = (int)(e >> 9);
            evaluate(x0 + v % VTX, y0 + (v / VTX) % VTY, t0 + v / (VTX * VTY), c);
        };
        static_assert(VTILE == 512, "queued pairs are (slot << 9 | voxel)");
        const int n_items = s_first[cnt];
        while (true) {
            int item = 0;
            if (lane == 0) item = atomicAdd(&s_counter, 1);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item >= n_items) break;
            const int c = s_owner[item];
            const int4 b = s_box[c];
            const int w = b.w & 0xff, h = (b.w >> 8) & 0xff, d = b.w >> 16;
            const int j = ((item - s_first[c]) << 5) + lane;
            bool keep = false;
            int vox = 0;
            if (j < w * h * d) {
                const int2 r = s_rcp[c];
                // exact: j < 512 and w, h <= 16, so the 16-bit reciprocals give floor
                const int q = (j * r.x) >> 16;  // j / w
                const int qx = b.x + (j - q * w);
                const int qt = (q * r.y) >> 16;  // q / h
                const int qy = b.y + (q - qt * h);
                const int qtt = b.z + qt;
                vox = ((qtt - t0) * VTY + (qy - y0)) * VTX + (qx - x0);
                if (s_prev[vox] != c) {  // else evaluated in pass 1
                    const VoxCluster &cd = cand[c];
                    const float lb = __fadd_rn(__fmul_rn(a.lam, own_dc(qx, qy, qtt, cd)),
                                               __fmul_rn(a.ms2, vspatial(qx, qy, qtt, cd)));
                    // s_best holds (D bits, slot); all ones (a NaN) until a D arrives
                    keep = !(lb > __uint_as_float((unsigned)(s_best[vox] >> 32)));
                    if (!keep) {  // cannot win: not walked (counted as the method's work)
                        my_samples += max(abs(qx - cd.ex), max(abs(qy - cd.ey), abs(qtt - cd.et))) + 1;
                        my_pairs += 1;
                    }
                }
            }
            const unsigned kept = __ballot_sync(0xffffffffu, keep);
            if (keep) wq[queued + __popc(kept & lanes_below)] = ((unsigned)c << 9) | (unsigned)vox;
            queued += __popc(kept);
            __syncwarp();
            if (queued >= 32) {
                const unsigned e = wq[lane];
                __syncwarp();
                if (lane < queued - 32) wq[lane] = wq[32 + lane];
                queued -= 32;
                __syncwarp();
                walk_queued(e);
            }
        }
        if (lane < queued) walk_queued(wq[lane]);
        __syncthreads();
        if (valid) {
            const unsigned long long bb = s_best[tid];
            // slot -> cluster index (the record's pad field holds k)
            if (bb != ~0ull) lab = cand[(int)(bb & 0xffffffffu)].pad;
        }
    } else {
        const float4 own = valid ? __ldg(a.plane + p) : make_float4(0.f, 0.f, 0.f, 0.f);
        float bestD = FLT_MAX;
        int bestk = INT_MAX;
        for (int i = 0; i < cnt; ++i) {
            const int k = a.tile_list[off + i];
            const VoxCluster cd = a.cdev[k];
            if (!valid || x < cd.xlo || x > cd.xhi || y < cd.ylo || y > cd.yhi || t < cd.tlo || t > cd.thi)
                continue;
            float sdc, sw;
            const int len = vpath_sums(a.plane, a.W, a.HW, x, y, t, cd.ex, cd.ey, cd.et, cd.L, cd.a, cd.b,
                                       sdc, sw);
            const float dcp = colour_dist(own, cd.L, cd.a, cd.b);
            const float ddx = (float)x - cd.xk, ddy = (float)y - cd.yk, ddt = (float)t - cd.tk;
            const float ds = fmaf(ddx, ddx, fmaf(ddy, ddy, ddt * ddt));
            const float D = scalp_distance(dcp, sdc, sw, len, a.lam, a.gamma, a.ms2, ds);
            if (D < bestD || (D == bestD && k < bestk)) {
                bestD = D;
                bestk = k;
            }
            my_samples += len;
            my_pairs += 1;
        }
        if (bestk != INT_MAX) lab = bestk;
    }
    if (valid) {
        if (lab >= 0) {
            a.labels[p] = lab;
        } else {
            lab = a.labels[p];  // no window reaches the voxel: keep its label
            atomicAdd(&a.ctr->orphans, 1);
        }
    }
    // a warp = 32 voxels of one frame: 16 columns x 2 rows
    const float4 own = valid ? __ldg(a.plane + p) : make_float4(0.f, 0.f, 0.f, 0.f);
    const int bx = x0, by = y0 + (ly & ~1), bt = t;
    vaggregate(a, valid, lab, bx, by, bt, lx, ly & 1, 0, own);
    if (a.count_samples) {
        for (int o = 16; o > 0; o >>= 1) {
            my_samples += __shfl_down_sync(0xffffffffu, my_samples, o);
            my_pairs += __shfl_down_sync(0xffffffffu, my_pairs, o);
        }
        if (lane == 0) {
            atomicAdd(&a.ctr->samples, (unsigned long long)my_samples);
            atomicAdd(&a.ctr->pairs, (unsigned long long)my_pairs);
        }
    }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
constexpr size_t VALIGN = 256;

size_t vcarve(size_t &cur, size_t bytes)
{
    const size_t at = (cur + VALIGN - 1) & ~(VALIGN - 1);
    cur = at + bytes;
    return at;
}

struct VLayout {
    size_t rgb, contour, plane, labels, st_n, st_sx, st_sy, st_st, st_col, st_end, cdev, acc, prev_win,
        proj, tile_count, tile_off, tile_cursor, tile_list, ctr, total;
    long long tile_cap;
    int n_tx, n_ty, n_tt, tpw_x, tpw_y, tpw_t;
};

// Tiles one window can span along an axis: the window holds at most
// floor(2r) + 1 consecutive voxels (one more allowed for rounding).
int vtiles_per_window(double r, int tile)
{
    const long long len = (long long)(2.0 * r) + 2;
    return (int)((len + tile - 1) / tile + 1);
}

bool vsizes_ok(int T, int H, int W, int K)
{
    if (T < 1 || H < 1 || W < 1 || K < 1) return false;
    const long long N = (long long)T * H * W;
    if (N > (1LL << 30) || W > 65535 || H > 65535 || T > 65535) return false;
    return K <= N;
}

void vgrid(int T, int H, int W, int K, int &nx, int &ny, int &nt, double &r)
{
    const double N = (double)T * (double)H * (double)W;
    r = std::cbrt(N / (double)K);
    const int d[3] = {W, H, T};
    int g[3];
    for (int i = 0; i < 3; ++i) {
        g[i] = (int)std::floor((double)d[i] / r + 0.5);
        g[i] = std::max(1, std::min(g[i], d[i]));
    }
    nx = g[0];
    ny = g[1];
    nt = g[2];
}

VLayout vmake_layout(int T, int H, int W, int K)
{
    VLayout L{};
    const size_t N = (size_t)T * H * W;
    int nx, ny, nt;
    double r;
    vgrid(T, H, W, K, nx, ny, nt, r);
    const size_t Keff = (size_t)nx * ny * nt;
    L.n_tx = (W + VTX - 1) / VTX;
    L.n_ty = (H + VTY - 1) / VTY;
    L.n_tt = (T + VTT - 1) / VTT;
    L.tpw_x = std::min(vtiles_per_window(r, VTX), L.n_tx);
    L.tpw_y = std::min(vtiles_per_window(r, VTY), L.n_ty);
    L.tpw_t = std::min(vtiles_per_window(r, VTT), L.n_tt);
    L.tile_cap = (long long)Keff * L.tpw_x * L.tpw_y * L.tpw_t;
    const size_t n_tiles = (size_t)L.n_tx * L.n_ty * L.n_tt;
    size_t cur = 0;
    L.rgb = vcarve(cur, 3 * N);
    L.contour = vcarve(cur, 4 * N);
    L.plane = vcarve(cur, 16 * N);
    L.labels = vcarve(cur, 4 * N);
    L.st_n = vcarve(cur, 8 * Keff);
    L.st_sx = vcarve(cur, 8 * Keff);
    L.st_sy = vcarve(cur, 8 * Keff);
    L.st_st = vcarve(cur, 8 * Keff);
    L.st_col = vcarve(cur, 16 * Keff);
    L.st_end = vcarve(cur, 16 * Keff);
    L.cdev = vcarve(cur, sizeof(VoxCluster) * Keff);
    L.acc = vcarve(cur, sizeof(VoxAcc) * Keff);
    L.prev_win = vcarve(cur, 24 * Keff);
    L.proj = vcarve(cur, 4 * Keff);
    L.tile_count = vcarve(cur, 4 * n_tiles);
    L.tile_off = vcarve(cur, 4 * (n_tiles + 1));
    L.tile_cursor = vcarve(cur, 4 * n_tiles);
    L.tile_list = vcarve(cur, 4 * (size_t)L.tile_cap);
    L.ctr = vcarve(cur, sizeof(DevCounters));
    L.total = (cur + VALIGN - 1) & ~(VALIGN - 1);
    return L;
}

}  // namespace
}  // namespace scalp

using namespace scalp;

struct scalp_vctx {
    int T, H, W, K;
    long long N;
    int nx, ny, nt, Keff;
    double r, gamma;
    float m;
    cudaStream_t st;
    unsigned char *ws;
    VLayout L;
    VoxArgs a;
    int iterations;
    // profiling: an event pair around each assignment launch
    bool profiling = false;
    std::vector<cudaEvent_t> ev;
    int ev_pending = 0;  // pairs recorded and not yet read
    double prof_ms = 0.0;
    long long prof_launches = 0;
};

namespace {

thread_local std::string g_verr;

int vfail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_verr = buf;
    scalp::set_last_error(buf);
    return code;
}

int vcheck(cudaError_t e, const char *what)
{
    return e == cudaSuccess ? SCALP_OK : vfail(SCALP_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Programmatic launches (each kernel placed while the one before drains),
// except around the profiling event records.
void venqueue_lists(scalp_vctx *c)
{
    const bool pdl = !c->profiling;
    pdl_launch(pdl, k_vscan, dim3(1), dim3(VSCAN_THREADS), 0, c->st, c->a);
    const long long slots = (long long)c->Keff * c->a.tpw_x * c->a.tpw_y * c->a.tpw_t;
    pdl_launch(pdl, k_vfill, dim3((unsigned)((slots + 255) / 256)), dim3(256), 0, c->st, c->a);
}

void venqueue_update(scalp_vctx *c, int from_acc, int whole)
{
    const bool pdl = !c->profiling;
    pdl_launch(pdl, k_vupdate, dim3((c->Keff + 63) / 64), dim3(64), 0, c->st, c->a, from_acc);
    if (from_acc)
        pdl_launch(pdl, k_vproject, dim3(std::min(c->Keff, 2 * 152)), dim3(VPROJ_THREADS), 0, c->st, c->a,
                   whole);
    venqueue_lists(c);
}

// The counters go to the thread's pinned status buffer behind the stream's
// work: one asynchronous copy and one synchronisation.
int vdevice_status(scalp_vctx *c)
{
    DevCounters local;
    DevCounters *h = pinned_status_buffer();
    if (!h) h = &local;
    int rc = vcheck(cudaMemcpyAsync(h, c->a.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->st),
                    "read counters");
    if (rc) return rc;
    rc = vcheck(cudaStreamSynchronize(c->st), "synchronise");
    if (rc) return rc;
    if (h->error) return vfail(SCALP_E_INTERNAL, "device-side check failed (code %d)", h->error);
    return SCALP_OK;
}

}  // namespace

extern "C" {

size_t scalp_voxel_workspace_bytes(int32_t T, int32_t H, int32_t W, int32_t K, const scalp_params *params)
{
    (void)params;
    if (!vsizes_ok(T, H, W, K)) return 0;
    return vmake_layout(T, H, W, K).total;
}

int scalp_voxel_init(scalp_vctx **out, const scalp_volume *vol, int32_t K, float m,
                     const scalp_params *params)
{
    if (!out) return vfail(SCALP_E_ARG, "out is NULL");
    *out = nullptr;
    if (!vol || !vol->rgb || !params) return vfail(SCALP_E_ARG, "volume, volume->rgb and params are required");
    if (!vsizes_ok(vol->T, vol->H, vol->W, K)) return vfail(SCALP_E_ARG, "invalid volume size or K");
    if (!(m > 0.0f)) return vfail(SCALP_E_ARG, "m must be > 0");
    if (params->storage != SCALP_STORAGE_F32) return vfail(SCALP_E_ARG, "supervoxels take FP32 planes only");
    if (params->prior != SCALP_PRIOR_INPUT) return vfail(SCALP_E_ARG, "supervoxels take the input prior only");
    if (!(params->sigma > 0.0f) || params->lambda < 0.0f || params->lambda > 1.0f)
        return vfail(SCALP_E_ARG, "need sigma > 0 and lambda in [0, 1]");
    const size_t need = scalp_voxel_workspace_bytes(vol->T, vol->H, vol->W, K, params);
    if (!params->workspace || params->workspace_bytes < need)
        return vfail(SCALP_E_NOMEM, "supervoxel workspace of %zu bytes needed", need);
    if (reinterpret_cast<uintptr_t>(params->workspace) % VALIGN)
        return vfail(SCALP_E_ARG, "workspace must be 256-byte aligned");
    scalp_vctx *c = new (std::nothrow) scalp_vctx();
    if (!c) return vfail(SCALP_E_NOMEM, "host allocation failed");
    c->T = vol->T; c->H = vol->H; c->W = vol->W; c->K = K; c->m = m;
    c->N = (long long)vol->T * vol->H * vol->W;
    vgrid(c->T, c->H, c->W, K, c->nx, c->ny, c->nt, c->r);
    c->Keff = c->nx * c->ny * c->nt;
    c->gamma = params->gamma < 0.0f ? 2.0 * c->r : (double)params->gamma;
    c->st = reinterpret_cast<cudaStream_t>(params->stream);
    c->ws = reinterpret_cast<unsigned char *>(params->workspace);
    c->L = vmake_layout(c->T, c->H, c->W, K);
    const VLayout &L = c->L;
    VoxArgs &a = c->a;
    a = VoxArgs{};
    a.T = c->T; a.H = c->H; a.W = c->W; a.K = K; a.Keff = c->Keff;
    a.nx = c->nx; a.ny = c->ny; a.nt = c->nt;
    a.N = c->N; a.HW = (long long)c->H * c->W;
    a.r = c->r;
    a.lam = params->lambda;
    a.gamma = (float)c->gamma;
    a.ms2 = (float)((double)m * (double)m / (c->r * c->r));
    a.n_tx = L.n_tx; a.n_ty = L.n_ty; a.n_tt = L.n_tt;
    a.tpw_x = L.tpw_x; a.tpw_y = L.tpw_y; a.tpw_t = L.tpw_t;
    a.tile_cap = L.tile_cap;
    a.plane = reinterpret_cast<const float4 *>(c->ws + L.plane);
    a.labels = reinterpret_cast<int *>(c->ws + L.labels);
    a.st_n = reinterpret_cast<long long *>(c->ws + L.st_n);
    a.st_sx = reinterpret_cast<long long *>(c->ws + L.st_sx);
    a.st_sy = reinterpret_cast<long long *>(c->ws + L.st_sy);
    a.st_st = reinterpret_cast<long long *>(c->ws + L.st_st);
    a.st_col = reinterpret_cast<float4 *>(c->ws + L.st_col);
    a.st_end = reinterpret_cast<int4 *>(c->ws + L.st_end);
    a.cdev = reinterpret_cast<VoxCluster *>(c->ws + L.cdev);
    a.acc = reinterpret_cast<VoxAcc *>(c->ws + L.acc);
    a.prev_win = reinterpret_cast<int *>(c->ws + L.prev_win);
    a.proj_list = reinterpret_cast<int *>(c->ws + L.proj);
    a.tile_count = reinterpret_cast<int *>(c->ws + L.tile_count);
    a.tile_off = reinterpret_cast<int *>(c->ws + L.tile_off);
    a.tile_cursor = reinterpret_cast<int *>(c->ws + L.tile_cursor);
    a.tile_list = reinterpret_cast<int *>(c->ws + L.tile_list);
    a.ctr = reinterpret_cast<DevCounters *>(c->ws + L.ctr);
    const uint8_t *rgb = vol->rgb;
    const float *con = vol->contour;
    const size_t N = (size_t)c->N;
    int rc = SCALP_OK;
    if (!vol->on_device) {
        rc = vcheck(cudaMemcpyAsync(c->ws + L.rgb, rgb, 3 * N, cudaMemcpyHostToDevice, c->st), "copy volume");
        rgb = c->ws + L.rgb;
        if (!rc && con) {
            rc = vcheck(cudaMemcpyAsync(c->ws + L.contour, con, 4 * N, cudaMemcpyHostToDevice, c->st),
                        "copy contour");
            con = reinterpret_cast<const float *>(c->ws + L.contour);
        }
    }
    const size_t n_tiles = (size_t)L.n_tx * L.n_ty * L.n_tt;
    if (!rc) rc = vcheck(cudaMemsetAsync(a.acc, 0, sizeof(VoxAcc) * c->Keff, c->st), "memset");
    if (!rc) rc = vcheck(cudaMemsetAsync(a.tile_count, 0, 4 * n_tiles, c->st), "memset");
    if (!rc) rc = vcheck(cudaMemsetAsync(a.cdev, 0, sizeof(VoxCluster) * c->Keff, c->st), "memset");
    if (!rc) rc = vcheck(cudaMemsetAsync(a.ctr, 0, sizeof(DevCounters), c->st), "memset");
    if (!rc) rc = vcheck(srgb_table(&a.lut, c->st), "transfer-function table");
    if (rc) {
        delete c;
        return rc;
    }
    k_vsetup<<<152 * 8, 256, 0, c->st>>>(a, rgb, con, params->sigma, reinterpret_cast<float4 *>(c->ws + L.plane));
    venqueue_update(c, 1, 1);
    rc = vcheck(cudaGetLastError(), "initialisation kernels");
    if (!rc) rc = vcheck(cudaStreamSynchronize(c->st), "initialisation");  // host staging is released
    if (rc) {
        delete c;
        return rc;
    }
    c->iterations = 0;
    *out = c;
    return SCALP_OK;
}

int scalp_voxel_iterate(scalp_vctx *c, int32_t n)
{
    if (!c || n < 0) return vfail(SCALP_E_ARG, "ctx is NULL or n < 0");
    for (int i = 0; i < n; ++i) {
        const unsigned tiles = (unsigned)(c->a.n_tx * c->a.n_ty * c->a.n_tt);
        const bool prof = c->profiling;
        if (prof) {
            while ((int)c->ev.size() < 2 * (c->ev_pending + 1)) {
                cudaEvent_t e;
                const int rc = vcheck(cudaEventCreate(&e), "profiling event");
                if (rc) return rc;
                c->ev.push_back(e);
            }
            cudaEventRecord(c->ev[2 * c->ev_pending], c->st);
        }
        pdl_launch(!prof, k_vassign, dim3(tiles), dim3(VTILE), 0, c->st, c->a);
        if (prof) cudaEventRecord(c->ev[2 * c->ev_pending++ + 1], c->st);
        venqueue_update(c, 1, 0);
        ++c->iterations;
    }
    return vcheck(cudaGetLastError(), "iteration kernels");
}

int scalp_voxel_labels(scalp_vctx *c, int32_t *out, int32_t out_on_device)
{
    if (!c || !out) return vfail(SCALP_E_ARG, "ctx or out is NULL");
    int rc = vcheck(cudaMemcpyAsync(out, c->a.labels, 4 * (size_t)c->N,
                                    out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st),
                    "copy labels");
    return rc ? rc : vdevice_status(c);
}

int scalp_voxel_get_info(const scalp_vctx *c, scalp_voxel_info *info)
{
    if (!c || !info) return vfail(SCALP_E_ARG, "ctx or info is NULL");
    info->T = c->T; info->H = c->H; info->W = c->W; info->K = c->K;
    info->nx = c->nx; info->ny = c->ny; info->nt = c->nt; info->Keff = c->Keff;
    info->r = c->r; info->gamma = c->gamma;
    info->iterations = c->iterations;
    return SCALP_OK;
}

int scalp_voxel_get_state(scalp_vctx *c, const scalp_voxel_state *s)
{
    if (!c || !s || !s->labels || !s->n || !s->sx || !s->sy || !s->st || !s->color || !s->endpoint)
        return vfail(SCALP_E_ARG, "ctx and every state array are required");
    const size_t K = (size_t)c->Keff;
    std::vector<float4> col(K);
    std::vector<int4> end(K);
    int rc = vcheck(cudaStreamSynchronize(c->st), "synchronise");
    if (!rc) rc = vcheck(cudaMemcpy(s->labels, c->a.labels, 4 * (size_t)c->N, cudaMemcpyDeviceToHost), "copy");
    if (!rc) rc = vcheck(cudaMemcpy(s->n, c->a.st_n, 8 * K, cudaMemcpyDeviceToHost), "copy");
    if (!rc) rc = vcheck(cudaMemcpy(s->sx, c->a.st_sx, 8 * K, cudaMemcpyDeviceToHost), "copy");
    if (!rc) rc = vcheck(cudaMemcpy(s->sy, c->a.st_sy, 8 * K, cudaMemcpyDeviceToHost), "copy");
    if (!rc) rc = vcheck(cudaMemcpy(s->st, c->a.st_st, 8 * K, cudaMemcpyDeviceToHost), "copy");
    if (!rc) rc = vcheck(cudaMemcpy(col.data(), c->a.st_col, 16 * K, cudaMemcpyDeviceToHost), "copy");
    if (!rc) rc = vcheck(cudaMemcpy(end.data(), c->a.st_end, 16 * K, cudaMemcpyDeviceToHost), "copy");
    if (rc) return rc;
    for (size_t k = 0; k < K; ++k) {
        s->color[3 * k] = col[k].x;
        s->color[3 * k + 1] = col[k].y;
        s->color[3 * k + 2] = col[k].z;
        s->endpoint[3 * k] = end[k].x;
        s->endpoint[3 * k + 1] = end[k].y;
        s->endpoint[3 * k + 2] = end[k].z;
    }
    return vdevice_status(c);
}

int scalp_voxel_set_state(scalp_vctx *c, const scalp_voxel_state *s)
{
    if (!c || !s || !s->labels || !s->n || !s->sx || !s->sy || !s->st || !s->color || !s->endpoint)
        return vfail(SCALP_E_ARG, "ctx and every state array are required");
    const size_t K = (size_t)c->Keff;
    for (size_t k = 0; k < K; ++k) {
        if (s->n[k] < 1 || s->n[k] > (1LL << 30))
            return vfail(SCALP_E_ARG, "cluster %zu has n outside [1, 2^30]", k);
        const long long n = s->n[k];
        if (s->sx[k] < 0 || s->sx[k] > n * (c->W - 1) || s->sy[k] < 0 || s->sy[k] > n * (c->H - 1) ||
            s->st[k] < 0 || s->st[k] > n * (c->T - 1))
            return vfail(SCALP_E_ARG, "barycenter of cluster %zu is outside the volume", k);
        const int32_t *e = s->endpoint + 3 * k;
        if (e[0] < 0 || e[0] >= c->W || e[1] < 0 || e[1] >= c->H || e[2] < 0 || e[2] >= c->T)
            return vfail(SCALP_E_ARG, "endpoint of cluster %zu is outside the volume", k);
    }
    for (long long p = 0; p < c->N; ++p)
        if (s->labels[p] < 0 || s->labels[p] >= c->Keff) return vfail(SCALP_E_ARG, "label out of range");
    std::vector<float4> col(K);
    std::vector<int4> end(K);
    for (size_t k = 0; k < K; ++k) {
        col[k] = make_float4((float)s->color[3 * k], (float)s->color[3 * k + 1], (float)s->color[3 * k + 2], 0.f);
        end[k] = make_int4(s->endpoint[3 * k], s->endpoint[3 * k + 1], s->endpoint[3 * k + 2], 0);
    }
    const size_t n_tiles = (size_t)c->L.n_tx * c->L.n_ty * c->L.n_tt;
    int rc = vcheck(cudaStreamSynchronize(c->st), "synchronise");
    if (!rc) rc = vcheck(cudaMemcpy(c->a.labels, s->labels, 4 * (size_t)c->N, cudaMemcpyHostToDevice), "copy");
    if (!rc) rc = vcheck(cudaMemcpy(c->a.st_n, s->n, 8 * K, cudaMemcpyHostToDevice), "copy");
    if (!rc) rc = vcheck(cudaMemcpy(c->a.st_sx, s->sx, 8 * K, cudaMemcpyHostToDevice), "copy");
    if (!rc) rc = vcheck(cudaMemcpy(c->a.st_sy, s->sy, 8 * K, cudaMemcpyHostToDevice), "copy");
    if (!rc) rc = vcheck(cudaMemcpy(c->a.st_st, s->st, 8 * K, cudaMemcpyHostToDevice), "copy");
    if (!rc) rc = vcheck(cudaMemcpy(c->a.st_col, col.data(), 16 * K, cudaMemcpyHostToDevice), "copy");
    if (!rc) rc = vcheck(cudaMemcpy(c->a.st_end, end.data(), 16 * K, cudaMemcpyHostToDevice), "copy");
    if (!rc) rc = vcheck(cudaMemset(c->a.acc, 0, sizeof(VoxAcc) * K), "memset");
    if (!rc) rc = vcheck(cudaMemset(c->a.tile_count, 0, 4 * n_tiles), "memset");
    if (rc) return rc;
    venqueue_update(c, 0, 0);
    rc = vcheck(cudaGetLastError(), "derive kernels");
    return rc ? rc : vdevice_status(c);
}

int scalp_voxel_count_samples(scalp_vctx *c, int32_t enable, int64_t *samples, int64_t *pairs)
{
    if (!c) return vfail(SCALP_E_ARG, "ctx is NULL");
    int rc = vcheck(cudaStreamSynchronize(c->st), "synchronise");
    DevCounters h;
    if (!rc) rc = vcheck(cudaMemcpy(&h, c->a.ctr, sizeof h, cudaMemcpyDeviceToHost), "read counters");
    if (rc) return rc;
    if (samples) *samples = (int64_t)h.samples;
    if (pairs) *pairs = (int64_t)h.pairs;
    if (enable >= 0) {
        if (enable) {
            unsigned long long z[2] = {0, 0};
            rc = vcheck(cudaMemcpy(&c->a.ctr->samples, z, sizeof z, cudaMemcpyHostToDevice), "reset counters");
            if (rc) return rc;
        }
        c->a.count_samples = enable != 0;
    }
    return SCALP_OK;
}

int scalp_voxel_profile(scalp_vctx *c, int32_t enable, double *ms, int64_t *launches)
{
    if (!c) return vfail(SCALP_E_ARG, "ctx is NULL");
    if (c->ev_pending) {
        const int rc = vcheck(cudaStreamSynchronize(c->st), "synchronise");
        if (rc) return rc;
        for (int i = 0; i < c->ev_pending; ++i) {
            float t = 0.f;
            const int r2 = vcheck(cudaEventElapsedTime(&t, c->ev[2 * i], c->ev[2 * i + 1]), "event time");
            if (r2) return r2;
            c->prof_ms += t;
            c->prof_launches += 1;
        }
        c->ev_pending = 0;
    }
    if (ms) *ms = c->prof_ms;
    if (launches) *launches = c->prof_launches;
    if (enable >= 0) {
        if (enable) {
            c->prof_ms = 0.0;
            c->prof_launches = 0;
        }
        c->profiling = enable != 0;
    }
    return SCALP_OK;
}

void scalp_voxel_destroy(scalp_vctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->st);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    delete c;
}

}  // extern "C"
