// scalp_phases.cuh -- the device bodies of one iteration's cluster update,
// projection (Eq. 4) and candidate lists, shared by the per-kernel launches
// (scalp_kernels.cu) and the persistent batched kernel (scalp_persistent.cu).
#pragma once

#include <cfloat>
#include <climits>

#include "scalp_internal.cuh"

namespace scalp {

// ---------------------------------------------------------------------------
// Windows.  Pixel p is a candidate of cluster k iff |x_p - x_k| <= r and
// |y_p - y_k| <= r (the (2r+1)x(2r+1) window of Algorithm 1), i.e.
// K*(n*x_p - Sx)^2 <= N*n^2 and likewise for y, evaluated exactly; each
// window becomes an inclusive integer range clipped to the image.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool in_window(long long v, long long n, long long s, long long N,
                                          long long K)
{
    __int128 d = (__int128)n * v - s;
    unsigned __int128 lhs = (unsigned __int128)K * (unsigned __int128)(d * d);
    unsigned __int128 rhs = (unsigned __int128)N * (unsigned __int128)n * (unsigned __int128)n;
    return lhs <= rhs;
}

__device__ inline bool window_range(long long n, long long s, long long N, long long K, double r,
                             int limit, int &lo, int &hi)
{
    long long l, h;
    window_start(s, n, r, limit, l, h);
    int guard = 0;
    while (!in_window(l, n, s, N, K) && guard++ < 64) ++l;
    guard = 0;
    while (!in_window(h, n, s, N, K) && guard++ < 64) --h;
    if (!in_window(l, n, s, N, K) || !in_window(h, n, s, N, K)) return false;
    lo = (int)max(0LL, l);
    hi = (int)min((long long)limit - 1, h);
    return true;
}

// ---------------------------------------------------------------------------
// Projection, Eq. 4: X_k^* = argmin over p in S_k of ||X_p - X_k||, compared
// exactly as (n*x - Sx)^2 + (n*y - Sy)^2 in integers (64-bit when the image
// size bounds them below 2^62, else 128-bit), ties to the smallest raster
// index.  Searches issue PROJ_BATCH label loads per thread before comparing
// them.
// ---------------------------------------------------------------------------
constexpr int PROJ_THREADS = 512;
constexpr int PROJ_BATCH = 8;

struct ProjBest {
    unsigned long long hi, lo;
    long long p;
};

__device__ __forceinline__ bool proj_less(const ProjBest &u, const ProjBest &v)
{
    return u.hi < v.hi || (u.hi == v.hi && (u.lo < v.lo || (u.lo == v.lo && u.p < v.p)));
}

__device__ __forceinline__ void proj_shfl_min(ProjBest &b)
{
    for (int o = 16; o > 0; o >>= 1) {
        ProjBest c;
        c.hi = __shfl_xor_sync(0xffffffffu, b.hi, o);
        c.lo = __shfl_xor_sync(0xffffffffu, b.lo, o);
        c.p = __shfl_xor_sync(0xffffffffu, b.p, o);
        if (proj_less(c, b)) b = c;
    }
}



// Candidate p (raster index, pixel (x, y)) for X_k^* of cluster (n, sx, sy).
__device__ __forceinline__ ProjBest proj_candidate(long long p, int x, int y, long long n,
                                                   long long sx, long long sy, bool small)
{
    ProjBest c;
    c.p = p;
    if (small) {
        const long long dx = n * x - sx, dy = n * y - sy;
        c.hi = 0;
        c.lo = (unsigned long long)(dx * dx) + (unsigned long long)(dy * dy);
    } else {
        const __int128 dx = (__int128)n * x - sx, dy = (__int128)n * y - sy;
        const unsigned __int128 d2 = (unsigned __int128)(dx * dx) + (unsigned __int128)(dy * dy);
        c.hi = (unsigned long long)(d2 >> 64);
        c.lo = (unsigned long long)d2;
    }
    return c;
}

// ---------------------------------------------------------------------------
// Cluster update (Algorithm 1) and everything derived from it, one thread per
// cluster.  With from_acc: the means over S_k from the integer sums (an empty
// cluster keeps its colour, barycenter and endpoint), the endpoint X_k rounded
// half-up, and a projection request (Eq. 4) when the pixel there is not
// labelled k; the sums are cleared for the next assignment.  Then, from the
// state: the window, the cluster record the assignment reads, and the count
// of each tile the window overlaps (for the candidate lists).  The window the
// last assignment used is kept for the projection search.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void update_cluster(const SolveArgs &a, int k, int from_acc)
{
    // every load that does not depend on another is issued first: the
    // previous window, the state (kept when the cluster received no pixel)
    // and the sums; the new state then stays in registers
    const ClusterDev old = a.cdev[k];
    long long n = a.st_n[k], sx = a.st_sx[k], sy = a.st_sy[k];
    float4 col = a.st_col[k];
    int2 e = a.st_end[k];
    bool check_projection = false;
    int label_at_end = k;
    if (from_acc && k == 0) {
        // the orphans of the assignment just finished decide the projection's
        // region; the count starts again for the next assignment
        a.ctr->proj_all = atomicExch(&a.ctr->orphans, 0) > 0;
    }
    if (from_acc) {
        const ClusterAcc c = a.acc[k];
        a.acc[k] = ClusterAcc{};
        if (c.n > 0) {
            n = (long long)c.n;
            sx = (long long)c.sx;
            sy = (long long)c.sy;
            a.st_n[k] = n;
            a.st_sx[k] = sx;
            a.st_sy[k] = sy;
            const double den = (double)n * (double)(1 << COLOR_FRAC_BITS);
            col = make_float4((float)((double)(long long)c.sL / den), (float)((double)(long long)c.sa / den),
                              (float)((double)(long long)c.sb / den), 0.f);
            a.st_col[k] = col;
            e = make_int2((int)((2 * sx + n) / (2 * n)), (int)((2 * sy + n) / (2 * n)));
            a.st_end[k] = e;
            // Eq. 4 is needed when the endpoint's pixel is not in S_k; the
            // label is read now and used last
            label_at_end = a.labels[(long long)e.y * a.W + e.x];
            check_projection = true;
        }
    }
    a.prev_win[k] = make_int4(old.xlo, old.xhi, old.ylo, old.yhi);
    ClusterDev cd;
    cd.L = col.x; cd.a = col.y; cd.b = col.z;
    cd.xk = (float)((double)sx / (double)n);
    cd.yk = (float)((double)sy / (double)n);
    cd.ex = e.x; cd.ey = e.y;
    cd.pad = k;
    const bool ok = window_range(n, sx, a.N, a.K, a.r, a.W, cd.xlo, cd.xhi) &&
                    window_range(n, sy, a.N, a.K, a.r, a.H, cd.ylo, cd.yhi);
    if (!ok) {
        atomicExch(&a.ctr->error, ERR_BAD_LABEL);
        cd.xlo = 1; cd.xhi = 0; cd.ylo = 1; cd.yhi = 0;
    }
    a.cdev[k] = cd;
    if (ok) {
        for (int ty = cd.ylo / TILE_Y; ty <= cd.yhi / TILE_Y; ++ty)
            for (int tx = cd.xlo / TILE_X; tx <= cd.xhi / TILE_X; ++tx)
                atomicAdd(&a.tile_count[ty * a.n_tx + tx], 1);
    }
    if (check_projection && label_at_end != k) {
        const int slot = atomicAdd(&a.ctr->nproj, 1);
        a.proj_list[slot] = k;
    }
}

// Eq. 4 for queued cluster j of one image by one warp, over the window the
// last assignment used (which holds S_k): the same argmin, with the same
// exact comparison and tie rule, as the CTA-wide search.
__device__ __forceinline__ void project_warp(const SolveArgs &a, int j)
{
    constexpr int BATCH = 4;
    const int lane = threadIdx.x & 31;
    const int k = a.proj_list[j];
    const long long n = a.st_n[k], sx = a.st_sx[k], sy = a.st_sy[k];
    const int4 w4 = a.prev_win[k];
    const int xlo = w4.x, ylo = w4.z;
    const int w = w4.y - w4.x + 1;
    const long long area = (long long)w * (w4.w - w4.z + 1);
    const RowDiv div(w, area);
    const double bound = (double)max(a.W, a.H);
    const bool small = 2.0 * (n * bound) * (n * bound) < 4.0e18;
    ProjBest b = {~0ull, ~0ull, LLONG_MAX};
    for (long long base = 0; base < area; base += 32 * BATCH) {
        int lab[BATCH];
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const long long i = base + u * 32 + lane;
            lab[u] = -1;
            if (i < area) {
                const long long r = div.row(i);
                lab[u] = a.labels[(long long)(ylo + (int)r) * a.W + xlo + (int)(i - r * w)];
            }
        }
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            if (lab[u] != k) continue;
            const long long i = base + u * 32 + lane;
            const long long r = div.row(i);
            const int y = ylo + (int)r, x = xlo + (int)(i - r * w);
            const ProjBest c = proj_candidate((long long)y * a.W + x, x, y, n, sx, sy, small);
            if (proj_less(c, b)) b = c;
        }
    }
    proj_shfl_min(b);
    if (lane == 0) {
        if (b.p == LLONG_MAX) {
            atomicExch(&a.ctr->error, ERR_BAD_LABEL);
        } else {
            const int ex = (int)(b.p % a.W), ey = (int)(b.p / a.W);
            a.st_end[k] = make_int2(ex, ey);
            a.cdev[k].ex = ex;
            a.cdev[k].ey = ey;
        }
    }
}

// Queued projections: S_k lies inside the window the last assignment used for
// cluster k, unless some pixel kept its old label for lack of any candidate;
// then (or with whole_image, at set-up) the whole image is searched.  One CTA
// per queued cluster.  Queue entries j0, j0 + stride, ... of one image.
__device__ __forceinline__ void project_cta(const SolveArgs &a, int whole_image, int j0, int stride)
{
    __shared__ ProjBest s_best[PROJ_THREADS / 32];
    const int nproj = a.ctr->nproj;
    const bool all = whole_image || a.ctr->proj_all;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double bound = (double)max(a.W, a.H);
    // (the step cannot overflow: a stride past the queue's end ends the loop)
    for (int j = j0; j < nproj; j = stride < nproj - j ? j + stride : nproj) {
        const int k = a.proj_list[j];
        const long long n = a.st_n[k], sx = a.st_sx[k], sy = a.st_sy[k];
        int xlo = 0, xhi = a.W - 1, ylo = 0, yhi = a.H - 1;
        if (!all) {
            const int4 w4 = a.prev_win[k];
            xlo = w4.x; xhi = w4.y; ylo = w4.z; yhi = w4.w;
        }
        const int w = xhi - xlo + 1;
        const long long area = (long long)w * (yhi - ylo + 1);
        const RowDiv div(w, area);
        const bool small = 2.0 * (n * bound) * (n * bound) < 4.0e18;
        ProjBest b = {~0ull, ~0ull, LLONG_MAX};
        for (long long base = 0; base < area; base += (long long)PROJ_THREADS * PROJ_BATCH) {
            int lab[PROJ_BATCH];
            long long idx[PROJ_BATCH];
#pragma unroll
            for (int u = 0; u < PROJ_BATCH; ++u) {
                const long long i = base + (long long)u * PROJ_THREADS + tid;
                lab[u] = -1;
                idx[u] = -1;
                if (i < area) {
                    const long long r = div.row(i);
                    const int y = ylo + (int)r, x = xlo + (int)(i - r * w);
                    idx[u] = (long long)y * a.W + x;
                    lab[u] = a.labels[idx[u]];
                }
            }
#pragma unroll
            for (int u = 0; u < PROJ_BATCH; ++u) {
                if (lab[u] != k) continue;
                const long long p = idx[u];
                const long long r = div.row(base + (long long)u * PROJ_THREADS + tid);
                const int y = ylo + (int)r, x = xlo + (int)(base + (long long)u * PROJ_THREADS + tid - r * w);
                const ProjBest c = proj_candidate(p, x, y, n, sx, sy, small);
                if (proj_less(c, b)) b = c;
            }
        }
        proj_shfl_min(b);
        if (lane == 0) s_best[warp] = b;
        __syncthreads();
        if (warp == 0) {
            b = lane < PROJ_THREADS / 32 ? s_best[lane] : ProjBest{~0ull, ~0ull, LLONG_MAX};
            proj_shfl_min(b);
            if (lane == 0) {
                if (b.p == LLONG_MAX) {
                    atomicExch(&a.ctr->error, ERR_BAD_LABEL);
                } else {
                    const int ex = (int)(b.p % a.W), ey = (int)(b.p / a.W);
                    a.st_end[k] = make_int2(ex, ey);
                    a.cdev[k].ex = ex;
                    a.cdev[k].ey = ey;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Per-tile candidate lists: exclusive scan of the tile counts, then one thread
// per (cluster, tile) slot files the cluster into each tile its window
// overlaps, at tile_off[t] + (a per-tile cursor).  The assignment CTA of tile
// t zeroes tile_count[t] and tile_cursor[t] once it has read its list (set-up
// and set_state zero them on the host side).  The lists touch no other
// counter, so they can run beside the projection: the update restarts the
// orphan count and the assignment the projection queue.
// ---------------------------------------------------------------------------

// tile_off from the counts and the overflow check.
__device__ __forceinline__ void publish_offsets(const SolveArgs &a, const int *off)
{
    const int n = a.n_tx * a.n_ty;
    for (int i = threadIdx.x; i <= n; i += blockDim.x) a.tile_off[i] = off[i];
    if (threadIdx.x == 0 && off[n] > a.tile_cap) atomicExch(&a.ctr->error, ERR_TILE_LIST_OVERFLOW);
}

constexpr int SCAN1_THREADS = 1024;

// tile_off of one image by one CTA of THREADS threads.
template <int THREADS = SCAN1_THREADS>
__device__ __forceinline__ void scan_tiles_cta(const SolveArgs &a)
{
    __shared__ int s_warp[32];
    cta_scan(a.tile_count, a.tile_off, a.n_tx * a.n_ty, THREADS, s_warp);
    if (threadIdx.x == 0) {
        const int n = a.n_tx * a.n_ty;
        if (a.tile_off[n] > a.tile_cap) atomicExch(&a.ctr->error, ERR_TILE_LIST_OVERFLOW);
    }
}

__device__ __forceinline__ void fill_slot(const SolveArgs &a, long long i)
{
    const long long slots = (long long)a.tpw_x * a.tpw_y;
    if (i >= (long long)a.Keff * slots) return;
    const int k = (int)(i / slots), j = (int)(i % slots);
    const ClusterDev cd = a.cdev[k];
    if (cd.xlo > cd.xhi) return;
    const int tx = cd.xlo / TILE_X + j % a.tpw_x, ty = cd.ylo / TILE_Y + j / a.tpw_x;
    if (tx > cd.xhi / TILE_X || ty > cd.yhi / TILE_Y) return;
    const int t = ty * a.n_tx + tx;
    const int pos = a.tile_off[t] + atomicAdd(&a.tile_cursor[t], 1);
    if (pos < a.tile_cap) a.tile_list[pos] = k;
}

}  // namespace scalp
