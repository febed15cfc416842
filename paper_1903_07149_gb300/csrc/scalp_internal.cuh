// scalp_internal.cuh -- device data layout and helpers shared by the libscalp
// kernels (never by the CPU oracle).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace scalp {

// Assignment tile: a CTA labels TILE_X x TILE_Y pixels.  For the reduction a
// warp takes 8 x 4 blocks of them (one pixel per lane), so the labels a warp
// sums are spatially coherent.
constexpr int TILE_X = 32;
constexpr int TILE_Y = 32;
constexpr int TILE_PIXELS = TILE_X * TILE_Y;
constexpr int WARP_BLOCK_X = 8;
constexpr int WARP_BLOCK_Y = 4;
// Candidate clusters of one tile held in shared memory.  A tile with more
// candidates (never seen on the regular grid) takes a slower per-pixel path.
constexpr int MAX_TILE_CANDIDATES = 128;
// Assignment CTAs: 512 threads, two per SM (one CTA's set-up, map building
// and tail overlap the other's path walks).
constexpr int ASSIGN_THREADS = 512;
constexpr int ASSIGN_CTAS_PER_SM = 2;
// Colour sums are kept as integers: value * 2^COLOR_FRAC_BITS, rounded.  CIELab
// of 8-bit sRGB has |L|, |a|, |b| < 108, so 32 such values sum below 2^31.
constexpr int COLOR_FRAC_BITS = 19;

// sRGB -> CIELab (Sec. II-A): the sRGB inverse transfer function (a 256-entry
// table `lin`), the D65 sRGB->XYZ matrix, normalisation by the XYZ of sRGB
// white (the matrix row sums), then CIE 1976 companding with the linear
// segment below (6/29)^3.
__host__ __device__ constexpr float rgb2xyz(int i)
{
    constexpr float m[9] = {0.4124564f, 0.3575761f, 0.1804375f,
                            0.2126729f, 0.7151522f, 0.0721750f,
                            0.0193339f, 0.1191920f, 0.9503041f};
    return m[i];
}

// Cube root on [(6/29)^3, 1], the range the companding takes it on (a
// normalised XYZ value is at most 1 up to rounding).  Newton-Raphson on the
// reciprocal cube root, y <- y (4 - t y^3) / 3, which needs no division,
// from a start that divides the float's bit pattern by three (the pattern
// is a piecewise-linear log2); 0x54A232A0 minimises the start's largest
// relative error over the range (3.4%).  Two steps, then c = t y^2 corrected
// once by (t - c^3) y^2 / 3, leave less than one ulp against the exact root
// (0.75 ulp at most over the floats of the range in an FP32 emulation).
__device__ __forceinline__ float cube_root(float t)
{
    const float third = 1.0f / 3.0f;
    float y = __uint_as_float(0x54A232A0u - __float_as_uint(t) / 3u);
#pragma unroll
    for (int i = 0; i < 2; ++i) y = (y * fmaf(-t, (y * y) * y, 4.0f)) * third;
    const float y2 = y * y;
    const float c = t * y2;
    return fmaf(fmaf(-c, c * c, t), y2 * third, c);
}

__device__ __forceinline__ float lab_f(float t)
{
    const float d3 = (6.0f / 29.0f) * (6.0f / 29.0f) * (6.0f / 29.0f);
    return t > d3 ? cube_root(t) : t * (841.0f / 108.0f) + (4.0f / 29.0f);
}

// CIELab of one sRGB pixel; lin = the 256-entry inverse transfer function.
// Each matrix row is divided by its sum at compile time, so the products are
// the normalised X/Xw, Y/Yw, Z/Zw.
__device__ __forceinline__ float3 srgb_to_lab(const float *lin, const uint8_t *px)
{
    constexpr float wx = rgb2xyz(0) + rgb2xyz(1) + rgb2xyz(2);
    constexpr float wy = rgb2xyz(3) + rgb2xyz(4) + rgb2xyz(5);
    constexpr float wz = rgb2xyz(6) + rgb2xyz(7) + rgb2xyz(8);
    const float R = lin[px[0]], G = lin[px[1]], B = lin[px[2]];
    const float tx = (rgb2xyz(0) / wx) * R + (rgb2xyz(1) / wx) * G + (rgb2xyz(2) / wx) * B;
    const float ty = (rgb2xyz(3) / wy) * R + (rgb2xyz(4) / wy) * G + (rgb2xyz(5) / wy) * B;
    const float tz = (rgb2xyz(6) / wz) * R + (rgb2xyz(7) / wz) * G + (rgb2xyz(8) / wz) * B;
    const float fx = lab_f(tx), fy = lab_f(ty), fz = lab_f(tz);
    return make_float3(116.0f * fy - 16.0f, 500.0f * (fx - fy), 200.0f * (fy - fz));
}

// Exclusive scan of in[0, n) into out[0, n] (out[n] = total) by one CTA of
// `threads` threads (a multiple of 32, at most 1024).  Each warp scans a
// contiguous segment 32 consecutive entries at a time (coalesced loads,
// conflict-free stores), carrying its running sum; the warps' totals are
// then scanned and each warp adds its offset.  s_warp holds 32 ints.
__device__ __forceinline__ void cta_scan(const int *in, int *out, int n, int threads, int *s_warp)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = threads / 32;
    const int seg = (n + nw - 1) / nw;
    const int b = min(n, wid * seg), e = min(n, b + seg);
    int carry = 0;
#pragma unroll 4
    for (int base = b; base < e; base += 32) {
        const int i = base + lane;
        const int v = i < e ? in[i] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        if (i < e) out[i] = carry + incl - v;
        carry += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0) s_warp[wid] = carry;
    __syncthreads();
    if (wid == 0) {  // inclusive scan of the warp totals
        int w = lane < nw ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += t;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const int off = wid ? s_warp[wid - 1] : 0;
    if (off)
        for (int i = b + lane; i < e; i += 32) out[i] += off;  // (each entry its own lane's)
    if (threadIdx.x == 0) out[n] = s_warp[31];
    __syncthreads();
}

// Row of index i in rows of w pixels: i / w by a 32-bit reciprocal
// (rcp = ceil(2^32 / w), exact while i * w < 2^32; the caller checks), else by
// a 64-bit division.
struct RowDiv {
    long long w;
    unsigned rcp;
    bool fast;
    __device__ __forceinline__ RowDiv(long long w_, long long area) : w(w_)
    {
        fast = w_ > 1 && (unsigned long long)area * (unsigned long long)w_ < (1ULL << 32);
        rcp = fast ? (unsigned)((0x100000000ULL + w_ - 1) / w_) : 0u;
    }
    __device__ __forceinline__ long long row(long long i) const
    {
        if (w == 1) return i;
        return fast ? (long long)__umulhi((unsigned)i, rcp) : i / w;
    }
};

// The start of an exact window search, floor(s/n - r) - 1 and ceil(s/n + r)
// + 1 for a coordinate in [0, lim): the searches then move inward with the
// exact integer test, so the start needs only an error below one.  For lim
// <= 2^20 it is taken in FP32, without FP64 divisions (slow on this part):
// s, n and their quotient each rounded leave at most 4e-7 relative, 0.42
// absolute; rounding r adds at most 0.07 and the subtraction 0.13, 0.62 in
// all.  Larger dimensions take FP64.
__device__ __forceinline__ void window_start(long long s, long long n, double r, int lim, long long &lo,
                                             long long &hi)
{
    if (lim <= (1 << 20)) {
        const float c = __fdividef((float)s, (float)n), rf = (float)r;
        lo = (long long)floorf(c - rf) - 1;
        hi = (long long)ceilf(c + rf) + 1;
    } else {
        const double c = (double)s / (double)n;
        lo = (long long)floor(c - r) - 1;
        hi = (long long)ceil(c + r) + 1;
    }
}

// Programmatic dependent launch: a kernel launched with pdl_launch() may be
// placed on the GPU while its predecessor in the stream is still draining.
// It calls pdl_wait() before it reads anything the predecessor wrote (the wait
// returns once the predecessor has completed and its writes are visible), and
// pdl_release() to let its own successor be placed early.  Both are no-ops
// for a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// What the assignment kernel reads about one cluster (48 bytes).
struct ClusterDev {
    float L, a, b;           // mean CIELab colour
    float xk, yk;            // barycenter X_k
    int ex, ey;              // path endpoint: X_k rounded half-up, or X_k^* (Eq. 4)
    int xlo, xhi, ylo, yhi;  // window of X_k, clipped to the image (inclusive)
    int pad;
};
static_assert(sizeof(ClusterDev) == 48, "ClusterDev layout");

// Per-cluster integer sums accumulated by one assignment (64 bytes).
struct ClusterAcc {
    unsigned long long n, sx, sy;  // count and coordinate sums
    unsigned long long sL, sa, sb; // two's-complement sums of fixed-point colour
    unsigned long long pad0, pad1;
};

// Counters and flags on the device.
struct DevCounters {
    int nproj;        // clusters queued for projection in this update
    int orphans;      // pixels no window reached in the last assignment
    int error;        // nonzero: a device-side check failed (code below)
    int timeout;      // nonzero: a bounded wait gave up
    unsigned long long samples;  // optional: path samples of the last assignment
    unsigned long long pairs;    // optional: (pixel, cluster) pairs evaluated
    unsigned long long map_rects;    // optional: (tile, cluster) rectangles walked on a map
    unsigned long long plane_rects;  // optional: ... walked on the plane in global memory
    unsigned prior_max;  // scratch: maximum of the gradient prior (float bits)
    int proj_all;        // the update saw orphans: the projection searches the image
    int n_labels;        // labels after the last connectivity enforcement
};
constexpr int ERR_TILE_LIST_OVERFLOW = 1;
constexpr int ERR_BAD_LABEL = 2;
constexpr int ERR_CCL_CHAIN = 3;

// Everything the per-iteration kernels need, by value.
struct SolveArgs {
    int H, W, K, Keff, nx, ny;
    long long N;
    double r;          // sqrt(N/K)
    float lam, gamma, sigma, ms2;  // ms2 = m^2 / r^2
    int n_tx, n_ty;    // tiles
    int map_cap;       // distance-map pairs per assignment CTA (0: every path on the plane)
    int pitch;         // plane row pitch in pixels (>= W, multiple of 4)
    // grid column of the set-up, floor(x * nx / W), as a multiply-high by
    // ceil(2^32 / W) where that is exact; 0: divide
    unsigned grid_rcp_x;
    int count_samples;
    int prune;         // 1: skip pairs whose lower bound exceeds the pixel's best D (0: evaluate all)
    const float4 *plane32;   // (L, a, b, w) per pixel, row pitch `pitch` [FP32 storage]
    const uint2 *plane16;    // the same as 4 x fp16                   [FP16 storage]
    int *labels;
    long long *st_n, *st_sx, *st_sy;   // cluster state
    float4 *st_col;
    int2 *st_end;
    ClusterDev *cdev;
    ClusterAcc *acc;
    int4 *prev_win;    // window (xlo, xhi, ylo, yhi) the last assignment used
    const float *lut;  // 256-entry inverse sRGB transfer function
    int *proj_list;
    int *tile_count, *tile_off, *tile_cursor, *tile_list;
    long long tile_cap;
    int tpw_x, tpw_y;  // bound on the tiles one window spans, per axis
    DevCounters *ctr;
};

// A batch: the argument blocks of `count` images in device memory, and prefix
// sums that map a flat index (tile, cluster, fill slot) to its image.
struct BatchArgs {
    const SolveArgs *args;
    const int *tile_base;   // count+1: prefix of n_tx*n_ty
    const int *clus_base;   // count+1: prefix of Keff
    const int *fill_base;   // count+1: prefix of Keff*tpw_x*tpw_y
    int count;
};

// Synchronisation words of a persistent batched launch (zeroed before each).
struct PersistSync {
    unsigned arrive;  // CTAs arrived at the current barrier
    unsigned gen;     // barriers completed
    unsigned queue;   // next tile of the assignment queue
    unsigned abort;   // a wait gave up: every CTA returns
};

// A persistent batched launch: n iterations of the batch in one launch.
struct PersistArgs {
    BatchArgs b;
    const int *order;       // count: the images in queue order
    const int *order_base;  // count+1: prefix of their tile counts, in that order
    PersistSync *sync;
    int total_tiles, total_clusters, total_fill, iters;
    long long wait_ns;      // bound on each barrier wait
    int hold;               // test hook: extra arrivals a barrier waits for (0)
};

// Static shared memory a persistent batched CTA may use beside the
// assignment's dynamic buffer (the map capacity leaves this much free).
constexpr int PERSIST_STATIC_SMEM = 1024;

// Image of flat index g: the last i with base[i] <= g (base[0] = 0).
__device__ __forceinline__ int batch_find(const int *base, int count, int g)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// A plane sample as stored (float4, or 4 x fp16 in a uint2) and as FP32.
__device__ __forceinline__ float4 sample_value(float4 v) { return v; }
__device__ __forceinline__ float4 sample_value(uint2 u)
{
    __half2 lo = *reinterpret_cast<__half2 *>(&u.x);
    __half2 hi = *reinterpret_cast<__half2 *>(&u.y);
    float2 a = __half22float2(lo), b = __half22float2(hi);
    return make_float4(a.x, a.y, b.x, b.y);
}

// Read-only global load of one plane sample, as FP32.
template <typename T>
__device__ __forceinline__ float4 fetch_sample(const T *q) { return sample_value(__ldg(q)); }

// The linear path of Sec. II-B between pixels p and e, walked from the
// lexicographically smaller end (x, then y) so the pixel set does not depend
// on the direction.  With ns = max(|dx|,|dy|) steps along the major axis, step
// i moves the minor coordinate by floor((2*i*d_minor + ns) / (2*ns)), i.e.
// i*d_minor/ns rounded half-up: the incremental integer form below keeps
// e = (2*i*d_minor + ns) mod 2*ns.
struct PathSetup {
    int ax, ay;        // start
    int ns, dmin;      // steps along the major axis, minor extent
    int major_sgn_y;   // for y-major paths: +1 / -1 direction of y; 0 for x-major
    int minor_sgn;     // direction of the minor axis (+1/-1)
    bool xmajor;
};

__device__ __forceinline__ PathSetup path_setup(int px, int py, int ex, int ey)
{
    PathSetup s;
    int ax, ay, bx, by;
    if (px < ex || (px == ex && py <= ey)) { ax = px; ay = py; bx = ex; by = ey; }
    else { ax = ex; ay = ey; bx = px; by = py; }
    int dx = bx - ax;
    int dy = by - ay;
    int ady = dy < 0 ? -dy : dy;
    int sgy = dy < 0 ? -1 : 1;
    s.ax = ax; s.ay = ay;
    if (dx >= ady) { s.xmajor = true; s.ns = dx; s.dmin = ady; s.minor_sgn = sgy; s.major_sgn_y = 0; }
    else { s.xmajor = false; s.ns = ady; s.dmin = dx; s.minor_sgn = 1; s.major_sgn_y = sgy; }
    return s;
}

// The stepping rule of every path (Sec. II-B): after sample i the walk has
// taken m_i = floor(1/2 + i dmin / ns) minor steps (per minor axis, for the
// 3-D paths of supervoxels).  Two forms of the carry (is step i -> i+1 a minor
// step?) give the same m_i; a debugging entry point walks both in lockstep.
//
// Error term: e starts at ns and grows by 2 dmin per step; a minor step is
// taken (and 2 ns removed) when e reaches 2 ns, so e = ns + 2 i dmin - 2 ns m_i.
struct ErrorTermCarry {
    int e, two_d, two_ns;
    __device__ __forceinline__ ErrorTermCarry(int dmin, int ns) : e(ns), two_d(2 * dmin), two_ns(2 * ns) {}
    __device__ __forceinline__ bool next()
    {
        e += two_d;
        if (e >= two_ns) {
            e -= two_ns;
            return true;
        }
        return false;
    }
};

// Fixed point: a 32-bit accumulator starts at 2^31 and adds S per step; its
// carry is the minor step.  With S = dmin 2^32 / ns + eps, the carry count
// after i steps is floor(1/2 + i dmin / ns + i eps / 2^32).  For 0 < eps <
// FIXED_STEP_EPS and ns <= FIXED_STEP_MAX_NS the excess i eps / 2^32 stays
// below 1 / (2 ns), the least distance from 1/2 + i dmin / ns up to the next
// integer when it is not one, so the count is m_i.  dmin = ns (exact slope
// 2^32) takes S = 2^32 - 1: the count is i + floor((2^31 - i) / 2^32) = i.
constexpr int FIXED_STEP_MAX_NS = 512;
constexpr uint32_t FIXED_STEP_EPS = 4610;
static_assert((double)FIXED_STEP_EPS * FIXED_STEP_MAX_NS * FIXED_STEP_MAX_NS < 2147483648.0,
              "i eps / 2^32 < 1 / (2 ns) for every i <= ns <= FIXED_STEP_MAX_NS");

// S for 0 <= dmin <= ns <= FIXED_STEP_MAX_NS.  The estimate dmin / ns * 2^32
// from the approximate reciprocal (at most 4 ulp: relative error below 2^-21,
// so within 2304 of the exact slope, itself below 2^32 - 2^23 when dmin < ns)
// is raised by 2305: then 0 < S - dmin 2^32 / ns < 4610 = FIXED_STEP_EPS.
__device__ __forceinline__ uint32_t fixed_step_slope(int dmin, int ns)
{
    if (dmin >= ns) return 0xffffffffu;  // also ns = 0: one sample, no step
    float inv;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"((float)ns));
    const float f = (float)dmin * inv * 4294967296.0f;
    return __float2uint_rz(f) + (FIXED_STEP_EPS / 2);
}
static_assert(FIXED_STEP_EPS / 2 == 2305, "the raise covers a 4-ulp reciprocal");

struct FixedPointCarry {
    uint32_t acc, S;
    __device__ __forceinline__ FixedPointCarry(int dmin, int ns) : acc(0x80000000u), S(fixed_step_slope(dmin, ns)) {}
    __device__ __forceinline__ bool next()
    {
        const uint32_t na = acc + S;
        const bool carry = na < acc;
        acc = na;
        return carry;
    }
};

// The address step of a 2-D path: smaj, plus smin on a minor step.
template <typename Carry>
struct PathStep {
    Carry c;
    int smaj, sboth;
    __device__ __forceinline__ PathStep(const PathSetup &s, int smaj_, int smin_)
        : c(s.dmin, s.ns), smaj(smaj_), sboth(smaj_ + smin_) {}
    __device__ __forceinline__ int next() { return c.next() ? sboth : smaj; }
};
using ErrorTermStep = PathStep<ErrorTermCarry>;
using FixedPointStep = PathStep<FixedPointCarry>;

// Steps through the |P| = ns + 1 samples of a path from its start `q`
// (an address or offset in any unit): each step adds smaj, plus smin on a
// minor step.  `visit` receives every sample address.
template <typename Step, typename Addr, typename Visit>
__device__ __forceinline__ int walk_with(Addr q, int smaj, int smin, const PathSetup &s, Visit &&visit)
{
    Step st(s, smaj, smin);
#pragma unroll 4
    for (int i = 0; i <= s.ns; ++i) {
        visit(q);
        q += st.next();
    }
    return s.ns + 1;
}

// The fixed-point rule in closed form: the carries after i steps are
// m_i = floor((2^31 + i S) / 2^32), so sample i lies at q + i smaj + m_i smin.
// The walk takes U samples at a time from the accumulator at the group's
// start (m of sample k of the group = the high word of acc + k S, one wide
// multiply-add each; the samples' addresses do not depend on one another) and
// then moves the start and the accumulator on by U steps.  Same samples, in
// the same order, as walk_with<FixedPointStep>; for ns <= FIXED_STEP_MAX_NS.
template <int U, typename Addr, typename Visit>
__device__ __forceinline__ int walk_grouped(Addr q, int smaj, int smin, const PathSetup &s, Visit &&visit)
{
    const uint32_t S = fixed_step_slope(s.dmin, s.ns);
    uint32_t acc = 0x80000000u;
    const int n = s.ns + 1;
    const auto at = [&](int k) {
        const uint32_t m = k == 0 ? 0u : (uint32_t)(((unsigned long long)S * (unsigned)k + acc) >> 32);
        return q + (Addr)(k * smaj) + (Addr)((int)m * smin);
    };
    int i = 0;
#pragma unroll 1
    for (; i + U <= n; i += U) {
#pragma unroll
        for (int k = 0; k < U; ++k) visit(at(k));
        const unsigned long long t = (unsigned long long)S * (unsigned)U + acc;
        acc = (uint32_t)t;
        q += (Addr)(U * smaj) + (Addr)((int)(t >> 32) * smin);
    }
#pragma unroll
    for (int k = 0; k < U - 1; ++k)
        if (i + k < n) visit(at(k));
    return n;
}

template <typename Addr, typename Visit>
__device__ __forceinline__ int walk_steps(Addr q, int smaj, int smin, const PathSetup &s,
                                          Visit &&visit)
{
    return walk_with<ErrorTermStep>(q, smaj, smin, s, visit);
}

// Element strides of the major and minor steps on a plane with row pitch `pitch`.
__device__ __forceinline__ void path_strides(const PathSetup &s, int pitch, int &smaj, int &smin)
{
    if (s.xmajor) { smaj = 1; smin = s.minor_sgn * pitch; }
    else { smaj = s.major_sgn_y * pitch; smin = 1; }
}

// Visits the pixels of the path on a plane with row pitch `pitch` whose
// element (0,0) is image pixel (ox, oy).  Returns |P|.
template <typename T, typename Visit>
__device__ __forceinline__ int walk_path(const T *__restrict__ base, int pitch, int ox, int oy,
                                         const PathSetup &s, Visit &&visit)
{
    int smaj, smin;
    path_strides(s, pitch, smaj, smin);
    const T *q = base + (long long)(s.ay - oy) * pitch + (s.ax - ox);
    return walk_steps(q, smaj, smin, s, visit);
}

// Squared CIELab distance d_c(q, C_k) of Eq. 1 between a sample and a
// cluster colour, in one fixed FP32 order (every walker and map uses it).
// The L and a differences are one packed FP32x2 subtraction (each half
// rounded to nearest, as two scalar subtractions would be).
__device__ __forceinline__ float colour_dist(float4 v, float cL, float ca, float cb)
{
    unsigned long long xy, cxy, d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(xy) : "f"(v.x), "f"(v.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(cxy) : "f"(cL), "f"(ca));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(xy), "l"(cxy));
    float dl, da;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(dl), "=f"(da) : "l"(d));
    const float db = v.z - cb;
    return fmaf(dl, dl, fmaf(da, da, db * db));
}

// Sums along the path of d_c(q, C_k) (Eq. 1) and of the contour factor w(q)
// (Eq. 2), in walk order.  Returns |P|.
template <typename T>
__device__ __forceinline__ int path_sums(const T *__restrict__ base, int pitch, int ox, int oy,
                                         const PathSetup &s, float cL, float ca, float cb,
                                         float &sum_dc, float &sum_w)
{
    float dc = 0.f, w = 0.f;
    int len = walk_path(base, pitch, ox, oy, s, [&](const T *q) {
        const float4 v = fetch_sample<T>(q);
        dc += colour_dist(v, cL, ca, cb);
        w += v.w;
    });
    sum_dc = dc;
    sum_w = w;
    return len;
}

// Eq. 1-3 assembled from the path sums.
__device__ __forceinline__ float scalp_distance(float dcp, float sum_dc, float sum_w, int len,
                                                float lam, float gamma, float ms2, float ds)
{
    // 1 / |P| from the hardware reciprocal (relative error below 2^-22: far
    // inside the FP32 rounding of the sums); every walker shares this code
    float inv;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"((float)len));
    float dcol = lam * dcp + (1.0f - lam) * (sum_dc * inv);
    float dcon = 1.0f + gamma * (sum_w * inv);
    return fmaf(dcol, dcon, ms2 * ds);
}

// ---------------------------------------------------------------------------
// Warp-aggregated segmented reduction.  Lanes holding the same key are summed
// with warp reductions and the group's first lane hands the sums to `sink`.
// Coordinates come relative to a warp-uniform base (bx, by) with offsets in
// [0, 31], so both offset sums pack into one 32-bit reduction; colour values
// are fixed point (x 2^COLOR_FRAC_BITS), small enough that a 32-lane sum fits
// in 32 bits.
template <class Sink>
__device__ __forceinline__ void warp_aggregate(bool valid, int key, int bx, int by, int dx, int dy,
                                               float4 v, Sink &&sink)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const float scale = (float)(1 << COLOR_FRAC_BITS);
    const int qL = valid ? __float2int_rn(v.x * scale) : 0;
    const int qa = valid ? __float2int_rn(v.y * scale) : 0;
    const int qb = valid ? __float2int_rn(v.z * scale) : 0;
    const unsigned qxy = valid ? (unsigned)dx | ((unsigned)dy << 16) : 0u;
    unsigned pending = __ballot_sync(FULL, valid);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int k = __shfl_sync(FULL, key, leader);
        const bool mine = valid && key == k;
        const unsigned grp = __ballot_sync(FULL, mine);
        const long long cnt = __popc(grp);
        const unsigned sxy = __reduce_add_sync(FULL, mine ? qxy : 0u);
        const long long sL = __reduce_add_sync(FULL, mine ? qL : 0);
        const long long sa = __reduce_add_sync(FULL, mine ? qa : 0);
        const long long sb = __reduce_add_sync(FULL, mine ? qb : 0);
        if (lane == leader)
            sink(k, cnt, cnt * bx + (long long)(sxy & 0xffffu), cnt * by + (long long)(sxy >> 16), sL,
                 sa, sb);
        pending &= ~grp;
    }
}

__device__ __forceinline__ void acc_add(ClusterAcc *c, long long n, long long sx, long long sy,
                                        long long sL, long long sa, long long sb)
{
    atomicAdd(&c->n, (unsigned long long)n);
    atomicAdd(&c->sx, (unsigned long long)sx);
    atomicAdd(&c->sy, (unsigned long long)sy);
    atomicAdd(&c->sL, (unsigned long long)sL);
    atomicAdd(&c->sa, (unsigned long long)sa);
    atomicAdd(&c->sb, (unsigned long long)sb);
}

// Sum straight into the global per-cluster sums.
__device__ __forceinline__ void warp_aggregate_global(bool valid, int label, int bx, int by, int dx,
                                                      int dy, float4 v, ClusterAcc *acc)
{
    warp_aggregate(valid, label, bx, by, dx, dy, v,
                   [&](int k, long long n, long long sx, long long sy, long long sL, long long sa,
                       long long sb) { acc_add(&acc[k], n, sx, sy, sL, sa, sb); });
}

__host__ __device__ inline long long ceil_div_ll(long long a, long long b) { return (a + b - 1) / b; }

// Upper bound on the tiles a window spans along one axis: the window holds at
// most floor(2r) + 1 consecutive pixels (one more is allowed for rounding of r).
__host__ __device__ inline int tiles_per_window(double r, int tile)
{
    long long len = (long long)(2.0 * r) + 2;
    return (int)((len + tile - 1) / tile + 1);
}

}  // namespace scalp
