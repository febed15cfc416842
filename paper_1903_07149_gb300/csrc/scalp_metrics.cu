// scalp_metrics.cu -- maps and scores computed from decompositions.
//
// scalp_quality_metrics: the superpixel metrics of Sec. III-A2 against a
// ground-truth segmentation: boundary recall (Eq. 5), achievable segmentation
// accuracy (Eq. 6), undersegmentation error (Eq. 7) and compactness (Eq. 8).
//
// scalp_boundary_map: the multi-scale boundary confidence map the paper's
// precision-recall evaluation uses (Sec. III-A2: boundary maps of the
// decompositions at several scales, averaged).  A pixel is a boundary pixel of
// a decomposition iff one of its 4-neighbours carries another label; the map
// is the fraction of the decompositions in which it is one.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>

#include "../../include/scalp.h"
#include "scalp_launch.h"

using namespace scalp;

namespace {

struct MapPtrs {
    const int *p[SCALP_MAX_MAPS];
};

__global__ void k_boundary_map(MapPtrs m, int count, int H, int W, float *__restrict__ out)
{
    const long long N = (long long)H * W;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        const int y = (int)((unsigned)p / (unsigned)W), x = (int)p - y * W;  // N <= 2^30
        int hits = 0;
        for (int i = 0; i < count; ++i) {
            const int *__restrict__ l = m.p[i];
            const int c = l[p];
            const bool b = (x > 0 && l[p - 1] != c) || (x < W - 1 && l[p + 1] != c) ||
                           (y > 0 && l[p - W] != c) || (y < H - 1 && l[p + W] != c);
            hits += b;
        }
        out[p] = (float)hits / (float)count;
    }
}

int metrics_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    scalp::set_last_error(buf);
    return code;
}

}  // namespace

extern "C" int scalp_boundary_map(const int32_t *const *labels, int32_t count, int32_t H, int32_t W,
                                  float *out, void *stream)
{
    if (!labels || !out) return metrics_fail(SCALP_E_ARG, "labels and out are required");
    if (count < 1 || count > SCALP_MAX_MAPS)
        return metrics_fail(SCALP_E_ARG, "count must be in [1, %d]", SCALP_MAX_MAPS);
    if (H < 1 || W < 1 || (long long)H * W > (1LL << 30)) return metrics_fail(SCALP_E_ARG, "bad H, W");
    MapPtrs m{};
    for (int i = 0; i < count; ++i) {
        if (!labels[i]) return metrics_fail(SCALP_E_ARG, "labels[%d] is NULL", i);
        m.p[i] = labels[i];
    }
    const long long N = (long long)H * W;
    const int blocks = (int)std::min<long long>((N + 255) / 256, 152 * 16);
    k_boundary_map<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(m, count, H, W, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return metrics_fail(SCALP_E_CUDA, "boundary map: %s", cudaGetErrorString(e));
    return SCALP_OK;
}

// ---------------------------------------------------------------------------
// Quality metrics, Eq. 5-8.  Boundary pixels: a 4-neighbour carries another
// label.  BR: ground-truth boundary pixels with a superpixel boundary pixel at
// Euclidean distance < eps.  ASA: sum over superpixels of the largest overlap
// with one segment, over N.  UE: sum over segments and the superpixels that
// meet them of |S_k - G_i|, over N.  CO: (1/N) sum 4 pi |S_k|^2 / |P(S_k)|^2,
// |P| = pixel edges between S_k and the rest (image border included).
// ---------------------------------------------------------------------------
namespace {

struct QualityWs {
    int *ov;                       // n_labels x n_gt overlaps
    unsigned long long *area, *perim;
    long long *best, *ue;          // per superpixel
    double *co;                    // per superpixel
    unsigned long long *counts;    // [0] gt boundary pixels, [1] hits
    double *result;                // br, asa, ue, co
};

__device__ __forceinline__ bool bnd(const int *__restrict__ l, int H, int W, int x, int y)
{
    const long long p = (long long)y * W + x;
    const int c = l[p];
    return (x > 0 && l[p - 1] != c) || (x < W - 1 && l[p + 1] != c) || (y > 0 && l[p - W] != c) ||
           (y < H - 1 && l[p + W] != c);
}

__global__ void k_quality_pixels(const int *__restrict__ lab, const int *__restrict__ gt, int n_gt,
                                 int H, int W, double eps, QualityWs w)
{
    const long long N = (long long)H * W;
    const int r = (int)ceil(eps);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        const int y = (int)((unsigned)p / (unsigned)W), x = (int)p - y * W;  // N <= 2^30
        const int k = lab[p];
        atomicAdd(&w.ov[(long long)k * n_gt + gt[p]], 1);
        atomicAdd(&w.area[k], 1ull);
        const unsigned e = (x == 0 || lab[p - 1] != k) + (x == W - 1 || lab[p + 1] != k) +
                           (y == 0 || lab[p - W] != k) + (y == H - 1 || lab[p + W] != k);
        if (e) atomicAdd(&w.perim[k], (unsigned long long)e);
        if (bnd(gt, H, W, x, y)) {
            atomicAdd(&w.counts[0], 1ull);
            bool found = false;
            for (int dy = -r; dy <= r && !found; ++dy)
                for (int dx = -r; dx <= r && !found; ++dx) {
                    const int qx = x + dx, qy = y + dy;
                    if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                    if (sqrt((double)(dx * dx + dy * dy)) >= eps) continue;
                    if (bnd(lab, H, W, qx, qy)) found = true;
                }
            if (found) atomicAdd(&w.counts[1], 1ull);
        }
    }
}

__global__ void k_quality_rows(int n_labels, int n_gt, QualityWs w)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_labels) return;
    const long long a = (long long)w.area[k];
    long long best = 0, ue = 0;
    for (int i = 0; i < n_gt; ++i) {
        const long long o = w.ov[(long long)k * n_gt + i];
        best = max(best, o);
        if (o > 0) ue += a - o;
    }
    w.best[k] = best;
    w.ue[k] = ue;
    const double pr = (double)w.perim[k];
    w.co[k] = a > 0 ? 4.0 * M_PI * (double)a * (double)a / (pr * pr) : 0.0;
}

// One CTA, a fixed summation order: deterministic.
__global__ void __launch_bounds__(1024) k_quality_total(int n_labels, long long N, QualityWs w)
{
    __shared__ long long s_best[1024], s_ue[1024];
    __shared__ double s_co[1024];
    long long b = 0, u = 0;
    double c = 0.0;
    for (int k = threadIdx.x; k < n_labels; k += 1024) {
        b += w.best[k];
        u += w.ue[k];
        c += w.co[k];
    }
    s_best[threadIdx.x] = b;
    s_ue[threadIdx.x] = u;
    s_co[threadIdx.x] = c;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s_best[threadIdx.x] += s_best[threadIdx.x + h];
            s_ue[threadIdx.x] += s_ue[threadIdx.x + h];
            s_co[threadIdx.x] += s_co[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned long long gb = w.counts[0], hit = w.counts[1];
        w.result[0] = gb ? (double)hit / (double)gb : 1.0;
        w.result[1] = (double)s_best[0] / (double)N;
        w.result[2] = (double)s_ue[0] / (double)N;
        w.result[3] = s_co[0] / (double)N;
    }
}

size_t quality_layout(int n_labels, int n_gt, QualityWs *w, unsigned char *base)
{
    size_t cur = 0;
    auto take = [&](size_t bytes) {
        const size_t off = (cur + 255) & ~(size_t)255;
        cur = off + bytes;
        return base ? base + off : nullptr;
    };
    unsigned char *ov = take((size_t)n_labels * n_gt * sizeof(int));
    unsigned char *area = take((size_t)n_labels * 8);
    unsigned char *perim = take((size_t)n_labels * 8);
    unsigned char *best = take((size_t)n_labels * 8);
    unsigned char *ue = take((size_t)n_labels * 8);
    unsigned char *co = take((size_t)n_labels * 8);
    unsigned char *counts = take(2 * 8);
    unsigned char *result = take(4 * 8);
    if (w) {
        w->ov = reinterpret_cast<int *>(ov);
        w->area = reinterpret_cast<unsigned long long *>(area);
        w->perim = reinterpret_cast<unsigned long long *>(perim);
        w->best = reinterpret_cast<long long *>(best);
        w->ue = reinterpret_cast<long long *>(ue);
        w->co = reinterpret_cast<double *>(co);
        w->counts = reinterpret_cast<unsigned long long *>(counts);
        w->result = reinterpret_cast<double *>(result);
    }
    return (cur + 255) & ~(size_t)255;
}

}  // namespace

extern "C" size_t scalp_quality_workspace_bytes(int32_t H, int32_t W, int32_t n_labels, int32_t n_gt)
{
    if (H < 1 || W < 1 || n_labels < 1 || n_gt < 1) return 0;
    if ((long long)n_labels * n_gt > (1LL << 28)) return 0;
    return quality_layout(n_labels, n_gt, nullptr, nullptr);
}

extern "C" int scalp_quality_metrics(const int32_t *labels, int32_t n_labels, const int32_t *gt,
                                     int32_t n_gt, int32_t H, int32_t W, double eps, void *workspace,
                                     size_t workspace_bytes, scalp_quality *out, void *stream)
{
    if (!labels || !gt || !out) return metrics_fail(SCALP_E_ARG, "labels, gt and out are required");
    if (!(eps > 0)) return metrics_fail(SCALP_E_ARG, "eps must be > 0");
    const size_t need = scalp_quality_workspace_bytes(H, W, n_labels, n_gt);
    if (need == 0) return metrics_fail(SCALP_E_ARG, "bad sizes (n_labels * n_gt <= 2^28)");
    if (!workspace || workspace_bytes < need)
        return metrics_fail(SCALP_E_NOMEM, "workspace of %zu bytes needed", need);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    QualityWs w;
    quality_layout(n_labels, n_gt, &w, reinterpret_cast<unsigned char *>(workspace));
    cudaError_t e = cudaMemsetAsync(workspace, 0, need, st);
    const long long N = (long long)H * W;
    if (e == cudaSuccess) {
        const int blocks = (int)std::min<long long>((N + 255) / 256, 152 * 16);
        k_quality_pixels<<<blocks, 256, 0, st>>>(labels, gt, n_gt, H, W, eps, w);
        k_quality_rows<<<(n_labels + 255) / 256, 256, 0, st>>>(n_labels, n_gt, w);
        k_quality_total<<<1, 1024, 0, st>>>(n_labels, N, w);
        e = cudaGetLastError();
    }
    double r[4];
    if (e == cudaSuccess) e = cudaMemcpyAsync(r, w.result, sizeof r, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return metrics_fail(SCALP_E_CUDA, "quality metrics: %s", cudaGetErrorString(e));
    out->br = r[0];
    out->asa = r[1];
    out->ue = r[2];
    out->co = r[3];
    return SCALP_OK;
}
