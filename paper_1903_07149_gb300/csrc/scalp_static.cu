// scalp_static.cu -- scalp_label_means_static(): per-superpixel means with no
// device allocation at all.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// that runs while another component owns the device memory budget, plugins
// that are given only the input and output buffers, or hosts where allocation
// would synchronise the device at a bad moment.  This entry point serves them.
// Its scratch (the integer sums and the sRGB table) is one file-scope
// __device__ array of fixed size, which every GPU that loads the library
// holds until the process exits.  The caller passes only the inputs and the
// output.
#include <algorithm>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/scalp.h"
#include "scalp_launch.h"

using namespace scalp;

namespace {

constexpr int MAX_DEVICES = 64;

// Scratch: SCALP_STATIC_MAX_LABELS cluster sums, then the 256-entry table.
struct StaticScratch {
    ClusterAcc sums[SCALP_STATIC_MAX_LABELS];
    float lut[256];
};
static_assert(offsetof(StaticScratch, sums) == 0, "the sums start the scratch");
static __device__ __align__(256) StaticScratch g_static_scratch;

std::mutex g_static_mutex;
StaticScratch *g_static_ptr[MAX_DEVICES];  // device address, per device, once known

// Errors are reported through scalp_last_error(NULL).
int static_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    scalp::set_last_error(buf);
    return code;
}

__global__ void k_static_table(StaticScratch *s)
{
    const int i = threadIdx.x;
    if (i < 256) {
        const double c = i / 255.0;
        s->lut[i] = (float)(c <= 0.04045 ? c / 12.92 : pow((c + 0.055) / 1.055, 2.4));
    }
}

// CIELab of 8-bit sRGB (the set-up kernel's conversion), then warp-aggregated
// integer sums per label into the static scratch.  Labels outside
// [0, n_labels) are skipped.
__global__ void __launch_bounds__(256)
    k_static_sums(const uint8_t *__restrict__ rgb, long long rgb_stride,
                  const int *__restrict__ labels, int H, int W, int n_labels, StaticScratch *s)
{
    __shared__ float lin[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) lin[i] = s->lut[i];
    __syncthreads();
    const long long segs_per_row = (W + 31) / 32;
    const long long n_segs = segs_per_row * H;
    const long long warps = (long long)gridDim.x * (blockDim.x / 32);
    for (long long seg = blockIdx.x * (long long)(blockDim.x / 32) + (threadIdx.x >> 5); seg < n_segs;
         seg += warps) {
        const int y = (int)(seg / segs_per_row);
        const int bx = (int)(seg % segs_per_row) * 32;
        const int x = bx + (threadIdx.x & 31);
        bool valid = x < W;
        int label = 0;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) {
            label = labels[(long long)y * W + x];
            valid = label >= 0 && label < n_labels;
            const float3 c = srgb_to_lab(lin, rgb + y * rgb_stride + 3 * (long long)x);
            v = make_float4(c.x, c.y, c.z, 0.f);
        }
        warp_aggregate_global(valid, valid ? label : 0, bx, y, x - bx, 0, v, s->sums);
    }
}

// out[6k .. 6k+5] = (n, mean L, mean a, mean b, mean x, mean y); zeros if n = 0.
__global__ void k_static_means(const StaticScratch *s, int n_labels, double *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_labels) return;
    const ClusterAcc c = s->sums[k];
    const long long n = (long long)c.n;
    double *o = out + 6LL * k;
    if (n == 0) {
        for (int i = 0; i < 6; ++i) o[i] = 0.0;
        return;
    }
    const double den = (double)n * (double)(1 << COLOR_FRAC_BITS);
    o[0] = (double)n;
    o[1] = (double)(long long)c.sL / den;
    o[2] = (double)(long long)c.sa / den;
    o[3] = (double)(long long)c.sb / den;
    o[4] = (double)(long long)c.sx / (double)n;
    o[5] = (double)(long long)c.sy / (double)n;
}

}  // namespace

extern "C" int scalp_label_means_static(const uint8_t *rgb, int64_t rgb_stride, const int32_t *labels,
                                        int32_t H, int32_t W, int32_t n_labels, double *out,
                                        void *stream)
{
    if (!rgb || !labels || !out) return static_fail(SCALP_E_ARG, "rgb, labels and out must be device pointers");
    if (H < 1 || W < 1 || (long long)H * W > (1LL << 30))
        return static_fail(SCALP_E_ARG, "need H, W >= 1 and H*W <= 2^30");
    if (n_labels < 1 || n_labels > SCALP_STATIC_MAX_LABELS)
        return static_fail(SCALP_E_ARG, "n_labels must be in [1, %d] (the fixed scratch holds %d)",
                           SCALP_STATIC_MAX_LABELS, SCALP_STATIC_MAX_LABELS);
    if (rgb_stride != 0 && rgb_stride < 3LL * W) return static_fail(SCALP_E_ARG, "rgb_stride < 3*W");
    const long long stride = rgb_stride ? rgb_stride : 3LL * W;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(SCALP_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return static_fail(SCALP_E_ARG, "device %d not supported", dev);
    StaticScratch *s;
    {
        // set-up, once per device, with that device current: the scratch's
        // device address (the symbol itself is only a host-side stand-in)
        // and the sRGB table
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess)
                return static_fail(SCALP_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            k_static_table<<<1, 256, 0, st>>>(static_cast<StaticScratch *>(p));
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // ready for any stream
            if (e != cudaSuccess) return static_fail(SCALP_E_CUDA, "table kernel: %s", cudaGetErrorString(e));
            g_static_ptr[dev] = static_cast<StaticScratch *>(p);
        }
        s = g_static_ptr[dev];
    }
    // the sums start at zero on every call
    e = cudaMemsetAsync(static_cast<void *>(s), 0, sizeof(ClusterAcc) * (size_t)n_labels, st);
    if (e != cudaSuccess) return static_fail(SCALP_E_CUDA, "clear scratch: %s", cudaGetErrorString(e));
    const long long n_segs = (long long)((W + 31) / 32) * H;
    const int blocks = (int)std::min<long long>((n_segs + 7) / 8, 152 * 16);
    k_static_sums<<<blocks, 256, 0, st>>>(rgb, stride, labels, H, W, n_labels, s);
    k_static_means<<<(n_labels + 255) / 256, 256, 0, st>>>(s, n_labels, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(SCALP_E_CUDA, "means kernels: %s", cudaGetErrorString(e));
    return SCALP_OK;
}
