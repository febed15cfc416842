// scalp_metrics.cu -- maps computed from decompositions.
//
// scalp_boundary_map: the multi-scale boundary confidence map the paper's
// precision-recall evaluation uses (Sec. III-A2: boundary maps of the
// decompositions at several scales, averaged).  A pixel is a boundary pixel of
// a decomposition iff one of its 4-neighbours carries another label; the map
// is the fraction of the decompositions in which it is one.
#include <algorithm>
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
        const int y = (int)(p / W), x = (int)(p - (long long)y * W);
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
