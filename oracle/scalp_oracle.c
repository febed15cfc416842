/*
 * scalp_oracle.c -- plain, slow, FP64 CPU oracle for SCALP
 * ("Superpixels with Contour Adherence using Linear Path", Giraud, Ta,
 * Papadakis, ICPR 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this file.  It shares no code, header,
 * table or helper with the CUDA library; neither includes the other.
 *
 * Everything is evaluated in double precision, in the order Algorithm 1 states
 * it: for each cluster C_k, for each pixel p of the (2r+1)x(2r+1) window
 * centred on X_k, compute D(p, C_k) (Eq. 3) and relabel p on a strict '<'.
 * Then update the clusters and, where needed, project their barycenters
 * (Eq. 4).
 *
 * Readings of points the paper leaves open:
 *   - CIELab: sRGB (IEC 61966-2-1) -> linear -> XYZ (D65 matrix) -> CIE 1976
 *     L*a*b*, with the reference white taken as the XYZ image of sRGB white.
 *   - Grid: r = sqrt(N/K); nx = max(1, round(W/r)), ny = max(1, round(H/r));
 *     pixel (x, y) starts in cell floor(y*ny/H)*nx + floor(x*nx/W).
 *   - Window: p is a candidate of C_k iff |x_p - x_k| <= r and |y_p - y_k| <= r,
 *     tested exactly as K*(n*x_p - Sx)^2 <= N*n^2 in 128-bit integers.
 *   - Path endpoint: X_k rounded half-up, floor((2*Sx + n) / (2n)), or X_k^*
 *     when projected.  The path holds both p and the endpoint; it is traced
 *     from the lexicographically smaller (x, then y) end so it is symmetric.
 *   - No candidate: the pixel keeps its previous label.  Empty cluster: its
 *     colour, barycenter and endpoint are kept.
 *   - Projection is triggered when the label at the rounded barycenter is not
 *     k; ties in Eq. 4 go to the smallest raster index.
 *   - Connectivity enforcement (not in the paper) follows a fixed
 *     component-merging rule, see orc_connectivity().
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* CIELab conversion (Sec. II-A: clustering runs in the CIELab space).       */
/* ------------------------------------------------------------------------ */

static double srgb_channel_to_linear(double c)
{
    /* IEC 61966-2-1 transfer function, inverted */
    if (c <= 0.04045) return c / 12.92;
    return pow((c + 0.055) / 1.055, 2.4);
}

static double cie_f(double t)
{
    /* CIE 1976 companding: cube root above (6/29)^3, linear segment below */
    const double d = 6.0 / 29.0;
    if (t > d * d * d) return cbrt(t);
    return t / (3.0 * d * d) + 4.0 / 29.0;
}

static const double M_SRGB_TO_XYZ[3][3] = {
    {0.4124564, 0.3575761, 0.1804375},
    {0.2126729, 0.7151522, 0.0721750},
    {0.0193339, 0.1191920, 0.9503041},
};

void orc_lab_from_rgb(const uint8_t *rgb, int64_t npix, double *L, double *A, double *B)
{
    double white[3];
    for (int i = 0; i < 3; i++)
        white[i] = M_SRGB_TO_XYZ[i][0] + M_SRGB_TO_XYZ[i][1] + M_SRGB_TO_XYZ[i][2];
    for (int64_t p = 0; p < npix; p++) {
        double lin[3], xyz[3];
        for (int c = 0; c < 3; c++) lin[c] = srgb_channel_to_linear(rgb[3 * p + c] / 255.0);
        for (int i = 0; i < 3; i++)
            xyz[i] = M_SRGB_TO_XYZ[i][0] * lin[0] + M_SRGB_TO_XYZ[i][1] * lin[1] +
                     M_SRGB_TO_XYZ[i][2] * lin[2];
        double fx = cie_f(xyz[0] / white[0]);
        double fy = cie_f(xyz[1] / white[1]);
        double fz = cie_f(xyz[2] / white[2]);
        L[p] = 116.0 * fy - 16.0;
        A[p] = 500.0 * (fx - fy);
        B[p] = 200.0 * (fy - fz);
    }
}

/* ------------------------------------------------------------------------ */
/* Regular grid (Sec. II-A; Algorithm 1, initialisation).                    */
/* ------------------------------------------------------------------------ */

void orc_grid_dims(int H, int W, int K, int *nx, int *ny)
{
    double N = (double)H * (double)W;
    double r = sqrt(N / (double)K);
    int gx = (int)floor((double)W / r + 0.5);
    int gy = (int)floor((double)H / r + 0.5);
    if (gx < 1) gx = 1;
    if (gy < 1) gy = 1;
    if (gx > W) gx = W;
    if (gy > H) gy = H;
    *nx = gx;
    *ny = gy;
}

/* ------------------------------------------------------------------------ */
/* Linear path (Sec. II-B), Bresenham's digital segment between two pixels. */
/* ------------------------------------------------------------------------ */

/* Writes the path pixels as (x, y) pairs into xy (capacity >= len) and
 * returns len = max(|dx|, |dy|) + 1.  Step i along the major axis moves the
 * minor coordinate by round-half-up(i * d_minor / d_major). */
int orc_path(int px, int py, int ex, int ey, int32_t *xy)
{
    int ax, ay, bx, by;
    if (px < ex || (px == ex && py <= ey)) {
        ax = px; ay = py; bx = ex; by = ey;
    } else {
        ax = ex; ay = ey; bx = px; by = py;
    }
    int dx = bx - ax; /* >= 0 by the ordering */
    int dy = by - ay;
    int ady = dy < 0 ? -dy : dy;
    int sy = dy < 0 ? -1 : 1;
    if (dx >= ady) {
        int ns = dx;
        for (int i = 0; i <= ns; i++) {
            int off = ns == 0 ? 0 : (int)((2LL * i * ady + ns) / (2LL * ns));
            xy[2 * i] = ax + i;
            xy[2 * i + 1] = ay + sy * off;
        }
        return ns + 1;
    } else {
        int ns = ady;
        for (int i = 0; i <= ns; i++) {
            int off = (int)((2LL * i * dx + ns) / (2LL * ns));
            xy[2 * i] = ax + off;
            xy[2 * i + 1] = ay + sy * i;
        }
        return ns + 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Solver state.                                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t H, W, K;      /* image size, requested number of superpixels */
    int32_t nx, ny, Keff; /* grid; Keff = nx*ny clusters */
    double m, lambda, sigma, gamma; /* gamma < 0 selects the default 2r */
    double r;             /* filled by orc_init: sqrt(N/K) */
    const double *L, *A, *B; /* CIELab planes, N each, row-major */
    const double *C;         /* contour prior in [0,1], N */
    int32_t *labels;      /* N */
    int64_t *n, *sx, *sy; /* Keff: |S_k| and the integer coordinate sums */
    double *cL, *cA, *cB; /* Keff: mean colour */
    int32_t *ex, *ey;     /* Keff: path endpoint (rounded or projected X_k) */
    int64_t orphans;      /* pixels with no candidate in the last assignment */
    int64_t projections;  /* clusters projected in the last update */
} orc_ctx;

/* |v - s/n| <= r with r^2 = N/K, i.e. K*(n*v - s)^2 <= N*n^2, exactly. */
static int in_window(int64_t v, int64_t n, int64_t s, int64_t N, int64_t K)
{
    i128 d = (i128)n * v - (i128)s;
    i128 lhs = (i128)K * d * d;
    i128 rhs = (i128)N * (i128)n * (i128)n;
    return lhs <= rhs;
}

int orc_in_window(int64_t v, int64_t n, int64_t s, int64_t N, int64_t K)
{
    return in_window(v, n, s, N, K);
}

static double dc_at(const orc_ctx *c, int64_t q, int k)
{
    double dl = c->L[q] - c->cL[k];
    double da = c->A[q] - c->cA[k];
    double db = c->B[q] - c->cB[k];
    return dl * dl + da * da + db * db;
}

/* D(p, C_k) of Eq. 3 with the colour term of Eq. 1 and the contour weight of
 * Eq. 2, all sums over the path P_p^k. */
double orc_distance(const orc_ctx *c, int px, int py, int k, int32_t *path_len)
{
    int64_t W = c->W;
    int maxlen = (c->W > c->H ? c->W : c->H) + 1;
    int32_t *xy = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)maxlen);
    int len = orc_path(px, py, c->ex[k], c->ey[k], xy);
    double sum_dc = 0.0, sum_w = 0.0;
    for (int i = 0; i < len; i++) {
        int64_t q = (int64_t)xy[2 * i + 1] * W + xy[2 * i];
        sum_dc += dc_at(c, q, k);
        double cq = c->C[q];
        sum_w += 1.0 - exp(-(cq * cq) / (c->sigma * c->sigma));
    }
    free(xy);
    int64_t p = (int64_t)py * W + px;
    double dc_path = c->lambda * dc_at(c, p, k) + (1.0 - c->lambda) * sum_dc / len;  /* Eq. 1 */
    double d_contour = 1.0 + c->gamma / len * sum_w;                                /* Eq. 2 */
    double xk = (double)c->sx[k] / (double)c->n[k];
    double yk = (double)c->sy[k] / (double)c->n[k];
    double ds = (px - xk) * (px - xk) + (py - yk) * (py - yk);
    if (path_len) *path_len = len;
    return dc_path * d_contour + ds * (c->m * c->m) / (c->r * c->r); /* Eq. 3 */
}

/* Eq. 4: X_k^* = argmin over p in S_k of ||X_p - X_k||, evaluated as
 * (n*x_p - Sx)^2 + (n*y_p - Sy)^2 in 128-bit integers; ties -> smallest raster
 * index.  Only called for clusters with n > 0 (so S_k is not empty). */
static void project_center(orc_ctx *c, int k)
{
    int64_t N = (int64_t)c->H * c->W;
    i128 best = -1;
    int64_t best_p = -1;
    for (int64_t p = 0; p < N; p++) {
        if (c->labels[p] != k) continue;
        int64_t x = p % c->W, y = p / c->W;
        i128 ddx = (i128)c->n[k] * x - c->sx[k];
        i128 ddy = (i128)c->n[k] * y - c->sy[k];
        i128 d2 = ddx * ddx + ddy * ddy;
        if (best_p < 0 || d2 < best) {
            best = d2;
            best_p = p;
        }
    }
    c->ex[k] = (int32_t)(best_p % c->W);
    c->ey[k] = (int32_t)(best_p / c->W);
}

/* Algorithm 1, last two steps: recompute [l_k, a_k, b_k, X_k] as means over
 * S_k, then project X_k when it is not inside S_k. */
void orc_update(orc_ctx *c)
{
    int64_t N = (int64_t)c->H * c->W;
    int K = c->Keff;
    int64_t *n = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *sx = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *sy = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    double *sl = (double *)calloc((size_t)K, sizeof(double));
    double *sa = (double *)calloc((size_t)K, sizeof(double));
    double *sb = (double *)calloc((size_t)K, sizeof(double));
    for (int64_t p = 0; p < N; p++) {
        int k = c->labels[p];
        n[k] += 1;
        sx[k] += p % c->W;
        sy[k] += p / c->W;
        sl[k] += c->L[p];
        sa[k] += c->A[p];
        sb[k] += c->B[p];
    }
    c->projections = 0;
    for (int k = 0; k < K; k++) {
        if (n[k] == 0) continue; /* empty cluster: unchanged */
        c->n[k] = n[k];
        c->sx[k] = sx[k];
        c->sy[k] = sy[k];
        c->cL[k] = sl[k] / (double)n[k];
        c->cA[k] = sa[k] / (double)n[k];
        c->cB[k] = sb[k] / (double)n[k];
        c->ex[k] = (int32_t)((2 * sx[k] + n[k]) / (2 * n[k]));
        c->ey[k] = (int32_t)((2 * sy[k] + n[k]) / (2 * n[k]));
        if (c->labels[(int64_t)c->ey[k] * c->W + c->ex[k]] != k) {
            project_center(c, k);
            c->projections++;
        }
    }
    free(n); free(sx); free(sy); free(sl); free(sa); free(sb);
}

/* Algorithm 1 initialisation: clusters from the regular grid, labels = cell. */
int orc_init(orc_ctx *c)
{
    int64_t N = (int64_t)c->H * c->W;
    if (c->H < 1 || c->W < 1 || c->K < 1 || c->K > N) return -1;
    c->r = sqrt((double)N / (double)c->K);
    if (c->gamma < 0) c->gamma = 2.0 * c->r;
    orc_grid_dims(c->H, c->W, c->K, &c->nx, &c->ny);
    c->Keff = c->nx * c->ny;
    for (int64_t p = 0; p < N; p++) {
        int64_t x = p % c->W, y = p / c->W;
        int cx = (int)(x * c->nx / c->W);
        int cy = (int)(y * c->ny / c->H);
        c->labels[p] = cy * c->nx + cx;
    }
    orc_update(c);
    c->orphans = 0;
    return 0;
}

/* Algorithm 1, assignment: d <- inf; for each C_k, for each p of its window,
 * relabel p when D(p, C_k) < d(p).  Pixels no window reaches keep their label.
 * dbest (optional, N) receives d(p). */
int64_t orc_assign(orc_ctx *c, double *dbest)
{
    int64_t N = (int64_t)c->H * c->W;
    double *d = (double *)malloc(sizeof(double) * (size_t)N);
    for (int64_t p = 0; p < N; p++) d[p] = INFINITY;
    for (int k = 0; k < c->Keff; k++) {
        double xk = (double)c->sx[k] / (double)c->n[k];
        double yk = (double)c->sy[k] / (double)c->n[k];
        int x0 = (int)floor(xk - c->r) - 1, x1 = (int)ceil(xk + c->r) + 1;
        int y0 = (int)floor(yk - c->r) - 1, y1 = (int)ceil(yk + c->r) + 1;
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 > c->W - 1) x1 = c->W - 1;
        if (y1 > c->H - 1) y1 = c->H - 1;
        for (int y = y0; y <= y1; y++) {
            if (!in_window(y, c->n[k], c->sy[k], N, c->K)) continue;
            for (int x = x0; x <= x1; x++) {
                if (!in_window(x, c->n[k], c->sx[k], N, c->K)) continue;
                double D = orc_distance(c, x, y, k, NULL);
                int64_t p = (int64_t)y * c->W + x;
                if (D < d[p]) {
                    d[p] = D;
                    c->labels[p] = k;
                }
            }
        }
    }
    int64_t orphans = 0;
    for (int64_t p = 0; p < N; p++) {
        if (d[p] == INFINITY) orphans++;
        if (dbest) dbest[p] = d[p];
    }
    free(d);
    c->orphans = orphans;
    return orphans;
}

int orc_iterate(orc_ctx *c, int iters)
{
    for (int it = 0; it < iters; it++) {
        orc_assign(c, NULL);
        orc_update(c);
    }
    return 0;
}

/* The same iterations with the assignment taken pixel by pixel, rows shared
 * out over `threads` OpenMP threads (the CPU baseline on all host cores).
 * For each pixel the clusters whose window holds it are visited in ascending
 * k with the strict '<' of Algorithm 1, so every label and distance equals
 * orc_assign's; the update is orc_update's, with the projections (each reads
 * the labels and writes only its own cluster's endpoint) run in parallel. */
static void update_parallel(orc_ctx *c, int threads)
{
    int64_t N = (int64_t)c->H * c->W;
    int K = c->Keff;
    int64_t *n = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *sx = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *sy = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    double *sl = (double *)calloc((size_t)K, sizeof(double));
    double *sa = (double *)calloc((size_t)K, sizeof(double));
    double *sb = (double *)calloc((size_t)K, sizeof(double));
    int *proj = (int *)malloc(sizeof(int) * (size_t)K);
    int nproj = 0;
    for (int64_t p = 0; p < N; p++) { /* raster order, as orc_update */
        int k = c->labels[p];
        n[k] += 1;
        sx[k] += p % c->W;
        sy[k] += p / c->W;
        sl[k] += c->L[p];
        sa[k] += c->A[p];
        sb[k] += c->B[p];
    }
    for (int k = 0; k < K; k++) {
        if (n[k] == 0) continue;
        c->n[k] = n[k];
        c->sx[k] = sx[k];
        c->sy[k] = sy[k];
        c->cL[k] = sl[k] / (double)n[k];
        c->cA[k] = sa[k] / (double)n[k];
        c->cB[k] = sb[k] / (double)n[k];
        c->ex[k] = (int32_t)((2 * sx[k] + n[k]) / (2 * n[k]));
        c->ey[k] = (int32_t)((2 * sy[k] + n[k]) / (2 * n[k]));
        if (c->labels[(int64_t)c->ey[k] * c->W + c->ex[k]] != k) proj[nproj++] = k;
    }
#pragma omp parallel for schedule(dynamic) num_threads(threads)
    for (int i = 0; i < nproj; i++) project_center(c, proj[i]);
    c->projections = nproj;
    free(n); free(sx); free(sy); free(sl); free(sa); free(sb); free(proj);
}

int64_t orc_assign_rows(orc_ctx *c, int threads)
{
    int64_t N = (int64_t)c->H * c->W;
    int32_t *out = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int64_t orphans = 0;
#pragma omp parallel num_threads(threads) reduction(+ : orphans)
    {
        int *cand = (int *)malloc(sizeof(int) * (size_t)c->Keff);
#pragma omp for schedule(dynamic)
        for (int y = 0; y < c->H; y++) {
            int nc = 0; /* clusters whose window holds row y, ascending k */
            for (int k = 0; k < c->Keff; k++)
                if (in_window(y, c->n[k], c->sy[k], N, c->K)) cand[nc++] = k;
            for (int x = 0; x < c->W; x++) {
                int64_t p = (int64_t)y * c->W + x;
                double best = INFINITY;
                int lab = c->labels[p];
                for (int i = 0; i < nc; i++) {
                    int k = cand[i];
                    if (!in_window(x, c->n[k], c->sx[k], N, c->K)) continue;
                    double D = orc_distance(c, x, y, k, NULL);
                    if (D < best) {
                        best = D;
                        lab = k;
                    }
                }
                if (best == INFINITY) orphans++;
                out[p] = lab;
            }
        }
        free(cand);
    }
    memcpy(c->labels, out, sizeof(int32_t) * (size_t)N);
    free(out);
    c->orphans = orphans;
    return orphans;
}

int orc_iterate_rows(orc_ctx *c, int iters, int threads)
{
    for (int it = 0; it < iters; it++) {
        orc_assign_rows(c, threads);
        update_parallel(c, threads);
    }
    return 0;
}

/* Label of each listed pixel as the assignment would give it, found by
 * testing every cluster's window (pixel-centric); used to check single pixels
 * of large images.  out_label gets the argmin (smallest k on ties, previous
 * label when no window covers the pixel), out_d its distance (inf if none). */
void orc_assign_pixels(const orc_ctx *c, const int64_t *pix, int64_t M, int32_t *out_label,
                       double *out_d)
{
    int64_t N = (int64_t)c->H * c->W;
    for (int64_t i = 0; i < M; i++) {
        int64_t p = pix[i];
        int x = (int)(p % c->W), y = (int)(p / c->W);
        double best = INFINITY;
        int lab = c->labels[p];
        for (int k = 0; k < c->Keff; k++) {
            if (!in_window(x, c->n[k], c->sx[k], N, c->K)) continue;
            if (!in_window(y, c->n[k], c->sy[k], N, c->K)) continue;
            double D = orc_distance(c, x, y, k, NULL);
            if (D < best) {
                best = D;
                lab = k;
            }
        }
        out_label[i] = lab;
        out_d[i] = best;
    }
}

/* ------------------------------------------------------------------------ */
/* Connectivity enforcement (not part of the paper).                         */
/*   1. 4-connected components of equal label; a component's seed is its     */
/*      smallest raster index.                                               */
/*   2. A component is small iff its size <= floor(N / (4K)).                */
/*   3. A small component whose seed s is not pixel 0 is absorbed by the     */
/*      component holding s-1 (if x(s) > 0) or s-W (otherwise); these have   */
/*      smaller seeds.  It takes the identity that component ends up with.   */
/*   4. Surviving components are numbered 0.. in raster order of seeds.      */
/* ------------------------------------------------------------------------ */

int32_t orc_connectivity(const int32_t *labels, int H, int W, int K, int32_t *out)
{
    int64_t N = (int64_t)H * W;
    int64_t *comp = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);  /* pixel -> component */
    int64_t *seed = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);  /* component -> seed */
    int64_t *size = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t p = 0; p < N; p++) comp[p] = -1;
    int64_t ncomp = 0;
    for (int64_t s = 0; s < N; s++) {
        if (comp[s] >= 0) continue;
        int64_t id = ncomp++;
        seed[id] = s;
        int64_t top = 0;
        stack[top++] = s;
        comp[s] = id;
        while (top > 0) {
            int64_t q = stack[--top];
            size[id]++;
            int64_t qx = q % W, qy = q / W;
            int64_t nb[4];
            int nn = 0;
            if (qx > 0) nb[nn++] = q - 1;
            if (qx < W - 1) nb[nn++] = q + 1;
            if (qy > 0) nb[nn++] = q - W;
            if (qy < H - 1) nb[nn++] = q + W;
            for (int j = 0; j < nn; j++) {
                int64_t t = nb[j];
                if (comp[t] < 0 && labels[t] == labels[q]) {
                    comp[t] = id;
                    stack[top++] = t;
                }
            }
        }
    }
    /* Components were discovered in raster order of their seeds, so a
     * component's absorbing neighbour always has a smaller id. */
    int64_t T = N / (4 * (int64_t)K);
    int64_t *final_id = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncomp);
    int64_t *number = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncomp);
    int32_t nlab = 0;
    for (int64_t id = 0; id < ncomp; id++) {
        int64_t s = seed[id];
        int small = size[id] <= T && s != 0;
        if (small) {
            int64_t nbp = (s % W) > 0 ? s - 1 : s - W;
            final_id[id] = final_id[comp[nbp]];
        } else {
            final_id[id] = id;
            number[id] = nlab++;
        }
    }
    for (int64_t p = 0; p < N; p++) out[p] = (int32_t)number[final_id[comp[p]]];
    free(comp); free(seed); free(size); free(stack); free(final_id); free(number);
    return nlab;
}

/* ------------------------------------------------------------------------ */
/* Multi-scale boundary map (Sec. III-A2: boundary maps of decompositions at  */
/* several scales are averaged into a confidence map).  Pixel p is a boundary */
/* pixel of a decomposition iff one of its 4-neighbours carries another      */
/* label; the map is the fraction of the `count` decompositions in which p is */
/* a boundary pixel: (number of decompositions) / count, in single precision. */
/* ------------------------------------------------------------------------ */

void orc_boundary_map(const int32_t *const *labels, int count, int H, int W, float *out)
{
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int64_t p = (int64_t)y * W + x;
            int hits = 0;
            for (int i = 0; i < count; i++) {
                const int32_t *l = labels[i];
                int b = 0;
                if (x > 0 && l[p - 1] != l[p]) b = 1;
                if (x < W - 1 && l[p + 1] != l[p]) b = 1;
                if (y > 0 && l[p - W] != l[p]) b = 1;
                if (y < H - 1 && l[p + W] != l[p]) b = 1;
                hits += b;
            }
            out[p] = (float)hits / (float)count;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Superpixel quality metrics against a ground-truth segmentation, Eq. 5-8.  */
/* Boundary pixels are pixels with a 4-neighbour of another label.           */
/*   BR  (Eq. 5): fraction of ground-truth boundary pixels p with a          */
/*        superpixel boundary pixel q at Euclidean distance ||p-q|| < eps.    */
/*   ASA (Eq. 6): sum over superpixels of the largest overlap with one        */
/*        ground-truth segment, over the number of pixels.                    */
/*   UE  (Eq. 7): sum over segments G_i and superpixels S_k meeting G_i of    */
/*        |S_k - G_i|, over the number of pixels.                             */
/*   CO  (Eq. 8): (1/|I|) sum_k 4 pi |S_k|^2 / |P(S_k)|^2, the perimeter      */
/*        being the number of pixel edges between S_k and the rest of the     */
/*        image, the image border included.                                   */
/* Labels in [0, n_labels), ground truth in [0, n_gt).                        */
/* ------------------------------------------------------------------------ */

static int is_boundary(const int32_t *l, int H, int W, int x, int y)
{
    int64_t p = (int64_t)y * W + x;
    if (x > 0 && l[p - 1] != l[p]) return 1;
    if (x < W - 1 && l[p + 1] != l[p]) return 1;
    if (y > 0 && l[p - W] != l[p]) return 1;
    if (y < H - 1 && l[p + W] != l[p]) return 1;
    return 0;
}

void orc_quality(const int32_t *labels, int n_labels, const int32_t *gt, int n_gt, int H, int W,
                 double eps, double *br, double *asa, double *ue, double *co)
{
    int64_t N = (int64_t)H * W;
    /* Eq. 5 */
    int r = (int)ceil(eps);
    int64_t gb = 0, hit = 0;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            if (!is_boundary(gt, H, W, x, y)) continue;
            gb++;
            int found = 0;
            for (int dy = -r; dy <= r && !found; dy++)
                for (int dx = -r; dx <= r && !found; dx++) {
                    int qx = x + dx, qy = y + dy;
                    if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                    if (sqrt((double)(dx * dx + dy * dy)) >= eps) continue;
                    if (is_boundary(labels, H, W, qx, qy)) found = 1;
                }
            hit += found;
        }
    *br = gb ? (double)hit / (double)gb : 1.0;
    /* overlaps |S_k n G_i| */
    int64_t *ov = (int64_t *)calloc((size_t)n_labels * (size_t)n_gt, sizeof(int64_t));
    int64_t *area = (int64_t *)calloc((size_t)n_labels, sizeof(int64_t));
    int64_t *perim = (int64_t *)calloc((size_t)n_labels, sizeof(int64_t));
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int64_t p = (int64_t)y * W + x;
            int k = labels[p];
            ov[(int64_t)k * n_gt + gt[p]]++;
            area[k]++;
            /* edges to each of the 4 sides: image border or another label */
            perim[k] += (x == 0 || labels[p - 1] != k) + (x == W - 1 || labels[p + 1] != k) +
                        (y == 0 || labels[p - W] != k) + (y == H - 1 || labels[p + W] != k);
        }
    /* Eq. 6 and Eq. 7 */
    int64_t asa_num = 0, ue_num = 0;
    for (int k = 0; k < n_labels; k++) {
        int64_t best = 0;
        for (int i = 0; i < n_gt; i++) {
            int64_t o = ov[(int64_t)k * n_gt + i];
            if (o > best) best = o;
            if (o > 0) ue_num += area[k] - o;
        }
        asa_num += best;
    }
    *asa = (double)asa_num / (double)N;
    *ue = (double)ue_num / (double)N;
    /* Eq. 8 */
    double s = 0.0;
    for (int k = 0; k < n_labels; k++) {
        if (area[k] == 0) continue;
        double a = (double)area[k], pr = (double)perim[k];
        s += 4.0 * M_PI * a * a / (pr * pr);
    }
    *co = s / (double)N;
    free(ov); free(area); free(perim);
}

/* ------------------------------------------------------------------------ */
/* A contour prior computed from the image itself.  Sec. II-E lets SCALP take
 * any soft prior with values in [0, 1] (or a binary one) from any contour
 * detector; the detector the paper uses needs trained models.  Reading used
 * here: the magnitude of the CIELab gradient, divided by its maximum over the
 * image (all zero when the image is flat).  Per channel and axis the
 * derivative is the central difference (f[i+1] - f[i-1]) / 2 inside the image,
 * the one-sided difference f[1] - f[0] or f[n-1] - f[n-2] at the two ends, and
 * 0 along an axis of length 1.  The magnitude is the Euclidean norm of the six
 * derivatives. */
static double axis_derivative(const double *f, int64_t stride, int i, int n)
{
    if (n < 2) return 0.0;
    if (i == 0) return f[stride] - f[0];
    if (i == n - 1) return f[0] - f[-stride];
    return (f[stride] - f[-stride]) / 2.0;
}

void orc_gradient_prior(const double *L, const double *A, const double *B, int H, int W,
                        double *out)
{
    const double *ch[3] = {L, A, B};
    double gmax = 0.0;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int64_t p = (int64_t)y * W + x;
            double s = 0.0;
            for (int c = 0; c < 3; c++) {
                double gx = axis_derivative(ch[c] + p, 1, x, W);
                double gy = axis_derivative(ch[c] + p, W, y, H);
                s += gx * gx + gy * gy;
            }
            out[p] = sqrt(s);
            if (out[p] > gmax) gmax = out[p];
        }
    int64_t N = (int64_t)H * W;
    for (int64_t p = 0; p < N; p++) out[p] = gmax > 0.0 ? out[p] / gmax : 0.0;
}

/* ======================================================================== */
/* Supervoxels: SCALP on a video volume (the extension the paper's           */
/* conclusion names as future work).  Readings, each the 2-D rule taken      */
/* axis by axis:                                                             */
/*   - volume T frames x H x W, voxel (x, y, t) at index (t*H + y)*W + x;    */
/*   - r = cbrt(N/K) (host C library); grid nx = max(1, round(W/r)),         */
/*     ny = max(1, round(H/r)), nt = max(1, round(T/r)); voxel starts in     */
/*     cell floor(t*nt/T)*ny*nx + floor(y*ny/H)*nx + floor(x*nx/W);          */
/*   - window: |v - s/n| <= r per axis with r the real cube root of N/K,    */
/*     i.e. K*|n*v - s|^3 <= N*n^3, decided exactly in 128-bit integers;     */
/*   - path: 3-D digital segment, traced from the lexicographically smaller  */
/*     end (x, then y, then t); the major axis is the one with the largest   */
/*     |delta| (ties: x, then y, then t); step i moves each other axis by    */
/*     round-half-up(i*|delta_j|/ns); |P| = ns + 1;                          */
/*   - D as Eq. 3 with the squared 3-D distance; projection (Eq. 4) in exact */
/*     integers, ties to the smallest voxel index; no connectivity step.     */
/* ======================================================================== */
typedef struct {
    int32_t T, H, W, K;
    int32_t nx, ny, nt, Keff;
    double m, lambda, sigma, gamma; /* gamma < 0 selects 2r */
    double r;                       /* filled by orc_vinit: cbrt(N/K) */
    const double *L, *A, *B, *C;    /* N each */
    int32_t *labels;                /* N */
    int64_t *n, *sx, *sy, *st;      /* Keff */
    double *cL, *cA, *cB;           /* Keff */
    int32_t *ex, *ey, *et;          /* Keff: path endpoint */
    int64_t orphans, projections;
} orc_vctx;

void orc_vgrid_dims(int T, int H, int W, int K, int *nx, int *ny, int *nt, double *r)
{
    double N = (double)T * (double)H * (double)W;
    double rr = cbrt(N / (double)K);
    int d[3] = {W, H, T}, g[3];
    for (int i = 0; i < 3; i++) {
        g[i] = (int)floor((double)d[i] / rr + 0.5);
        if (g[i] < 1) g[i] = 1;
        if (g[i] > d[i]) g[i] = d[i];
    }
    *nx = g[0];
    *ny = g[1];
    *nt = g[2];
    *r = rr;
}

int orc_vpath(int px, int py, int pt, int ex, int ey, int et, int32_t *xyz)
{
    int p[3] = {px, py, pt}, e[3] = {ex, ey, et}, a[3], b[3];
    int p_first = px < ex || (px == ex && (py < ey || (py == ey && pt <= et)));
    for (int j = 0; j < 3; j++) {
        a[j] = p_first ? p[j] : e[j];
        b[j] = p_first ? e[j] : p[j];
    }
    int ad[3], sg[3], major = 0;
    for (int j = 0; j < 3; j++) {
        int d = b[j] - a[j];
        ad[j] = d < 0 ? -d : d;
        sg[j] = d < 0 ? -1 : 1;
        if (ad[j] > ad[major]) major = j;
    }
    int ns = ad[major];
    for (int i = 0; i <= ns; i++)
        for (int j = 0; j < 3; j++) {
            int off = j == major ? i : (ns ? (2 * i * ad[j] + ns) / (2 * ns) : 0);
            xyz[3 * i + j] = a[j] + sg[j] * off;
        }
    return ns + 1;
}

/* |v - s/n| <= r with r^3 = N/K, i.e. K*|n*v - s|^3 <= N*n^3, exactly.  A
 * volume holds at most 2^30 voxels, so r <= 2^10 and n, N <= 2^30: a distance
 * |n*v - s| above 2^10*n is outside, and below it both q^3 and N*n^3 are at
 * most 2^120; K*q^3 <= N*n^3 holds iff q^3 <= floor(N*n^3 / K) (q^3 is an
 * integer). */
static int vin_window(int64_t v, int64_t n, int64_t s, int64_t N, int64_t K)
{
    i128 d = (i128)n * v - (i128)s;
    u128 q = (u128)(d < 0 ? -d : d);
    if (q > (u128)n * 1024u) return 0;
    u128 rhs = (u128)N * (u128)n * (u128)n * (u128)n / (u128)K;
    return q * q * q <= rhs;
}

int orc_vin_window(int64_t v, int64_t n, int64_t s, int64_t N, int64_t K)
{
    return vin_window(v, n, s, N, K);
}

static double vdc_at(const orc_vctx *c, int64_t q, int k)
{
    double dl = c->L[q] - c->cL[k];
    double da = c->A[q] - c->cA[k];
    double db = c->B[q] - c->cB[k];
    return dl * dl + da * da + db * db;
}

double orc_vdistance(const orc_vctx *c, int x, int y, int t, int k, int32_t *path_len)
{
    int64_t W = c->W, H = c->H;
    int maxd = c->W > c->H ? c->W : c->H;
    if (c->T > maxd) maxd = c->T;
    int32_t *xyz = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(maxd + 1));
    int len = orc_vpath(x, y, t, c->ex[k], c->ey[k], c->et[k], xyz);
    double sum_dc = 0.0, sum_w = 0.0;
    for (int i = 0; i < len; i++) {
        int64_t q = ((int64_t)xyz[3 * i + 2] * H + xyz[3 * i + 1]) * W + xyz[3 * i];
        sum_dc += vdc_at(c, q, k);
        double cq = c->C[q];
        sum_w += 1.0 - exp(-(cq * cq) / (c->sigma * c->sigma));
    }
    free(xyz);
    int64_t p = ((int64_t)t * H + y) * W + x;
    double dc_path = c->lambda * vdc_at(c, p, k) + (1.0 - c->lambda) * sum_dc / len; /* Eq. 1 */
    double d_contour = 1.0 + c->gamma / len * sum_w;                               /* Eq. 2 */
    double xk = (double)c->sx[k] / (double)c->n[k];
    double yk = (double)c->sy[k] / (double)c->n[k];
    double tk = (double)c->st[k] / (double)c->n[k];
    double ds = (x - xk) * (x - xk) + (y - yk) * (y - yk) + (t - tk) * (t - tk);
    if (path_len) *path_len = len;
    return dc_path * d_contour + ds * (c->m * c->m) / (c->r * c->r); /* Eq. 3 */
}

static void vproject_center(orc_vctx *c, int k)
{
    int64_t N = (int64_t)c->T * c->H * c->W, HW = (int64_t)c->H * c->W;
    i128 best = -1;
    int64_t best_p = -1;
    for (int64_t p = 0; p < N; p++) {
        if (c->labels[p] != k) continue;
        int64_t t = p / HW, y = (p % HW) / c->W, x = p % c->W;
        i128 dx = (i128)c->n[k] * x - c->sx[k];
        i128 dy = (i128)c->n[k] * y - c->sy[k];
        i128 dt = (i128)c->n[k] * t - c->st[k];
        i128 d2 = dx * dx + dy * dy + dt * dt;
        if (best_p < 0 || d2 < best) {
            best = d2;
            best_p = p;
        }
    }
    c->ex[k] = (int32_t)(best_p % c->W);
    c->ey[k] = (int32_t)((best_p % HW) / c->W);
    c->et[k] = (int32_t)(best_p / HW);
}

void orc_vupdate(orc_vctx *c)
{
    int64_t N = (int64_t)c->T * c->H * c->W, HW = (int64_t)c->H * c->W;
    int K = c->Keff;
    int64_t *n = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *sx = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *sy = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *st = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    double *sl = (double *)calloc((size_t)K, sizeof(double));
    double *sa = (double *)calloc((size_t)K, sizeof(double));
    double *sb = (double *)calloc((size_t)K, sizeof(double));
    for (int64_t p = 0; p < N; p++) {
        int k = c->labels[p];
        n[k] += 1;
        sx[k] += p % c->W;
        sy[k] += (p % HW) / c->W;
        st[k] += p / HW;
        sl[k] += c->L[p];
        sa[k] += c->A[p];
        sb[k] += c->B[p];
    }
    c->projections = 0;
    for (int k = 0; k < K; k++) {
        if (n[k] == 0) continue; /* empty cluster: unchanged */
        c->n[k] = n[k];
        c->sx[k] = sx[k];
        c->sy[k] = sy[k];
        c->st[k] = st[k];
        c->cL[k] = sl[k] / (double)n[k];
        c->cA[k] = sa[k] / (double)n[k];
        c->cB[k] = sb[k] / (double)n[k];
        c->ex[k] = (int32_t)((2 * sx[k] + n[k]) / (2 * n[k]));
        c->ey[k] = (int32_t)((2 * sy[k] + n[k]) / (2 * n[k]));
        c->et[k] = (int32_t)((2 * st[k] + n[k]) / (2 * n[k]));
        if (c->labels[((int64_t)c->et[k] * c->H + c->ey[k]) * c->W + c->ex[k]] != k) {
            vproject_center(c, k);
            c->projections++;
        }
    }
    free(n); free(sx); free(sy); free(st); free(sl); free(sa); free(sb);
}

int orc_vinit(orc_vctx *c)
{
    int64_t N = (int64_t)c->T * c->H * c->W, HW = (int64_t)c->H * c->W;
    if (c->T < 1 || c->H < 1 || c->W < 1 || c->K < 1 || c->K > N) return -1;
    if (N > ((int64_t)1 << 30)) return -1; /* the window test's 128-bit bound */
    orc_vgrid_dims(c->T, c->H, c->W, c->K, &c->nx, &c->ny, &c->nt, &c->r);
    if (c->gamma < 0) c->gamma = 2.0 * c->r;
    c->Keff = c->nx * c->ny * c->nt;
    for (int64_t p = 0; p < N; p++) {
        int64_t t = p / HW, y = (p % HW) / c->W, x = p % c->W;
        int cx = (int)(x * c->nx / c->W);
        int cy = (int)(y * c->ny / c->H);
        int ct = (int)(t * c->nt / c->T);
        c->labels[p] = (ct * c->ny + cy) * c->nx + cx;
    }
    orc_vupdate(c);
    c->orphans = 0;
    return 0;
}

/* Window bounds along one axis: every v in [lo, hi] of [0, lim) passes (the
 * window is an interval; the double bounds only seed the exact search). */
static void vwindow(const orc_vctx *c, int64_t n, int64_t s, int lim, int *lo, int *hi)
{
    int64_t N = (int64_t)c->T * c->H * c->W;
    double ctr = (double)s / (double)n;
    int a = (int)floor(ctr - c->r) - 1, b = (int)ceil(ctr + c->r) + 1;
    if (a < 0) a = 0;
    if (b > lim - 1) b = lim - 1;
    while (a <= b && !vin_window(a, n, s, N, c->K)) a++;
    while (b >= a && !vin_window(b, n, s, N, c->K)) b--;
    *lo = a;
    *hi = b;
}

int64_t orc_vassign(orc_vctx *c, double *dbest)
{
    int64_t N = (int64_t)c->T * c->H * c->W;
    double *d = (double *)malloc(sizeof(double) * (size_t)N);
    for (int64_t p = 0; p < N; p++) d[p] = INFINITY;
    for (int k = 0; k < c->Keff; k++) {
        int x0, x1, y0, y1, t0, t1;
        vwindow(c, c->n[k], c->sx[k], c->W, &x0, &x1);
        vwindow(c, c->n[k], c->sy[k], c->H, &y0, &y1);
        vwindow(c, c->n[k], c->st[k], c->T, &t0, &t1);
        for (int t = t0; t <= t1; t++)
            for (int y = y0; y <= y1; y++)
                for (int x = x0; x <= x1; x++) {
                    double D = orc_vdistance(c, x, y, t, k, NULL);
                    int64_t p = ((int64_t)t * c->H + y) * c->W + x;
                    if (D < d[p]) {
                        d[p] = D;
                        c->labels[p] = k;
                    }
                }
    }
    int64_t orphans = 0;
    for (int64_t p = 0; p < N; p++) {
        if (d[p] == INFINITY) orphans++;
        if (dbest) dbest[p] = d[p];
    }
    free(d);
    c->orphans = orphans;
    return orphans;
}

int orc_viterate(orc_vctx *c, int iters)
{
    for (int it = 0; it < iters; it++) {
        orc_vassign(c, NULL);
        orc_vupdate(c);
    }
    return 0;
}
