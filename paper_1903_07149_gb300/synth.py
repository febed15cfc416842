"""Seeded synthetic inputs shaped like the paper's workloads.

The paper evaluates on the Berkeley Segmentation Dataset (321x481 RGB images,
Sec. III-A1) with a contour prior from a structured-forest edge detector
(Sec. III-A3).  Neither is available here, so these generators stand in for
them: a seeded Voronoi partition gives piecewise-homogeneous colour regions, and
the partition's own boundaries, blurred and noised, give a soft contour map in
[0, 1] (Sec. II-E allows any soft or binary prior).

This module holds none of SCALP's arithmetic.  It is the one module that both
the CUDA path's tests and the CPU oracle's tests draw their inputs from.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "Workload",
    "voronoi_image",
    "single_image_config",
    "batch_configs",
    "batch_images",
    "serving_arrivals",
    "voronoi_video",
    "WORKLOADS",
    "VIDEO_WORKLOADS",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    H: int
    W: int
    K: int
    n_cells: int
    gradient: bool
    noise_sigma: float
    seed: int
    iters: int = 10


# Single-image workloads.  "bsd" copies the BSD image shape (Sec. III-A1);
# "hd" and "uhd" are the larger single-image sizes the throughput is quoted on.
WORKLOADS = {
    "bsd_321x481_k400": Workload("bsd_321x481_k400", 321, 481, 400, 40, False, 8.0, 1000),
    "hd_1080x1920_k2000": Workload("hd_1080x1920_k2000", 1080, 1920, 2000, 300, True, 6.0, 1001),
    "uhd_2160x3840_k10000": Workload("uhd_2160x3840_k10000", 2160, 3840, 10000, 1200, True, 6.0, 1002),
}


def _gauss_kernel(sigma: float, radius: int) -> np.ndarray:
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    return k / k.sum()


def _blur_reflect(img: np.ndarray, sigma: float = 1.0, radius: int = 3) -> np.ndarray:
    """Separable Gaussian blur with mirror (reflect, edge sample repeated) borders."""
    k = _gauss_kernel(sigma, radius)
    out = img.astype(np.float64)
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (radius, radius)
        p = np.pad(out, pad, mode="symmetric")
        acc = np.zeros_like(out)
        n = out.shape[axis]
        for i, w in enumerate(k):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(i, i + n)
            acc += w * p[tuple(sl)]
        out = acc
    return out


def _voronoi_cells(H: int, W: int, seeds_xy: np.ndarray) -> np.ndarray:
    """Nearest-seed index for every pixel centre (x, y)."""
    from scipy.spatial import cKDTree

    tree = cKDTree(seeds_xy)
    ys, xs = np.mgrid[0:H, 0:W]
    pts = np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.float64)
    _, idx = tree.query(pts, k=1, workers=-1)
    return idx.reshape(H, W).astype(np.int32)


def voronoi_image(H: int, W: int, n_cells: int, *, gradient: bool, noise_sigma: float,
                  seed: int, contour_noise: float = 0.05):
    """Return (rgb uint8 HxWx3, contour float32 HxW in [0,1], cells int32 HxW).

    * n_cells seeds uniform in [0,W)x[0,H); every pixel takes its nearest seed.
    * gradient=False: one uniform random colour per cell in [0,255]^3.
      gradient=True: a base colour uniform in [40,215]^3 plus a linear ramp,
      a 3x2 matrix with entries U[-40,40] per cell radius R=sqrt(HW/n_cells)
      applied to (pixel - seed)/R.
    * then additive Gaussian noise N(0, noise_sigma^2), rounded and clipped.
    * contour: 1 where a 4-neighbour lies in another cell, blurred with a
      sigma=1 Gaussian (radius 3), divided by its maximum, plus U[0,0.05),
      clipped to [0,1].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    seeds = np.stack([rng.uniform(0, W, n_cells), rng.uniform(0, H, n_cells)], axis=1)
    cells = _voronoi_cells(H, W, seeds)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    if gradient:
        base = rng.uniform(40, 215, size=(n_cells, 3))
        G = rng.uniform(-40, 40, size=(n_cells, 3, 2))
        R = np.sqrt(H * W / n_cells)
        dx = (xs - seeds[cells, 0]) / R
        dy = (ys - seeds[cells, 1]) / R
        col = base[cells] + G[cells, :, 0] * dx[..., None] + G[cells, :, 1] * dy[..., None]
    else:
        base = rng.uniform(0, 255, size=(n_cells, 3))
        col = base[cells]
    col = col + rng.normal(0.0, noise_sigma, size=col.shape)
    rgb = np.clip(np.rint(col), 0, 255).astype(np.uint8)

    edge = np.zeros((H, W), dtype=np.float64)
    diff_x = cells[:, 1:] != cells[:, :-1]
    diff_y = cells[1:, :] != cells[:-1, :]
    edge[:, 1:][diff_x] = 1.0
    edge[:, :-1][diff_x] = 1.0
    edge[1:, :][diff_y] = 1.0
    edge[:-1, :][diff_y] = 1.0
    blurred = _blur_reflect(edge, 1.0, 3)
    mx = blurred.max()
    if mx > 0:
        blurred = blurred / mx
    contour = np.clip(blurred + rng.uniform(0.0, contour_noise, size=(H, W)), 0.0, 1.0)
    return rgb, contour.astype(np.float32), cells


def single_image_config(name: str):
    """(workload, rgb, contour) for one of the named single-image workloads."""
    w = WORKLOADS[name]
    rgb, contour, _ = voronoi_image(w.H, w.W, w.n_cells, gradient=w.gradient,
                                    noise_sigma=w.noise_sigma, seed=w.seed)
    return w, rgb, contour


def small_image(H: int, W: int, seed: int, n_cells: int | None = None, gradient: bool = True):
    """A small test image built like the HD workload (for parity tests)."""
    if n_cells is None:
        n_cells = max(2, (H * W) // 4000)
    rgb, contour, cells = voronoi_image(H, W, n_cells, gradient=gradient, noise_sigma=6.0,
                                        seed=seed)
    return rgb, contour, cells


def batch_configs(n_images: int = 64, seed: int = 3000):
    """Sizes of the uneven batch: H~U{240..1080}, W~U{320..1920}, grid step
    S~U[12,30], K=round(HW/S^2); cells scale with area like the HD workload."""
    out = []
    for i in range(n_images):
        rng = np.random.Generator(np.random.PCG64(seed + i))
        H = int(rng.integers(240, 1081))
        W = int(rng.integers(320, 1921))
        S = float(rng.uniform(12.0, 30.0))
        K = max(1, int(round(H * W / (S * S))))
        n_cells = max(2, int(round(300 * H * W / 2_073_600)))
        out.append(Workload(f"batch{i}_{H}x{W}_k{K}", H, W, K, n_cells, True, 6.0, seed + i))
    return out


def batch_images(workloads):
    """(rgb list, contour list) for a list of workloads (e.g. batch_configs())."""
    rgbs, cons = [], []
    for w in workloads:
        rgb, con, _ = voronoi_image(w.H, w.W, w.n_cells, gradient=w.gradient,
                                    noise_sigma=w.noise_sigma, seed=w.seed)
        rgbs.append(rgb)
        cons.append(con)
    return rgbs, cons


def serving_arrivals(n_requests: int = 2000, rate_hz: float = 500.0, seed: int = 4000):
    """Poisson arrival times (s) and a size class per request: 0 = batch mix, 1 = UHD."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    kind = (rng.uniform(size=n_requests) < 0.10).astype(np.int32)
    return np.cumsum(gaps), kind


# Video volumes for the supervoxel form: (T, H, W, K, n_cells, seed).
VIDEO_WORKLOADS = {
    "video_32x240x320_k2000": (32, 240, 320, 2000, 40, 5000),
}


def voronoi_video(T: int, H: int, W: int, n_cells: int, *, seed: int, noise_sigma: float = 6.0,
                  contour_noise: float = 0.05):
    """Return (rgb uint8 TxHxWx3, contour float32 TxHxW in [0,1], cells int32 TxHxW).

    Moving Voronoi cells: seeds uniform in [0,W)x[0,H) drift with a velocity
    uniform in [-1.5, 1.5] pixels per frame (reflected at the borders); every
    voxel takes its frame's nearest seed.  Colours as the gradient images of
    voronoi_image (base U[40,215]^3 plus a per-cell linear ramp), then Gaussian
    noise.  The contour of each frame is its cell boundary, blurred, normalised
    and noised as in voronoi_image."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = np.stack([rng.uniform(0, W, n_cells), rng.uniform(0, H, n_cells)], axis=1)
    vel = rng.uniform(-1.5, 1.5, size=(n_cells, 2))
    base = rng.uniform(40, 215, size=(n_cells, 3))
    G = rng.uniform(-40, 40, size=(n_cells, 3, 2))
    R = np.sqrt(H * W / n_cells)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    rgb = np.empty((T, H, W, 3), np.uint8)
    contour = np.empty((T, H, W), np.float32)
    cells = np.empty((T, H, W), np.int32)
    for t in range(T):
        p = pos + vel * t
        for j, lim in ((0, W), (1, H)):  # reflect into [0, lim)
            period = 2.0 * lim
            q = np.mod(p[:, j], period)
            p[:, j] = np.where(q < lim, q, period - q - 1e-9)
        c = _voronoi_cells(H, W, p)
        col = base[c] + G[c, :, 0] * ((xs - p[c, 0]) / R)[..., None] + G[c, :, 1] * ((ys - p[c, 1]) / R)[..., None]
        col = col + rng.normal(0.0, noise_sigma, size=col.shape)
        rgb[t] = np.clip(np.rint(col), 0, 255).astype(np.uint8)
        edge = np.zeros((H, W))
        dx = c[:, 1:] != c[:, :-1]
        dy = c[1:, :] != c[:-1, :]
        edge[:, 1:][dx] = 1.0
        edge[:, :-1][dx] = 1.0
        edge[1:, :][dy] = 1.0
        edge[:-1, :][dy] = 1.0
        b = _blur_reflect(edge, 1.0, 3)
        if b.max() > 0:
            b = b / b.max()
        contour[t] = np.clip(b + rng.uniform(0.0, contour_noise, size=(H, W)), 0.0, 1.0)
        cells[t] = c
    return rgb, contour, cells
