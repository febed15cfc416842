"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

None of these compares the oracle with itself: each checks a closed form, an
invariant, a special case the paper states, a library routine, published
colour values, or brute force on tiny inputs.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact_rationals import cube_root_convergents
from paper_1903_07149_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# CIELab (Sec. II-A names CIELab; the conversion itself is the sRGB/CIE
# standard).  Published L*a*b* of the sRGB primaries under D65.
# --------------------------------------------------------------------------
def test_lab_published_values():
    rgb = np.array([[255, 255, 255], [0, 0, 0], [255, 0, 0], [0, 255, 0], [0, 0, 255]],
                   np.uint8)
    L, A, B = oracle.lab_from_rgb(rgb)
    assert abs(L[0] - 100) < 1e-9 and abs(A[0]) < 1e-9 and abs(B[0]) < 1e-9
    assert abs(L[1]) < 1e-12 and abs(A[1]) < 1e-12 and abs(B[1]) < 1e-12
    expected = {2: (53.2408, 80.0925, 67.2032), 3: (87.7347, -86.1827, 83.1793),
                4: (32.2970, 79.1875, -107.8602)}
    for i, (l, a, b) in expected.items():
        assert abs(L[i] - l) < 2e-3 and abs(A[i] - a) < 2e-3 and abs(B[i] - b) < 2e-3


def test_lab_gray_axis_and_monotone():
    v = np.arange(256, dtype=np.uint8)
    rgb = np.stack([v, v, v], axis=1)
    L, A, B = oracle.lab_from_rgb(rgb)
    assert np.all(np.abs(A) < 1e-9) and np.all(np.abs(B) < 1e-9)
    assert np.all(np.diff(L) > 0)
    # Low end is the linear segment of both transfer functions:
    # Y = (v/255)/12.92 and L = 116 * (Y/(3*(6/29)^2) + 4/29) - 16 = (29/3)^3 * Y
    Y = (1 / 255) / 12.92
    assert abs(L[1] - (29 / 3) ** 3 * Y) < 1e-9


# --------------------------------------------------------------------------
# Grid (Sec. II-A: blocks of size r = sqrt(N/k)).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("H,W,K,exp", [(321, 481, 400, (24, 16)), (1080, 1920, 2000, (60, 34)),
                                       (2160, 3840, 10000, (133, 75)), (64, 96, 24, (6, 4)),
                                       (5, 5, 25, (5, 5)), (1, 7, 1, (3, 1))])
def test_grid_dims(H, W, K, exp):
    assert oracle.grid_dims(H, W, K) == exp


# --------------------------------------------------------------------------
# Linear path (Sec. II-B; Bresenham's digital segment).
# --------------------------------------------------------------------------
def _check_path(p, e):
    pts = oracle.path(p, e)
    dx, dy = e[0] - p[0], e[1] - p[1]
    ns = max(abs(dx), abs(dy))
    assert len(pts) == ns + 1
    s = {tuple(q) for q in pts}
    assert len(s) == ns + 1
    assert tuple(p) in s and tuple(e) in s
    # 8-connected, one step along the major axis each time
    steps = np.abs(np.diff(pts, axis=0))
    if ns:
        assert np.all(steps.max(axis=1) == 1)
    # every pixel is a nearest lattice point to the exact segment in its
    # major-axis column: |minor - exact| <= 1/2
    if ns:
        major = 0 if abs(dx) >= abs(dy) else 1
        for q in pts:
            t = Fraction(int(q[major] - p[major]), int(e[major] - p[major]))
            exact = p[1 - major] + t * (e[1 - major] - p[1 - major])
            assert abs(q[1 - major] - exact) <= Fraction(1, 2)
    # symmetric: the same set from either end
    back = {tuple(q) for q in oracle.path(e, p)}
    assert back == s


def test_path_properties_exhaustive_small():
    for ex in range(-6, 7):
        for ey in range(-6, 7):
            _check_path((0, 0), (ex, ey))
            _check_path((3, 5), (3 + ex, 5 + 2 * ey))


def test_path_properties_random():
    rng = np.random.default_rng(7)
    for _ in range(300):
        p = tuple(int(v) for v in rng.integers(0, 80, 2))
        e = tuple(int(v) for v in rng.integers(0, 80, 2))
        _check_path(p, e)


# --------------------------------------------------------------------------
# Window test (Algorithm 1: a (2r+1)x(2r+1) window centred on X_k).
# --------------------------------------------------------------------------
def test_window_predicate_exact():
    rng = np.random.default_rng(3)
    for _ in range(3000):
        N = int(rng.integers(10, 10_000_000))
        K = int(rng.integers(1, min(N, 20000) + 1))
        n = int(rng.integers(1, 5000))
        s = int(rng.integers(0, n * 4000))
        xk = Fraction(s, n)
        r2 = Fraction(N, K)
        # probe the integers around the window edge
        r = math.sqrt(N / K)
        for v in {math.floor(xk - r) - 1, math.floor(xk - r), math.ceil(xk - r),
                  math.floor(xk + r), math.ceil(xk + r), math.ceil(xk + r) + 1}:
            assert oracle.in_window(v, n, s, N, K) == ((v - xk) ** 2 <= r2)
    # huge clusters do not overflow
    N, K = 8_294_400, 10_000
    assert oracle.in_window(3839, N, N * 1919 + N // 2, N, K) is False
    assert oracle.in_window(1919, N, N * 1919 + N // 2, N, K) is True


# --------------------------------------------------------------------------
# Distance, Eq. 1-3, on hand-worked examples.
# --------------------------------------------------------------------------
def _golden_solver(g, lam, gamma):
    lab = tuple(np.array(g[c], dtype=np.float64) for c in ("L", "a", "b"))
    s = oracle.Solver(lab, np.array(g["C"], dtype=np.float64), g["K"], m=g["m"], lam=lam,
                      sigma=g["sigma"], gamma=gamma)
    for c in g["clusters"]:
        k = c["k"]
        s.n[k], s.sx[k], s.sy[k] = c["n"], c["sx"], c["sy"]
        s.cL[k], s.cA[k], s.cB[k] = c["color"]
        s.ex[k], s.ey[k] = c["endpoint"]
    return s


def test_distance_worked_examples():
    with open(os.path.join(GOLDEN, "distance_worked_examples.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        s = _golden_solver(g, case["lambda"], case["gamma"])
        assert s.r == 2.0
        c = g["clusters"][case["k"]]
        pth = oracle.path(tuple(case["p"]), tuple(c["endpoint"]))
        assert sorted(map(tuple, pth)) == sorted(map(tuple, case["path"]))
        D, plen = s.distance(case["p"][0], case["p"][1], case["k"])
        assert plen == len(case["path"])
        assert abs(D - case["D"]) <= 1e-12 * abs(case["D"]), case["name"]


# --------------------------------------------------------------------------
# Special case stated below Eq. 3: lambda=1, gamma=0 gives SLIC.
# A plain SLIC, written here with numpy, must give the same labels.
# --------------------------------------------------------------------------
def _slic_numpy(L, A, B, K, iters, m):
    H, W = L.shape
    N = H * W
    nx, ny = oracle.grid_dims(H, W, K)
    ys, xs = np.mgrid[0:H, 0:W]
    lab = (ys * ny // H) * nx + (xs * nx // W)
    feats = np.stack([L, A, B], axis=-1)

    def means(lab):
        Kc = nx * ny
        cnt = np.bincount(lab.ravel(), minlength=Kc)
        sx = np.bincount(lab.ravel(), weights=xs.ravel(), minlength=Kc).astype(np.int64)
        sy = np.bincount(lab.ravel(), weights=ys.ravel(), minlength=Kc).astype(np.int64)
        col = np.stack([np.bincount(lab.ravel(), weights=feats[..., c].ravel(), minlength=Kc)
                        for c in range(3)], axis=1)
        return cnt, sx, sy, col

    n, sx, sy, col = means(lab)
    col = col / n[:, None]
    for _ in range(iters):
        best = np.full((H, W), np.inf)
        new = lab.copy()
        for k in range(nx * ny):
            # window: K*(n*v - S)^2 <= N*n^2 per axis, with Python ints
            inx = K * (n[k] * xs - sx[k]) ** 2 <= N * n[k] ** 2
            iny = K * (n[k] * ys - sy[k]) ** 2 <= N * n[k] ** 2
            win = inx & iny
            dc = ((feats - col[k]) ** 2).sum(-1)
            ds = (xs - sx[k] / n[k]) ** 2 + (ys - sy[k] / n[k]) ** 2
            D = dc + ds * m * m * K / N
            upd = win & (D < best)
            best[upd] = D[upd]
            new[upd] = k
        lab = new
        n2, sx2, sy2, col2 = means(lab)
        keep = n2 > 0
        n[keep], sx[keep], sy[keep] = n2[keep], sx2[keep], sy2[keep]
        col[keep] = col2[keep] / n2[keep, None]
    return lab


def test_slic_special_case():
    rgb, contour, _ = synth.small_image(40, 56, seed=11, n_cells=6)
    L, A, B = oracle.lab_from_rgb(rgb)
    K = 14
    s = oracle.Solver((L, A, B), contour, K, lam=1.0, gamma=0.0)
    ref = _slic_numpy(L, A, B, K, iters=4, m=10.0)
    for it in range(4):
        s.iterate(1)
    # the two differ only by the order of FP64 roundings in d_s*m^2/r^2;
    # exact ties are impossible on this noisy image
    assert np.array_equal(s.labels, ref)


# --------------------------------------------------------------------------
# Constant image, no contour: D = m^2/r^2 * d_s.  With r an integer that
# divides H and W the grid is a fixed point (cells are the Voronoi regions of
# their centres under the window test).
# --------------------------------------------------------------------------
def test_constant_image_fixed_point():
    H, W, K = 64, 96, 24  # r = 16, 6 x 4 cells of 16 x 16
    lab = (np.full((H, W), 50.0), np.full((H, W), 10.0), np.full((H, W), -5.0))
    s = oracle.Solver(lab, np.zeros((H, W)), K)
    assert s.r == 16.0 and s.grid == (6, 4)
    ys, xs = np.mgrid[0:H, 0:W]
    cells = (ys // 16) * 6 + xs // 16
    c0 = s.centers().copy()
    assert np.allclose(c0[:, 0], (np.arange(24) % 6) * 16 + 7.5)
    assert np.allclose(c0[:, 1], (np.arange(24) // 6) * 16 + 7.5)
    for _ in range(3):
        s.iterate(1)
        assert np.array_equal(s.labels, cells)
        assert np.array_equal(s.centers(), c0)
        assert np.allclose(s.colors(), [50.0, 10.0, -5.0])
        assert s.projections == 0


# --------------------------------------------------------------------------
# Contour wall: a full column with C=1 and a large gamma.  A path that
# crosses the wall costs far more than one that does not, so no superpixel
# straddles it (Sec. II-D: the term keeps pixels from clusters behind a
# contour).
# --------------------------------------------------------------------------
def test_contour_wall_not_crossed():
    H, W, K = 48, 64, 12  # r = 16, 4 x 3 cells
    rng = np.random.default_rng(5)
    rgb = rng.integers(90, 166, size=(H, W, 3)).astype(np.uint8)
    C = np.zeros((H, W))
    wall = 31  # cells span x in [0,16),[16,32),..; the wall is inside one cell
    C[:, wall] = 1.0
    lab = oracle.lab_from_rgb(rgb)
    s = oracle.Solver(lab, C, K, gamma=1e4)
    for _ in range(4):
        s.iterate(1)
        left = set(np.unique(s.labels[:, :wall]))
        right = set(np.unique(s.labels[:, wall + 1:]))
        assert not (left & right)
    # with gamma=0 the same image does straddle the wall
    s0 = oracle.Solver(lab, C, K, gamma=0.0)
    s0.iterate(1)
    assert set(np.unique(s0.labels[:, :wall])) & set(np.unique(s0.labels[:, wall + 1:]))


# --------------------------------------------------------------------------
# Brute force on tiny images: D is evaluated here, independently, for every
# (pixel, cluster) pair without a window.  Wherever the global winner's window
# holds the pixel, the windowed oracle must pick it.
# --------------------------------------------------------------------------
def _brute_D(L, A, B, C, st, K, m, lam, sigma, gamma, x, y, k):
    H, W = L.shape
    N = H * W
    pts = oracle.path((x, y), (int(st["ex"][k]), int(st["ey"][k])))
    col = np.array([st["cL"][k], st["cA"][k], st["cB"][k]])

    def dc(q):
        return ((np.array([L[q[1], q[0]], A[q[1], q[0]], B[q[1], q[0]]]) - col) ** 2).sum()

    sdc = sum(dc(q) for q in pts)
    sw = sum(1 - math.exp(-C[q[1], q[0]] ** 2 / sigma ** 2) for q in pts)
    xk, yk = st["sx"][k] / st["n"][k], st["sy"][k] / st["n"][k]
    ds = (x - xk) ** 2 + (y - yk) ** 2
    return (lam * dc((x, y)) + (1 - lam) * sdc / len(pts)) * (1 + gamma * sw / len(pts)) + \
        ds * m * m / (N / K)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bruteforce_tiny(seed):
    H, W, K = 24, 32, 8
    rgb, C, _ = synth.small_image(H, W, seed=100 + seed, n_cells=5)
    lab = oracle.lab_from_rgb(rgb)
    s = oracle.Solver(lab, C, K)
    s.iterate(2)
    st = s.state()
    s.assign()
    N = H * W
    checked = 0
    for y in range(H):
        for x in range(W):
            Ds = [_brute_D(*lab, C, st, K, 10.0, 0.5, 0.25, s.gamma, x, y, k)
                  for k in range(s.Keff)]
            kbest = int(np.argmin(Ds))
            if (K * (st["n"][kbest] * x - st["sx"][kbest]) ** 2 <= N * st["n"][kbest] ** 2 and
                    K * (st["n"][kbest] * y - st["sy"][kbest]) ** 2 <= N * st["n"][kbest] ** 2):
                assert s.labels[y, x] == kbest
                checked += 1
    assert checked > 0.6 * N


# --------------------------------------------------------------------------
# The pixel-centric assignment (used to check single pixels of large images)
# against the cluster-centric loop of Algorithm 1, on every pixel.
# --------------------------------------------------------------------------
def _assign_both(s):
    """(labels, d) of the whole-image assignment and of assign_pixels over
    every pixel, both from the solver's current state (left unchanged)."""
    st = s.state()
    lab_px, d_px = s.assign_pixels(np.arange(s.N))
    d = s.assign(return_d=True)
    lab = s.labels.copy()
    s.set_state(st)
    return lab.ravel(), d.ravel(), lab_px, d_px


def test_assign_pixels_equals_assign_random_states():
    for seed, (H, W, K, iters) in enumerate([(24, 32, 8, 2), (37, 29, 15, 1), (16, 50, 40, 3)]):
        rgb, C, _ = synth.small_image(H, W, seed=140 + seed, n_cells=6)
        s = oracle.Solver(oracle.lab_from_rgb(rgb), C, K)
        s.iterate(iters)
        lab, d, lab_px, d_px = _assign_both(s)
        assert np.array_equal(lab, lab_px)
        assert np.array_equal(d, d_px)  # the same D(p, C_k), bit for bit
        assert np.all(np.isfinite(d))


def test_assign_pixels_orphans_keep_label():
    # every barycenter moved into the top-left quarter: the pixels of the other
    # corner lie in no window and keep their previous label, with d = inf
    H, W, K = 40, 40, 16
    rgb, C, _ = synth.small_image(H, W, seed=150, n_cells=6)
    s = oracle.Solver(oracle.lab_from_rgb(rgb), C, K)
    st = s.state()
    rng = np.random.default_rng(151)
    for k in range(s.Keff):
        x, y = (int(v) for v in rng.integers(0, 10, 2))
        n = int(st["n"][k])
        st["sx"][k], st["sy"][k] = n * x, n * y
        st["ex"][k], st["ey"][k] = x, y
    st["labels"] = rng.integers(0, s.Keff, (H, W)).astype(np.int32)
    s.set_state(st)
    lab, d, lab_px, d_px = _assign_both(s)
    orphan = np.isinf(d)
    assert orphan.sum() > 100 and (~orphan).sum() > 100
    assert np.array_equal(lab, lab_px) and np.array_equal(np.isinf(d_px), orphan)
    assert np.array_equal(d[~orphan], d_px[~orphan])
    assert np.array_equal(lab[orphan], st["labels"].ravel()[orphan])


def test_assign_pixels_exact_ties_go_to_smallest_k():
    # constant colour equal to every cluster's, no contour: D is m^2/r^2 d_s
    # plus path terms that vanish.  Clusters 1 and 2 sit at (10 - 3, 10) and
    # (10 + 3, 10): the pixels of column 10 are at equal distance from both
    # (exact ties); cluster 0 and the rest are far off.  The strict '<' in
    # ascending k gives every tie to cluster 1.
    H, W, K = 30, 40, 12
    lab3 = (np.full((H, W), 40.0), np.full((H, W), 5.0), np.full((H, W), -7.0))
    s = oracle.Solver(lab3, np.zeros((H, W)), K)
    st = s.state()
    where = {1: (7, 10), 2: (13, 10)}
    for k in range(s.Keff):
        x, y = where.get(k, (39 - (k % 3), 29 - (k % 2)))
        n = 50
        st["n"][k], st["sx"][k], st["sy"][k] = n, n * x, n * y
        st["ex"][k], st["ey"][k] = x, y
    st["cL"][:], st["cA"][:], st["cB"][:] = 40.0, 5.0, -7.0
    s.set_state(st)
    lab, d, lab_px, d_px = _assign_both(s)
    assert np.array_equal(lab, lab_px) and np.array_equal(d, d_px)
    ties = 0
    for y in range(H):
        D1, _ = s.distance(10, y, 1)
        D2, _ = s.distance(10, y, 2)
        assert D1 == D2
        p = y * W + 10
        if np.isfinite(d[p]) and d[p] == D1:
            assert lab[p] == 1
            ties += 1
    assert ties >= 10


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_iterate_rows_equals_iterate(threads):
    # the CPU baseline's row-parallel iterations give Algorithm 1's state, bit
    # for bit, on any number of threads (projections included)
    H, W, K = 45, 61, 20
    rgb, C, _ = synth.small_image(H, W, seed=160, n_cells=7)
    lab = oracle.lab_from_rgb(rgb)
    a = oracle.Solver(lab, C, K)
    b = oracle.Solver(lab, C, K)
    projected = 0
    for _ in range(4):
        a.iterate(1)
        b.iterate_rows(1, threads)
        projected += a.projections
        assert b.projections == a.projections and b.orphans == a.orphans
        sa, sb = a.state(), b.state()
        for key in sa:
            assert np.array_equal(sa[key], sb[key]), key
    assert projected > 0


# --------------------------------------------------------------------------
# Update (Algorithm 1: means over S_k) against numpy reductions.
# --------------------------------------------------------------------------
def test_update_means():
    rgb, C, _ = synth.small_image(60, 80, seed=21)
    L, A, B = oracle.lab_from_rgb(rgb)
    s = oracle.Solver((L, A, B), C, 30)
    s.iterate(3)
    lab = s.labels.ravel()
    ys, xs = np.mgrid[0:60, 0:80]
    cnt = np.bincount(lab, minlength=s.Keff)
    nz = cnt > 0
    assert np.array_equal(s.n[nz], cnt[nz])
    assert np.array_equal(s.sx[nz], np.bincount(lab, weights=xs.ravel(), minlength=s.Keff)[nz]
                          .astype(np.int64))
    assert np.array_equal(s.sy[nz], np.bincount(lab, weights=ys.ravel(), minlength=s.Keff)[nz]
                          .astype(np.int64))
    for arr, plane in ((s.cL, L), (s.cA, A), (s.cB, B)):
        ref = np.bincount(lab, weights=plane.ravel(), minlength=s.Keff)[nz] / cnt[nz]
        assert np.allclose(arr[nz], ref, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# Projection, Eq. 4: a superpixel whose barycenter lies outside it.
# --------------------------------------------------------------------------
def test_projection_ring():
    H, W, K = 30, 30, 4
    lab = (np.full((H, W), 50.0), np.zeros((H, W)), np.zeros((H, W)))
    s = oracle.Solver(lab, np.zeros((H, W)), K)
    ys, xs = np.mgrid[0:H, 0:W]
    # label 0: a ring around (14.5, 14.5) with a slot, label 1: everything else
    rr = (xs - 14.5) ** 2 + (ys - 14.5) ** 2
    ring = (rr >= 49) & (rr <= 100) & ~((xs > 14) & (ys >= 13) & (ys <= 16))
    labels = np.where(ring, 0, 1).astype(np.int32)
    s.labels[...] = labels
    s.update()
    assert s.projections >= 1
    n, sx, sy = ring.sum(), xs[ring].sum(), ys[ring].sum()
    assert s.n[0] == n and s.sx[0] == sx and s.sy[0] == sy
    ex_r, ey_r = (2 * sx + n) // (2 * n), (2 * sy + n) // (2 * n)
    assert labels[ey_r, ex_r] != 0
    d2 = [((Fraction(int(x)) - Fraction(int(sx), int(n))) ** 2 +
           (Fraction(int(y)) - Fraction(int(sy), int(n))) ** 2, y * W + x)
          for y, x in zip(ys[ring], xs[ring])]
    best = min(d2)
    assert (s.ey[0] * W + s.ex[0]) == best[1]
    assert labels[s.ey[0], s.ex[0]] == 0


# --------------------------------------------------------------------------
# Connectivity enforcement: scipy's connected-component labelling plus the
# merge rule written out here, and the invariants the rule guarantees.
# --------------------------------------------------------------------------
def _connectivity_scipy(labels, K):
    from scipy import ndimage

    H, W = labels.shape
    N = H * W
    comp = np.full((H, W), -1, np.int64)
    nxt = 0
    for v in np.unique(labels):
        cc, n = ndimage.label(labels == v)  # 4-connectivity by default
        m = cc > 0
        comp[m] = cc[m] - 1 + nxt
        nxt += n
    flat = comp.ravel()
    seeds = np.full(nxt, N, np.int64)
    np.minimum.at(seeds, flat, np.arange(N))
    sizes = np.bincount(flat, minlength=nxt)
    T = N // (4 * K)
    order = np.argsort(seeds)
    final = {}
    number = {}
    for c in order:
        s = seeds[c]
        if sizes[c] <= T and s != 0:
            nb = s - 1 if s % W else s - W
            final[c] = final[flat[nb]]
        else:
            final[c] = c
            number[c] = len(number)
    return np.array([number[final[c]] for c in flat], np.int32).reshape(H, W), len(number)


@pytest.mark.parametrize("seed", range(6))
def test_connectivity_vs_scipy(seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(5, 40)), int(rng.integers(5, 40))
    base = rng.integers(0, 6, size=(H // 3 + 1, W // 3 + 1))
    labels = np.kron(base, np.ones((3, 3), int))[:H, :W]
    noise = rng.uniform(size=(H, W)) < 0.15
    labels = np.where(noise, rng.integers(0, 6, size=(H, W)), labels).astype(np.int32)
    K = int(rng.integers(2, 12))
    out, n = oracle.connectivity(labels, K)
    ref, nref = _connectivity_scipy(labels, K)
    assert n == nref
    assert np.array_equal(out, ref)


def test_connectivity_invariants():
    rgb, C, _ = synth.small_image(90, 120, seed=31)
    s, out, n = oracle.solve(rgb, C, 60, iters=3)
    from scipy import ndimage

    H, W = out.shape
    T = H * W // (4 * 60)
    assert out.min() == 0 and out.max() == n - 1
    first = []
    for v in range(n):
        m = out == v
        _, ncc = ndimage.label(m)
        assert ncc == 1  # every output superpixel is 4-connected
        idx = np.flatnonzero(m.ravel())
        first.append(idx[0])
        if idx[0] != 0:
            assert m.sum() > T
    assert first == sorted(first)  # numbered in raster order of their seeds


# --------------------------------------------------------------------------
# Multi-scale boundary map (Sec. III-A2): averaged boundary indicators.
# --------------------------------------------------------------------------
def _boundary_numpy(lab):
    b = np.zeros(lab.shape, bool)
    dx = lab[:, 1:] != lab[:, :-1]
    dy = lab[1:, :] != lab[:-1, :]
    b[:, 1:] |= dx
    b[:, :-1] |= dx
    b[1:, :] |= dy
    b[:-1, :] |= dy
    return b


def test_boundary_map_closed_forms():
    two = np.zeros((5, 8), np.int32)
    two[:, 5:] = 1
    m = oracle.boundary_map([two])
    expected = np.zeros((5, 8), np.float32)
    expected[:, 4:6] = 1.0
    assert np.array_equal(m, expected)
    checker = (np.add.outer(np.arange(6), np.arange(7)) % 2).astype(np.int32)
    assert np.all(oracle.boundary_map([checker]) == 1.0)
    assert np.all(oracle.boundary_map([np.full((4, 4), 3, np.int32)]) == 0.0)


def test_boundary_map_vs_numpy_average():
    rng = np.random.default_rng(4)
    maps = [np.kron(rng.integers(0, 9, size=(8, 10)), np.ones((4, 5), int)).astype(np.int32)
            for _ in range(5)]
    ref = np.mean([_boundary_numpy(m) for m in maps], axis=0).astype(np.float32)
    got = oracle.boundary_map(maps)
    assert np.allclose(got, ref, atol=1e-7)
    counts = np.sum([_boundary_numpy(m) for m in maps], axis=0)
    assert np.array_equal(got, (counts.astype(np.float32) / np.float32(5)))


def test_multiscale_ladder():
    Ks = oracle.multiscale_K()
    assert len(Ks) == 12 and Ks[0] == 6 and Ks[-1] == 600
    ratios = np.array(Ks[1:]) / np.array(Ks[:-1])
    assert np.all(np.abs(ratios - 100 ** (1 / 11)) < 0.12)  # geometric up to rounding


# --------------------------------------------------------------------------
# Quality metrics, Eq. 5-8, against closed forms and an independent numpy /
# scipy formulation.
# --------------------------------------------------------------------------
def test_quality_identity_and_single_superpixel():
    rng = np.random.default_rng(8)
    gt = np.kron(rng.integers(0, 6, size=(5, 6)), np.ones((6, 7), int)).astype(np.int32)
    q = oracle.quality(gt, gt)
    assert q["br"] == 1.0 and q["asa"] == 1.0 and q["ue"] == 0.0
    one = np.zeros_like(gt)
    q = oracle.quality(one, gt)
    sizes = np.bincount(gt.ravel())
    sizes = sizes[sizes > 0]
    N = gt.size
    assert q["asa"] == sizes.max() / N
    assert q["ue"] == pytest.approx(len(sizes) * N / N - 1.0)  # sum_i (N - |G_i|) / N
    assert q["br"] == 0.0


def test_compactness_closed_forms():
    assert oracle.quality(np.zeros((9, 9), np.int32), np.zeros((9, 9), np.int32))["co"] == \
        pytest.approx(np.pi / 4)
    n = 13
    assert oracle.quality(np.zeros((1, n), np.int32), np.zeros((1, n), np.int32))["co"] == \
        pytest.approx(4 * np.pi * n / (2 * n + 2) ** 2)
    blocks = np.kron(np.arange(12).reshape(3, 4), np.ones((5, 5), int)).astype(np.int32)
    assert oracle.quality(blocks, blocks)["co"] == pytest.approx(np.pi / 4)


def test_boundary_recall_distance_is_strict():
    H, W, c = 12, 20, 8
    gt = np.zeros((H, W), np.int32)
    gt[:, c:] = 1            # ground-truth boundary pixels: columns c-1 and c
    s = np.zeros((H, W), np.int32)
    s[:, c + 2:] = 1         # superpixel boundary pixels: columns c+1 and c+2
    # column c is at distance 1 (hit); column c-1 at distance 2, not < 2 (miss)
    assert oracle.quality(s, gt)["br"] == 0.5
    s1 = np.zeros((H, W), np.int32)
    s1[:, c + 1:] = 1
    assert oracle.quality(s1, gt)["br"] == 1.0


def _quality_numpy(lab, gt, eps=2.0):
    from scipy import ndimage

    N = lab.size
    bs, bg = _boundary_numpy(lab), _boundary_numpy(gt)
    dist = ndimage.distance_transform_edt(~bs)
    br = (dist[bg] < eps).mean() if bg.any() else 1.0
    k, i = lab.ravel(), gt.ravel()
    ov = np.zeros((k.max() + 1, i.max() + 1), np.int64)
    np.add.at(ov, (k, i), 1)
    area = ov.sum(1)
    asa = ov.max(1).sum() / N
    ue = ((area[:, None] - ov) * (ov > 0)).sum() / N
    pad = np.pad(lab, 1, constant_values=-1)
    edges = np.zeros(k.max() + 1, np.int64)
    for sl in ((slice(1, -1), slice(0, -2)), (slice(1, -1), slice(2, None)),
               (slice(0, -2), slice(1, -1)), (slice(2, None), slice(1, -1))):
        diff = pad[sl] != lab
        np.add.at(edges, lab[diff], 1)
    nz = area > 0
    co = (4 * np.pi * area[nz] ** 2 / edges[nz] ** 2).sum() / N
    return dict(br=br, asa=asa, ue=ue, co=co)


def test_quality_vs_numpy_scipy():
    rgb, C, cells = synth.small_image(70, 90, seed=41, n_cells=6)
    s, out, n = oracle.solve(rgb, C, 40, iters=3)
    got = oracle.quality(out, cells)
    ref = _quality_numpy(out, cells)
    for key in ("br", "asa", "ue", "co"):
        assert got[key] == pytest.approx(ref[key], rel=1e-12, abs=1e-12), key


# --------------------------------------------------------------------------
# Contour prior computed from the image (Sec. II-E allows any soft prior):
# the CIELab gradient magnitude over its maximum.
# --------------------------------------------------------------------------
def _gradient_prior_numpy(lab):
    """The same prior through numpy.gradient (central differences inside,
    one-sided at the ends), an independent implementation."""
    g2 = np.zeros(lab[0].shape)
    for f in lab:
        for axis in (0, 1):
            if f.shape[axis] > 1:
                g2 += np.gradient(f, axis=axis) ** 2
    g = np.sqrt(g2)
    return g / g.max() if g.max() > 0 else g


@pytest.mark.parametrize("shape", [(9, 13), (1, 11), (12, 1), (2, 2), (31, 17)])
def test_gradient_prior_vs_numpy(shape):
    rng = np.random.default_rng(sum(shape))
    lab = tuple(rng.normal(scale=20.0, size=shape) for _ in range(3))
    got = oracle.gradient_prior(lab)
    assert np.allclose(got, _gradient_prior_numpy(lab), rtol=1e-12, atol=1e-12)


def test_gradient_prior_linear_ramp_is_one():
    # a plane linear in x and y has the same gradient everywhere, the borders
    # included (one-sided differences of a linear function are its slope)
    ys, xs = np.mgrid[0:7, 0:10].astype(np.float64)
    lab = (3.0 * xs + 4.0 * ys, np.zeros((7, 10)), -2.0 * xs)
    assert np.allclose(oracle.gradient_prior(lab), 1.0, rtol=0, atol=1e-15)


def test_gradient_prior_step_and_flat():
    c1, c2 = (30, 200, 90), (220, 40, 10)
    rgb = np.zeros((6, 10, 3), np.uint8)
    rgb[:, :5] = c1
    rgb[:, 5:] = c2
    C = oracle.gradient_prior(oracle.lab_from_rgb(rgb))
    want = np.zeros((6, 10))
    want[:, 4:6] = 1.0  # the two columns whose central difference spans the step
    assert np.array_equal(C, want)
    # a step after the first column: the one-sided difference there is twice
    # the central one next to it
    rgb[:, 1:] = c2
    rgb[:, :1] = c1
    C = oracle.gradient_prior(oracle.lab_from_rgb(rgb))
    assert np.allclose(C[:, 0], 1.0, atol=1e-15) and np.allclose(C[:, 1], 0.5, atol=1e-15)
    assert np.all(C[:, 2:] == 0)
    flat = np.full((5, 8, 3), 77, np.uint8)
    assert np.all(oracle.gradient_prior(oracle.lab_from_rgb(flat)) == 0)


# --------------------------------------------------------------------------
# Supervoxels (SCALP on (T, H, W) volumes; the readings are the 2-D ones taken
# axis by axis).
# --------------------------------------------------------------------------
def test_vpath_properties():
    from fractions import Fraction

    rng = np.random.default_rng(5)
    pts = rng.integers(0, 9, size=(600, 6))
    pts = np.concatenate([pts, [[3, 3, 3, 3, 3, 3], [0, 0, 0, 8, 8, 8], [0, 8, 0, 8, 0, 8],
                                [2, 5, 1, 6, 1, 3]]])
    for q in pts:
        p, e = tuple(int(v) for v in q[:3]), tuple(int(v) for v in q[3:])
        P = oracle.vpath(p, e)
        d = [abs(e[j] - p[j]) for j in range(3)]
        ns = max(d)
        assert len(P) == ns + 1
        # traced from the lexicographically smaller end (x, then y, then t)
        a, b = (p, e) if p <= e else (e, p)
        assert tuple(P[0]) == a and tuple(P[-1]) == b
        # symmetric: the other direction gives the same voxel sequence
        assert np.array_equal(oracle.vpath(e, p), P)
        major = int(np.argmax(d))  # the first largest |delta|: x, then y, then t
        for i, v in enumerate(P):
            for j in range(3):
                sgn = 1 if b[j] >= a[j] else -1
                off = sgn * (int(v[j]) - a[j])
                if j == major:
                    assert off == i
                else:
                    # the nearest integer to the exact segment point, half up
                    exact = Fraction(i * d[j], ns) if ns else Fraction(0)
                    assert off == int((exact + Fraction(1, 2)).__floor__())


def test_vpath_reduces_to_2d_path():
    rng = np.random.default_rng(6)
    for _ in range(300):
        x0, y0, x1, y1, t = (int(v) for v in rng.integers(0, 12, 5))
        P3 = oracle.vpath((x0, y0, t), (x1, y1, t))
        P2 = oracle.path((x0, y0), (x1, y1))
        assert np.array_equal(P3[:, :2], P2) and np.all(P3[:, 2] == t)


def test_vconstant_volume_fixed_point():
    # 16^3 voxels, K = 64: r = 4, a 4x4x4 grid of 4^3 cells; a constant image
    # with no contour leaves only the spatial term, and the grid is a fixed point
    T = H = W = 16
    rgb = np.full((T, H, W, 3), 120, np.uint8)
    s = oracle.VSolver(oracle.lab_from_rgb(rgb), np.zeros((T, H, W)), 64)
    assert s.r == 4.0 and s.grid == (4, 4, 4)
    cells = s.labels.copy()
    n0, sx0 = s.n.copy(), s.sx.copy()
    s.iterate(3)
    assert np.array_equal(s.labels, cells) and np.array_equal(s.n, n0) and np.array_equal(s.sx, sx0)
    assert s.projections == 0


def _vaxis_in_window(v, n, sv, N, K):
    """|v - sv/n| <= r with r^3 = N/K, in rational arithmetic (cubing both
    non-negative sides): |v - sv/n|^3 <= N/K."""
    return abs(Fraction(v) - Fraction(sv, n)) ** 3 <= Fraction(N, K)


def _vwindow_mask(s, k, T, H, W):
    """Voxels of cluster k's window: per axis |v - X_k| <= cbrt(N/K), exactly."""
    n, N = int(s.n[k]), T * H * W
    def axis(length, sv):
        return np.array([_vaxis_in_window(v, n, sv, N, s.K) for v in range(length)])
    return (axis(T, int(s.st[k]))[:, None, None] & axis(H, int(s.sy[k]))[None, :, None]
            & axis(W, int(s.sx[k]))[None, None, :])


def test_cube_root_convergents_helper():
    # the helper's first convergents of 2^(1/3) = [1; 3, 1, 5, 1, 1, 4, 1, 1, 8, ...]
    conv = cube_root_convergents(2, 6)
    assert conv[:6] == [(1, 1), (4, 3), (5, 4), (29, 23), (34, 27), (63, 50)]
    for p, q in conv:
        assert abs(p / q - 2 ** (1 / 3)) < 1 / q ** 2
    assert cube_root_convergents(27, 3)[0] == (3, 1)


def test_vwindow_predicate_exact():
    """The supervoxel window |v - s/n| <= r, r^3 = N/K, against rational
    arithmetic: random values, exact edges (N/K a perfect cube), values within
    1e-12 of an irrational edge (convergents of the cube root), huge clusters."""
    rng = np.random.default_rng(31)
    for _ in range(3000):
        N = int(rng.integers(10, 1 << 30))
        K = int(rng.integers(1, min(N, 200000) + 1))
        n = int(rng.integers(1, 1 << 20))
        s = int(rng.integers(0, n * 4000))
        r = (N / K) ** (1 / 3)
        xk = s / n
        for v in {math.floor(xk - r) - 1, math.floor(xk - r), math.ceil(xk - r),
                  math.floor(xk + r), math.ceil(xk + r), math.ceil(xk + r) + 1}:
            assert oracle.vin_window(v, n, s, N, K) == _vaxis_in_window(v, n, s, N, K)
    # N/K a perfect cube: r = 3 exactly, and |v - s/n| = 3 is inside, 3 + 1/n not
    for n in (1, 7, 1000, 1 << 29):
        for v in (10, 100):
            assert oracle.vin_window(v, n, n * (v - 3), 27 * 5, 5)
            assert oracle.vin_window(v, n, n * (v + 3), 27 * 5, 5)
            assert not oracle.vin_window(v, n, n * (v - 3) - 1, 27 * 5, 5)
            assert not oracle.vin_window(v, n, n * (v + 3) + 1, 27 * 5, 5)
    # |v - s/n| = p/q, a convergent of cbrt(a): alternately just inside and
    # just outside the edge, closer than double rounding of r can resolve
    checked_close = 0
    for a in (2, 3, 5, 7, 10, 100, 999):
        for p, q in cube_root_convergents(a, 40):
            if q > (1 << 29) or p > 1024 * q:
                break
            N, K = a * 1000, 1000
            n = q
            for v, s in ((5, 5 * q - p), (5, 5 * q + p)):  # n*v - s = +p and -p
                want = Fraction(p, q) ** 3 <= a
                assert oracle.vin_window(v, n, s, N, K) == want
                assert _vaxis_in_window(v, n, s, N, K) == want
            if abs(p / q - a ** (1 / 3)) < 1e-12 * a ** (1 / 3):
                checked_close += 1
    assert checked_close >= 10
    # huge clusters: n = 2^30 voxels, K = 1 (r = 2^10): the window's extreme
    # values and one past them, without overflow
    N, K, n = 1 << 30, 1, 1 << 30
    assert oracle.vin_window(1024, n, 0, N, K) and not oracle.vin_window(1025, n, 0, N, K)
    assert oracle.vin_window(0, n, 1024 * n, N, K) and not oracle.vin_window(0, n, 1025 * n, N, K)
    assert not oracle.vin_window(65535, n, 0, N, K)


def test_vslic_special_case():
    # lambda = 1, gamma = 0: D = d_c(p, C_k) + m^2/r^2 d_s, a plain 3-D SLIC
    # assignment, computed here in numpy over every cluster whose window holds p
    rng = np.random.default_rng(7)
    T, H, W = 4, 14, 18
    rgb = rng.integers(0, 256, (T, H, W, 3), dtype=np.uint8)
    lab = oracle.lab_from_rgb(rgb)
    s = oracle.VSolver(lab, rng.uniform(size=(T, H, W)), 10, lam=1.0, gamma=0.0)
    s.iterate(1)
    st = s.state()
    s.assign()
    tt, yy, xx = np.meshgrid(np.arange(T), np.arange(H), np.arange(W), indexing="ij")
    best = np.full((T, H, W), np.inf)
    lab_ref = st["labels"].copy()
    for k in range(s.Keff):
        if st["n"][k] == 0:
            continue
        m = _vwindow_mask(s, k, T, H, W)
        n = st["n"][k]
        dc = ((lab[0] - st["cL"][k]) ** 2 + (lab[1] - st["cA"][k]) ** 2 + (lab[2] - st["cB"][k]) ** 2)
        ds = (xx - st["sx"][k] / n) ** 2 + (yy - st["sy"][k] / n) ** 2 + (tt - st["st"][k] / n) ** 2
        D = dc + (10.0 ** 2 / s.r ** 2) * ds
        take = m & (D < best)
        best[take] = D[take]
        lab_ref[take] = k
    assert np.array_equal(s.labels, lab_ref)


def test_vbruteforce_tiny():
    rng = np.random.default_rng(8)
    T, H, W = 3, 8, 10
    rgb = rng.integers(0, 256, (T, H, W, 3), dtype=np.uint8)
    s = oracle.VSolver(oracle.lab_from_rgb(rgb), rng.uniform(size=(T, H, W)), 8)
    s.iterate(2)
    st = s.state()
    s.assign()
    for t in range(T):
        for y in range(H):
            for x in range(W):
                best, kb = np.inf, int(st["labels"][t, y, x])
                for k in range(s.Keff):
                    if st["n"][k] == 0 or not _vwindow_mask(s, k, T, H, W)[t, y, x]:
                        continue
                    D, _ = s.distance(x, y, t, k)
                    if D < best:
                        best, kb = D, k
                assert s.labels[t, y, x] == kb


def test_vupdate_and_projection():
    rng = np.random.default_rng(9)
    T, H, W = 5, 12, 16
    rgb = rng.integers(0, 256, (T, H, W, 3), dtype=np.uint8)
    lab = oracle.lab_from_rgb(rgb)
    s = oracle.VSolver(lab, np.zeros((T, H, W)), 12)
    # a label map where cluster 0 is a hollow box: its barycenter lies outside it
    labels = np.ones((T, H, W), np.int32)
    labels[:, 2:10, 3:13] = 0
    labels[1:4, 4:8, 5:11] = 2
    st = s.state()
    st["labels"] = labels
    s.set_state(st)
    s.update()
    tt, yy, xx = np.meshgrid(np.arange(T), np.arange(H), np.arange(W), indexing="ij")
    for k in range(3):
        m = labels == k
        n = int(m.sum())
        assert s.n[k] == n and s.sx[k] == xx[m].sum() and s.sy[k] == yy[m].sum()
        assert s.st[k] == tt[m].sum()
        assert s.cL[k] == pytest.approx(lab[0][m].mean(), rel=1e-12, abs=1e-12)
        sx, sy, stt = int(xx[m].sum()), int(yy[m].sum()), int(tt[m].sum())
        e = ((2 * sx + n) // (2 * n), (2 * sy + n) // (2 * n), (2 * stt + n) // (2 * n))
        if labels[e[2], e[1], e[0]] != k:
            # Eq. 4 by brute force in exact integers, ties to the smallest index
            d2 = [((n * x - sx) ** 2 + (n * y - sy) ** 2 + (n * t - stt) ** 2, (t * H + y) * W + x, (x, y, t))
                  for t, y, x in zip(tt[m], yy[m], xx[m])]
            e = min(d2)[2]
        assert (s.ex[k], s.ey[k], s.et[k]) == tuple(int(v) for v in e), k
    assert s.projections >= 1
