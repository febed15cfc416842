"""FP64 CPU oracle for SCALP -- test infrastructure only.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py may
import this package.  The product path (the CUDA library and its binding) never
imports it, and it shares no code with that library.

The arithmetic lives in ``scalp_oracle.c`` (plain C, double precision, the steps
of Algorithm 1 in the paper's order).  This module compiles it with gcc and
marshals numpy arrays to it; it adds no arithmetic of its own.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scalp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: no fused multiply-add, so x86-64 and aarch64 hosts give
# the same bits.
# -fopenmp: the row-parallel iterations of the CPU baseline (orc_iterate_rows).
CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, a second or two)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Ctx(ctypes.Structure):
    _fields_ = [
        ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("K", ctypes.c_int32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("Keff", ctypes.c_int32),
        ("m", ctypes.c_double), ("lam", ctypes.c_double), ("sigma", ctypes.c_double),
        ("gamma", ctypes.c_double), ("r", ctypes.c_double),
        ("L", ctypes.c_void_p), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
        ("C", ctypes.c_void_p),
        ("labels", ctypes.c_void_p),
        ("n", ctypes.c_void_p), ("sx", ctypes.c_void_p), ("sy", ctypes.c_void_p),
        ("cL", ctypes.c_void_p), ("cA", ctypes.c_void_p), ("cB", ctypes.c_void_p),
        ("ex", ctypes.c_void_p), ("ey", ctypes.c_void_p),
        ("orphans", ctypes.c_int64), ("projections", ctypes.c_int64),
    ]


class _VCtx(ctypes.Structure):
    _fields_ = [
        ("T", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("K", ctypes.c_int32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nt", ctypes.c_int32),
        ("Keff", ctypes.c_int32),
        ("m", ctypes.c_double), ("lam", ctypes.c_double), ("sigma", ctypes.c_double),
        ("gamma", ctypes.c_double), ("r", ctypes.c_double),
        ("L", ctypes.c_void_p), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
        ("C", ctypes.c_void_p),
        ("labels", ctypes.c_void_p),
        ("n", ctypes.c_void_p), ("sx", ctypes.c_void_p), ("sy", ctypes.c_void_p),
        ("st", ctypes.c_void_p),
        ("cL", ctypes.c_void_p), ("cA", ctypes.c_void_p), ("cB", ctypes.c_void_p),
        ("ex", ctypes.c_void_p), ("ey", ctypes.c_void_p), ("et", ctypes.c_void_p),
        ("orphans", ctypes.c_int64), ("projections", ctypes.c_int64),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            L.orc_lab_from_rgb.argtypes = [P, ctypes.c_int64, P, P, P]
            L.orc_grid_dims.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]
            L.orc_path.argtypes = [ctypes.c_int] * 4 + [P]
            L.orc_path.restype = ctypes.c_int
            L.orc_in_window.argtypes = [ctypes.c_int64] * 5
            L.orc_in_window.restype = ctypes.c_int
            L.orc_distance.argtypes = [ctypes.POINTER(_Ctx), ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, P]
            L.orc_distance.restype = ctypes.c_double
            L.orc_update.argtypes = [ctypes.POINTER(_Ctx)]
            L.orc_init.argtypes = [ctypes.POINTER(_Ctx)]
            L.orc_init.restype = ctypes.c_int
            L.orc_assign.argtypes = [ctypes.POINTER(_Ctx), P]
            L.orc_assign.restype = ctypes.c_int64
            L.orc_iterate.argtypes = [ctypes.POINTER(_Ctx), ctypes.c_int]
            L.orc_iterate_rows.argtypes = [ctypes.POINTER(_Ctx), ctypes.c_int, ctypes.c_int]
            L.orc_assign_rows.argtypes = [ctypes.POINTER(_Ctx), ctypes.c_int]
            L.orc_assign_rows.restype = ctypes.c_int64
            L.orc_assign_pixels.argtypes = [ctypes.POINTER(_Ctx), P, ctypes.c_int64, P, P]
            L.orc_connectivity.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
            L.orc_connectivity.restype = ctypes.c_int32
            L.orc_boundary_map.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
            L.orc_quality.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, P, P, P, P]
            L.orc_gradient_prior.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, P]
            L.orc_vgrid_dims.argtypes = [ctypes.c_int] * 4 + [P, P, P, P]
            L.orc_vpath.argtypes = [ctypes.c_int] * 6 + [P]
            L.orc_vpath.restype = ctypes.c_int
            L.orc_vin_window.argtypes = [ctypes.c_int64] * 5
            L.orc_vin_window.restype = ctypes.c_int
            L.orc_vdistance.argtypes = [ctypes.POINTER(_VCtx)] + [ctypes.c_int] * 4 + [P]
            L.orc_vdistance.restype = ctypes.c_double
            L.orc_vupdate.argtypes = [ctypes.POINTER(_VCtx)]
            L.orc_vinit.argtypes = [ctypes.POINTER(_VCtx)]
            L.orc_vinit.restype = ctypes.c_int
            L.orc_vassign.argtypes = [ctypes.POINTER(_VCtx), P]
            L.orc_vassign.restype = ctypes.c_int64
            L.orc_viterate.argtypes = [ctypes.POINTER(_VCtx), ctypes.c_int]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def lab_from_rgb(rgb: np.ndarray):
    """sRGB uint8 (..., 3) -> (L, a, b) float64 planes of the same leading shape."""
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
    shape = rgb.shape[:-1]
    n = int(np.prod(shape))
    L = np.empty(n); A = np.empty(n); B = np.empty(n)
    lib().orc_lab_from_rgb(_ptr(rgb), n, _ptr(L), _ptr(A), _ptr(B))
    return L.reshape(shape), A.reshape(shape), B.reshape(shape)


def grid_dims(H: int, W: int, K: int):
    nx = ctypes.c_int(); ny = ctypes.c_int()
    lib().orc_grid_dims(H, W, K, ctypes.byref(nx), ctypes.byref(ny))
    return nx.value, ny.value


def path(p, e):
    """Pixels of the linear path between p=(x, y) and e=(x, y), as an (n, 2) array."""
    n = max(abs(p[0] - e[0]), abs(p[1] - e[1])) + 1
    xy = np.empty(2 * n, dtype=np.int32)
    m = lib().orc_path(int(p[0]), int(p[1]), int(e[0]), int(e[1]), _ptr(xy))
    assert m == n
    return xy.reshape(n, 2)


def in_window(v: int, n: int, s: int, N: int, K: int) -> bool:
    return bool(lib().orc_in_window(v, n, s, N, K))


def connectivity(labels: np.ndarray, K: int):
    """Connectivity enforcement of a (H, W) int32 label map -> (labels, n_labels)."""
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    H, W = labels.shape
    out = np.empty_like(labels)
    n = lib().orc_connectivity(_ptr(labels), H, W, K, _ptr(out))
    return out, int(n)


def boundary_map(label_maps):
    """Average boundary indicator of several (H, W) label maps -> float32 (H, W)."""
    maps = [np.ascontiguousarray(m, dtype=np.int32) for m in label_maps]
    H, W = maps[0].shape
    ptrs = (ctypes.c_void_p * len(maps))(*[m.ctypes.data for m in maps])
    out = np.empty((H, W), np.float32)
    lib().orc_boundary_map(ctypes.cast(ptrs, ctypes.c_void_p), len(maps), H, W, _ptr(out))
    return out


def quality(labels, gt, eps: float = 2.0):
    """BR, ASA, UE, CO (Eq. 5-8) of a label map against a ground truth."""
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    gt = np.ascontiguousarray(gt, dtype=np.int32)
    H, W = labels.shape
    out = [ctypes.c_double() for _ in range(4)]
    lib().orc_quality(_ptr(labels), int(labels.max()) + 1, _ptr(gt), int(gt.max()) + 1, H, W,
                      float(eps), *[ctypes.byref(v) for v in out])
    return dict(zip(("br", "asa", "ue", "co"), (v.value for v in out)))


def gradient_prior(lab):
    """Contour prior from the image: CIELab gradient magnitude / its maximum.
    ``lab`` = (L, a, b) float64 (H, W) planes, e.g. from lab_from_rgb."""
    L, A, B = (np.ascontiguousarray(x, dtype=np.float64) for x in lab)
    H, W = L.shape
    out = np.empty((H, W))
    lib().orc_gradient_prior(_ptr(L), _ptr(A), _ptr(B), H, W, _ptr(out))
    return out


def multiscale_K(k_min: int = 6, k_max: int = 600, scales: int = 12):
    """Geometric scale ladder k_min .. k_max (the paper's 12 scales, 6 to 600)."""
    return [int(round(k_min * (k_max / k_min) ** (i / (scales - 1)))) for i in range(scales)]


class Solver:
    """One SCALP solve held in numpy arrays, stepped by the C oracle.

    ``lab`` = (L, a, b) float64 planes (H, W); ``contour`` float (H, W) in [0,1].
    """

    def __init__(self, lab, contour, K: int, m: float = 10.0, lam: float = 0.5,
                 sigma: float = 0.25, gamma: float = -1.0):
        L, A, B = (np.ascontiguousarray(x, dtype=np.float64) for x in lab)
        self.H, self.W = L.shape
        self.N = self.H * self.W
        self.K = int(K)
        self.L, self.A, self.B = L, A, B
        self.C = np.ascontiguousarray(contour, dtype=np.float64)
        nx, ny = grid_dims(self.H, self.W, self.K)
        Keff = nx * ny
        self.labels = np.zeros((self.H, self.W), dtype=np.int32)
        self.n = np.zeros(Keff, np.int64); self.sx = np.zeros(Keff, np.int64)
        self.sy = np.zeros(Keff, np.int64)
        self.cL = np.zeros(Keff); self.cA = np.zeros(Keff); self.cB = np.zeros(Keff)
        self.ex = np.zeros(Keff, np.int32); self.ey = np.zeros(Keff, np.int32)
        c = _Ctx()
        c.H, c.W, c.K = self.H, self.W, self.K
        c.m, c.lam, c.sigma, c.gamma = m, lam, sigma, gamma
        for name in ("L", "A", "B", "C", "labels", "n", "sx", "sy", "cL", "cA", "cB",
                     "ex", "ey"):
            setattr(c, name, _ptr(getattr(self, name)))
        self._c = c
        rc = lib().orc_init(ctypes.byref(c))
        if rc != 0:
            raise ValueError("invalid SCALP arguments")
        assert c.Keff == Keff

    # -- state ---------------------------------------------------------------
    @property
    def r(self) -> float:
        return self._c.r

    @property
    def gamma(self) -> float:
        return self._c.gamma

    @property
    def Keff(self) -> int:
        return self._c.Keff

    @property
    def grid(self):
        return self._c.nx, self._c.ny

    @property
    def orphans(self) -> int:
        return self._c.orphans

    @property
    def projections(self) -> int:
        return self._c.projections

    def centers(self):
        """(Keff, 2) barycenters X_k = (Sx/n, Sy/n)."""
        return np.stack([self.sx / self.n, self.sy / self.n], axis=1)

    def colors(self):
        return np.stack([self.cL, self.cA, self.cB], axis=1)

    def endpoints(self):
        return np.stack([self.ex, self.ey], axis=1)

    def state(self):
        """Copy of the cluster state and labels (the data one iteration reads)."""
        return dict(labels=self.labels.copy(), n=self.n.copy(), sx=self.sx.copy(),
                    sy=self.sy.copy(), cL=self.cL.copy(), cA=self.cA.copy(),
                    cB=self.cB.copy(), ex=self.ex.copy(), ey=self.ey.copy())

    def set_state(self, st):
        for k, v in st.items():
            getattr(self, k)[...] = v

    # -- Algorithm 1 steps ---------------------------------------------------
    def assign(self, return_d: bool = False):
        d = np.empty((self.H, self.W)) if return_d else None
        lib().orc_assign(ctypes.byref(self._c), _ptr(d) if return_d else None)
        return d

    def update(self):
        lib().orc_update(ctypes.byref(self._c))

    def iterate(self, iters: int = 1):
        lib().orc_iterate(ctypes.byref(self._c), int(iters))

    def iterate_rows(self, iters: int = 1, threads: int = 0):
        """The same iterations with the assignment pixel by pixel over rows on
        `threads` OpenMP threads (0: every host core)."""
        lib().orc_iterate_rows(ctypes.byref(self._c), int(iters), int(threads or os.cpu_count()))

    def assign_rows(self, threads: int = 0):
        lib().orc_assign_rows(ctypes.byref(self._c), int(threads or os.cpu_count()))

    def distance(self, x: int, y: int, k: int):
        """D(p, C_k) of Eq. 3 for p=(x, y); returns (D, |P|)."""
        n = ctypes.c_int32()
        D = lib().orc_distance(ctypes.byref(self._c), int(x), int(y), int(k), ctypes.byref(n))
        return D, n.value

    def assign_pixels(self, pix):
        pix = np.ascontiguousarray(pix, dtype=np.int64)
        lab = np.empty(len(pix), np.int32)
        d = np.empty(len(pix))
        lib().orc_assign_pixels(ctypes.byref(self._c), _ptr(pix), len(pix), _ptr(lab), _ptr(d))
        return lab, d


def solve(rgb: np.ndarray, contour: np.ndarray, K: int, iters: int = 10, m: float = 10.0,
          lam: float = 0.5, sigma: float = 0.25, gamma: float = -1.0, enforce: bool = True):
    """Full SCALP run: Lab, grid init, iters x (assign, update), connectivity."""
    lab = lab_from_rgb(rgb)
    s = Solver(lab, contour, K, m=m, lam=lam, sigma=sigma, gamma=gamma)
    s.iterate(iters)
    if enforce:
        out, n = connectivity(s.labels, K)
        return s, out, n
    return s, s.labels.copy(), int(s.Keff)


# ---------------------------------------------------------------------------
# Supervoxels: SCALP on a (T, H, W) volume (the extension the paper's
# conclusion names), stepped by the C oracle.
# ---------------------------------------------------------------------------
def vgrid_dims(T: int, H: int, W: int, K: int):
    """(nx, ny, nt, r) of the 3-D grid, r = cbrt(N/K)."""
    v = [ctypes.c_int() for _ in range(3)]
    r = ctypes.c_double()
    lib().orc_vgrid_dims(T, H, W, K, *(ctypes.byref(x) for x in v), ctypes.byref(r))
    return v[0].value, v[1].value, v[2].value, r.value


def vpath(p, e):
    """Voxels (x, y, t) of the 3-D linear path between p and e, as an (n, 3) array."""
    n = max(abs(p[i] - e[i]) for i in range(3)) + 1
    xyz = np.empty(3 * n, dtype=np.int32)
    m = lib().orc_vpath(*(int(v) for v in p), *(int(v) for v in e), _ptr(xyz))
    assert m == n
    return xyz.reshape(n, 3)


def vin_window(v: int, n: int, s: int, N: int, K: int) -> bool:
    """|v - s/n| <= cbrt(N/K), the supervoxel window along one axis."""
    return bool(lib().orc_vin_window(v, n, s, N, K))


class VSolver:
    """One supervoxel solve.  ``lab`` = (L, a, b) float64 (T, H, W) volumes,
    ``contour`` float (T, H, W) in [0, 1]."""

    def __init__(self, lab, contour, K: int, m: float = 10.0, lam: float = 0.5,
                 sigma: float = 0.25, gamma: float = -1.0):
        L, A, B = (np.ascontiguousarray(x, dtype=np.float64) for x in lab)
        self.T, self.H, self.W = L.shape
        self.N = L.size
        self.K = int(K)
        self.L, self.A, self.B = L, A, B
        self.C = np.ascontiguousarray(contour, dtype=np.float64)
        nx, ny, nt, _ = vgrid_dims(self.T, self.H, self.W, self.K)
        Keff = nx * ny * nt
        self.labels = np.zeros((self.T, self.H, self.W), dtype=np.int32)
        for name in ("n", "sx", "sy", "st"):
            setattr(self, name, np.zeros(Keff, np.int64))
        for name in ("cL", "cA", "cB"):
            setattr(self, name, np.zeros(Keff))
        for name in ("ex", "ey", "et"):
            setattr(self, name, np.zeros(Keff, np.int32))
        c = _VCtx()
        c.T, c.H, c.W, c.K = self.T, self.H, self.W, self.K
        c.m, c.lam, c.sigma, c.gamma = m, lam, sigma, gamma
        for name in ("L", "A", "B", "C", "labels", "n", "sx", "sy", "st", "cL", "cA", "cB",
                     "ex", "ey", "et"):
            setattr(c, name, _ptr(getattr(self, name)))
        self._c = c
        if lib().orc_vinit(ctypes.byref(c)) != 0:
            raise ValueError("invalid supervoxel arguments")
        assert c.Keff == Keff

    @property
    def r(self) -> float:
        return self._c.r

    @property
    def gamma(self) -> float:
        return self._c.gamma

    @property
    def Keff(self) -> int:
        return self._c.Keff

    @property
    def grid(self):
        return self._c.nx, self._c.ny, self._c.nt

    @property
    def orphans(self) -> int:
        return self._c.orphans

    @property
    def projections(self) -> int:
        return self._c.projections

    def state(self):
        return {k: getattr(self, k).copy() for k in
                ("labels", "n", "sx", "sy", "st", "cL", "cA", "cB", "ex", "ey", "et")}

    def set_state(self, st):
        for k, v in st.items():
            getattr(self, k)[...] = v

    def assign(self, return_d: bool = False):
        d = np.empty((self.T, self.H, self.W)) if return_d else None
        lib().orc_vassign(ctypes.byref(self._c), _ptr(d) if return_d else None)
        return d

    def update(self):
        lib().orc_vupdate(ctypes.byref(self._c))

    def iterate(self, iters: int = 1):
        lib().orc_viterate(ctypes.byref(self._c), int(iters))

    def distance(self, x: int, y: int, t: int, k: int):
        n = ctypes.c_int32()
        D = lib().orc_vdistance(ctypes.byref(self._c), int(x), int(y), int(t), int(k),
                                ctypes.byref(n))
        return D, n.value
