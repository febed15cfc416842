"""ctypes binding of libscalp (include/scalp.h).

The functions below carry the C names and do argument marshalling only: every
step of SCALP runs in the CUDA kernels of libscalp.  PyTorch supplies device
memory (the workspace, inputs and outputs) and streams.  There is no CPU
fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libscalp.so")

SCALP_OK = 0
SCALP_E_ARG = -1
SCALP_E_NOMEM = -2
SCALP_E_CUDA = -3
SCALP_E_TIMEOUT = -4
SCALP_E_STATE = -5
SCALP_E_INTERNAL = -6
STORAGE = {"f32": 0, "f16": 1}
BATCH_LAUNCH = {"flat": 0, "persistent": 1, "persistent_cost": 2}
PRIOR = {"input": 0, "gradient": 1}


class ScalpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libscalp error {code}: {msg}")
        self.code = code


class scalp_image(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("rgb", ctypes.c_void_p),
                ("rgb_stride", ctypes.c_int64), ("on_device", ctypes.c_int32)]


class scalp_contour(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("stride", ctypes.c_int64)]


class scalp_params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_float), ("sigma", ctypes.c_float), ("gamma", ctypes.c_float),
                ("storage", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("global_walk", ctypes.c_int32), ("prior", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t)]


class scalp_info(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("K", ctypes.c_int32),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("Keff", ctypes.c_int32),
                ("r", ctypes.c_double), ("gamma", ctypes.c_double), ("map_pairs", ctypes.c_int32),
                ("iterations", ctypes.c_int32)]


class scalp_quality(ctypes.Structure):
    _fields_ = [("br", ctypes.c_double), ("asa", ctypes.c_double), ("ue", ctypes.c_double),
                ("co", ctypes.c_double)]


class scalp_volume(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("rgb", ctypes.c_void_p), ("contour", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class scalp_voxel_info(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("K", ctypes.c_int32),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nt", ctypes.c_int32),
                ("Keff", ctypes.c_int32), ("r", ctypes.c_double), ("gamma", ctypes.c_double),
                ("iterations", ctypes.c_int32)]


class scalp_voxel_state(ctypes.Structure):
    _fields_ = [("labels", ctypes.c_void_p), ("n", ctypes.c_void_p), ("sx", ctypes.c_void_p),
                ("sy", ctypes.c_void_p), ("st", ctypes.c_void_p), ("color", ctypes.c_void_p),
                ("endpoint", ctypes.c_void_p)]


class scalp_state(ctypes.Structure):
    _fields_ = [("labels", ctypes.c_void_p), ("n", ctypes.c_void_p), ("sx", ctypes.c_void_p),
                ("sy", ctypes.c_void_p), ("color", ctypes.c_void_p), ("endpoint", ctypes.c_void_p)]


# Every symbol include/scalp.h declares.
EXPORTS = (
    "scalp_default_params", "scalp_workspace_bytes", "scalp_init", "scalp_reload",
    "scalp_iterate", "scalp_labels", "scalp_get_info", "scalp_get_state", "scalp_set_state",
    "scalp_clusters", "scalp_server_inject_status",
    "scalp_debug_paths", "scalp_profile", "scalp_count_samples", "scalp_sync",
    "scalp_last_error", "scalp_destroy", "scalp_label_means_static",
    "scalp_batch_workspace_bytes", "scalp_batch_init", "scalp_batch_reload", "scalp_batch_iterate",
    "scalp_batch_labels", "scalp_batch_get_state", "scalp_batch_get_info", "scalp_batch_destroy",
    "scalp_batch_set_launch", "scalp_batch_get_launch", "scalp_batch_set_wait",
    "scalp_batch_count_samples", "scalp_batch_profile", "scalp_batch_autotune",
    "scalp_server_reserve_bytes", "scalp_server_create", "scalp_server_submit", "scalp_server_step",
    "scalp_server_poll", "scalp_server_stats", "scalp_server_destroy", "scalp_boundary_map",
    "scalp_server_set_step_budget",
    "scalp_quality_workspace_bytes", "scalp_quality_metrics",
    "scalp_gradient_prior_workspace_bytes", "scalp_gradient_prior",
    "scalp_voxel_workspace_bytes", "scalp_voxel_init", "scalp_voxel_iterate", "scalp_voxel_labels",
    "scalp_voxel_get_info", "scalp_voxel_get_state", "scalp_voxel_set_state",
    "scalp_voxel_count_samples", "scalp_voxel_profile", "scalp_voxel_destroy",
)

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libscalp.so (built by paper_1903_07149_gb300.build); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise FileNotFoundError(
                f"{path} is missing: build it with `python -m paper_1903_07149_gb300.build`")
        L = ctypes.CDLL(path)
        P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sig = {
            "scalp_default_params": (None, [ctypes.POINTER(scalp_params)]),
            "scalp_workspace_bytes": (ctypes.c_size_t, [I32, I32, I32, ctypes.POINTER(scalp_params)]),
            "scalp_init": (ctypes.c_int, [ctypes.POINTER(P), ctypes.POINTER(scalp_image),
                                          ctypes.POINTER(scalp_contour), I32, ctypes.c_float,
                                          ctypes.POINTER(scalp_params)]),
            "scalp_reload": (ctypes.c_int, [P, ctypes.POINTER(scalp_image),
                                            ctypes.POINTER(scalp_contour)]),
            "scalp_iterate": (ctypes.c_int, [P, I32]),
            "scalp_labels": (ctypes.c_int, [P, P, I32, I32, ctypes.POINTER(I32)]),
            "scalp_get_info": (ctypes.c_int, [P, ctypes.POINTER(scalp_info)]),
            "scalp_get_state": (ctypes.c_int, [P, ctypes.POINTER(scalp_state)]),
            "scalp_clusters": (ctypes.c_int, [P, P, ctypes.POINTER(I32)]),
            "scalp_set_state": (ctypes.c_int, [P, ctypes.POINTER(scalp_state)]),
            "scalp_debug_paths": (ctypes.c_int, [P, P, I32, P, I32, P]),
            "scalp_profile": (ctypes.c_int, [P, I32, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(I64)]),
            "scalp_count_samples": (ctypes.c_int, [P, I32, ctypes.POINTER(I64),
                                                   ctypes.POINTER(I64), ctypes.POINTER(I64),
                                                   ctypes.POINTER(I64)]),
            "scalp_sync": (ctypes.c_int, [P]),
            "scalp_last_error": (ctypes.c_char_p, [P]),
            "scalp_destroy": (None, [P]),
            "scalp_label_means_static": (ctypes.c_int, [P, I64, P, I32, I32, I32, P, P]),
            "scalp_batch_workspace_bytes": (ctypes.c_size_t, [I32, P, P, P, ctypes.POINTER(scalp_params)]),
            "scalp_batch_init": (ctypes.c_int, [ctypes.POINTER(P), I32, P, P, P, P,
                                                ctypes.POINTER(scalp_params)]),
            "scalp_batch_reload": (ctypes.c_int, [P, P, P]),
            "scalp_batch_iterate": (ctypes.c_int, [P, I32]),
            "scalp_batch_labels": (ctypes.c_int, [P, P, I32, I32, P]),
            "scalp_batch_get_state": (ctypes.c_int, [P, I32, ctypes.POINTER(scalp_state)]),
            "scalp_batch_get_info": (ctypes.c_int, [P, I32, ctypes.POINTER(scalp_info)]),
            "scalp_batch_destroy": (None, [P]),
            "scalp_batch_set_launch": (ctypes.c_int, [P, I32]),
            "scalp_batch_get_launch": (ctypes.c_int, [P, ctypes.POINTER(I32), ctypes.POINTER(I32)]),
            "scalp_batch_set_wait": (ctypes.c_int, [P, I64, I32]),
            "scalp_batch_count_samples": (ctypes.c_int, [P, I32, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
            "scalp_batch_profile": (ctypes.c_int, [P, I32, ctypes.POINTER(ctypes.c_double),
                                                   ctypes.POINTER(I64)]),
            "scalp_batch_autotune": (ctypes.c_int, [P, P, P, I32, ctypes.c_char_p, ctypes.POINTER(I32),
                                                    P, ctypes.POINTER(I32)]),
            "scalp_server_reserve_bytes": (ctypes.c_size_t, [I32]),
            "scalp_server_create": (ctypes.c_int, [ctypes.POINTER(P), P, ctypes.c_size_t, I32,
                                                   ctypes.POINTER(scalp_params)]),
            "scalp_server_submit": (ctypes.c_int, [P, ctypes.POINTER(scalp_image),
                                                   ctypes.POINTER(scalp_contour), I32, ctypes.c_float,
                                                   I32, I32, P, ctypes.POINTER(ctypes.c_uint64)]),
            "scalp_server_step": (ctypes.c_int, [P, ctypes.POINTER(I32)]),
            "scalp_server_set_step_budget": (ctypes.c_int, [P, I64]),
            "scalp_server_poll": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.POINTER(I32),
                                                 ctypes.POINTER(I32)]),
            "scalp_server_stats": (ctypes.c_int, [P, ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_size_t)]),
            "scalp_server_inject_status": (ctypes.c_int, [P, ctypes.c_uint64, I32, I32]),
            "scalp_server_destroy": (None, [P]),
            "scalp_boundary_map": (ctypes.c_int, [P, I32, I32, I32, P, P]),
            "scalp_quality_workspace_bytes": (ctypes.c_size_t, [I32, I32, I32, I32]),
            "scalp_gradient_prior_workspace_bytes": (ctypes.c_size_t, [I32, I32, I32, I32]),
            "scalp_voxel_workspace_bytes": (ctypes.c_size_t, [I32, I32, I32, I32, ctypes.POINTER(scalp_params)]),
            "scalp_voxel_init": (ctypes.c_int, [ctypes.POINTER(P), ctypes.POINTER(scalp_volume), I32,
                                                ctypes.c_float, ctypes.POINTER(scalp_params)]),
            "scalp_voxel_iterate": (ctypes.c_int, [P, I32]),
            "scalp_voxel_labels": (ctypes.c_int, [P, P, I32]),
            "scalp_voxel_get_info": (ctypes.c_int, [P, ctypes.POINTER(scalp_voxel_info)]),
            "scalp_voxel_get_state": (ctypes.c_int, [P, ctypes.POINTER(scalp_voxel_state)]),
            "scalp_voxel_set_state": (ctypes.c_int, [P, ctypes.POINTER(scalp_voxel_state)]),
            "scalp_voxel_count_samples": (ctypes.c_int, [P, I32, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
            "scalp_voxel_profile": (ctypes.c_int, [P, I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64)]),
            "scalp_voxel_destroy": (None, [P]),
            "scalp_gradient_prior": (ctypes.c_int, [ctypes.POINTER(scalp_image), P, I64, I32, P, P,
                                                    ctypes.c_size_t]),
            "scalp_quality_metrics": (ctypes.c_int, [P, I32, P, I32, I32, I32, ctypes.c_double, P,
                                                     ctypes.c_size_t, ctypes.POINTER(scalp_quality), P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _check(rc: int, ctx=None):
    if rc != SCALP_OK:
        msg = load().scalp_last_error(ctx).decode(errors="replace")
        raise ScalpError(rc, msg)


# --- C names, argument marshalling only -------------------------------------
def scalp_default_params() -> scalp_params:
    p = scalp_params()
    load().scalp_default_params(ctypes.byref(p))
    return p


def scalp_workspace_bytes(H: int, W: int, K: int, params: scalp_params) -> int:
    return int(load().scalp_workspace_bytes(H, W, K, ctypes.byref(params)))


def scalp_init(image: scalp_image, contour: scalp_contour, K: int, m: float,
               params: scalp_params) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(load().scalp_init(ctypes.byref(ctx), ctypes.byref(image), ctypes.byref(contour),
                             int(K), float(m), ctypes.byref(params)))
    return ctx


def scalp_reload(ctx, image: scalp_image, contour: scalp_contour):
    _check(load().scalp_reload(ctx, ctypes.byref(image), ctypes.byref(contour)), ctx)


def scalp_iterate(ctx, n: int):
    _check(load().scalp_iterate(ctx, int(n)), ctx)


def scalp_labels(ctx, out_ptr: int, out_on_device: bool, enforce: bool) -> int:
    n = ctypes.c_int32()
    _check(load().scalp_labels(ctx, ctypes.c_void_p(out_ptr), int(out_on_device), int(enforce),
                               ctypes.byref(n)), ctx)
    return n.value


def scalp_get_info(ctx) -> scalp_info:
    info = scalp_info()
    _check(load().scalp_get_info(ctx, ctypes.byref(info)), ctx)
    return info


def scalp_get_state(ctx, state: scalp_state):
    _check(load().scalp_get_state(ctx, ctypes.byref(state)), ctx)


def scalp_set_state(ctx, state: scalp_state):
    _check(load().scalp_set_state(ctx, ctypes.byref(state)), ctx)


def scalp_clusters(ctx, Keff: int) -> np.ndarray:
    """(Keff, 5) float32 cluster descriptors (l, a, b, x, y) of Sec. II-A."""
    out = np.empty((Keff, 5), np.float32)
    k = ctypes.c_int32()
    _check(load().scalp_clusters(ctx, out.ctypes.data, ctypes.byref(k)), ctx)
    assert k.value == Keff
    return out


def scalp_debug_paths(ctx, pairs: np.ndarray, stride_xy: int):
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 4)
    M = len(pairs)
    out_xy = np.full((M, stride_xy), -1, dtype=np.int32)
    out_len = np.zeros(M, dtype=np.int32)
    _check(load().scalp_debug_paths(ctx, pairs.ctypes.data, M, out_xy.ctypes.data, stride_xy,
                                    out_len.ctypes.data), ctx)
    return out_xy, out_len


def scalp_profile(ctx, enable: int):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().scalp_profile(ctx, int(enable), ctypes.byref(ms), ctypes.byref(n)), ctx)
    return ms.value, n.value


def scalp_count_samples(ctx, enable: int, rects: bool = False):
    """(samples, pairs) of the last assignment, plus (map_rects, plane_rects)
    when rects; enable 1 resets and counts, 0 stops, -1 only reads."""
    v = [ctypes.c_int64() for _ in range(4)]
    _check(load().scalp_count_samples(ctx, int(enable), *(ctypes.byref(x) for x in v)), ctx)
    out = tuple(x.value for x in v)
    return out if rects else out[:2]


def scalp_sync(ctx):
    _check(load().scalp_sync(ctx), ctx)


def scalp_destroy(ctx):
    load().scalp_destroy(ctx)


def scalp_label_means_static(rgb_ptr: int, rgb_stride: int, labels_ptr: int, H: int, W: int,
                             n_labels: int, out_ptr: int, stream_ptr: int):
    """Per-label means with no device allocation (device pointers in and out)."""
    _check(load().scalp_label_means_static(ctypes.c_void_p(rgb_ptr), int(rgb_stride),
                                           ctypes.c_void_p(labels_ptr), int(H), int(W),
                                           int(n_labels), ctypes.c_void_p(out_ptr),
                                           ctypes.c_void_p(stream_ptr)))


# --- convenience wrapper over the C calls -------------------------------------
class Segmenter:
    """One SCALP solve on the current CUDA device.

    rgb: (H, W, 3) uint8, a CUDA tensor or a host numpy array / CPU tensor.
    contour: (H, W) float32 in [0,1] on the same side, or None.
    The workspace is a torch uint8 CUDA tensor owned by this object.
    """

    def __init__(self, rgb, contour, K: int, m: float = 10.0, lam: float = 0.5,
                 sigma: float = 0.25, gamma: float = -1.0, storage: str = "f32",
                 use_graph: bool = True, global_walk: bool = False, stream=None, prune: bool = True,
                 prior: str = "input"):
        import torch

        self._torch = torch
        H, W = int(rgb.shape[0]), int(rgb.shape[1])
        self.H, self.W, self.K = H, W, int(K)
        p = scalp_default_params()
        p.lambda_, p.sigma, p.gamma = lam, sigma, gamma
        p.storage = STORAGE[storage]
        p.use_graph = int(use_graph)
        p.global_walk = int(global_walk) | (0 if prune else 2)
        p.prior = PRIOR[prior]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        p.stream = self.stream.cuda_stream
        nbytes = scalp_workspace_bytes(H, W, K, p)
        if nbytes == 0:
            raise ScalpError(SCALP_E_ARG, "invalid sizes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        p.workspace = self.workspace.data_ptr()
        p.workspace_bytes = nbytes
        self.params = p
        img, con, self._keep = self._marshal(rgb, contour)
        self.ctx = scalp_init(img, con, K, m, p)
        self.info = scalp_get_info(self.ctx)

    def _marshal(self, rgb, contour):
        torch = self._torch
        keep = []
        if isinstance(rgb, torch.Tensor) and rgb.is_cuda:
            rgb = rgb.contiguous()
            keep.append(rgb)
            img = scalp_image(rgb.shape[0], rgb.shape[1], rgb.data_ptr(), 0, 1)
            con = scalp_contour(None, 0)
            if contour is not None:
                c = contour.to(device=rgb.device, dtype=torch.float32).contiguous()
                keep.append(c)
                con = scalp_contour(c.data_ptr(), 0)
        else:
            a = np.ascontiguousarray(np.asarray(rgb), dtype=np.uint8)
            keep.append(a)
            img = scalp_image(a.shape[0], a.shape[1], a.ctypes.data, 0, 0)
            con = scalp_contour(None, 0)
            if contour is not None:
                c = np.ascontiguousarray(np.asarray(contour), dtype=np.float32)
                keep.append(c)
                con = scalp_contour(c.ctypes.data, 0)
        return img, con, keep

    def reload(self, rgb, contour):
        img, con, self._keep = self._marshal(rgb, contour)
        scalp_reload(self.ctx, img, con)

    def iterate(self, n: int = 1):
        scalp_iterate(self.ctx, n)

    def labels(self, enforce: bool = True, out=None):
        """Labels as a (H, W) int32 array: into `out` (a CUDA tensor or a numpy
        array) if given, else a new numpy array.  Returns (labels, n_labels)."""
        torch = self._torch
        if out is None:
            out = np.empty((self.H, self.W), dtype=np.int32)
        if isinstance(out, torch.Tensor):
            assert out.is_cuda and out.dtype == torch.int32 and out.is_contiguous()
            n = scalp_labels(self.ctx, out.data_ptr(), True, enforce)
        else:
            assert out.dtype == np.int32 and out.flags["C_CONTIGUOUS"]
            n = scalp_labels(self.ctx, out.ctypes.data, False, enforce)
        return out, n

    def get_state(self):
        K = self.info.Keff
        st = dict(labels=np.empty((self.H, self.W), np.int32), n=np.empty(K, np.int64),
                  sx=np.empty(K, np.int64), sy=np.empty(K, np.int64),
                  color=np.empty((K, 3), np.float64), endpoint=np.empty((K, 2), np.int32))
        scalp_get_state(self.ctx, scalp_state(*(st[k].ctypes.data for k in
                                                ("labels", "n", "sx", "sy", "color", "endpoint"))))
        return st

    def set_state(self, st):
        arrs = dict(labels=np.ascontiguousarray(st["labels"], np.int32),
                    n=np.ascontiguousarray(st["n"], np.int64),
                    sx=np.ascontiguousarray(st["sx"], np.int64),
                    sy=np.ascontiguousarray(st["sy"], np.int64),
                    color=np.ascontiguousarray(st["color"], np.float64),
                    endpoint=np.ascontiguousarray(st["endpoint"], np.int32))
        scalp_set_state(self.ctx, scalp_state(*(arrs[k].ctypes.data for k in
                                                ("labels", "n", "sx", "sy", "color", "endpoint"))))

    def clusters(self):
        """(Keff, 5) float32: per cluster (l_k, a_k, b_k, x_k, y_k), Sec. II-A."""
        return scalp_clusters(self.ctx, self.info.Keff)

    def debug_paths(self, pairs, stride_xy: int | None = None):
        if stride_xy is None:
            stride_xy = 2 * (max(self.H, self.W) + 1)
        return scalp_debug_paths(self.ctx, pairs, stride_xy)

    def profile(self, enable: int):
        return scalp_profile(self.ctx, enable)

    def count_samples(self, enable: int, rects: bool = False):
        return scalp_count_samples(self.ctx, enable, rects)

    def sync(self):
        scalp_sync(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            scalp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- batches -----------------------------------------------------------------
def scalp_batch_workspace_bytes(H, W, K, params: scalp_params) -> int:
    H = np.ascontiguousarray(H, np.int32); W = np.ascontiguousarray(W, np.int32)
    K = np.ascontiguousarray(K, np.int32)
    return int(load().scalp_batch_workspace_bytes(len(H), H.ctypes.data, W.ctypes.data,
                                                  K.ctypes.data, ctypes.byref(params)))


def scalp_batch_init(images, contours, K, m, params: scalp_params) -> ctypes.c_void_p:
    n = len(images)
    imgs = (scalp_image * n)(*images)
    cons = (scalp_contour * n)(*contours) if contours is not None else None
    K = np.ascontiguousarray(K, np.int32)
    m = np.ascontiguousarray(m, np.float32)
    b = ctypes.c_void_p()
    _check(load().scalp_batch_init(ctypes.byref(b), n, ctypes.cast(imgs, ctypes.c_void_p),
                                   ctypes.cast(cons, ctypes.c_void_p) if cons is not None else None,
                                   K.ctypes.data, m.ctypes.data, ctypes.byref(params)))
    return b


def scalp_batch_reload(batch, images, contours):
    n = len(images)
    imgs = (scalp_image * n)(*images)
    cons = (scalp_contour * n)(*contours) if contours is not None else None
    _check(load().scalp_batch_reload(batch, ctypes.cast(imgs, ctypes.c_void_p),
                                     ctypes.cast(cons, ctypes.c_void_p) if cons is not None else None))


def scalp_batch_iterate(batch, n: int):
    _check(load().scalp_batch_iterate(batch, int(n)))


def scalp_batch_labels(batch, out_ptrs, out_on_device: bool, enforce: bool):
    n = len(out_ptrs)
    ptrs = (ctypes.c_void_p * n)(*out_ptrs)
    nl = np.zeros(n, np.int32)
    _check(load().scalp_batch_labels(batch, ctypes.cast(ptrs, ctypes.c_void_p), int(out_on_device),
                                     int(enforce), nl.ctypes.data))
    return nl


def scalp_batch_get_state(batch, index: int, state: scalp_state):
    _check(load().scalp_batch_get_state(batch, int(index), ctypes.byref(state)))


def scalp_batch_get_info(batch, index: int) -> scalp_info:
    info = scalp_info()
    _check(load().scalp_batch_get_info(batch, int(index), ctypes.byref(info)))
    return info


def scalp_batch_destroy(batch):
    load().scalp_batch_destroy(batch)


class Batch:
    """Many SCALP solves of uneven size on the current CUDA device.

    rgbs: list of (H_i, W_i, 3) uint8 CUDA tensors (or numpy arrays in host
    memory, copied in by the library); contours: list of (H_i, W_i) float32
    arrays on the same side, or None; Ks: list of K_i.
    """

    def __init__(self, rgbs, contours, Ks, m: float = 10.0, lam: float = 0.5, sigma: float = 0.25,
                 gamma: float = -1.0, storage: str = "f32", use_graph: bool = True,
                 global_walk: bool = False, stream=None, prior: str = "input"):
        import torch

        self._torch = torch
        self.count = len(rgbs)
        self.shapes = [(int(r.shape[0]), int(r.shape[1])) for r in rgbs]
        p = scalp_default_params()
        p.lambda_, p.sigma, p.gamma = lam, sigma, gamma
        p.storage = STORAGE[storage]
        p.use_graph = int(use_graph)
        p.global_walk = int(global_walk)
        p.prior = PRIOR[prior]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        p.stream = self.stream.cuda_stream
        H = [s[0] for s in self.shapes]
        W = [s[1] for s in self.shapes]
        nbytes = scalp_batch_workspace_bytes(H, W, Ks, p)
        if nbytes == 0:
            raise ScalpError(SCALP_E_ARG, "invalid batch sizes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        p.workspace = self.workspace.data_ptr()
        p.workspace_bytes = nbytes
        self.params = p
        imgs, cons, self._keep = self._marshal(rgbs, contours)
        self.batch = scalp_batch_init(imgs, cons, Ks, [m] * self.count, p)
        self.infos = [scalp_batch_get_info(self.batch, i) for i in range(self.count)]

    def _marshal(self, rgbs, contours):
        torch = self._torch
        keep, imgs, cons = [], [], []
        for i, r in enumerate(rgbs):
            c = None if contours is None else contours[i]
            if isinstance(r, np.ndarray):
                r = np.ascontiguousarray(r, dtype=np.uint8)
                keep.append(r)
                imgs.append(scalp_image(r.shape[0], r.shape[1], r.ctypes.data, 0, 0))
                if c is not None:
                    c = np.ascontiguousarray(c, dtype=np.float32)
                    keep.append(c)
                cons.append(scalp_contour(None if c is None else c.ctypes.data, 0))
                continue
            r = r.contiguous()
            keep.append(r)
            imgs.append(scalp_image(r.shape[0], r.shape[1], r.data_ptr(), 0, 1))
            if c is None:
                cons.append(scalp_contour(None, 0))
            else:
                c = c.to(device=r.device, dtype=torch.float32).contiguous()
                keep.append(c)
                cons.append(scalp_contour(c.data_ptr(), 0))
        return imgs, cons, keep

    def reload(self, rgbs, contours):
        imgs, cons, self._keep = self._marshal(rgbs, contours)
        scalp_batch_reload(self.batch, imgs, cons)

    def iterate(self, n: int = 1):
        scalp_batch_iterate(self.batch, n)

    def labels(self, enforce: bool = True, outs=None):
        """Labels of every image: into `outs` (CUDA int32 tensors) if given,
        else new numpy arrays.  Returns (labels list, n_labels array)."""
        torch = self._torch
        if outs is None:
            outs = [np.empty(s, dtype=np.int32) for s in self.shapes]
        on_dev = isinstance(outs[0], torch.Tensor)
        ptrs = [o.data_ptr() if on_dev else o.ctypes.data for o in outs]
        n = scalp_batch_labels(self.batch, ptrs, on_dev, enforce)
        return outs, n

    def set_launch(self, mode: str):
        """'flat', 'persistent' or 'persistent_cost' (scalp_batch_set_launch)."""
        _check(load().scalp_batch_set_launch(self.batch, BATCH_LAUNCH[mode]))

    def get_launch(self):
        m, g = ctypes.c_int32(), ctypes.c_int32()
        _check(load().scalp_batch_get_launch(self.batch, ctypes.byref(m), ctypes.byref(g)))
        return {v: k for k, v in BATCH_LAUNCH.items()}[m.value], g.value

    def set_wait(self, limit_ns: int = 2_000_000_000, hold: int = 0):
        _check(load().scalp_batch_set_wait(self.batch, int(limit_ns), int(hold)))

    def count_samples(self, enable: int):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(load().scalp_batch_count_samples(self.batch, int(enable), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def profile(self, enable: int):
        """(ms, launches) of the batched assignment launches since timing was
        enabled (none in a persistent launch mode)."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(load().scalp_batch_profile(self.batch, int(enable), ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def autotune(self, rgbs, contours, iters: int = 10, cache_path=None):
        """Times each launch mode and keeps the fastest (the batch is left
        freshly reloaded).  Returns (mode, {mode: ms}, from_cache)."""
        imgs, cons, keep = self._marshal(rgbs, contours)
        arr_i = (scalp_image * self.count)(*imgs)
        arr_c = (scalp_contour * self.count)(*cons)
        m, hit = ctypes.c_int32(), ctypes.c_int32()
        ms = (ctypes.c_float * 3)()
        path = cache_path.encode() if cache_path else None
        _check(load().scalp_batch_autotune(self.batch, ctypes.cast(arr_i, ctypes.c_void_p),
                                           ctypes.cast(arr_c, ctypes.c_void_p), int(iters), path,
                                           ctypes.byref(m), ctypes.cast(ms, ctypes.c_void_p),
                                           ctypes.byref(hit)))
        self._keep = keep
        names = {v: k for k, v in BATCH_LAUNCH.items()}
        return names[m.value], {names[i]: ms[i] for i in range(3) if ms[i] >= 0}, bool(hit.value)

    def get_state(self, index: int):
        info = self.infos[index]
        K = info.Keff
        st = dict(labels=np.empty((info.H, info.W), np.int32), n=np.empty(K, np.int64),
                  sx=np.empty(K, np.int64), sy=np.empty(K, np.int64),
                  color=np.empty((K, 3), np.float64), endpoint=np.empty((K, 2), np.int32))
        scalp_batch_get_state(self.batch, index, scalp_state(*(st[k].ctypes.data for k in
                                                               ("labels", "n", "sx", "sy", "color",
                                                                "endpoint"))))
        return st

    def close(self):
        if getattr(self, "batch", None):
            scalp_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- serving -------------------------------------------------------------------
def scalp_server_reserve_bytes(max_slots: int) -> int:
    return int(load().scalp_server_reserve_bytes(int(max_slots)))


def scalp_server_create(pool_ptr: int, pool_bytes: int, max_slots: int, params: scalp_params):
    s = ctypes.c_void_p()
    _check(load().scalp_server_create(ctypes.byref(s), ctypes.c_void_p(pool_ptr), int(pool_bytes),
                                      int(max_slots), ctypes.byref(params)))
    return s


def scalp_server_submit(server, image: scalp_image, contour: scalp_contour, K: int, m: float,
                        iters: int, enforce: bool, labels_out_ptr: int):
    """Request id, or None when the request does not fit now (SCALP_E_NOMEM)."""
    rid = ctypes.c_uint64()
    rc = load().scalp_server_submit(server, ctypes.byref(image), ctypes.byref(contour), int(K),
                                    float(m), int(iters), int(enforce),
                                    ctypes.c_void_p(labels_out_ptr), ctypes.byref(rid))
    if rc == SCALP_E_NOMEM:
        return None
    _check(rc)
    return rid.value


def scalp_server_step(server) -> int:
    n = ctypes.c_int32()
    _check(load().scalp_server_step(server, ctypes.byref(n)))
    return n.value


def scalp_server_poll(server, rid: int):
    """(done, n_labels).  A request that failed raises ScalpError with
    .done = True (it has been released)."""
    done = ctypes.c_int32()
    nl = ctypes.c_int32()
    rc = load().scalp_server_poll(server, ctypes.c_uint64(rid), ctypes.byref(done), ctypes.byref(nl))
    if rc != SCALP_OK:
        err = ScalpError(rc, load().scalp_last_error(None).decode(errors="replace"))
        err.done = bool(done.value)
        raise err
    return bool(done.value), nl.value


def scalp_server_inject_status(server, rid: int, error: int = 0, timeout: int = 0):
    _check(load().scalp_server_inject_status(server, ctypes.c_uint64(rid), int(error), int(timeout)))


def scalp_server_stats(server):
    n = ctypes.c_int32()
    f = ctypes.c_size_t()
    _check(load().scalp_server_stats(server, ctypes.byref(n), ctypes.byref(f)))
    return n.value, f.value


def scalp_server_destroy(server):
    load().scalp_server_destroy(server)


class Server:
    """Continuous batching of SCALP solves within a device memory budget."""

    def __init__(self, budget_bytes: int, max_slots: int = 1024, storage: str = "f32", m: float = 10.0,
                 iters: int = 10, enforce: bool = True, stream=None, step_pixels: int = 0):
        """step_pixels > 0: each step iterates the requests with the least
        remaining work within that many pixels (scalp_server_set_step_budget)."""
        import torch

        self._torch = torch
        p = scalp_default_params()
        p.storage = STORAGE[storage]
        self.stream = stream if stream is not None else torch.cuda.Stream()
        p.stream = self.stream.cuda_stream
        self.params = p
        self.pool = torch.empty(int(budget_bytes), dtype=torch.uint8, device="cuda")
        self.server = scalp_server_create(self.pool.data_ptr(), int(budget_bytes), max_slots, p)
        if step_pixels:
            _check(load().scalp_server_set_step_budget(self.server, int(step_pixels)))
        self.m, self.iters, self.enforce = m, iters, enforce
        self._keep = {}

    def submit(self, rgb, contour, K: int):
        """rgb (H, W, 3) uint8 and contour (H, W) float32, CUDA tensors.  Returns
        (id, pinned host labels tensor) or None when the request must wait."""
        torch = self._torch
        rgb = rgb.contiguous()
        img = scalp_image(rgb.shape[0], rgb.shape[1], rgb.data_ptr(), 0, 1)
        con = scalp_contour(None, 0)
        keep = [rgb]
        if contour is not None:
            c = contour.contiguous()
            keep.append(c)
            con = scalp_contour(c.data_ptr(), 0)
        out = torch.empty((rgb.shape[0], rgb.shape[1]), dtype=torch.int32, pin_memory=True)
        rid = scalp_server_submit(self.server, img, con, K, self.m, self.iters, self.enforce,
                                  out.data_ptr())
        if rid is None:
            return None
        self._keep[rid] = (keep, out)
        return rid, out

    def step(self) -> int:
        return scalp_server_step(self.server)

    def poll(self, rid: int):
        try:
            done, n = scalp_server_poll(self.server, rid)
        except ScalpError as e:
            if getattr(e, "done", False):
                self._keep.pop(rid, None)
            raise
        if done:
            self._keep.pop(rid, None)
        return done, n

    def inject_status(self, rid: int, error: int = 0, timeout: int = 0):
        """Test hook: request rid completes as if a device-side check failed."""
        scalp_server_inject_status(self.server, rid, error, timeout)

    def stats(self):
        return scalp_server_stats(self.server)

    def close(self):
        if getattr(self, "server", None):
            scalp_server_destroy(self.server)
            self.server = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- multi-scale boundary map ---------------------------------------------------
def scalp_boundary_map(label_ptrs, H: int, W: int, out_ptr: int, stream_ptr: int):
    n = len(label_ptrs)
    ptrs = (ctypes.c_void_p * n)(*label_ptrs)
    _check(load().scalp_boundary_map(ctypes.cast(ptrs, ctypes.c_void_p), n, int(H), int(W),
                                     ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream_ptr)))


def multiscale_K(k_min: int = 6, k_max: int = 600, scales: int = 12):
    """The scale ladder: scales values of K from k_min to k_max, geometric."""
    return [int(round(k_min * (k_max / k_min) ** (i / (scales - 1)))) for i in range(scales)]


def multiscale_boundaries(rgb, contour, Ks, iters: int = 10, storage: str = "f32", stream=None):
    """Solves one image (CUDA tensors) at every K of Ks as one batch and returns
    (boundary confidence map (H, W) float32 CUDA tensor, list of label tensors)."""
    import torch

    stream = stream if stream is not None else torch.cuda.current_stream()
    H, W = int(rgb.shape[0]), int(rgb.shape[1])
    b = Batch([rgb] * len(Ks), None if contour is None else [contour] * len(Ks), Ks,
              storage=storage, stream=stream)
    try:
        b.iterate(iters)
        outs = [torch.empty((H, W), dtype=torch.int32, device="cuda") for _ in Ks]
        b.labels(enforce=True, outs=outs)
        bmap = torch.empty((H, W), dtype=torch.float32, device="cuda")
        scalp_boundary_map([o.data_ptr() for o in outs], H, W, bmap.data_ptr(), stream.cuda_stream)
        stream.synchronize()
    finally:
        b.close()
    return bmap, outs


# --- quality metrics ----------------------------------------------------------------
def scalp_quality_workspace_bytes(H: int, W: int, n_labels: int, n_gt: int) -> int:
    return int(load().scalp_quality_workspace_bytes(int(H), int(W), int(n_labels), int(n_gt)))


def gradient_prior(rgb, out=None, stream=None):
    """Contour prior from the image on the GPU (scalp_gradient_prior): the
    CIELab gradient magnitude over its maximum, (H, W) float32 in [0, 1].

    rgb: (H, W, 3) uint8 CUDA tensor; out: optional (H, W) float32 CUDA tensor.
    Returns the output tensor (work enqueued on `stream`, not synchronised)."""
    import torch

    rgb = rgb.contiguous()
    H, W = int(rgb.shape[0]), int(rgb.shape[1])
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=rgb.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    L = load()
    nbytes = L.scalp_gradient_prior_workspace_bytes(H, W, 1, 1)
    if nbytes == 0:
        raise ScalpError(SCALP_E_ARG, "invalid sizes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=rgb.device)
    img = scalp_image(H, W, rgb.data_ptr(), 0, 1)
    _check(L.scalp_gradient_prior(ctypes.byref(img), out.data_ptr(), out.stride(0), 1,
                                  st.cuda_stream, ws.data_ptr(), nbytes), None)
    out._scalp_keep = (rgb, ws)  # the enqueued kernels read both
    return out


def quality_metrics(labels, gt, eps: float = 2.0, stream=None):
    """BR, ASA, UE, CO (Eq. 5-8) of a CUDA int32 label map against a CUDA int32
    ground truth, both (H, W).  Returns a dict."""
    import torch

    stream = stream if stream is not None else torch.cuda.current_stream()
    H, W = int(labels.shape[0]), int(labels.shape[1])
    n_labels = int(labels.max().item()) + 1
    n_gt = int(gt.max().item()) + 1
    nbytes = scalp_quality_workspace_bytes(H, W, n_labels, n_gt)
    if nbytes == 0:
        raise ScalpError(SCALP_E_ARG, "invalid sizes for the quality metrics")
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    q = scalp_quality()
    lab = labels.contiguous()
    g = gt.contiguous()
    _check(load().scalp_quality_metrics(ctypes.c_void_p(lab.data_ptr()), n_labels,
                                        ctypes.c_void_p(g.data_ptr()), n_gt, H, W, float(eps),
                                        ctypes.c_void_p(ws.data_ptr()), nbytes, ctypes.byref(q),
                                        ctypes.c_void_p(stream.cuda_stream)))
    return {"br": q.br, "asa": q.asa, "ue": q.ue, "co": q.co}


class VoxelSegmenter:
    """Supervoxels (SCALP on a (T, H, W) video volume) on the current CUDA device.

    rgb: (T, H, W, 3) uint8 CUDA tensor; contour: (T, H, W) float32 CUDA tensor
    in [0, 1], or None.  The workspace is a torch CUDA tensor owned here.
    """

    def __init__(self, rgb, contour, K: int, m: float = 10.0, lam: float = 0.5,
                 sigma: float = 0.25, gamma: float = -1.0, stream=None):
        import torch

        self._torch = torch
        T, H, W = (int(v) for v in rgb.shape[:3])
        self.T, self.H, self.W, self.K = T, H, W, int(K)
        p = scalp_default_params()
        p.lambda_, p.sigma, p.gamma = lam, sigma, gamma
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        p.stream = self.stream.cuda_stream
        L = load()
        nbytes = L.scalp_voxel_workspace_bytes(T, H, W, int(K), ctypes.byref(p))
        if nbytes == 0:
            raise ScalpError(SCALP_E_ARG, "invalid sizes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        p.workspace, p.workspace_bytes = self.workspace.data_ptr(), nbytes
        rgb = rgb.contiguous()
        con = contour.to(device=rgb.device, dtype=torch.float32).contiguous() if contour is not None else None
        vol = scalp_volume(T, H, W, rgb.data_ptr(), con.data_ptr() if con is not None else None, 1)
        ctx = ctypes.c_void_p()
        _check(L.scalp_voxel_init(ctypes.byref(ctx), ctypes.byref(vol), int(K), float(m), ctypes.byref(p)))
        self.ctx = ctx
        info = scalp_voxel_info()
        _check(L.scalp_voxel_get_info(self.ctx, ctypes.byref(info)))
        self.info = info

    @property
    def Keff(self) -> int:
        return self.info.Keff

    def iterate(self, n: int = 1):
        _check(load().scalp_voxel_iterate(self.ctx, int(n)))

    def labels(self, out=None):
        """(T, H, W) int32 labels: into `out` (a CUDA tensor) if given, else a numpy array."""
        if out is not None:
            _check(load().scalp_voxel_labels(self.ctx, out.data_ptr(), 1))
            return out
        a = np.empty((self.T, self.H, self.W), np.int32)
        _check(load().scalp_voxel_labels(self.ctx, a.ctypes.data, 0))
        return a

    def _state_arrays(self):
        K = self.Keff
        return dict(labels=np.empty((self.T, self.H, self.W), np.int32), n=np.empty(K, np.int64),
                    sx=np.empty(K, np.int64), sy=np.empty(K, np.int64), st=np.empty(K, np.int64),
                    color=np.empty((K, 3), np.float64), endpoint=np.empty((K, 3), np.int32))

    @staticmethod
    def _struct(d):
        return scalp_voxel_state(*(np.ascontiguousarray(d[k]).ctypes.data for k in
                                   ("labels", "n", "sx", "sy", "st", "color", "endpoint")))

    def get_state(self):
        d = self._state_arrays()
        s = self._struct(d)
        _check(load().scalp_voxel_get_state(self.ctx, ctypes.byref(s)))
        return d

    def set_state(self, d):
        d = {k: np.ascontiguousarray(v, dtype=self._state_arrays()[k].dtype) for k, v in d.items()}
        s = self._struct(d)
        _check(load().scalp_voxel_set_state(self.ctx, ctypes.byref(s)))

    def count_samples(self, enable: int):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(load().scalp_voxel_count_samples(self.ctx, int(enable), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def profile(self, enable: int):
        """(ms, launches) of the assignment launches since profiling was enabled."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(load().scalp_voxel_profile(self.ctx, int(enable), ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def close(self):
        if getattr(self, "ctx", None):
            load().scalp_voxel_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
