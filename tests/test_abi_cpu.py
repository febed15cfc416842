"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/scalp.h declares, and rejects bad arguments on the host
before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1903_07149_gb300 import build as scalp_build
from paper_1903_07149_gb300 import scalp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    scalp_build.build()
    return scalp.load()


def _declared_functions():
    with open(os.path.join(ROOT, "include", "scalp.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(scalp_[a-z_]+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(scalp.EXPORTS) == declared


def test_default_params(lib):
    p = scalp.scalp_default_params()
    assert p.lambda_ == 0.5 and p.sigma == 0.25 and p.gamma < 0
    assert p.storage == 0 and p.use_graph == 1 and p.global_walk == 0


def test_workspace_bytes(lib):
    p = scalp.scalp_default_params()
    small = scalp.scalp_workspace_bytes(321, 481, 400, p)
    big = scalp.scalp_workspace_bytes(1080, 1920, 2000, p)
    assert 0 < small < big
    # planes, labels and the connectivity buffers dominate: > 40 bytes/pixel
    assert big > 40 * 1080 * 1920
    p.storage = 1
    assert scalp.scalp_workspace_bytes(1080, 1920, 2000, p) < big
    p.storage = 0
    for H, W, K in [(0, 5, 1), (5, 0, 1), (5, 5, 0), (5, 5, 26), (1 << 16, 1 << 15, 10)]:
        assert scalp.scalp_workspace_bytes(H, W, K, p) == 0


def _init(lib, H=8, W=8, K=4, m=10.0, rgb=True, ws=True, **over):
    p = scalp.scalp_default_params()
    for k, v in over.items():
        setattr(p, k, v)
    buf = np.zeros((max(H, 1), max(W, 1), 3), np.uint8)
    img = scalp.scalp_image(H, W, buf.ctypes.data if rgb else None, 0, 0)
    con = scalp.scalp_contour(None, 0)
    if ws:
        p.workspace = None
        p.workspace_bytes = 0
    ctx = ctypes.c_void_p()
    rc = lib.scalp_init(ctypes.byref(ctx), ctypes.byref(img), ctypes.byref(con), K, m,
                        ctypes.byref(p))
    return rc, ctx, lib.scalp_last_error(None).decode()


def test_init_rejects_bad_arguments_on_host(lib):
    assert _init(lib, K=0)[0] == scalp.SCALP_E_ARG
    assert _init(lib, K=65)[0] == scalp.SCALP_E_ARG
    assert _init(lib, H=0)[0] == scalp.SCALP_E_ARG
    assert _init(lib, m=0.0)[0] == scalp.SCALP_E_ARG
    assert _init(lib, m=float("nan"))[0] == scalp.SCALP_E_ARG
    assert _init(lib, rgb=False)[0] == scalp.SCALP_E_ARG
    assert _init(lib, lambda_=1.5)[0] == scalp.SCALP_E_ARG
    assert _init(lib, sigma=0.0)[0] == scalp.SCALP_E_ARG
    assert _init(lib, storage=3)[0] == scalp.SCALP_E_ARG
    rc, ctx, msg = _init(lib)  # valid, but no workspace given
    assert rc == scalp.SCALP_E_NOMEM and "workspace" in msg
    assert not ctx.value


def test_null_context_calls(lib):
    assert lib.scalp_iterate(None, 1) == scalp.SCALP_E_ARG
    assert lib.scalp_sync(None) == scalp.SCALP_E_ARG
    ms, n = ctypes.c_double(-1.0), ctypes.c_int64(-1)
    assert lib.scalp_profile(None, 1, ctypes.byref(ms), ctypes.byref(n)) == scalp.SCALP_E_ARG
    # a NULL batch is refused before anything is read or written
    assert lib.scalp_batch_iterate(None, 1) == scalp.SCALP_E_ARG
    assert lib.scalp_batch_profile(None, 1, ctypes.byref(ms), ctypes.byref(n)) == scalp.SCALP_E_ARG
    assert (ms.value, n.value) == (-1.0, -1)
    a, b = ctypes.c_int64(-1), ctypes.c_int64(-1)
    assert lib.scalp_batch_count_samples(None, 1, ctypes.byref(a), ctypes.byref(b)) == scalp.SCALP_E_ARG
    assert (a.value, b.value) == (-1, -1)
    lib.scalp_destroy(None)  # no-op
    lib.scalp_batch_destroy(None)  # no-op
