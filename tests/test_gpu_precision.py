"""Precision statement per workload: FP32 and FP16-storage solves (10
iterations from the grid, free-running) against the FP64 oracle run the same
way, through the C ABI.  Reported per storage: label agreement, and the
barycenter and colour errors over all clusters and over the clusters whose
final pixel set matches.

Bars: FP32 reaches >= 99.9% label agreement (the metric's bar) with every
matching cluster's barycenter exact and colour within 1e-4 relative.  FP16
storage rounds L, a, b and the contour factor to 2^-11 relative, so near-ties
flip and the flips move centres over ten iterations; its agreement is stated,
and gated at the level measured on GB300 (it does not meet the 99.9% bar)."""
import numpy as np
import pytest

import oracle
from paper_1903_07149_gb300 import build as scalp_build
from paper_1903_07149_gb300 import synth

pytestmark = pytest.mark.gpu

COLOR_RTOL = 1e-4


@pytest.fixture(scope="module")
def S():
    import torch

    assert torch.cuda.is_available()
    scalp_build.build()
    from paper_1903_07149_gb300 import scalp

    scalp.load()
    return scalp


@pytest.fixture(scope="module")
def oracle_runs():
    """FP64 oracle after 10 iterations (row-parallel on every host core; equal
    to Algorithm 1's loop bit for bit, pinned on the CPU) per workload."""
    out = {}
    for name in ("bsd_321x481_k400", "hd_1080x1920_k2000"):
        w, rgb, con = synth.single_image_config(name)
        s = oracle.Solver(oracle.lab_from_rgb(rgb), con, w.K)
        s.iterate_rows(w.iters)
        out[name] = (w, rgb, con, s)
    return out


def precision_stats(g, orc):
    """Agreement and errors of a GPU state g against the oracle solver orc."""
    diff = g["labels"] != orc.labels
    bad = np.unique(np.concatenate([g["labels"][diff], orc.labels[diff]]))
    # clusters holding pixels whose pixel set is the same on both sides (an
    # empty cluster keeps whatever state its history left it)
    present = np.unique(orc.labels)
    same = np.setdiff1d(present, bad)
    cg = np.stack([g["sx"] / g["n"], g["sy"] / g["n"]], axis=1)
    co = orc.centers()
    dcen = np.hypot(*(cg - co).T)
    ref = orc.colors()
    dcol = np.max(np.abs(g["color"] - ref) / np.maximum(np.abs(ref), 1), axis=1)
    return {"agreement": float(1.0 - diff.mean()), "clusters": int(orc.Keff),
            "clusters_same_pixels": int(len(same)),
            "centre_err_max_px": float(dcen.max()), "centre_err_p99_px": float(np.percentile(dcen, 99)),
            "centre_err_max_px_same": float(dcen[same].max()) if len(same) else 0.0,
            "colour_rel_err_max_same": float(dcol[same].max()) if len(same) else 0.0,
            "same": same}


@pytest.mark.parametrize("name", ["bsd_321x481_k400", "hd_1080x1920_k2000"])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_precision_statement(S, oracle_runs, name, storage):
    import torch

    w, rgb, con, orc = oracle_runs[name]
    seg = S.Segmenter(torch.from_numpy(rgb).cuda(), torch.from_numpy(con).cuda(), w.K, storage=storage)
    seg.iterate(w.iters)
    g = seg.get_state()
    st = precision_stats(g, orc)
    same = st.pop("same")
    print(f"{name} {storage}: {st}")
    if storage == "f32":
        assert st["agreement"] >= 0.999, st
        assert st["centre_err_max_px_same"] == 0.0, st
        assert st["colour_rel_err_max_same"] <= COLOR_RTOL, st
    else:
        assert st["agreement"] >= 0.96, st
        assert st["colour_rel_err_max_same"] <= 2e-3, st
    assert len(same) > 0
    seg.close()
