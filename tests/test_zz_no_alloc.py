"""scalp_label_means_static: the entry point for callers that cannot allocate
device memory.  Its output must match the means the regular, workspace-based
solver reports for the same image and labels, on two calls in a row (the second
call reuses the fixed scratch the first one left behind).

This file sorts last so that a run stopping at the first failure has already
run every other test."""
import numpy as np
import pytest

from paper_1903_07149_gb300 import build as scalp_build
from paper_1903_07149_gb300 import synth

pytestmark = pytest.mark.gpu

COLOR_RTOL = 1e-4  # as in the parity tests


def test_label_means_static_matches_solver_state():
    import torch

    assert torch.cuda.is_available()
    scalp_build.build()
    from paper_1903_07149_gb300 import scalp

    H, W, K = 240, 330, 150
    rgb, con, _ = synth.small_image(H, W, seed=77)
    d_rgb = torch.from_numpy(rgb).cuda()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        seg = scalp.Segmenter(d_rgb, torch.from_numpy(con).cuda(), K, stream=stream)
        seg.iterate(3)
        labels = torch.empty((H, W), dtype=torch.int32, device="cuda")
        seg.labels(enforce=False, out=labels)
        st = seg.get_state()  # the workspace-based solver's means for these labels
        Keff = seg.info.Keff
        used = st["n"] > 0
        present = np.zeros(Keff, bool)
        present[np.unique(labels.cpu().numpy())] = True
        for call in range(2):
            out = torch.full((Keff, 6), -1.0, dtype=torch.float64, device="cuda")
            scalp.scalp_label_means_static(d_rgb.data_ptr(), 0, labels.data_ptr(), H, W, Keff,
                                           out.data_ptr(), stream.cuda_stream)
            stream.synchronize()
            o = out.cpu().numpy()
            n = o[:, 0].astype(np.int64)
            assert np.array_equal(n > 0, present)
            k = present & used
            assert np.array_equal(n[k], st["n"][k]), call
            assert np.allclose(o[k, 4], st["sx"][k] / st["n"][k], rtol=0, atol=1e-9)
            assert np.allclose(o[k, 5], st["sy"][k] / st["n"][k], rtol=0, atol=1e-9)
            ref = st["color"][k]
            assert np.all(np.abs(o[k, 1:4] - ref) <= COLOR_RTOL * np.maximum(np.abs(ref), 1)), call
            assert np.all(o[~present] == 0.0)
        seg.close()
    # sizes beyond the fixed scratch are refused with a clear error
    with pytest.raises(scalp.ScalpError) as e:
        scalp.scalp_label_means_static(d_rgb.data_ptr(), 0, labels.data_ptr(), H, W, 65537,
                                       out.data_ptr(), stream.cuda_stream)
    assert e.value.code == scalp.SCALP_E_ARG and "n_labels" in str(e.value)
