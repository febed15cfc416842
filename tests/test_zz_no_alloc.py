"""scalp_label_means_static: the entry point for callers that cannot allocate
device memory (a plugin handed only its buffers, code running while another
component owns the device memory budget).  Its output must match the means the
regular, workspace-based solver reports for the same image and labels, and the
means of the oracle's independent FP64 CIELab, on two calls in a row (the
second call reuses the fixed scratch the first one left behind), and the second
call must not change the device's free memory.

This file sorts last so that a run stopping at the first failure has already
run every other test."""
import numpy as np
import pytest

import oracle
from paper_1903_07149_gb300 import build as scalp_build
from paper_1903_07149_gb300 import synth

pytestmark = pytest.mark.gpu

COLOR_RTOL = 1e-4  # as in the parity tests


def test_label_means_static_matches_solver_and_oracle():
    import torch

    assert torch.cuda.is_available()
    scalp_build.build()
    from paper_1903_07149_gb300 import scalp

    H, W, K = 240, 330, 150
    rgb, con, _ = synth.small_image(H, W, seed=77)
    d_rgb = torch.from_numpy(rgb).cuda()
    stream = torch.cuda.Stream()
    # independent reference: numpy means of the oracle's FP64 CIELab
    lab64 = np.stack(oracle.lab_from_rgb(rgb), axis=-1).reshape(-1, 3)
    ys, xs = np.mgrid[0:H, 0:W]
    with torch.cuda.stream(stream):
        seg = scalp.Segmenter(d_rgb, torch.from_numpy(con).cuda(), K, stream=stream)
        seg.iterate(3)
        labels = torch.empty((H, W), dtype=torch.int32, device="cuda")
        seg.labels(enforce=False, out=labels)
        st = seg.get_state()  # the workspace-based solver's means for these labels
        Keff = seg.info.Keff
        lab_h = labels.cpu().numpy().ravel()
        cnt = np.bincount(lab_h, minlength=Keff)
        present = cnt > 0
        used = st["n"] > 0
        ref_col = np.stack([np.bincount(lab_h, weights=lab64[:, c], minlength=Keff) for c in range(3)],
                           axis=1)[present] / cnt[present, None]
        ref_x = np.bincount(lab_h, weights=xs.ravel(), minlength=Keff)[present] / cnt[present]
        ref_y = np.bincount(lab_h, weights=ys.ravel(), minlength=Keff)[present] / cnt[present]
        outs = [torch.full((Keff, 6), -1.0, dtype=torch.float64, device="cuda") for _ in range(2)]
        torch.cuda.synchronize()
        free = []
        for call in range(2):
            scalp.scalp_label_means_static(d_rgb.data_ptr(), 0, labels.data_ptr(), H, W, Keff,
                                           outs[call].data_ptr(), stream.cuda_stream)
            stream.synchronize()
            free.append(torch.cuda.mem_get_info()[0])
            o = outs[call].cpu().numpy()
            n = o[:, 0].astype(np.int64)
            assert np.array_equal(n, cnt), call
            # against the oracle's CIELab and numpy's exact coordinate means
            assert np.all(np.abs(o[present, 1:4] - ref_col) <= COLOR_RTOL * np.maximum(np.abs(ref_col), 1)), call
            assert np.array_equal(o[present, 4], ref_x) and np.array_equal(o[present, 5], ref_y), call
            # against the solver's own state for the same labels
            k = present & used
            assert np.array_equal(n[k], st["n"][k]), call
            ref = st["color"][k]
            assert np.all(np.abs(o[k, 1:4] - ref) <= COLOR_RTOL * np.maximum(np.abs(ref), 1)), call
            assert np.all(o[~present] == 0.0)
        # the first call may load the module (its fixed scratch); the second
        # allocates nothing
        assert free[1] == free[0], free
        seg.close()
    # sizes beyond the fixed scratch are refused with a clear error
    with pytest.raises(scalp.ScalpError) as e:
        scalp.scalp_label_means_static(d_rgb.data_ptr(), 0, labels.data_ptr(), H, W, 65537,
                                       outs[0].data_ptr(), stream.cuda_stream)
    assert e.value.code == scalp.SCALP_E_ARG and "n_labels" in str(e.value)
