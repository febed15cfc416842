"""Contour prior computed from the image on the GPU (scalp_gradient_prior):
element-wise against the oracle, host/device forms, and its use inside a
solve (params.prior = SCALP_PRIOR_GRADIENT).

Tolerance: the GPU converts sRGB to CIELab in FP32 (relative error ~1e-7 of
values up to ~100, so ~1e-5 absolute per channel) and forms the six
differences, their norm and the division by the maximum in FP32; the oracle
does all of it in FP64.  The prior is a ratio in [0, 1] of norms of such
differences, so 1e-5 absolute covers the FP32 error with margin."""
import numpy as np
import pytest

import oracle
from paper_1903_07149_gb300 import build as scalp_build
from paper_1903_07149_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def S():
    import torch

    assert torch.cuda.is_available()
    scalp_build.build()
    from paper_1903_07149_gb300 import scalp

    scalp.load()
    return scalp


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (29, 1), (2, 2), (9, 33), (150, 230), (321, 481)])
def test_prior_matches_oracle(S, H, W):
    import torch

    rgb, _, _ = synth.small_image(H, W, seed=H * 1000 + W, n_cells=max(2, H * W // 800))
    want = oracle.gradient_prior(oracle.lab_from_rgb(rgb))
    got = S.gradient_prior(torch.from_numpy(rgb).cuda())
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    assert got.shape == (H, W) and got.dtype == np.float32
    assert np.all((got >= 0) & (got <= 1))
    assert np.max(np.abs(got - want)) <= TOL


def test_prior_step_exact(S):
    import torch

    rgb = np.zeros((40, 70, 3), np.uint8)
    rgb[:, :33] = (30, 200, 90)
    rgb[:, 33:] = (220, 40, 10)
    got = S.gradient_prior(torch.from_numpy(rgb).cuda()).cpu().numpy()
    want = np.zeros((40, 70), np.float32)
    want[:, 32:34] = 1.0  # both columns hold the same FP32 difference, the maximum
    assert np.array_equal(got, want)
    flat = np.full((17, 23, 3), 91, np.uint8)
    assert np.all(S.gradient_prior(torch.from_numpy(flat).cuda()).cpu().numpy() == 0)


def test_prior_host_and_strided_forms(S):
    import ctypes

    import torch

    rgb, _, _ = synth.small_image(64, 90, seed=7)
    dev = S.gradient_prior(torch.from_numpy(rgb).cuda()).cpu().numpy()
    L = S.load()
    nbytes = L.scalp_gradient_prior_workspace_bytes(64, 90, 0, 0)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = np.full((64, 100), -1.0, np.float32)  # row stride 100 floats
    a = np.ascontiguousarray(rgb)
    img = S.scalp_image(64, 90, a.ctypes.data, 0, 0)
    rc = L.scalp_gradient_prior(ctypes.byref(img), out.ctypes.data, 100, 0,
                                torch.cuda.current_stream().cuda_stream, ws.data_ptr(), nbytes)
    assert rc == S.SCALP_OK
    assert np.array_equal(out[:, :90], dev) and np.all(out[:, 90:] == -1.0)
    # a workspace one byte short is refused
    rc = L.scalp_gradient_prior(ctypes.byref(img), out.ctypes.data, 100, 0,
                                torch.cuda.current_stream().cuda_stream, ws.data_ptr(), nbytes - 1)
    assert rc == S.SCALP_E_NOMEM


def test_solve_with_gradient_prior(S):
    """A solve that computes its prior equals one handed the same prior."""
    import torch

    rgb, _, _ = synth.small_image(150, 230, seed=11)
    t = torch.from_numpy(rgb).cuda()
    prior = S.gradient_prior(t)
    a = S.Segmenter(t, None, 120, prior="gradient")
    b = S.Segmenter(t, prior, 120)
    a.iterate(5)
    b.iterate(5)
    la, na = a.labels(enforce=True)
    lb, nb = b.labels(enforce=True)
    assert na == nb and np.array_equal(la, lb)
    with pytest.raises(S.ScalpError):
        S.Segmenter(t, prior, 120, prior="gradient")
    a.close(); b.close()


def test_gradient_prior_one_step_parity(S):
    """One assignment with the GPU prior, against the oracle run on the
    oracle's own prior of the same image (same state).  Near-tie bound: the
    priors differ by <= 1e-5 (TOL); w = 1 - exp(-C^2/sigma^2) has slope at most
    sqrt(2/e)/sigma = 3.43 at sigma = 0.25, so each w and their path mean move
    by <= 3.5e-5, and the contour factor 1 + gamma*mean(w) (gamma = 2r = 33.9
    here) by <= 1.2e-3 relative: a flip is accepted below a 2e-3 gap."""
    import torch

    from test_gpu_parity import check_one_step, to_gpu_state

    rgb, _, _ = synth.small_image(150, 230, seed=12)
    C = oracle.gradient_prior(oracle.lab_from_rgb(rgb))
    orc = oracle.Solver(oracle.lab_from_rgb(rgb), C, 120)
    orc.iterate(2)
    st = orc.state()
    seg = S.Segmenter(torch.from_numpy(rgb).cuda(), None, 120, prior="gradient")
    seg.set_state(to_gpu_state(st))
    seg.iterate(1)
    g = seg.get_state()
    orc.assign()
    check_one_step(orc, g["labels"], orc.labels, st, near_tie=2e-3)
    seg.close()
