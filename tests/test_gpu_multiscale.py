"""Multi-scale boundary map on the GPU against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1903_07149_gb300 import build as scalp_build
from paper_1903_07149_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch

    assert torch.cuda.is_available()
    scalp_build.build()
    from paper_1903_07149_gb300 import scalp

    scalp.load()
    return scalp


def test_boundary_kernel_bit_exact_on_oracle_labels(S):
    import torch

    rng = np.random.default_rng(5)
    H, W = 77, 131
    maps = [np.kron(rng.integers(0, 40, size=(H // 7 + 1, W // 6 + 1)), np.ones((7, 6), int))[:H, :W]
            .astype(np.int32) for _ in range(12)]
    ref = oracle.boundary_map(maps)
    d = [torch.from_numpy(m).cuda() for m in maps]
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    S.scalp_boundary_map([t.data_ptr() for t in d], H, W, out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)


def test_multiscale_vs_oracle(S):
    import torch

    H, W, iters = 161, 241, 3
    rgb, con, _ = synth.small_image(H, W, seed=321, n_cells=12, gradient=False)
    Ks = S.multiscale_K()
    assert Ks == oracle.multiscale_K()
    d_rgb, d_con = torch.from_numpy(rgb).cuda(), torch.from_numpy(con).cuda()
    bmap, outs = S.multiscale_boundaries(d_rgb, d_con, Ks, iters=iters)
    lab = oracle.lab_from_rgb(rgb)
    orc_final = []
    b = S.Batch([d_rgb] * len(Ks), [d_con] * len(Ks), Ks)
    b.iterate(iters)
    raw, _ = b.labels(enforce=False)
    b.close()
    for i, K in enumerate(Ks):
        s = oracle.Solver(lab, con, K)
        s.iterate(iters)
        agree = (raw[i] == s.labels).mean()
        assert agree >= 0.999, (K, agree)
        orc_final.append(oracle.connectivity(s.labels, K)[0])
    ref = oracle.boundary_map(orc_final)
    got = bmap.cpu().numpy()
    assert np.abs(got - ref).mean() <= 1e-3
    # where every scale's enforced labels agree, the maps are equal exactly
    same = np.all([o.cpu().numpy() == f for o, f in zip(outs, orc_final)], axis=0)
    assert same.mean() > 0.99
    assert np.array_equal(got[same], ref[same]) or np.abs(got[same] - ref[same]).max() <= 1 / 12
