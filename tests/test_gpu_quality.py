"""Quality metrics (Eq. 5-8) on the GPU against the oracle, on oracle-made
decompositions of synthetic images whose Voronoi cells are the ground truth."""
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


@pytest.mark.parametrize("seed,K", [(51, 60), (52, 250)])
def test_quality_matches_oracle(S, seed, K):
    import torch

    rgb, C, cells = synth.small_image(180, 260, seed=seed, n_cells=10)
    s, out, n = oracle.solve(rgb, C, K, iters=4)
    ref = oracle.quality(out, cells)
    got = S.quality_metrics(torch.from_numpy(out).cuda(), torch.from_numpy(cells).cuda())
    assert got["br"] == ref["br"] and got["asa"] == ref["asa"] and got["ue"] == ref["ue"]
    assert got["co"] == pytest.approx(ref["co"], rel=1e-12)


def test_quality_of_gpu_decomposition_is_sane(S):
    import torch

    rgb, C, cells = synth.small_image(240, 320, seed=53, n_cells=12)
    seg = S.Segmenter(torch.from_numpy(rgb).cuda(), torch.from_numpy(C).cuda(), 300)
    seg.iterate(10)
    out = torch.empty((240, 320), dtype=torch.int32, device="cuda")
    seg.labels(enforce=True, out=out)
    q = S.quality_metrics(out, torch.from_numpy(cells).cuda())
    assert 0.9 < q["asa"] <= 1.0 and 0.0 <= q["ue"] < 0.5 and 0.5 < q["br"] <= 1.0
    assert 0.2 < q["co"] < np.pi / 4 + 1e-9
    seg.close()
