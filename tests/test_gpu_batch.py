"""Batched solves: many images of uneven size and K in one set of launches give
exactly (bit for bit) what each image gives when solved alone."""
import numpy as np
import pytest

from paper_1903_07149_gb300 import build as scalp_build
from paper_1903_07149_gb300 import synth

pytestmark = pytest.mark.gpu

# (H, W, K): ragged tiles, tiny images, images whose map boxes overflow the
# shared-memory map buffer (some paths walk the plane in global memory),
# K = 1 and K = N
SIZES = [(150, 230, 120), (97, 131, 40), (240, 320, 400), (33, 47, 1), (100, 140, 2),
         (64, 96, 24), (7, 9, 63), (181, 263, 300)]


@pytest.fixture(scope="module")
def S():
    import torch

    assert torch.cuda.is_available()
    scalp_build.build()
    from paper_1903_07149_gb300 import scalp

    scalp.load()
    return scalp


def _inputs():
    import torch

    rgbs, cons = [], []
    for i, (H, W, K) in enumerate(SIZES):
        rgb, con, _ = synth.small_image(H, W, seed=500 + i, n_cells=max(2, H * W // 3000))
        rgbs.append(torch.from_numpy(rgb).cuda())
        cons.append(torch.from_numpy(con).cuda())
    return rgbs, cons


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_equals_alone(S, storage):
    import torch

    rgbs, cons = _inputs()
    Ks = [k for _, _, k in SIZES]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = S.Batch(rgbs, cons, Ks, storage=storage, stream=stream)
        assert all(info.map_pairs > 0 for info in b.infos)
        b.iterate(4)
        b.iterate(3)  # a second graph length
        raw, _ = b.labels(enforce=False)
        final, nfinal = b.labels(enforce=True)
        for i, (H, W, K) in enumerate(SIZES):
            s = S.Segmenter(rgbs[i], cons[i], K, storage=storage, stream=stream)
            s.iterate(7)
            lab, _ = s.labels(enforce=False)
            assert np.array_equal(raw[i], lab), i
            out, n = s.labels(enforce=True)
            assert n == nfinal[i] and np.array_equal(final[i], out), i
            sa, sb = s.get_state(), b.get_state(i)
            for k in ("n", "sx", "sy", "color", "endpoint"):
                assert np.array_equal(sa[k], sb[k]), (i, k)
            s.close()
        b.close()


def test_batch_reload_and_device_outputs(S):
    import torch

    rgbs, cons = _inputs()
    Ks = [k for _, _, k in SIZES]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = S.Batch(rgbs, cons, Ks, stream=stream)
        b.iterate(3)
        first, n1 = b.labels(enforce=True)
        b.reload(rgbs, cons)  # the same inputs again: the same result
        b.iterate(3)
        outs = [torch.empty(r.shape[:2], dtype=torch.int32, device="cuda") for r in rgbs]
        second, n2 = b.labels(enforce=True, outs=outs)
        assert np.array_equal(n1, n2)
        for a_, b_ in zip(first, second):
            assert np.array_equal(a_, b_.cpu().numpy())
        b.close()
