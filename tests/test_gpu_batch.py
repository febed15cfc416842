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


def _inputs(seed=500):
    import torch

    rgbs, cons = [], []
    for i, (H, W, K) in enumerate(SIZES):
        rgb, con, _ = synth.small_image(H, W, seed=seed + i, n_cells=max(2, H * W // 3000))
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


def test_batch_reload_new_and_host_inputs(S):
    """A batch set up on one set of images and reloaded with another of the
    same sizes gives what each new image gives alone, into device buffers that
    change between calls and into host memory; reloaded from host copies of
    the first set, it gives the first result again."""
    import torch

    rgbs_a, cons_a = _inputs(500)
    rgbs_b, cons_b = _inputs(900)
    Ks = [k for _, _, k in SIZES]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = S.Batch(rgbs_a, cons_a, Ks, stream=stream)
        b.iterate(3)
        first, n_first = b.labels(enforce=True)
        b.reload(rgbs_b, cons_b)
        b.iterate(3)
        raw, _ = b.labels(enforce=False)
        outs1 = [torch.full(r.shape[:2], -7, dtype=torch.int32, device="cuda") for r in rgbs_b]
        outs2 = [torch.full(r.shape[:2], -7, dtype=torch.int32, device="cuda") for r in rgbs_b]
        _, n1 = b.labels(enforce=True, outs=outs1)
        _, n2 = b.labels(enforce=True, outs=outs2)
        host, n3 = b.labels(enforce=True)
        for i, (H, W, K) in enumerate(SIZES):
            s = S.Segmenter(rgbs_b[i], cons_b[i], K, stream=stream)
            s.iterate(3)
            lab, _ = s.labels(enforce=False)
            assert np.array_equal(raw[i], lab), i
            out, n = s.labels(enforce=True)
            assert n == n1[i] == n2[i] == n3[i], i
            assert np.array_equal(outs1[i].cpu().numpy(), out), i
            assert np.array_equal(outs2[i].cpu().numpy(), out), i
            assert np.array_equal(host[i], out), i
            s.close()
        b.reload([r.cpu().numpy() for r in rgbs_a], [c.cpu().numpy() for c in cons_a])
        b.iterate(3)
        again, n_again = b.labels(enforce=True)
        assert np.array_equal(n_first, n_again)
        for x, y in zip(first, again):
            assert np.array_equal(x, y)
        b.close()


def test_batch_gradient_prior(S):
    """With the prior computed from each image (an odd number of images), a
    batch gives what each image gives alone, also after a reload."""
    import torch

    rgbs, _ = _inputs(700)
    sizes = SIZES[:5]
    rgbs = rgbs[:5]
    Ks = [k for _, _, k in sizes]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = S.Batch(rgbs, None, Ks, stream=stream, prior="gradient")
        b.iterate(4)
        first, n_first = b.labels(enforce=True)
        b.reload(rgbs, None)
        b.iterate(4)
        again, n_again = b.labels(enforce=True)
        assert np.array_equal(n_first, n_again)
        for i, (H, W, K) in enumerate(sizes):
            s = S.Segmenter(rgbs[i], None, K, stream=stream, prior="gradient")
            s.iterate(4)
            out, n = s.labels(enforce=True)
            assert n == n_first[i], i
            assert np.array_equal(first[i], out), i
            assert np.array_equal(again[i], out), i
            s.close()
        b.close()


def _alone_vs_batch(S, sizes, Ks, seed, iters=3):
    import torch

    rgbs, cons = [], []
    for i, (H, W) in enumerate(sizes):
        rgb, con, _ = synth.small_image(H, W, seed=seed + i, n_cells=max(2, H * W // 600))
        rgbs.append(torch.from_numpy(rgb).cuda())
        cons.append(torch.from_numpy(con).cuda())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = S.Batch(rgbs, cons, Ks, stream=stream)
        b.iterate(iters)
        raw, _ = b.labels(enforce=False)
        final, nfinal = b.labels(enforce=True)
        for i, K in enumerate(Ks):
            s = S.Segmenter(rgbs[i], cons[i], K, stream=stream)
            s.iterate(iters)
            lab, _ = s.labels(enforce=False)
            assert np.array_equal(raw[i], lab), (i, sizes[i], K)
            out, n = s.labels(enforce=True)
            assert n == nfinal[i] and np.array_equal(final[i], out), (i, sizes[i], K)
            s.close()
        b.close()


def test_many_small_images(S):
    """48 images of random size from 1x1 to 89x89 (many without tile borders in
    one or both directions) and random K: every flat launch maps its blocks to
    the right image."""
    rng = np.random.default_rng(123)
    sizes = [(int(rng.integers(1, 90)), int(rng.integers(1, 90))) for _ in range(48)]
    Ks = [int(rng.integers(1, min(H * W, 40) + 1)) for H, W in sizes]
    _alone_vs_batch(S, sizes, Ks, seed=1200)


def test_batch_of_single_tiles(S):
    """Every image fits in one 32x32 tile, so the border pass of the batch has
    no work at all and is not launched."""
    rng = np.random.default_rng(321)
    sizes = [(int(rng.integers(1, 33)), int(rng.integers(1, 33))) for _ in range(20)]
    Ks = [int(rng.integers(1, min(H * W, 12) + 1)) for H, W in sizes]
    _alone_vs_batch(S, sizes, Ks, seed=1300)
