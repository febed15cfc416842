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


def test_projection_work_lists(S):
    """A batch that takes both of the projection's work lists: 40 images of
    256x256 with K = 1024 (grid step 8, 17x17 windows: thousands of queued
    clusters, one warp each) and 4 of 480x640 with K = 20 (windows far above
    4096 pixels: one CTA each).  Labels, counts, sums, colours and endpoints
    equal each image solved alone."""
    import torch

    sizes = [(256, 256)] * 40 + [(480, 640)] * 4
    Ks = [1024] * 40 + [20] * 4
    rgbs, cons = [], []
    for i, (H, W) in enumerate(sizes):
        rgb, con, _ = synth.small_image(H, W, seed=1400 + i, n_cells=max(2, H * W // 600))
        rgbs.append(torch.from_numpy(rgb).cuda())
        cons.append(torch.from_numpy(con).cuda())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = S.Batch(rgbs, cons, Ks, stream=stream)
        b.iterate(4)
        raw, _ = b.labels(enforce=False)
        projected = 0
        for i, K in enumerate(Ks):
            s = S.Segmenter(rgbs[i], cons[i], K, stream=stream)
            s.iterate(4)
            lab, _ = s.labels(enforce=False)
            assert np.array_equal(raw[i], lab), (i, sizes[i], K)
            sa, sb = s.get_state(), b.get_state(i)
            for k in ("n", "sx", "sy", "color", "endpoint"):
                assert np.array_equal(sa[k], sb[k]), (i, k)
            if i < 40:  # clusters the last update queued: endpoint != rounded barycenter
                n = sb["n"]
                half_up = (2 * sb["sx"] + n) // np.maximum(2 * n, 1), (2 * sb["sy"] + n) // np.maximum(2 * n, 1)
                projected += int(((n > 0) & ((sb["endpoint"][:, 0] != half_up[0]) |
                                             (sb["endpoint"][:, 1] != half_up[1]))).sum())
            s.close()
        b.close()
    # the warp list needs more queued clusters than four per CTA (304 CTAs)
    assert projected > 4 * 2 * 152, projected


def test_more_tiles_than_the_lists_scan_holds(S):
    """A 3008x4224 image has 12,408 tiles, more than the single-image list
    kernel scans in shared memory (12,287): its lists come from the separate
    scan and fill kernels beside the projection.  Solved alone it equals the
    same image in a batch of one, whose lists a batch builds per image."""
    import torch

    H, W, K = 3008, 4224, 3000
    rgb, con, _ = synth.small_image(H, W, seed=1500, n_cells=400)
    d_rgb, d_con = torch.from_numpy(rgb).cuda(), torch.from_numpy(con).cuda()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = S.Segmenter(d_rgb, d_con, K, stream=stream)
        s.iterate(3)
        lab, _ = s.labels(enforce=False)
        b = S.Batch([d_rgb], [d_con], [K], stream=stream)
        b.iterate(3)
        raw, _ = b.labels(enforce=False)
        assert np.array_equal(raw[0], lab)
        sa, sb = s.get_state(), b.get_state(0)
        for k in ("n", "sx", "sy", "color", "endpoint"):
            assert np.array_equal(sa[k], sb[k]), k
        s.close()
        b.close()


def test_batch_of_single_tiles(S):
    """Every image fits in one 32x32 tile, so the border pass of the batch has
    no work at all and is not launched."""
    rng = np.random.default_rng(321)
    sizes = [(int(rng.integers(1, 33)), int(rng.integers(1, 33))) for _ in range(20)]
    Ks = [int(rng.integers(1, min(H * W, 12) + 1)) for H, W in sizes]
    _alone_vs_batch(S, sizes, Ks, seed=1300)


def _batch_result(b):
    raw, _ = b.labels(enforce=False)
    final, n = b.labels(enforce=True)
    states = [b.get_state(i) for i in range(b.count)]
    return raw, final, n, states


def _assert_same(r1, r2):
    raw1, fin1, n1, st1 = r1
    raw2, fin2, n2, st2 = r2
    assert np.array_equal(n1, n2)
    for i in range(len(raw1)):
        assert np.array_equal(raw1[i], raw2[i]), i
        assert np.array_equal(fin1[i], fin2[i]), i
        for k in ("n", "sx", "sy", "color", "endpoint"):
            assert np.array_equal(st1[i][k], st2[i][k]), (i, k)


def test_batch_profile_times_each_assignment(S):
    """Timing the batched assignment launches (events around each one, the
    programmatic overlap off meanwhile) counts one launch per iteration,
    also across graph replays of two lengths, changes no result, and times
    nothing in a persistent launch mode, whose assignment runs inside one
    kernel."""
    import torch

    rgbs, cons = _inputs()
    Ks = [k for _, _, k in SIZES]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = S.Batch(rgbs, cons, Ks, stream=stream)
        b.iterate(4)
        b.iterate(3)
        ref = _batch_result(b)
        b.reload(rgbs, cons)
        assert b.profile(1) == (0.0, 0)
        b.iterate(4)
        b.iterate(3)
        ms, n = b.profile(-1)  # read, keep timing
        assert n == 7 and ms > 0.0
        _assert_same(ref, _batch_result(b))
        b.reload(rgbs, cons)
        b.iterate(7)
        ms2, n2 = b.profile(0)
        assert n2 == 14 and ms2 > ms
        assert b.profile(-1) == (ms2, n2)  # stopped: nothing more is added
        b.reload(rgbs, cons)
        b.iterate(7)
        assert b.profile(-1) == (ms2, n2)
        _assert_same(ref, _batch_result(b))
        b.set_launch("persistent")
        b.reload(rgbs, cons)
        b.profile(1)
        b.iterate(7)
        assert b.profile(0) == (0.0, 0)
        _assert_same(ref, _batch_result(b))
        b.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_persistent_launch_equals_flat(S, storage):
    """All iterations of the batch in one cooperative launch (tiles from a
    queue, grid-wide barriers between the phases), the queue in batch order
    and by descending grid step: bit-identical to the per-kernel launches,
    also after a reload and across two calls of different lengths; the
    device-counted path samples agree too."""
    import torch

    rgbs, cons = _inputs()
    Ks = [k for _, _, k in SIZES]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = S.Batch(rgbs, cons, Ks, storage=storage, stream=stream)
        b.count_samples(1)
        b.iterate(4)
        b.iterate(3)
        ref_samples = b.count_samples(0)
        ref = _batch_result(b)
        for mode in ("persistent", "persistent_cost"):
            b.set_launch(mode)
            m, grid = b.get_launch()
            assert m == mode and grid >= torch.cuda.get_device_properties(0).multi_processor_count
            b.reload(rgbs, cons)
            b.count_samples(1)
            b.iterate(4)
            b.iterate(3)
            assert b.count_samples(0) == ref_samples
            _assert_same(ref, _batch_result(b))
        b.set_launch("flat")
        b.reload(rgbs, cons)
        b.iterate(7)
        _assert_same(ref, _batch_result(b))
        b.close()


def test_persistent_wait_runs_out_and_batch_recovers(S):
    """A barrier wait that can never complete (the test hold: one more arrival
    than there are CTAs, nothing faulted) runs out after its 20 ms limit:
    every CTA returns, the labels call reports SCALP_E_TIMEOUT, and after a
    reload the batch gives the right result again."""
    import time

    import torch

    rgbs, cons = _inputs()
    Ks = [k for _, _, k in SIZES]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ref_b = S.Batch(rgbs, cons, Ks, stream=stream)
        ref_b.iterate(3)
        ref = _batch_result(ref_b)
        ref_b.close()
        b = S.Batch(rgbs, cons, Ks, stream=stream)
        b.set_launch("persistent")
        b.set_wait(20_000_000, hold=1)
        t0 = time.perf_counter()
        b.iterate(3)
        with pytest.raises(S.ScalpError) as e:
            b.labels(enforce=True)
        assert e.value.code == S.SCALP_E_TIMEOUT
        assert time.perf_counter() - t0 < 30.0
        b.set_wait()  # default limit, no hold
        b.reload(rgbs, cons)
        b.iterate(3)
        _assert_same(ref, _batch_result(b))
        b.close()


def test_autotune_chooses_and_caches(S, tmp_path):
    """The autotuner times every launch mode, keeps the fastest, leaves the
    batch freshly reloaded (its solve then equals the flat one) and writes
    its choice to the JSON cache, which a second batch of the same shape
    class then reads without trials."""
    import json

    import torch

    rgbs, cons = _inputs()
    Ks = [k for _, _, k in SIZES]
    cache = str(tmp_path / "autotune.json")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ref_b = S.Batch(rgbs, cons, Ks, stream=stream)
        ref_b.iterate(5)
        ref = _batch_result(ref_b)
        ref_b.close()
        b = S.Batch(rgbs, cons, Ks, stream=stream)
        mode, ms, hit = b.autotune(rgbs, cons, iters=5, cache_path=cache)
        assert not hit and set(ms) == {"flat", "persistent", "persistent_cost"}
        assert ms[mode] == min(ms.values())
        assert b.get_launch()[0] == mode
        b.iterate(5)
        _assert_same(ref, _batch_result(b))
        b.close()
        with open(cache) as f:
            entries = json.load(f)
        assert len(entries) == 1 and list(entries.values())[0]["mode"] == S.BATCH_LAUNCH[mode]
        b2 = S.Batch(rgbs, cons, Ks, stream=stream)
        mode2, ms2, hit2 = b2.autotune(rgbs, cons, iters=5, cache_path=cache)
        assert hit2 and mode2 == mode and ms2 == {}
        b2.iterate(5)
        _assert_same(ref, _batch_result(b2))
        b2.close()
