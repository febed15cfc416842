"""Serving: requests admitted into a memory-bounded server while others are
in flight give exactly what each image gives alone."""
import time

import numpy as np
import pytest

from paper_1903_07149_gb300 import build as scalp_build
from paper_1903_07149_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [(150, 230, 120), (97, 131, 40), (240, 320, 400), (33, 47, 1), (100, 140, 2),
         (64, 96, 24), (181, 263, 300), (300, 420, 500), (120, 160, 90), (211, 97, 60)]


@pytest.fixture(scope="module")
def S():
    import torch

    assert torch.cuda.is_available()
    scalp_build.build()
    from paper_1903_07149_gb300 import scalp

    scalp.load()
    return scalp


@pytest.mark.parametrize("storage,step_pixels", [("f32", 0), ("f16", 0), ("f32", 60000)])
def test_serving_mix_equals_alone(S, storage, step_pixels):
    """step_pixels > 0: each step iterates only the least remaining work
    within the budget; every request still gets all its iterations."""
    import torch

    imgs = []
    for i, (H, W, K) in enumerate(SIZES):
        rgb, con, _ = synth.small_image(H, W, seed=900 + i, n_cells=max(2, H * W // 3000))
        imgs.append((torch.from_numpy(rgb).cuda(), torch.from_numpy(con).cuda(), K))
    p = S.scalp_default_params()
    p.storage = S.STORAGE[storage]
    need = [S.scalp_workspace_bytes(H, W, K, p) for H, W, K in SIZES]
    # room for about three requests at a time: later ones wait for memory
    budget = S.scalp_server_reserve_bytes(8) + 3 * max(need) + (1 << 20)
    stream = torch.cuda.Stream()
    srv = S.Server(budget, max_slots=8, storage=storage, iters=6, stream=stream, step_pixels=step_pixels)
    pending = list(range(len(SIZES)))
    inflight, results, waited, steps = {}, {}, 0, 0
    t_end = time.monotonic() + 120.0  # the host runs ahead: idle steps spin
    while pending or inflight:
        # two new arrivals per step, while memory and slots allow
        for _ in range(2):
            if not pending:
                break
            i = pending[0]
            r = srv.submit(*imgs[i])
            if r is None:
                waited += 1
                break
            pending.pop(0)
            inflight[r[0]] = (i, r[1])
        steps += srv.step() > 0
        for rid in list(inflight):
            done, n = srv.poll(rid)
            if done:
                i, out = inflight.pop(rid)
                results[i] = (out.numpy().copy(), n)
        assert steps < 500 and time.monotonic() < t_end
    assert waited > 0  # admission was bounded by memory
    with torch.cuda.stream(stream):
        for i, (rgb, con, K) in enumerate(imgs):
            s = S.Segmenter(rgb, con, K, storage=storage, stream=stream)
            s.iterate(6)
            ref, nref = s.labels(enforce=True)
            out, n = results[i]
            assert n == nref and np.array_equal(out, ref), i
            s.close()
    srv.close()


def test_serving_zero_iterations(S):
    """Requests with no iterations never join a step: each is retired by the
    next step call, and its delivery must wait for its own set-up (on a side
    stream).  Their labels equal solves with no iterations."""
    import torch

    sizes = SIZES[:5]
    imgs = []
    for i, (H, W, K) in enumerate(sizes):
        rgb, con, _ = synth.small_image(H, W, seed=950 + i, n_cells=max(2, H * W // 3000))
        imgs.append((torch.from_numpy(rgb).cuda(), torch.from_numpy(con).cuda(), K))
    p = S.scalp_default_params()
    need = [S.scalp_workspace_bytes(H, W, K, p) for H, W, K in sizes]
    budget = S.scalp_server_reserve_bytes(8) + sum(need) + (1 << 20)
    stream = torch.cuda.Stream()
    srv = S.Server(budget, max_slots=8, storage="f32", iters=0, stream=stream)
    inflight = {}
    for i, im in enumerate(imgs):
        r = srv.submit(*im)
        assert r is not None
        inflight[r[0]] = (i, r[1])
    assert srv.step() == 0  # nothing to iterate; all retire
    results = {}
    t_end = time.monotonic() + 60.0
    while inflight:
        for rid in list(inflight):
            done, n = srv.poll(rid)
            if done:
                i, out = inflight.pop(rid)
                results[i] = (out.numpy().copy(), n)
        assert time.monotonic() < t_end
    with torch.cuda.stream(stream):
        for i, (rgb, con, K) in enumerate(imgs):
            s = S.Segmenter(rgb, con, K, storage="f32", stream=stream)
            ref, nref = s.labels(enforce=True)
            out, n = results[i]
            assert n == nref and np.array_equal(out, ref), i
            s.close()
    srv.close()


def test_two_servers_two_threads(S):
    """Two servers on streams of different priority, each driven by its own
    host thread (the serving benchmark's configuration), with step budgets:
    every delivered request equals the image solved alone."""
    import threading

    import torch

    imgs = []
    for i, (H, W, K) in enumerate(SIZES):
        rgb, con, _ = synth.small_image(H, W, seed=980 + i, n_cells=max(2, H * W // 3000))
        imgs.append((torch.from_numpy(rgb).cuda(), torch.from_numpy(con).cuda(), K))
    p = S.scalp_default_params()
    p.storage = S.STORAGE["f16"]
    need = [S.scalp_workspace_bytes(H, W, K, p) for H, W, K in SIZES]
    split = 40000  # pixels: smaller requests to the high-priority server
    device = torch.cuda.current_device()
    lanes = []
    for prio, mine in ((-5, [i for i, (H, W, _) in enumerate(SIZES) if H * W <= split]),
                       (0, [i for i, (H, W, _) in enumerate(SIZES) if H * W > split])):
        st = torch.cuda.Stream(priority=prio)
        budget = S.scalp_server_reserve_bytes(8) + sum(need[i] for i in mine) + (1 << 20)
        srv = S.Server(budget, max_slots=8, storage="f16", iters=5, stream=st, step_pixels=30000)
        lanes.append((srv, mine))
    results, errors = {}, []

    def drive(srv, mine):
        try:
            torch.cuda.set_device(device)
            inflight = {}
            for i in mine:
                r = srv.submit(*imgs[i])
                assert r is not None
                inflight[r[0]] = (i, r[1])
            t_end = time.monotonic() + 60.0
            while inflight:
                srv.step()
                for rid in list(inflight):
                    done, n = srv.poll(rid)
                    if done:
                        i, out = inflight.pop(rid)
                        results[i] = (out.numpy().copy(), n)
                assert time.monotonic() < t_end
        except Exception as exc:
            errors.append(exc)

    threads = [threading.Thread(target=drive, args=lane) for lane in lanes]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for i, (rgb, con, K) in enumerate(imgs):
            s = S.Segmenter(rgb, con, K, storage="f16", stream=stream)
            s.iterate(5)
            ref, nref = s.labels(enforce=True)
            out, n = results[i]
            assert n == nref and np.array_equal(out, ref), i
            s.close()
    for srv, _ in lanes:
        srv.close()


def test_serving_failed_request_is_released(S):
    """A request whose device-side status reports a failure (injected on the
    host: no GPU fault is made) is delivered as failed, with its pool region
    and slot released: the server then admits as many requests as before and
    their results are unaffected."""
    import torch

    H, W, K = 150, 230, 120
    rgb, con, _ = synth.small_image(H, W, seed=950)
    img = (torch.from_numpy(rgb).cuda(), torch.from_numpy(con).cuda(), K)
    p = S.scalp_default_params()
    need = S.scalp_workspace_bytes(H, W, K, p)
    budget = S.scalp_server_reserve_bytes(2) + 2 * need + (1 << 20)
    stream = torch.cuda.Stream()
    srv = S.Server(budget, max_slots=2, iters=3, stream=stream)
    _, free0 = srv.stats()

    def run(inject):
        ids = [srv.submit(*img)[0] for _ in range(2)]
        assert srv.submit(*img) is None  # both slots taken
        for rid, (err, tmo) in zip(ids, inject):
            if err or tmo:
                srv.inject_status(rid, err, tmo)
        out = {}
        for _ in range(200):
            srv.step()
            for rid in ids:
                if rid in out:
                    continue
                try:
                    done, n = srv.poll(rid)
                except S.ScalpError as e:
                    assert e.done
                    out[rid] = e.code
                    continue
                if done:
                    out[rid] = n
            if len(out) == 2:
                break
        return [out[r] for r in ids]

    res = run([(7, 0), (0, 1)])
    assert res == [S.SCALP_E_INTERNAL, S.SCALP_E_TIMEOUT]
    in_flight, free1 = srv.stats()
    assert in_flight == 0 and free1 == free0
    res = run([(0, 0), (0, 0)])  # slots and memory are back; results are right
    with torch.cuda.stream(stream):
        s = S.Segmenter(*img, stream=stream)
        s.iterate(3)
        _, nref = s.labels(enforce=True)
        s.close()
    assert res == [nref, nref]
    srv.close()
