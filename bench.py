#!/usr/bin/env python3
"""SCALP throughput benchmark (Mpix*iter/s) on GB300.

One step = one whole solve of the workload: load the image (CIELab, contour
factor, grid clusters), 10 iterations of assignment + update + projection,
connectivity enforcement, labels written to device memory.  Inputs are resident
in HBM when the timed region starts; L2 is flushed (256 MB write) before every
timed step, outside its events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): independent replicas, one solve per rank per step, no
collective on the data path (the images are independent).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpix·iter/s, plain FP32 vs batched FP16-storage, at ≥99.9% oracle label agreement"
UNIT = "Mpix*iter/s"
DEFAULT_WORKLOAD = "hd_1080x1920_k2000"
SMS = 152
FP32_LANES_PER_SM = 128
SMEM_BYTES_PER_CLK_PER_SM = 128  # 32 banks x 4 bytes
FALLBACK_SM_MHZ = 2070.0
# Algorithmic work of the assignment, as the method states it:
#  * each path sample gathers one (L, a, b, w) pixel: 16 bytes stored in FP32,
#    8 in FP16 (the binding roof: on-chip load bandwidth);
#  * FP32 flops: per sample 3 sub, 3 mul-add (counted as 6) and 2 adds, about
#    10 counted conservatively; per evaluated (pixel, cluster) pair about 30
#    (own colour distance, spatial distance, Eq. 1-3 assembly, comparison).
FLOPS_PER_SAMPLE = 10
FLOPS_PER_PAIR = 30
# The FP32 lane operations counted per sample / pair in the earlier line
# (kept as a secondary figure): 7 and 20.
LANE_OPS_PER_SAMPLE = 7
LANE_OPS_PER_PAIR = 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--storage", choices=["f32", "f16"], default="f32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP16-storage, batched and serving forms")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving form")
    ap.add_argument("--only-form", choices=["gradient_prior", "supervoxels", "serving", "batched"],
                    help="diagnostics: run only this form and print its result (not the benchmark line)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        import statistics

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# Kernels per step: reload = set-up (with the grid clusters' sums), update,
# projection, candidate lists;
# each iteration = assignment (with the sums), update, projection, candidate
# lists.  The lists are one kernel up to 12,287 tiles, else a scan and a fill.
FALLBACK_HBM_GBS = 6800.0


def list_launches(H: int, W: int) -> int:
    tiles = -(-H // 32) * -(-W // 32)
    return 1 if tiles <= 12287 else 2


def reload_launches(H: int, W: int) -> int:
    return 3 + list_launches(H, W)


def iter_launches(H: int, W: int) -> int:
    return 3 + list_launches(H, W)


def rank_max(x: float, device: str = "cuda") -> float:
    """Max of a per-rank number over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as td

    if not (td.is_available() and td.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: float, world: int, slowest_ms: float) -> float:
    """Mpix*iter/s of the whole job: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (slowest_ms / 1e3) / 1e6


def ccl_launches(H: int, W: int) -> int:
    """Connectivity kernels: tile-local, border (when there is more than one
    tile), flatten/count, link, resolve/count, chunk scan, numbering, output."""
    return 7 + (1 if H > 32 or W > 32 else 0)


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("scalp_assign.cu", "scalp_assign_tile.cuh", "scalp_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1903_07149_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(storage: str):
    """DRAM bytes per assignment launch from the committed ncu summary, or None
    when the kernel source changed since those counters were taken."""
    path = os.path.join(ROOT, "profiles", "assign_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(storage)
        if e and e.get("kernel_hash") == kernel_hash():
            return e.get("bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def assign_roofline(samples, pairs, pixels, launch_s, storage, sm_mhz, clk_measured=True, traffic=None):
    """Roofline of one assignment launch from its algorithmic work: the path
    samples' gathered bytes against the shared-memory load peak (the binding
    roof), FP32 flops against the FMA peak, and the compulsory HBM bytes
    against the measured copy bandwidth.  Peaks other than HBM are derived
    from unit counts and the SM clock (no measured figure exists for them)."""
    bps = 16 if storage == "f32" else 8
    clk = f"{sm_mhz:.0f} MHz ({'nvidia-smi clocks.max.sm' if clk_measured else 'fallback'})"
    smem_peak = SMEM_BYTES_PER_CLK_PER_SM * SMS * sm_mhz * 1e6 / 1e9
    fma_peak = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    lane_peak = SMS * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    ok = launch_s and launch_s > 0
    smem = samples * bps / launch_s / 1e9 if ok else None
    flops = (FLOPS_PER_SAMPLE * samples + FLOPS_PER_PAIR * pairs) / launch_s / 1e12 if ok else None
    lane = (LANE_OPS_PER_SAMPLE * samples + LANE_OPS_PER_PAIR * pairs) / launch_s / 1e12 if ok else None
    peaks = measured_peaks() or {}
    hbm_peak = peaks.get("hbm_gbs") or FALLBACK_HBM_GBS
    hbm = pixels * (bps + 8) / launch_s / 1e9 if ok else None
    return {
        "bound": "smem", "kernel": "k_assign", "achieved": smem, "peak": smem_peak, "unit": "GB/s",
        "frac": smem / smem_peak if ok else None, "traffic": traffic,
        "peak_source": f"derived: {SMEM_BYTES_PER_CLK_PER_SM} B/clk/SM shared-memory loads x {SMS} SMs x {clk}",
        "algorithmic": {"samples_per_launch": samples, "pairs_per_launch": pairs,
                        "bytes_per_sample": bps, "flops_per_sample": FLOPS_PER_SAMPLE,
                        "flops_per_pair": FLOPS_PER_PAIR},
        "launch_ms": launch_s * 1e3 if ok else None,
        "alu": {"achieved": flops, "peak": fma_peak, "unit": "TFLOP/s",
                "frac": flops / fma_peak if ok else None,
                "peak_source": f"derived: {SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 (FMA) x {clk}"},
        "alu_lane_ops": {"achieved": lane, "peak": lane_peak, "unit": "T op/s",
                         "frac": lane / lane_peak if ok else None,
                         "ops_per_sample": LANE_OPS_PER_SAMPLE, "ops_per_pair": LANE_OPS_PER_PAIR},
        "hbm_compulsory": {"achieved": hbm, "peak": hbm_peak, "unit": "GB/s",
                           "frac": hbm / hbm_peak if ok else None,
                           "bytes_per_pixel": bps + 8,
                           "peak_source": "measured (MEASURED_PEAKS.json)" if peaks.get("hbm_gbs")
                           else "fallback 6.8 TB/s"},
    }


# ---------------------------------------------------------------------------
# CPU legs: the only place bench.py runs the oracle (the CPU baseline, the
# reference arm and the FP64 labels the precision statement compares with).
# ---------------------------------------------------------------------------
def host_cpu():
    """(threads the oracle uses, CPU model) of this host."""
    n = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform

    return n, f"{model or 'unknown'} ({platform.machine()})"


def cpu_baseline_oracle(w, rgb, con, budget_s: float = 20.0, runs: int = 3):
    """The FP64 oracle as it stands on every host core (its row-parallel
    iterations, bit-identical to Algorithm 1's loop), on a bounded sample:
    grid initialisation then as many whole-image iterations as fit about
    budget_s / runs seconds; the median of `runs` such runs."""
    import statistics

    import oracle

    cores, model = host_cpu()
    lab = oracle.lab_from_rgb(rgb)
    N = w.H * w.W
    vals, iters = [], []
    for _ in range(runs):
        s = oracle.Solver(lab, con, w.K)
        done, t_iter = 0, 0.0
        while True:
            t0 = time.perf_counter()
            s.iterate_rows(1, cores)
            t_iter += time.perf_counter() - t0
            done += 1
            if t_iter * (done + 1) / done > budget_s / runs or done >= w.iters:
                break
        vals.append(N * done / t_iter / 1e6)
        iters.append(done)
    return {"value": statistics.median(vals), "unit": UNIT, "cores": cores, "cpu": model,
            "kind": "oracle", "runs": vals,
            "sample": f"median of {runs} runs, each {iters[0]} whole-image iteration(s) of {w.name} "
                      f"from the grid state (FP64 C oracle, rows over {cores} OpenMP threads)"}


def cpu_precision_statement(gpu_states, cores):
    """Label agreement and centre / colour errors of GPU solves against the
    FP64 oracle run the same way (10 iterations from the grid, free-running).
    gpu_states: {key: (workload, rgb, contour, {storage: state})}."""
    import numpy as np

    import oracle

    out = {}
    for key, (w, rgb, con, states) in gpu_states.items():
        orc = oracle.Solver(oracle.lab_from_rgb(rgb), con, w.K)
        t0 = time.perf_counter()
        orc.iterate_rows(w.iters, cores)
        t_orc = time.perf_counter() - t0
        co, ref = orc.centers(), orc.colors()
        row = {"H": w.H, "W": w.W, "K": w.K, "Keff": int(orc.Keff), "iters": w.iters,
               "oracle_s": t_orc}
        for storage, g in states.items():
            diff = g["labels"] != orc.labels
            bad = np.unique(np.concatenate([g["labels"][diff], orc.labels[diff]]))
            same = np.setdiff1d(np.unique(orc.labels), bad)  # non-empty, same pixels
            cg = np.stack([g["sx"] / g["n"], g["sy"] / g["n"]], axis=1)
            dcen = np.hypot(*(cg - co).T)
            dcol = np.max(np.abs(g["color"] - ref) / np.maximum(np.abs(ref), 1), axis=1)
            row[storage] = {
                "label_agreement": float(1.0 - diff.mean()),
                "meets_99_9": bool(1.0 - diff.mean() >= 0.999),
                "clusters_same_pixels": int(len(same)),
                "centre_err_max_px": float(dcen.max()),
                "centre_err_p99_px": float(np.percentile(dcen, 99)),
                "centre_err_max_px_same_pixels": float(dcen[same].max()) if len(same) else None,
                "colour_rel_err_max_same_pixels": float(dcol[same].max()) if len(same) else None,
            }
        out[key] = row
    return out


def line_config(w, world: int) -> dict:
    """The workload both arms name (same keys and values in both lines)."""
    return {"workload": w.name, "H": w.H, "W": w.W, "K": w.K, "iters": w.iters,
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}


def run_reference(args):
    """The reference arm: the FP64 oracle (there is no reference code), on
    every host core, on the same workload; each step is one whole-image
    iteration (a bounded sample of the workload's 10-iteration solve)."""
    world, rank, local = dist_env()
    if rank != 0:
        return
    from paper_1903_07149_gb300 import synth
    import oracle

    cores, model = host_cpu()
    w, rgb, con = synth.single_image_config(args.workload)
    lab = oracle.lab_from_rgb(rgb)
    N = w.H * w.W
    s = oracle.Solver(lab, con, w.K)
    for _ in range(args.warmup):
        s.iterate_rows(1, cores)
    t = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        s.iterate_rows(1, cores)
        t += time.perf_counter() - t0
    value = N * args.steps / t / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": line_config(w, world),
        "timing": "each step is one whole-image iteration of the FP64 CPU oracle "
                  f"(rows over {cores} OpenMP threads)",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu": model, "kind": "oracle",
                         "sample": f"{args.steps} whole-image iterations of {w.name}, "
                                   f"after {args.warmup} warm-up iterations"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_batch(args, storage: str, flush, batch_imgs, sm_mhz=None):
    """The batched form: 64 images of uneven size and K (H~U{240..1080},
    W~U{320..1920}, grid step S~U[12,30]) solved together, 10 iterations each;
    one step = reload + 10 batched iterations + connectivity for all images.
    The launch mode (per-kernel launches replayed as a graph, or one
    persistent launch with the queue in batch order or by grid step) is
    chosen by the library's autotuner first; every mode's time is reported."""
    import tempfile

    import torch

    from paper_1903_07149_gb300 import scalp

    ws, rgbs, cons = batch_imgs
    d_rgb = [torch.from_numpy(r).cuda() for r in rgbs]
    d_con = [torch.from_numpy(c).cuda() for c in cons]
    outs = [torch.empty((w.H, w.W), dtype=torch.int32, device="cuda") for w in ws]
    stream = torch.cuda.Stream()
    pix = sum(w.H * w.W for w in ws)
    iters = ws[0].iters
    with torch.cuda.stream(stream), tempfile.TemporaryDirectory() as tmp:
        b = scalp.Batch(d_rgb, d_con, [w.K for w in ws], storage=storage, stream=stream)
        mode, trial_ms, _ = b.autotune(d_rgb, d_con, iters=iters, cache_path=os.path.join(tmp, "tune.json"))

        def step():
            b.reload(d_rgb, d_con)
            b.iterate(iters)
            b.labels(enforce=True, outs=outs)

        for _ in range(args.warmup):
            step()
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev0[i].record(stream)
            step()
            ev1[i].record(stream)
        torch.cuda.synchronize()
        # the iteration loop alone (the batched kernels), for the split and
        # the roofline, and the path samples of those iterations
        b.reload(d_rgb, d_con)
        b.count_samples(1)
        flush.zero_()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        b.iterate(iters)
        t1.record(stream)
        torch.cuda.synchronize()
        samples, pairs = b.count_samples(0)
        # the same iterations once more with each assignment launch bracketed
        # by events (flat launches only: a persistent launch runs the
        # assignment inside one kernel)
        assign_s = None
        if mode == "flat":
            b.reload(d_rgb, d_con)
            b.profile(1)
            flush.zero_()
            b.iterate(iters)
            a_ms, a_n = b.profile(0)
            if a_n:
                assign_s = a_ms / a_n / 1e3
        b.close()
    total_ms = sum(a.elapsed_time(c) for a, c in zip(ev0, ev1))
    it_s = t0.elapsed_time(t1) / 1e3 / iters
    clk_args = dict(clk_measured=sm_mhz is not None)
    whole = assign_roofline(samples / iters, pairs / iters, pix, it_s, storage, sm_mhz or FALLBACK_SM_MHZ,
                            **clk_args)
    whole_iteration = {"achieved": whole["achieved"], "frac": whole["frac"], "iteration_ms": it_s * 1e3,
                       "note": "the same samples over the whole iteration (assignment, update, "
                               "projection, lists)"}
    if assign_s:
        roof = assign_roofline(samples / iters, pairs / iters, pix, assign_s, storage,
                               sm_mhz or FALLBACK_SM_MHZ, **clk_args)
        roof["kernel"] = "k_assign_batch"
        roof["note"] = "per assignment launch (CUDA events around each launch, one launch per iteration)"
    else:
        roof = whole
        roof["kernel"] = "k_batch_persistent" if mode != "flat" else "k_assign_batch"
        roof["note"] = whole_iteration["note"]
    roof["whole_iteration"] = whole_iteration
    return {"value": pix * iters * args.steps / (total_ms / 1e3) / 1e6, "unit": UNIT,
            "ms_per_step": total_ms / args.steps, "images": len(ws), "mpix": pix / 1e6,
            "iters": iters, "storage": storage, "launch": mode,
            "autotune_ms_per_mode": {k: v for k, v in trial_ms.items()},
            "iterations_only_mpix_iter_s": pix * iters / (it_s * iters) / 1e6,
            "roofline": roof,
            "workload": "64 images, H~U{240..1080}, W~U{320..1920}, S~U[12,30], K=round(HW/S^2)"}


def measure_serving(args, batch_imgs, n_requests: int = 2000, rate_hz: float = 500.0,
                    budget_gb: float = 40.0, storage: str = "f16", step_mpix: float = 4.0,
                    split_mpix: float = 4.0, large_first: bool = False, serial: bool = True,
                    large_step_mpix: float | None = None, equal_priority: bool = False,
                    large_solo: bool = True, age_ms: float | None = 5.0):
    """The serving form: Poisson arrivals at rate_hz over the batch size mix
    plus 10% 2160x3840 images, admitted into servers with a device memory
    budget; each request gets 10 iterations and connectivity enforcement.
    With split_mpix > 0 two lanes share the GPU: requests of at most
    split_mpix Mpix go to a continuous-batching server, larger ones (with
    large_solo) are solved whole, one at a time, each as reload + graph-replayed
    iterations + connectivity on a context of their own, or (without) go to a
    second server.  Each lane has its own host thread (the library's blocking
    calls release the interpreter lock) and stream; the small requests' stream
    has the higher priority unless large_first (or equal_priority).  step_mpix
    > 0 sets each server's step budget (least remaining work first).  Latency = delivery of its labels (host, pinned) - arrival.
    Compared with serial plain-FP32 solves of the same request stream (first
    come, first served, one at a time)."""
    import collections
    import threading

    import numpy as np
    import torch

    from paper_1903_07149_gb300 import scalp, synth

    ws, rgbs, cons = batch_imgs
    uhd = []
    for seed in (1002, 1003):
        w = synth.WORKLOADS["uhd_2160x3840_k10000"]
        rgb, con, _ = synth.voronoi_image(w.H, w.W, w.n_cells, gradient=True, noise_sigma=6.0, seed=seed)
        uhd.append((torch.from_numpy(rgb).cuda(), torch.from_numpy(con).cuda(), w.K))
    small = [(torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(), w.K)
             for w, r, c in zip(ws, rgbs, cons)]
    arrivals, kind = synth.serving_arrivals(n_requests, rate_hz, seed=4000)
    reqs = [uhd[i % 2] if kind[i] else small[i % len(small)] for i in range(n_requests)]
    pix = [int(r[0].shape[0]) * int(r[0].shape[1]) for r in reqs]
    iters = 10
    device = torch.cuda.current_device()

    # lanes: (server, stream, queue); a request goes to the first lane whose
    # size bound holds it
    if split_mpix > 0:
        # bound, stream priority, pool share; with large_first the rare large
        # requests (which set the tail) get the high-priority stream
        hi, lo = (0, 0) if equal_priority else (-5, 0)
        specs = [(split_mpix * 1e6, lo if large_first else hi, 0.25),
                 (float("inf"), hi if large_first else lo, 0.75)]
    else:
        specs = [(float("inf"), 0, 1.0)]
    lanes = []
    for bound, prio, share in specs:
        st = torch.cuda.Stream(priority=prio)
        budget = step_mpix if (bound != float("inf") or large_step_mpix is None) else large_step_mpix
        if large_solo and bound == float("inf"):
            srv = None  # whole solves one at a time (below)
        else:
            srv = scalp.Server(int(budget_gb * share * (1 << 30)), max_slots=1024, storage=storage,
                               iters=iters, stream=st, step_pixels=int(budget * 1e6))
        lanes.append((bound, srv, st, collections.deque()))
    # the solo lane: each large request is one whole solve (reload, graph-replayed
    # iterations, connectivity) on its own stream, in arrival order; one
    # context per distinct image size and K, made up front
    # With age_ms, a large request that has waited longer than that runs on a
    # high-priority stream of its own (aging), so a burst of large requests
    # cannot be held back indefinitely by the small ones.
    solo = {}
    st_boost = torch.cuda.Stream(priority=-5) if (large_solo and age_ms is not None) else None
    if large_solo:
        st_solo = lanes[-1][2]
        for st_k in [st_solo] + ([st_boost] if st_boost is not None else []):
            with torch.cuda.stream(st_k):
                for rgb, con, K in uhd:
                    seg = scalp.Segmenter(rgb, con, K, storage=storage, stream=st_k)
                    out = torch.empty((rgb.shape[0], rgb.shape[1]), dtype=torch.int32, pin_memory=True)
                    seg.iterate(iters)
                    seg.labels(enforce=True, out=out.numpy())
                    solo[(rgb.data_ptr(), K, st_k is st_boost)] = (seg, out)

    def lane_of(i):
        return next(k for k, l in enumerate(lanes) if pix[i] <= l[0])

    # warm the pinned-memory cache and the kernels with a few requests per lane
    for k, (_, srv, _, _) in enumerate(lanes):
        if srv is None:
            continue
        mine = [i for i in range(n_requests) if lane_of(i) == k][:8]
        warm = {r[0] for r in (srv.submit(*reqs[i]) for i in mine) if r}
        while warm:
            srv.step()
            warm = {rid for rid in warm if not srv.poll(rid)[0]}
    torch.cuda.synchronize()

    lat = np.zeros(n_requests)
    finished = threading.Event()
    errors = []
    t0 = time.perf_counter()

    def drive(srv, queue):
        try:
            torch.cuda.set_device(device)
            inflight = {}
            while not (finished.is_set() and not queue and not inflight):
                while queue:  # admit in arrival order while memory and slots allow
                    r = srv.submit(*reqs[queue[0]])
                    if r is None:
                        break
                    inflight[r[0]] = queue.popleft()
                if inflight:
                    srv.step()
                else:
                    time.sleep(20e-6)
                for rid in list(inflight):
                    done, _ = srv.poll(rid)
                    if done:
                        i = inflight.pop(rid)
                        lat[i] = time.perf_counter() - t0 - arrivals[i]
        except Exception as exc:  # reported after the join
            errors.append(exc)

    def drive_solo(st, queue):
        try:
            torch.cuda.set_device(device)
            while not (finished.is_set() and not queue):
                if not queue:
                    time.sleep(20e-6)
                    continue
                i = queue.popleft()
                rgb, con, K = reqs[i]
                boost = age_ms is not None and (time.perf_counter() - t0 - arrivals[i]) * 1e3 > age_ms
                seg, out = solo[(rgb.data_ptr(), K, boost)]
                with torch.cuda.stream(st_boost if boost else st):
                    seg.reload(rgb, con)
                    seg.iterate(iters)
                    seg.labels(enforce=True, out=out.numpy())
                lat[i] = time.perf_counter() - t0 - arrivals[i]
        except Exception as exc:  # reported after the join
            errors.append(exc)

    threads = [threading.Thread(target=drive, args=(srv, q)) if srv is not None
               else threading.Thread(target=drive_solo, args=(st, q)) for _, srv, st, q in lanes]
    for t in threads:
        t.start()
    for i in range(n_requests):  # dispatch at the arrival times
        wait = arrivals[i] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        lanes[lane_of(i)][3].append(i)
    finished.set()
    for t in threads:
        t.join()
    wall = time.perf_counter() - t0
    if errors:
        raise errors[0]
    for _, srv, _, _ in lanes:
        if srv is not None:
            srv.close()
    for seg, _ in solo.values():
        seg.close()
    stream = lanes[0][2]
    tot = sum(pix) * iters / 1e6
    res = {
        "requests": n_requests, "rate_hz": rate_hz, "budget_gb": budget_gb, "storage": storage,
        "step": (f"least remaining work first, at most {step_mpix:g} Mpix per step" if step_mpix
                 else "every request in flight each step"),
        "lanes": (("requests <= %g Mpix on a continuous-batching server, larger ones solved whole one at a "
                   "time (graph-replayed iterations) on a %s-priority stream%s, one host thread each"
                   % (split_mpix, "higher" if large_first else "lower",
                      "" if age_ms is None else f"; a large request waiting over {age_ms:g} ms runs on a "
                      "high-priority stream")) if (split_mpix and large_solo) else
                  (f"requests <= {split_mpix:g} Mpix on one server, larger ones on another, one host thread "
                   f"each; the {'larger' if large_first else 'smaller'} requests' stream has the higher priority")
                  if split_mpix else "one server"),
        "mix": "64 sizes of the batch mix + 10% 2160x3840", "iters": iters,
        "value": tot / wall, "unit": UNIT, "wall_s": wall,
        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "p99_small_ms": float(np.percentile(lat[np.array(pix) <= 4e6], 99) * 1e3),
        "p99_large_ms": float(np.percentile(lat[np.array(pix) > 4e6], 99) * 1e3),
    }
    if not serial:
        return res

    # serial plain-FP32 solves of the same stream
    lat_s = np.zeros(n_requests)
    segs = {}
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i, (rgb, con, K) in enumerate(reqs):
            now = time.perf_counter() - t0
            if arrivals[i] > now:
                time.sleep(arrivals[i] - now)
            key = (rgb.data_ptr(), K)
            if key not in segs:
                segs[key] = scalp.Segmenter(rgb, con, K, storage="f32", stream=stream)
            s = segs[key]
            s.reload(rgb, con)
            s.iterate(iters)
            out = torch.empty((rgb.shape[0], rgb.shape[1]), dtype=torch.int32, pin_memory=True)
            s.labels(enforce=True, out=out.numpy())
            lat_s[i] = time.perf_counter() - t0 - arrivals[i]
    wall_s = time.perf_counter() - t0
    for s in segs.values():
        s.close()
    res["serial_f32"] = {"value": tot / wall_s, "unit": UNIT, "wall_s": wall_s,
                         "p50_ms": float(np.percentile(lat_s, 50) * 1e3),
                         "p99_ms": float(np.percentile(lat_s, 99) * 1e3)}
    return res


def measure_serving_sweep(args, batch_imgs, rates=(500.0, 1000.0, 1500.0, 2000.0), n_requests: int = 1000):
    """The serving form at rising Poisson rates (same size mix): delivered
    Mpix*iter/s and latency per rate; where the delivered rate stops
    following the offered one, the form is at capacity."""
    out = []
    for rate in rates:
        r = measure_serving(args, batch_imgs, n_requests=n_requests, rate_hz=rate, serial=False)
        offered = r["value"] * r["wall_s"] / (n_requests / rate)
        out.append({"rate_hz": rate, "offered_mpix_iter_s": offered, "delivered_mpix_iter_s": r["value"],
                    "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "wall_s": r["wall_s"]})
    return out


def measure_multiscale(args, flush, storage: str = "f32"):
    """The multi-scale boundary map of Sec. III-A2 on the 321x481 workload: the
    image solved at 12 scales (K = 6 .. 600, geometric) as one batch, 10
    iterations, connectivity, then the averaged boundary map."""
    import torch

    from paper_1903_07149_gb300 import scalp, synth

    w, rgb, con = synth.single_image_config("bsd_321x481_k400")
    Ks = scalp.multiscale_K()
    d_rgb, d_con = torch.from_numpy(rgb).cuda(), torch.from_numpy(con).cuda()
    stream = torch.cuda.Stream()
    outs = [torch.empty((w.H, w.W), dtype=torch.int32, device="cuda") for _ in Ks]
    bmap = torch.empty((w.H, w.W), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        b = scalp.Batch([d_rgb] * len(Ks), [d_con] * len(Ks), Ks, storage=storage, stream=stream)

        def step():
            b.reload([d_rgb] * len(Ks), [d_con] * len(Ks))
            b.iterate(w.iters)
            b.labels(enforce=True, outs=outs)
            scalp.scalp_boundary_map([o.data_ptr() for o in outs], w.H, w.W, bmap.data_ptr(),
                                     stream.cuda_stream)

        for _ in range(args.warmup):
            step()
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev0[i].record(stream)
            step()
            ev1[i].record(stream)
        torch.cuda.synchronize()
        b.close()
    total_ms = sum(a.elapsed_time(c) for a, c in zip(ev0, ev1))
    return {"value": len(Ks) * w.H * w.W * w.iters * args.steps / (total_ms / 1e3) / 1e6,
            "unit": UNIT, "ms_per_map": total_ms / args.steps, "scales": Ks,
            "workload": w.name, "storage": storage}


def measure_quality(w, rgb, con, cells):
    """Superpixel metrics (Eq. 5-8) of the HD decomposition against its Voronoi
    cells, for SCALP's defaults and for the SLIC special case (lambda = 1,
    gamma = 0, stated below Eq. 3): the ablation of Fig. 4(a) on synthetic
    ground truth."""
    import torch

    from paper_1903_07149_gb300 import scalp

    d_rgb, d_con = torch.from_numpy(rgb).cuda(), torch.from_numpy(con).cuda()
    gt = torch.from_numpy(cells).cuda()
    res = {}
    for name, lam, gamma in (("scalp", 0.5, -1.0), ("slic", 1.0, 0.0)):
        seg = scalp.Segmenter(d_rgb, d_con, w.K, lam=lam, gamma=gamma)
        seg.iterate(w.iters)
        out = torch.empty((w.H, w.W), dtype=torch.int32, device="cuda")
        _, n = seg.labels(enforce=True, out=out)
        q = scalp.quality_metrics(out, gt)
        q["n_superpixels"] = int(n)
        res[name] = q
        seg.close()
    res["ground_truth"] = f"the {int(cells.max()) + 1} Voronoi cells of the synthetic image"
    return res


def measure_prior(args, w, rgb, con, cells, flush):
    """The contour prior computed from the image on the GPU (Sec. II-E takes any
    soft prior): its throughput on the workload's image, and the superpixel
    metrics of SCALP driven by it, by the workload's own prior and by none
    (C = 0): the influence of the prior (Fig. 4(b)) on synthetic ground truth."""
    import torch

    from paper_1903_07149_gb300 import scalp

    d_rgb = torch.from_numpy(rgb).cuda()
    out = torch.empty((w.H, w.W), dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    n_iter = max(args.steps, 5)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            scalp.gradient_prior(d_rgb, out, stream=stream)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n_iter)]
        torch.cuda.synchronize()
        for i in range(n_iter):
            flush.zero_()
            ev[2 * i].record(stream)
            scalp.gradient_prior(d_rgb, out, stream=stream)
            ev[2 * i + 1].record(stream)
        torch.cuda.synchronize()
    ms = sum(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(n_iter)) / n_iter
    # algorithmic bytes: rgb read (3 B) and the prior written (4 B) by the first
    # pass, read and written again (8 B) by the normalisation
    bytes_px = 15
    peaks = measured_peaks() or {}
    hbm = peaks.get("hbm_gbs")
    source = "measured (MEASURED_PEAKS.json)"
    if not hbm:
        hbm, source = FALLBACK_HBM_GBS, "fallback 6.8 TB/s (no measured peaks file)"
    gbs = w.H * w.W * bytes_px / (ms / 1e3) / 1e9
    res = {"workload": w.name, "ms": ms, "Mpix_per_s": w.H * w.W / (ms / 1e3) / 1e6,
           "launches": 2, "roofline": {"bound": "hbm", "achieved": gbs, "unit": "GB/s",
                                        "peak": hbm, "frac": gbs / hbm, "peak_source": source,
                                        "bytes_per_pixel": bytes_px}}
    gt = torch.from_numpy(cells).cuda()
    d_con = torch.from_numpy(con).cuda()
    quality = {}
    for name, contour, prior in (("gradient_prior", None, "gradient"), ("input_prior", d_con, "input"),
                                 ("no_prior", None, "input")):
        seg = scalp.Segmenter(d_rgb, contour, w.K, prior=prior)
        seg.iterate(w.iters)
        lab = torch.empty((w.H, w.W), dtype=torch.int32, device="cuda")
        _, n = seg.labels(enforce=True, out=lab)
        q = scalp.quality_metrics(lab, gt)
        q["n_superpixels"] = int(n)
        quality[name] = q
        seg.close()
    res["quality"] = quality
    return res


def measure_voxel(args, flush):
    """Supervoxels on a synthetic video volume (moving Voronoi cells): whole
    solves (set-up + 10 iterations, labels in device memory), Mvox*iter/s, and
    the assignment's work against the FP32 lane peak as in the 2-D line."""
    import torch

    from paper_1903_07149_gb300 import scalp, synth

    name = "video_32x240x320_k2000"
    T, H, W, K, n_cells, seed = synth.VIDEO_WORKLOADS[name]
    rgb, con, _ = synth.voronoi_video(T, H, W, n_cells, seed=seed)
    d_rgb, d_con = torch.from_numpy(rgb).cuda(), torch.from_numpy(con).cuda()
    out = torch.empty((T, H, W), dtype=torch.int32, device="cuda")
    iters = 10
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        def step():
            seg = scalp.VoxelSegmenter(d_rgb, d_con, K, stream=stream)
            seg.iterate(iters)
            seg.labels(out=out)
            return seg

        for _ in range(max(args.warmup, 1)):
            step().close()
        n_steps = max(args.steps // 2, 2)
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(n_steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(n_steps)]
        torch.cuda.synchronize()
        for i in range(n_steps):
            flush.zero_()
            ev0[i].record(stream)
            step().close()
            ev1[i].record(stream)
        torch.cuda.synchronize()
        # work of one iteration, counted on the device, the iteration time,
        # and the assignment's own time per launch (event pairs around it)
        seg = step()
        seg.count_samples(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        seg.iterate(1)
        e1.record(stream)
        samples, pairs = seg.count_samples(0)
        torch.cuda.synchronize()
        it_ms = e0.elapsed_time(e1)
        seg.profile(1)
        seg.iterate(iters)
        a_ms, a_n = seg.profile(0)
        keff = seg.Keff
        seg.close()
    ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1)) / n_steps
    N = T * H * W
    launch_s = a_ms / max(a_n, 1) / 1e3
    roof = assign_roofline(samples, pairs, N, launch_s, "f32", FALLBACK_SM_MHZ, clk_measured=False)
    roof["kernel"] = "k_vassign"
    roof["note"] = "the assignment launch alone (CUDA events around it); samples gathered from global memory"
    return {"workload": name, "T": T, "H": H, "W": W, "K": K, "Keff": keff, "iters": iters,
            "value": N * iters / (ms / 1e3) / 1e6, "unit": "Mvox*iter/s", "ms_per_solve": ms,
            "iteration_ms": it_ms, "assign_ms_per_launch": launch_s * 1e3,
            "samples_per_iteration": samples, "pairs_per_iteration": pairs, "roofline": roof}


def measure_single_form(args, w, rgb, con, storage: str, flush, steps=None, sm_mhz=None):
    """Plain single-image solves with the given plane storage: whole solves
    (reload, 10 iterations, connectivity), then the assignment's time per
    launch (a second pass with event records) and its path samples (counted
    on the device), for its roofline; also returns the solver state after
    one solve (for the precision statement)."""
    import torch

    from paper_1903_07149_gb300 import scalp

    steps = steps or args.steps
    stream = torch.cuda.Stream()
    d_rgb = torch.from_numpy(rgb).cuda()
    d_con = torch.from_numpy(con).cuda()
    out = torch.empty((w.H, w.W), dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        seg = scalp.Segmenter(d_rgb, d_con, w.K, storage=storage, stream=stream)

        def step():
            seg.reload(d_rgb, d_con)
            seg.iterate(w.iters)
            seg.labels(enforce=True, out=out)

        for _ in range(args.warmup):
            step()
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        torch.cuda.synchronize()
        for i in range(steps):
            flush.zero_()
            ev0[i].record(stream)
            step()
            ev1[i].record(stream)
        torch.cuda.synchronize()
        seg.profile(1)  # a second pass for the assignment's time per launch
        for i in range(steps):
            flush.zero_()
            step()
        torch.cuda.synchronize()
        ms_assign, n_assign = seg.profile(0)
        seg.count_samples(1)
        seg.reload(d_rgb, d_con)
        seg.iterate(w.iters)
        samples, pairs = seg.count_samples(0)
        state = seg.get_state()
        seg.close()
    total_ms = sum(a.elapsed_time(c) for a, c in zip(ev0, ev1))
    t_launch = ms_assign / max(n_assign, 1) / 1e3
    roof = assign_roofline(samples / w.iters, pairs / w.iters, w.H * w.W, t_launch, storage,
                           sm_mhz or FALLBACK_SM_MHZ, clk_measured=sm_mhz is not None,
                           traffic=traffic_per_launch(storage) if w.name == DEFAULT_WORKLOAD else None)
    return {"value": w.H * w.W * w.iters * steps / (total_ms / 1e3) / 1e6, "unit": UNIT,
            "ms_per_step": total_ms / steps, "storage": storage, "workload": w.name,
            "assign_ms_per_launch": t_launch * 1e3, "roofline": roof}, state


def measure_uhd_precision_form(args, flush, sm_mhz):
    """The precision form's own workload: 2160x3840, K=10000, 10 iterations,
    FP16 planes beside FP32 planes on the same input."""
    from paper_1903_07149_gb300 import synth

    w, rgb, con = synth.single_image_config("uhd_2160x3840_k10000")
    res, states = {}, {}
    for storage in ("f32", "f16"):
        res[storage], states[storage] = measure_single_form(args, w, rgb, con, storage, flush,
                                                            steps=max(args.steps // 2, 3), sm_mhz=sm_mhz)
    res["f16_over_f32"] = res["f16"]["value"] / res["f32"]["value"]
    return res, (w, rgb, con, states)


def batch_sample_states(bws, rgbs, cons, count: int = 4):
    """Solver states of the first `count` images of the batch mix, solved as
    one batch in each storage (10 iterations, free-running)."""
    import torch

    from paper_1903_07149_gb300 import scalp

    out = {}
    ws = bws[:count]
    d_rgb = [torch.from_numpy(r).cuda() for r in rgbs[:count]]
    d_con = [torch.from_numpy(c).cuda() for c in cons[:count]]
    states = {}
    for storage in ("f32", "f16"):
        b = scalp.Batch(d_rgb, d_con, [w.K for w in ws], storage=storage)
        b.iterate(ws[0].iters)
        states[storage] = [b.get_state(i) for i in range(count)]
        b.close()
    for i, w in enumerate(ws):
        out[f"batch_image_{i}"] = (w, rgbs[i], cons[i], {st: states[st][i] for st in states})
    return out


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    dist = world > 1
    if dist:
        import torch.distributed as td

        td.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1903_07149_gb300 import build as scalp_build
    from paper_1903_07149_gb300 import scalp, synth

    scalp_build.build()
    w, rgb, con = synth.single_image_config(args.workload)
    N, iters = w.H * w.W, w.iters
    stream = torch.cuda.Stream()
    d_rgb = torch.from_numpy(rgb).cuda()
    d_con = torch.from_numpy(con).cuda()
    out = torch.empty((w.H, w.W), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    seg = scalp.Segmenter(d_rgb, d_con, w.K, storage=args.storage, stream=stream)

    def step():
        seg.reload(d_rgb, d_con)
        seg.iterate(iters)
        return seg.labels(enforce=True, out=out)[1]

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        # path samples of one step, for the roofline's algorithmic work
        seg.count_samples(1)
        step()
        samples, pairs = seg.count_samples(0)
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if dist:
            td.barrier()
        torch.cuda.synchronize()
        clocks = Clocks(local)
        clocks.start()
        for i in range(args.steps):
            flush.zero_()
            ev0[i].record(stream)
            n_labels = step()
            ev1[i].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        # the same steps again with the assignment launches bracketed by events
        # (those records break the programmatic launch chain around them, so
        # the throughput above is timed without them)
        seg.profile(1)
        for i in range(args.steps):
            flush.zero_()
            step()
        torch.cuda.synchronize()
        ms_assign, assign_launches = seg.profile(0)
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_ms = rank_max(sum(step_ms))
    value = whole_job_value(N * iters * args.steps, world, total_ms)

    # end to end through the public API: pinned host buffers in, labels out.
    # Two solves in flight, as a throughput user would run them: each host
    # thread drives one context on its own stream (the library's blocking
    # calls release the interpreter lock), so one step's copies overlap the
    # other's kernels.  Every step uploads its inputs, flushes L2 and reads
    # its labels back inside the timed region.
    e2e = None
    if not args.no_e2e:
        import threading

        h_rgb = torch.from_numpy(rgb).pin_memory()
        h_con = torch.from_numpy(con).pin_memory()
        a_rgb, a_con = h_rgb.numpy(), h_con.numpy()
        streams = [stream, torch.cuda.Stream()]
        segs = [seg, scalp.Segmenter(d_rgb, d_con, w.K, storage=args.storage, stream=streams[1])]
        outs = [torch.empty((w.H, w.W), dtype=torch.int32, pin_memory=True).numpy() for _ in range(2)]
        flushes = [flush, torch.empty_like(flush)]
        errors = []

        def run(j, n):
            try:
                torch.cuda.set_device(local)
                with torch.cuda.stream(streams[j]):
                    for _ in range(n):
                        flushes[j].zero_()
                        segs[j].reload(a_rgb, a_con)
                        segs[j].iterate(iters)
                        segs[j].labels(enforce=True, out=outs[j])
            except Exception as exc:  # reported after the join
                errors.append(exc)

        for j in range(2):
            run(j, 1)
        torch.cuda.synchronize()
        if dist:
            td.barrier()
        t0 = time.perf_counter()
        threads = [threading.Thread(target=run, args=(j, (args.steps + 1 - j) // 2)) for j in range(2)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        torch.cuda.synchronize()
        t_e2e = rank_max(time.perf_counter() - t0)
        if errors:
            raise errors[0]
        segs[1].close()
        e2e = {"value": whole_job_value(N * iters * args.steps, world, t_e2e * 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(rgb.nbytes + con.nbytes),
               "d2h_bytes_per_step": int(w.H * w.W * 4),
               "pipeline": "two contexts on two streams, one host thread each"}

    if rank != 0:
        if dist:
            td.destroy_process_group()
        return

    # roofline of the dominant kernel (the assignment)
    t_launch = ms_assign / max(assign_launches, 1) / 1e3
    sm_max = (clk or {}).get("sm_max_mhz")
    roofline = assign_roofline(samples / iters, pairs / iters, N, t_launch, args.storage,
                               sm_max or FALLBACK_SM_MHZ, clk_measured=sm_max is not None,
                               traffic=traffic_per_launch(args.storage))
    roofline["launches"] = assign_launches
    peaks = measured_peaks()
    if peaks:
        roofline["measured_peaks"] = peaks
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": line_config(w, world),
        "timing": {"form": "plain single image", "storage": args.storage,
                   "step": "reload + 10 iterations + connectivity + labels in device memory",
                   "l2": "flushed (256 MB write) before each timed step"},
        "n_labels": int(n_labels),
        "clocks": clk, "e2e": e2e,
        "gpu_launches": args.steps * (reload_launches(w.H, w.W) + iter_launches(w.H, w.W) * iters
                                      + ccl_launches(w.H, w.W)),
        "roofline": roofline,
    }
    precision_inputs = {}
    if not args.no_forms:
        from paper_1903_07149_gb300 import synth

        other = "f16" if args.storage == "f32" else "f32"
        bws = synth.batch_configs()
        batch_imgs = (bws, *synth.batch_images(bws))
        single_other, st_other = measure_single_form(args, w, rgb, con, other, flush, sm_mhz=sm_max)
        line["forms"] = {
            f"single_{other}": single_other,
            "batched_f16": measure_batch(args, "f16", flush, batch_imgs, sm_max),
            "batched_f32": measure_batch(args, "f32", flush, batch_imgs, sm_max),
        }
        uhd, uhd_states = measure_uhd_precision_form(args, flush, sm_max)
        line["forms"]["uhd_2160x3840_k10000"] = uhd
        line["forms"]["multiscale_boundary_map"] = measure_multiscale(args, flush)
        _, _, cells = synth.voronoi_image(w.H, w.W, w.n_cells, gradient=w.gradient,
                                          noise_sigma=w.noise_sigma, seed=w.seed)
        line["forms"]["quality_eq5_8"] = measure_quality(w, rgb, con, cells)
        line["forms"]["gradient_prior"] = measure_prior(args, w, rgb, con, cells, flush)
        line["forms"]["supervoxels"] = measure_voxel(args, flush)
        if not args.no_serving:
            line["forms"]["serving"] = measure_serving(args, batch_imgs)
            line["forms"]["serving"]["rate_sweep"] = measure_serving_sweep(args, batch_imgs)
        # GPU states for the precision statement (computed in the CPU leg)
        seg.reload(d_rgb, d_con)
        seg.iterate(iters)
        st_main = seg.get_state()
        w0, rgb0, con0 = synth.single_image_config("bsd_321x481_k400")
        st0 = {}
        for storage in ("f32", "f16"):
            s0 = scalp.Segmenter(torch.from_numpy(rgb0).cuda(), torch.from_numpy(con0).cuda(), w0.K,
                                 storage=storage)
            s0.iterate(w0.iters)
            st0[storage] = s0.get_state()
            s0.close()
        precision_inputs = {w0.name: (w0, rgb0, con0, st0),
                            w.name: (w, rgb, con, {args.storage: st_main, other: st_other}),
                            "uhd_2160x3840_k10000": uhd_states}
        precision_inputs.update(batch_sample_states(*batch_imgs))
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_oracle(w, rgb, con)
        if precision_inputs:
            line["precision_vs_fp64_oracle"] = cpu_precision_statement(
                precision_inputs, line["cpu_baseline"]["cores"])
    print(json.dumps(line), flush=True)
    seg.close()
    if dist:
        td.destroy_process_group()


def run_form(args):
    import torch

    from paper_1903_07149_gb300 import build as scalp_build
    from paper_1903_07149_gb300 import synth

    scalp_build.build()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    if args.only_form == "supervoxels":
        res = measure_voxel(args, flush)
    elif args.only_form == "serving":
        bws = synth.batch_configs()
        imgs = (bws, *synth.batch_images(bws))
        res = {"default": measure_serving(args, imgs),
               "default_4000": measure_serving(args, imgs, n_requests=4000),
               "no_aging": measure_serving(args, imgs, age_ms=None, serial=False),
               "solo_equal_priority": measure_serving(args, imgs, equal_priority=True, age_ms=None, serial=False),
               "two_servers_large_first": measure_serving(args, imgs, large_solo=False, large_first=True,
                                                          age_ms=None, serial=False),
               "one_server": measure_serving(args, imgs, step_mpix=0.0, split_mpix=0.0, large_solo=False,
                                             age_ms=None, serial=False),
               "sweep": measure_serving_sweep(args, imgs)}
    elif args.only_form == "batched":
        bws = synth.batch_configs()
        imgs = (bws, *synth.batch_images(bws))
        res = {st: measure_batch(args, st, flush, imgs) for st in ("f16", "f32")}
        res["multiscale"] = measure_multiscale(args, flush)
    else:
        w, rgb, con = synth.single_image_config(args.workload)
        _, _, cells = synth.voronoi_image(w.H, w.W, w.n_cells, gradient=w.gradient,
                                          noise_sigma=w.noise_sigma, seed=w.seed)
        res = measure_prior(args, w, rgb, con, cells, flush)
    print(json.dumps({"form": args.only_form, "result": res}))


def main():
    args = parse()
    if args.only_form:
        run_form(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
