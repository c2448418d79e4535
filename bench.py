#!/usr/bin/env python
"""Benchmark of the tFFR adjoint on the 4096-pulse x 4096-frequency stripmap
workload (16,714,266 Stolt-mapped samples -> 4096 x 4096 image), one JSON line.

One step = one tFFR reconstruction of a batch of samples that is already in
HBM: tffr_set_points (coordinate reduction + pulse rows), tffr_weights
(frame weights + threshold) and tffr_adjoint (range spread, azimuth taps +
row FFT, column FFT + deapodisation).  The forward twin is timed on its own
(key "forward").  Inputs per step (402 MB of coordinates and samples) exceed
the 129 MB L2, so no flush is inserted between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs its own copy of the workload (independent
images, no collective on the data path); rank 0 prints value = total samples
over all ranks / max-over-ranks time.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "NU samples/s, tFFR adjoint, 16.7M samples->4096^2 image, rel-L2<=1e-5; HBM %"
UNIT = "NU samples/s"
WORKLOAD = "stripmap_4096"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a stage's
# kernel on this workload, from one ncu capture of that kernel; an entry is removed
# when its kernel changes, and a stage without one reports null.
DRAM_TRAFFIC = {
    ("col_fft", "pulse_rows"): 227_163_136,     # k_adj_cols_pulse<13, 1>
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.gpu_id = gpu_id

    def __enter__(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, ms_max: float) -> float:
    """Units per second over all ranks: each rank processes its own units (weak
    scaling), and the job takes as long as the slowest rank."""
    return world * units_per_rank / (ms_max * 1e-3)


def gpu_id_for_smi(local_rank: int):
    try:
        import torch
        u = str(torch.cuda.get_device_properties(local_rank).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[local_rank] if vis else str(local_rank)


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_sample_time(wl, D, n_pix: int, n_w: int, seed: int = 0):
    """Time the oracle on n_w weight evaluations and n_pix image pixels; return per-unit seconds.

    D: the oracle's weights for all samples (computed once by the caller, outside the timing).
    """
    import numpy as np
    import oracle
    g = np.random.default_rng(seed)
    sel = g.integers(0, wl.N, n_w)
    t0 = time.perf_counter()
    oracle.tffr_weights(wl.lam_x[sel], wl.M)
    t_w = (time.perf_counter() - t0) / n_w
    jx, jy = g.integers(0, wl.M, n_pix), g.integers(0, wl.M, n_pix)
    t0 = time.perf_counter()
    if n_pix:
        oracle.adjoint_pixels(wl.lam_x, wl.lam_y, wl.values, D, wl.M, wl.M, jx, jy)
    t_p = (time.perf_counter() - t0) / max(n_pix, 1)
    return t_w, t_p


def cpu_baseline(wl, D, budget_s: float = 15.0):
    import oracle
    t_w, t_p1 = oracle_sample_time(wl, D, 2, 200000, seed=1)
    n_pix = int(max(2, min(4096, budget_s / max(t_p1, 1e-6))))
    t_w, t_p = oracle_sample_time(wl, D, n_pix, 2000000, seed=2)
    full = t_w * wl.N + t_p * wl.M * wl.M
    return {"value": wl.N / full, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "FP64 oracle: tFFR weights on 2,000,000 of the %d samples and the direct sum of "
                      "Eq. (fstraight) at %d random pixels of the %dx%d image; full-image time "
                      "extrapolated (weights x N, sum x M^2 pixels) = %.0f s" % (wl.N, n_pix, wl.M, wl.M, full)}


def run_reference(args, world, rank):
    """The FP64 oracle on the host cores, each step a bounded sample of the workload:
    weights on 200,000 samples and the direct sum at 4 x cores pixels (so OpenMP keeps
    every core busy).  value = the workload's samples per second, extrapolated from the
    per-pixel and per-weight costs; ms_per_step = the measured time of one sample step."""
    if rank != 0:
        return 0
    import oracle
    from synth import make_workload
    wl = make_workload(WORKLOAD)
    D = oracle.tffr_weights(wl.lam_x, wl.M)
    cores = oracle.threads()
    n_pix, n_w = 4 * cores, 200000

    def step(i):
        return oracle_sample_time(wl, D, n_pix, n_w, seed=100 + i)

    for i in range(args.warmup):
        step(i)
    tw = tp = 0.0
    t0 = time.perf_counter()
    for i in range(args.steps):
        a, b = step(args.warmup + i)
        tw += a
        tp += b
    wall = (time.perf_counter() - t0) / args.steps
    tw /= args.steps
    tp /= args.steps
    full = tw * wl.N + tp * wl.M * wl.M
    value = wl.N / full
    sample = ("each step: FP64 oracle weights on %d samples + direct sum at %d pixels (%d threads); "
              "throughput extrapolated to the full %d-sample, %dx%d image (%.0f s per image)"
              % (n_w, n_pix, cores, wl.N, wl.M, wl.M, full))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": wl.N, "image": "%dx%d" % (wl.M, wl.M),
                       "step": "bounded sample: %d pixels + %d weights" % (n_pix, n_w),
                       "full_image_s_extrapolated": full},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

SECTION_S = 1.0          # minimum device time of each side section (--section-s)


def timed_ms(run, stream, world, min_s: float | None = None, min_iters: int = 3):
    """Mean milliseconds per call of run() (its work ordered on `stream`), over at least
    min_iters calls and about min_s seconds of device time, max over ranks."""
    import torch
    if min_s is None:
        min_s = SECTION_S
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    run()
    torch.cuda.synchronize()
    ev0.record(stream)
    run()
    ev1.record(stream)
    torch.cuda.synchronize()
    one = max(ev0.elapsed_time(ev1), 1e-3)
    iters = max(min_iters, int(min_s * 1e3 / one) + 1)
    barrier(world)
    ev0.record(stream)
    for _ in range(iters):
        run()
    ev1.record(stream)
    torch.cuda.synchronize()
    return max_over_ranks(ev0.elapsed_time(ev1) / iters, world), iters


def golden_crop():
    """The FP64 oracle's 256 x 256 centre crop of this workload's image, stored by
    tests/golden/make_golden.py, and the crop's pixel box; (None, None) when absent."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", "stripmap_4096_crop256.npy")
    if not os.path.exists(path):
        return None, None
    return np.load(path), (2048 - 128, 2048 - 128, 256, 256)


def crop_rel_l2(img, ref, box):
    import numpy as np
    if ref is None:
        return None
    jx0, jy0, nx, ny = box
    got = img[jy0:jy0 + ny, jx0:jx0 + nx].cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    from paper_1910_10908_gb300 import Plan
    from synth import make_workload

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = make_workload(WORKLOAD)
    N, M = wl.N, wl.M
    lx = torch.from_numpy(wl.lam_x).to(dev)
    ly = torch.from_numpy(wl.lam_y).to(dev)
    vals = torch.from_numpy(wl.values).to(dev)
    img = torch.empty((M, M), dtype=torch.complex64, device=dev)
    plan = Plan(M, values="c64", device=dev)
    stream = plan.stream

    def step():
        # set_points + weights + adjoint in one library call (tffr_reconstruct)
        plan.reconstruct(lx, ly, vals, out=img)

    def step_three_calls():
        plan.set_points(lx, ly)
        plan.weights(count=False)
        plan.adjoint(vals, out=img)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    info = plan.info()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    step()
    ev1.record(stream)
    torch.cuda.synchronize()
    est_ms = ev0.elapsed_time(ev1)

    # ---- timed region: exactly K steps per region, device events on the plan's stream.  When
    # K steps last under a second the region is repeated (back to back, each exactly K steps)
    # so that the clock sampler sees the load; ms_per_step is the median over the regions. ----
    region_ms = 1e3 * SECTION_S
    repeats = max(1, int(region_ms / max(est_ms * args.steps, 1e-3)) + 1) if args.steps * est_ms < region_ms else 1
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(repeats)]
    launches0 = plan.info()["kernel_launches"]
    with ClockSampler(gpu_id_for_smi(local)) as clk:
        barrier(world)
        torch.cuda.synchronize()
        for e0, e1 in evs:
            e0.record(stream)
            for _ in range(args.steps):
                step()
            e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    launches = (plan.info()["kernel_launches"] - launches0) // repeats
    ms = statistics.median(e0.elapsed_time(e1) / args.steps for e0, e1 in evs)
    ms_max = max_over_ranks(ms, world)
    value = whole_job_rate(N, world, ms_max)

    # ---- per-kernel times: a separate pass with stage events on the stream ----
    kp = 200 if SECTION_S >= 1.0 else 5
    plan.profile(True)
    for _ in range(kp):
        step()
    torch.cuda.synchronize()
    stages = plan.profile_read()
    plan.profile(False)

    # algorithmic bytes per launch: each input read once, each output written
    # once.  points: both coordinate arrays (16 B/sample).  weights: nothing,
    # D is evaluated inside the spread.  spread: lambda_x + value (16 B/sample)
    # in, pulse-row buffers (8 B/cell) out.  row_fft: row buffers in, the
    # intermediate out ([P][M] in pulse-row order, [2M][M] in fine-row order).
    # col_fft: intermediate in, M x M image out.
    hbm, peak_kind = peaks()
    R = int(info["row_cells"])
    pulse = bool(info["pulse_order"])
    T_bytes = 8 * M * (int(info["n_rows"]) if pulse else 2 * M)
    alg = {
        "points": N * 16,
        "weights": 0,
        "spread": N * 16 + 8 * R,
        "row_fft": 8 * R + T_bytes,
        "col_fft": T_bytes + 8 * M * M,
    }
    kern = {}
    for name, b in alg.items():
        tot, cnt = stages[name]
        if cnt:
            per = tot / cnt
            kern[name] = {"ms": per, "alg_bytes": b}
            if b:
                kern[name].update(gbs=b / (per * 1e-3) / 1e9, frac=b / (per * 1e-3) / 1e9 / hbm)
    hot = max(("spread", "row_fft", "col_fft"), key=lambda k: kern[k]["ms"])
    roof = {"bound": "hbm", "kernel": hot, "achieved": kern[hot]["gbs"], "peak": hbm, "unit": "GB/s",
            "frac": kern[hot]["frac"], "peak_source": peak_kind,
            "traffic": DRAM_TRAFFIC.get((hot, "pulse_rows" if pulse else "fine_rows"))}

    # ---- forward twin, timed on its own ----
    yout = torch.empty(N, dtype=torch.complex64, device=dev)
    fwd_ms, _ = timed_ms(lambda: plan.forward(img, out=yout), stream, world)
    three_ms, _ = timed_ms(step_three_calls, stream, world)

    # ---- end to end through host buffers ----
    # Every step copies its inputs in from pinned host memory and its image out
    # to pinned host memory.  Two plans on two streams take the steps in turn,
    # so that one step's copies overlap the other plan's kernels (set_points
    # waits for its own stream only), and the next step's input copies are
    # enqueued before this step's call, which waits on the host for its scan's
    # read-back; the events bracket both streams.
    h_lx = torch.from_numpy(wl.lam_x).pin_memory()
    h_ly = torch.from_numpy(wl.lam_y).pin_memory()
    h_v = torch.from_numpy(wl.values).pin_memory()
    streams = [stream, torch.cuda.Stream(device=dev)]
    with torch.cuda.stream(streams[1]):
        plan_b = Plan(M, values="c64", device=dev)
    plans = [plan, plan_b]
    d_in = [(torch.empty_like(lx), torch.empty_like(ly), torch.empty_like(vals)) for _ in range(2)]
    d_img = [img, torch.empty_like(img)]
    h_img = [torch.empty((M, M), dtype=torch.complex64).pin_memory() for _ in range(2)]

    def e2e_copy_in(k):
        d_lx, d_ly, d_v = d_in[k]
        with torch.cuda.stream(streams[k]):
            d_lx.copy_(h_lx, non_blocking=True)
            d_ly.copy_(h_ly, non_blocking=True)
            d_v.copy_(h_v, non_blocking=True)

    def e2e_call_and_copy_out(k):
        d_lx, d_ly, d_v = d_in[k]
        plans[k].reconstruct(d_lx, d_ly, d_v, out=d_img[k])
        with torch.cuda.stream(streams[k]):
            h_img[k].copy_(d_img[k], non_blocking=True)

    def e2e_run(k):
        # k steps taking the two plans in turn, bracketed by events on the first stream
        ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        joined = torch.cuda.Event()
        ev_a.record(streams[0])
        streams[1].wait_event(ev_a)
        e2e_copy_in(0)
        for i in range(k):
            if i + 1 < k:
                e2e_copy_in((i + 1) % 2)               # behind step i - 1 on its stream
            e2e_call_and_copy_out(i % 2)
        joined.record(streams[1])
        streams[0].wait_event(joined)
        ev_b.record(streams[0])
        torch.cuda.synchronize()
        return ev_a.elapsed_time(ev_b)

    e2e_run(4)
    e2e_iters = max(8, int(1e3 * SECTION_S / max(e2e_run(8) / 8, 1e-3)))
    barrier(world)
    e2e_ms = max_over_ranks(e2e_run(e2e_iters) / e2e_iters, world)
    h2d = int(h_lx.numel() * 8 + h_ly.numel() * 8 + h_v.numel() * 8)
    d2h = int(h_img[0].numel() * 8)

    # the same copies alone (no kernels), inputs in on one stream while the
    # previous step's image goes out on the other: the host link's floor for
    # the end-to-end step
    def copies_run(k):
        ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        joined = torch.cuda.Event()
        ev_a.record(streams[0])
        streams[1].wait_event(ev_a)
        for i in range(k):
            d_lx, d_ly, d_v = d_in[i % 2]
            with torch.cuda.stream(streams[0]):
                d_lx.copy_(h_lx, non_blocking=True)
                d_ly.copy_(h_ly, non_blocking=True)
                d_v.copy_(h_v, non_blocking=True)
            with torch.cuda.stream(streams[1]):
                h_img[i % 2].copy_(d_img[i % 2], non_blocking=True)
        joined.record(streams[1])
        streams[0].wait_event(joined)
        ev_b.record(streams[0])
        torch.cuda.synchronize()
        return ev_a.elapsed_time(ev_b)

    copies_run(4)
    floor_iters = max(8, int(1e3 * SECTION_S / max(copies_run(8) / 8, 1e-3)))
    copy_floor_ms = max_over_ranks(copies_run(floor_iters) / floor_iters, world)
    plan_b.close()
    del h_lx, h_ly, h_v, h_img, d_in

    # ---- comparison only: cuFFT (torch.fft) on the 2M x 2M grid a plain NUFFT transforms ----
    # (never on the path; the two pruned passes above also apply the azimuth
    # taps, the deapodisation and the crop)
    grid = torch.randn((2 * M, 2 * M), dtype=torch.complex64, device=dev)
    with torch.cuda.stream(stream):
        cufft_ms, _ = timed_ms(lambda: torch.fft.ifft2(grid, norm="forward"), stream, world)
    fft_compare = {"cufft_ifft2_%dx%d_c64_ms" % (2 * M, 2 * M): cufft_ms,
                   "tffr_x_pass_plus_column_pass_ms": kern["row_fft"]["ms"] + kern["col_fft"]["ms"]}
    del grid

    # ---- a batch of 64 uneven sub-aperture patches ----
    from paper_1910_10908_gb300.batched import PatchBatch
    from synth import patch_batch
    pb = patch_batch(64)
    patches = [(m, m, torch.from_numpy(plx).to(dev), torch.from_numpy(ply).to(dev)) for m, plx, ply, _ in pb]
    timings = {}
    # baseline: 64 plain adjoint calls one after the other on one stream
    with PatchBatch(patches, streams=1, persistent=False) as seq:
        for k, (_, _, _, pv) in enumerate(pb):
            seq.load(k, torch.from_numpy(pv).to(dev))
        timings["sequential"], _ = timed_ms(seq.adjoint_eager, seq.stream, world)
    with PatchBatch(patches) as batch:
        for k, (_, _, _, pv) in enumerate(pb):
            batch.load(k, torch.from_numpy(pv).to(dev))
        timings["per_plan_8_streams"], _ = timed_ms(batch.adjoint_eager, batch.stream, world)
        timings["persistent"], _ = timed_ms(batch.adjoint, batch.stream, world)
        tuned = batch.tune(reps=10 if SECTION_S >= 1.0 else 1)
        timings["persistent_tuned"], _ = timed_ms(batch.adjoint, batch.stream, world)
        batch.capture()
        timings["graph"], _ = timed_ms(batch.replay, batch.stream, world)
        batch.wait()
        batched = {"patches": len(pb), "samples": batch.samples,
                   "sides": sorted({m for m, _, _, _ in pb}),
                   "step": "the adjoint of every patch (points and weights set once)",
                   "sequential_ms": timings["sequential"],
                   "per_plan_8_streams_ms": timings["per_plan_8_streams"],
                   "persistent_ms": timings["persistent"], "persistent_tuned_ms": timings["persistent_tuned"],
                   "graph_ms": timings["graph"],
                   "launches_per_step": 1 + tuned["n_classes"],
                   "spread_ms": tuned["spread_ms"],
                   "autotuned": [{k: c[k] for k in ("side", "patches", "blocks", "ms")} for c in tuned["classes"]],
                   "value": whole_job_rate(batch.samples, world, timings["graph"]), "unit": UNIT}
    del pb, patches

    # ---- differentiable tFFR and the normal operator on the 2048^2 workload ----
    wl2 = make_workload("stripmap_2048")
    M2 = wl2.M
    plan_n = Plan(M2, values="c64", device=dev)
    plan_n.set_points(torch.from_numpy(wl2.lam_x).to(dev), torch.from_numpy(wl2.lam_y).to(dev))
    plan_n.weights(count=False)
    t0 = time.perf_counter()
    plan_n.normal_setup()
    setup_s = time.perf_counter() - t0
    f_n = torch.randn((M2, M2), dtype=torch.complex64, device=dev)
    g_n = torch.empty_like(f_n)
    y_n = torch.empty(wl2.N, dtype=torch.complex64, device=dev)
    v2 = torch.from_numpy(wl2.values).to(dev)
    gD = torch.empty(wl2.N, dtype=torch.float32, device=dev)

    def via_samples():
        plan_n.forward(f_n, out=y_n, apply_weights=False)
        plan_n.adjoint(y_n, out=g_n)

    sn = plan_n.stream
    normal = {"stripmap_2048": {"N": wl2.N, "image": "%dx%d" % (M2, M2), "setup_s": setup_s,
                                "toeplitz_ms": timed_ms(lambda: plan_n.normal(f_n, out=g_n), sn, world)[0],
                                "forward_adjoint_ms": timed_ms(via_samples, sn, world)[0]}}
    cg_out = torch.empty_like(f_n)
    diff = {"workload": "stripmap_2048", "N": wl2.N, "image": "%dx%d" % (M2, M2),
            "image_ms": timed_ms(lambda: plan_n.adjoint(v2, out=g_n), sn, world)[0],
            "grad_values_ms": timed_ms(lambda: plan_n.forward(f_n, out=y_n), sn, world)[0],
            "grad_weights_ms": timed_ms(lambda: plan_n.weight_grad(f_n, v2, out=gD), sn, world)[0],
            "cg20_toeplitz_ms": timed_ms(lambda: plan_n.cg(v2, 20, toeplitz=True, out=cg_out, residuals=False),
                                         sn, world, min_iters=3)[0],
            "cg20_forward_adjoint_ms": timed_ms(lambda: plan_n.cg(v2, 20, toeplitz=False, out=cg_out,
                                                                  residuals=False), sn, world, min_iters=3)[0]}
    _, hist = plan_n.cg(v2, 20, toeplitz=True, out=cg_out)
    diff["cg20_residual_ratio"] = hist[-1] / hist[0]
    del wl2, v2, gD
    # denser sampling: the 4096 x 4096 pulse/frequency grid on the same 2048^2 image
    from synth import stolt_points
    dlx, dly, _ = stolt_points(4096, 4096, M2)
    plan_n.set_points(torch.from_numpy(dlx).to(dev), torch.from_numpy(dly).to(dev))
    plan_n.weights(count=False)
    y_n = torch.empty(dlx.shape[0], dtype=torch.complex64, device=dev)
    plan_n.normal_setup()
    normal["stolt_4096x4096_on_2048"] = {"N": int(dlx.shape[0]), "image": "%dx%d" % (M2, M2),
                                         "toeplitz_ms": timed_ms(lambda: plan_n.normal(f_n, out=g_n), sn, world)[0],
                                         "forward_adjoint_ms": timed_ms(via_samples, sn, world)[0]}
    plan_n.close()
    del dlx, dly

    # ---- reduced-precision sample storage (4 B per sample, FP32 arithmetic) ----
    variants = {}
    for vt in ("f16", "bf16"):
        if vt == "f16":
            v_low = vals.to(torch.complex32)
        else:
            v_low = torch.view_as_real(vals).to(torch.bfloat16).contiguous()
        plan_v = Plan(M, values=vt, device=dev)
        img_v = torch.empty_like(img)

        def step_v():
            plan_v.reconstruct(lx, ly, v_low, out=img_v)

        ms_v, _ = timed_ms(step_v, plan_v.stream, world)
        variants[vt] = {"value": whole_job_rate(N, world, ms_v), "unit": UNIT, "ms_per_step": ms_v,
                        "bytes_per_sample_in": 12, "image": img_v}
        plan_v.close()

    line = None
    if rank == 0:
        # accuracy of the timed configuration: every pixel of the FP64 oracle's stored 256^2 centre crop
        ref, box = golden_crop()
        precision = {}
        for vt, d in variants.items():
            d["rel_l2_vs_fp64_oracle_crop256"] = crop_rel_l2(d.pop("image"), ref, box)
            precision[vt] = d
        base = None
        if world == 1:
            import oracle
            base = cpu_baseline(wl, oracle.tffr_weights(wl.lam_x, M))
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "image": "%dx%d" % (M, M), "pulses": wl.n_pulses,
                       "freqs": wl.n_freq, "sigma": 2, "width": 6, "beta": info["beta"], "values": "c64",
                       "layout": "rows" if info["layout"] == 2 else "general", "pulse_rows": info["n_rows"],
                       "pass_order": "pulse_rows" if pulse else "fine_rows",
                       "step": "set_points+weights+adjoint (one tffr_reconstruct call)",
                       "l2": "inputs (402 MB/step) larger than L2",
                       "timed_regions": repeats,
                       "parallelism": "independent images per GPU" if world > 1 else "single GPU"},
            "roofline": roof,
            "kernels": kern,
            "pixels_per_s": world * M * M / (ms_max * 1e-3),
            "adjoint_only_samples_per_s": N / (sum(stages[k][0] / max(stages[k][1], 1)
                                                   for k in ("spread", "row_fft", "col_fft")) * 1e-3),
            "forward": {"value": N / (fwd_ms * 1e-3), "unit": UNIT, "ms": fwd_ms},
            "step_as_three_calls": {"ms": three_ms, "value": N / (three_ms * 1e-3), "unit": UNIT,
                                    "calls": "tffr_set_points, tffr_weights, tffr_adjoint"},
            "accuracy": {"rel_l2_vs_fp64_oracle_crop256": crop_rel_l2(img, ref, box),
                         "pixels": 0 if ref is None else int(ref.size),
                         "reference": "tests/golden/stripmap_4096_crop256.npy (FP64 direct sum, centre crop)"},
            "precision_variants": precision,
            "batched_patches": batched,
            "differentiable": diff,
            "normal_operator": normal,
            "fft_comparison": fft_compare,
            "e2e": {"value": whole_job_rate(N, world, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
                    "steps": e2e_iters,
                    "overlap": "two plans on two streams: one step's copies overlap the other's kernels; the next "
                               "step's inputs are enqueued before this step's call",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "copy_floor_ms": copy_floor_ms, "of_copy_floor": copy_floor_ms / e2e_ms,
                    "copy_floor": "the same copies with no kernels, in and out on two streams at once"},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        if base is not None:
            line["cpu_baseline"] = base
    plan.close()
    if line is not None:
        print(json.dumps(line), flush=True)
    barrier(world)
    return 0


def run_step_only(args, local):
    """W + K steps of the main workload (set_points + weights + adjoint) and one forward
    twin, with nothing else on the device: the process ncu captures."""
    import torch

    from paper_1910_10908_gb300 import Plan
    from synth import make_workload

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = make_workload(WORKLOAD)
    lx = torch.from_numpy(wl.lam_x).to(dev)
    ly = torch.from_numpy(wl.lam_y).to(dev)
    vals = torch.from_numpy(wl.values).to(dev)
    with Plan(wl.M, values="c64", device=dev) as plan:
        img = torch.empty((wl.M, wl.M), dtype=torch.complex64, device=dev)
        for _ in range(args.warmup + args.steps):
            plan.reconstruct(lx, ly, vals, out=img)
        plan.forward(img)
        torch.cuda.synchronize()
    print(json.dumps({"step_only": True, "steps": args.warmup + args.steps, "N": wl.N}), flush=True)
    return 0


def run_batch_only(args, local):
    """W + K persistent adjoints of the 64-patch batch, nothing else on the device."""
    import torch

    from paper_1910_10908_gb300.batched import PatchBatch
    from synth import patch_batch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pb = patch_batch(64)
    with PatchBatch([(m, m, torch.from_numpy(lx).to(dev), torch.from_numpy(ly).to(dev))
                     for m, lx, ly, _ in pb]) as batch:
        for k, (_, _, _, v) in enumerate(pb):
            batch.load(k, torch.from_numpy(v).to(dev))
        for _ in range(args.warmup + args.steps):
            batch.adjoint()
        batch.wait()
        print(json.dumps({"batch_only": True, "adjoints": args.warmup + args.steps, "info": batch.info()}),
              flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="tffr", choices=["tffr", "reference"])
    ap.add_argument("--step-only", action="store_true",
                    help="run W + K steps of the main workload and nothing else (for ncu captures)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run W + K persistent adjoints of the 64-patch batch and nothing else (for ncu captures)")
    ap.add_argument("--section-s", type=float, default=1.0,
                    help="minimum timed length of each side section and of the main timed region (s); "
                         "the main region still times exactly K steps per repeat")
    args = ap.parse_args()
    global SECTION_S
    SECTION_S = max(0.0, args.section_s)
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        rc = run_reference(args, world, rank)
    elif args.step_only:
        rc = run_step_only(args, local)
    elif args.batch_only:
        rc = run_batch_only(args, local)
    else:
        rc = run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
