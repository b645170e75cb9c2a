#!/usr/bin/env python
"""Throughput benchmark of the GB300 seed-scanning track finder.

Headline (one step = one CUDA-graph replay of the batched configuration):
256 events, each a 104.97 MeV/c e- of 1-3 turns with 30-200 hits in the
finite-solenoid field map (451 x 1001 samples at 2 mm) plus DIO-like noise at
an occupancy uniform in 5-20 %, each with a seed grid of log-uniform 10^4-10^6
seeds around its first turn (~5.7e7 coarse seeds); ten scan rounds (the
coarse grid plus nine zoom rounds of 4 x 3^5 seeds at halved steps) with up to
3500 RKN steps of 2 mm and 3 turn partitions, and the hit classification of
every event's best seed, all in one CUDA graph.  value = seeds/s (coarse and
zoom seeds of all events over the replay's CUDA-event time); the roofline is
the coarse-round scan launch inside the graph against the FP32 FMA throughput
measured on the same GPU.  Inputs are seeded synthetic events generated on
the host.

Legs (timed separately, reported beside the headline):
  multi_turn: the single-event multi-turn configuration (circle Hough
    512 x 512 int32 -> a 10^6-seed grid -> ten rounds -> classification),
    eight distinct events in flight, and its one-event latency;
  single_turn: the uniform-field single-turn configuration (4000 seeds);
  refine: the 64 best seeds of each of 1024 distinct 3-turn events (65536
    seeds), five Gauss-Newton iterations, checkpointed adjoint gradient;
  sweep: 64 events at 30 % occupancy with 10^7 seeds in one CUDA graph, the
    batched Hough, and the FP32 steppers against the FP64 GPU stepper to 6 m;
  bidirectional, split_ab, event_loop: the ranked extensions.

--profile-case runs only the multi-turn leg on a 240000-seed coarse grid
(--profile-case full: on its 10^6-seed grid; with --profile-split also the
two-kernel A/B leg on the same event), --profile-batched N one eager
call of the batched step on its first N events (fixed launch shape, no
autotuning, so that the first scan-kernel launch is that call's coarse round),
and --profile-refine N only the refine leg on N events, for profiler captures;
their lines are marked as such and are not benchmark results.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the headline workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "seeds/s and RKN steps/s at 1 GB300 (frac. of FP32 peak) vs FP64 CPU oracle; refine seeds/s"
WORKLOAD = ("batched scan: 256 events in one CUDA-graph replay per step; per event a 104.97 MeV/c e- of 1-3 turns "
            "(30-200 hits) plus 5-20 % DIO-like occupancy in the solenoid map 451x1001 @ 2 mm, and a seed grid of "
            "log-uniform 10^4-10^6 seeds around its first turn (~5.7e7 coarse seeds in all); 10 scan rounds "
            "(coarse + 9 zoom x 4 x 3^5), RKN h=2 mm, <=3500 steps, 3 partitions; hit classification of every "
            "event's best seed")
WORKLOAD_MULTI_TURN = ("single multi-turn 104.97 MeV e- event, solenoid map 451x1001 @ 2 mm, 10% DIO-like occupancy; "
                       "circle Hough 512x512 -> 10^6-seed grid (10 theta0 x 40 z0 x 10 px0 x 10 py0 x 25 pz0); "
                       "10 scan rounds (coarse + 9 zoom x 4 x 3^5); RKN h=2 mm, <=3500 steps, 3 partitions; "
                       "hit classification of the best seed")
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per Blackwell SM
SCAN_SHAPES = [(256, 16), (256, 32), (128, 16), (128, 32)]   # order of cdc_tune_scan's timings
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the coarse-round scan launch of each workload
# from one single-pass ncu capture of this benchmark's own launch; valid only for the kernel sources it was
# taken on (csrc_digest: SHA-256 over the scan kernel's sources without comments), else null.
TRAFFIC = {
    "batched": {"bytes": 3974706176 + 8637271552, "shape": "128x32",
                "csrc_sha256": "8e79243e112a36e8eb454c4e15b9aaba8195532ee9fcfbacd4fb956d002a745b"},
    "multi_turn": {"bytes": 67645184 + 82392832, "shape": "256x32",
                   "csrc_sha256": None},
}
# Executed FP32 operations per RKN step of the coarse-round kernel (FFMA = 2; ncu on the reduced
# 240000-seed case, a per-step property of the code), same validity rule; the bench scales it by the
# measured launch.
FP32_COUNTS = {"fp32_ops_per_rkn_step": 247.9, "fma_pipe_active_pct": 41.9,
               "csrc_sha256": "8e79243e112a36e8eb454c4e15b9aaba8195532ee9fcfbacd4fb956d002a745b"}
FFMA_ITERS = 4096                # iterations of the FP32 throughput kernel (~4 ms on a GB300)


def csrc_digest() -> str:
    """SHA-256 over the sources the recorded scan-kernel counters depend on:
    the translation units that define and launch the scan kernel (scan.cu,
    capi.cu) and every header they include, with comments and whitespace
    removed, so that a comment edit, or a code edit in another translation
    unit (refine.cu, hough.cu, ...), keeps a measurement valid and an edit of
    the scan kernel's own code voids it."""
    import hashlib
    import re
    d = os.path.join(ROOT, "paper_1908_01949_gb300", "csrc")
    files, todo = set(), [os.path.join(d, "scan.cu"), os.path.join(d, "capi.cu")]
    while todo:
        f = os.path.normpath(todo.pop())
        if f in files:
            continue
        files.add(f)
        with open(f, encoding="utf-8") as fh:
            for inc in re.findall(r'^\s*#\s*include\s+"([^"]+)"', fh.read(), flags=re.M):
                todo.append(os.path.join(os.path.dirname(f), inc))
    h = hashlib.sha256()
    for f in sorted(files, key=lambda f: os.path.relpath(f, ROOT)):
        h.update(os.path.relpath(f, ROOT).encode())
        with open(f, encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()


def recorded(entry):
    """A recorded ncu figure if it was taken on the current kernel sources, else None."""
    return entry if entry and entry.get("csrc_sha256") == csrc_digest() else None


H, MAX_STEPS, LAM, MAX_PART, K, N_ROUNDS, N_ZOOM, MAX_DRIFT = 2.0, 3500, 4.0, 3, 8, 10, 4, 8.0
NC_CUT = 20                      # common hits of the entrance and exit scans (sec. 2.2)


def flops_per_step(kind: int) -> int:
    """Algorithmic FP32 operations of one classical RKN step (FMA = 2):
    field evaluation (map, x3): rho^2 3, sqrt 1, 1/rho 1, cell coordinates 4,
    bilinear Bz and Br 6 + 6, Br/rho 1, Bx, By 2 = 24; k = lam t x B (x4): 12;
    stage points t2, rm, t3, t4, re: 42; position update 21, direction update
    15.  The compensation of the FP32 state (Kahan, 24) and the wire lookup
    are not counted."""
    field = 24 if kind == 1 else 0
    return 3 * field + 4 * 12 + 42 + 21 + 15


# ------------------------------------------------------------------ helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                power.append(float(r[3]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


THROTTLE_REJECT = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clock_rejection(clocks):
    """Why a timed region's clock record rejects its number, else None: a
    hardware or thermal slowdown seen during it, or SM clocks held well below
    their maximum with no reason reported (a leftover clock lock).  A power cap
    (sw_power_cap) is kept and stays noted in the record."""
    bad = [r for r in clocks.get("reasons", []) if r in THROTTLE_REJECT]
    if bad:
        return "throttled: " + ", ".join(bad)
    sm, smax = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    if sm and smax and sm < 0.85 * smax and not clocks.get("reasons"):
        return f"SM clock {sm:.0f} of {smax:.0f} MHz with no reason reported"
    return None


def timed_region(run, sampler, sync, dist=None, device=None):
    """run() between barriers and device synchronisations under the clock
    sampler.  If any rank's clock record rejects the run, every rank runs it
    once more and the second run is kept, with the reason the first was
    rejected in the clock record."""
    def once():
        if dist:
            dist.barrier()
        sync()
        sampler.start()
        out = run()
        if dist:
            dist.barrier()
        return out, sampler.stop()

    out, clocks = once()
    why = clock_rejection(clocks)
    if reduce_max(1.0 if why else 0.0, dist, device) > 0.0:
        out, clocks = once()
        clocks["first_run_rejected"] = why or "clock record of another rank"
    return out, clocks


def grid_for_tuning(ctx, ne, off, wid, hp, acc, cand, ncand, grid, hflags, stream):
    """The step's seed grid (Hough output), computed once before tuning."""
    ctx.cdc_hough_seeds(ne, off, wid, hp, acc, cand, ncand, grid, hflags, stream)
    return grid


def guarded(name, fn):
    """Run one secondary leg; a failure is reported in its place instead of
    losing the benchmark line."""
    try:
        return fn()
    except Exception as e:  # noqa: BLE001 - the leg's error is the report
        import traceback
        traceback.print_exc()
        return {"error": f"{name}: {type(e).__name__}: {e}"}


def reduce_max(value: float, dist=None, device=None) -> float:
    """Max over ranks of a per-rank time: the slowest rank sets the step time."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world_size: int, units_per_rank_step: float, ms_per_step: float) -> float:
    """Whole-job throughput: every rank processes its own units each step
    (weak scaling), over the slowest rank's step time."""
    return world_size * units_per_rank_step / (ms_per_step / 1e3)


def make_workload(rank: int):
    """Rank r scans its own event (event sharding: events are independent, so
    the data path has no collective)."""
    import cdc_synth as S
    g = S.make_geometry()
    fm = S.solenoid_map()
    _, _, ev = S.cfg2_case(rank, fm, occupancy=0.10)
    return g, fm, ev


_GEN_FIELD = None


def _gen_init():
    global _GEN_FIELD
    import cdc_synth as S
    _GEN_FIELD = S.solenoid_map()


def _gen_cfg3(i):
    import cdc_synth as S
    return S.cfg3_event(i, _GEN_FIELD)


def _gen_cfg5(i):
    import cdc_synth as S
    return S.cfg5_event(i, _GEN_FIELD)


def make_batched_workload(n_events, first=0, gen=_gen_cfg3):
    """Events generated by a spawn pool (host only)."""
    import multiprocessing as mp
    import cdc_synth as S
    with mp.get_context("spawn").Pool(min(os.cpu_count() or 1, 32), initializer=_gen_init) as pool:
        out = pool.map(gen, range(first, first + n_events), chunksize=1)
    return [ev for ev, _ in out], np.concatenate([gr for _, gr in out]), S


def graph_scan(tr, off_t, wid_t, dr_t, gr_t, sp, warmup):
    """The whole scan call (all rounds, all events) captured in one CUDA graph."""
    import torch
    side = torch.cuda.Stream(device=tr.dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        tr.scan(off_t, wid_t, dr_t, gr_t, sp, want_hits=True, stream=side)
    side.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        out = tr.scan(off_t, wid_t, dr_t, gr_t, sp, want_hits=True, stream=side)
    for _ in range(max(warmup, 3)):
        graph.replay()
    torch.cuda.synchronize()
    return graph, out


def time_graph(graph, out, flush, reps):
    import torch
    times = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times), int(out["steps"].sum())



def fp32_peak(tr, sampler):
    """Measured FP32 FMA throughput of this GPU (cdc_fp32_peak: every SM at full
    occupancy, eight independent FMA chains per thread), best of three
    launches, with the SM clock sampled meanwhile; and the figure the unit
    counts and the maximum clock give, for reference."""
    import torch
    tr.ctx.cdc_fp32_peak(256)                                     # warm-up (clock ramp)
    sampler.start()
    runs = [tr.ctx.cdc_fp32_peak(FFMA_ITERS) for _ in range(3)]
    clocks = sampler.stop()
    best = max(runs, key=lambda r: r[0])
    props = torch.cuda.get_device_properties(tr.dev)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    units = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    return {"tflops": best[0], "ms": best[1], "runs_tflops": [r[0] for r in runs], "clocks": clocks,
            "units_tflops": units,
            "units_basis": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                           f"{sm_max:.0f} MHz",
            "kernel": "cdc_fp32_peak: 8 independent FFMA chains per thread x 16 x "
                      f"{FFMA_ITERS} iterations, full occupancy on every SM, CUDA-event timed, best of 3"}


def roofline(kernel, steps, ms, peak, traffic_key, shape):
    """ALU roofline of a coarse-round scan launch: 198 algorithmic FP32
    operations (FMA = 2) per executed RKN step over the launch's CUDA-event
    time, against the measured FP32 FMA throughput."""
    f_step = flops_per_step(1)
    achieved = f_step * steps / (ms / 1e3) / 1e12
    tr = recorded(TRAFFIC.get(traffic_key))
    fc = recorded(FP32_COUNTS)
    executed = fc["fp32_ops_per_rkn_step"] * steps / (ms / 1e3) / 1e12 if fc else None
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak["tflops"], "unit": "TFLOP/s",
            "frac": achieved / peak["tflops"], "traffic": tr["bytes"] if tr else None,
            "peak_basis": "measured on this GPU in this run (cdc_fp32_peak, FFMA throughput)",
            "peak_units": peak["units_tflops"], "frac_of_units": achieved / peak["units_tflops"],
            "launch_ms": ms, "rkn_steps": steps, "flops_per_rkn_step": f_step,
            "traffic_note": (f"DRAM bytes of this launch from one ncu capture at launch shape {tr['shape']} "
                             f"(this run's shape {shape[0]}x{shape[1]}; the shapes run the same per-seed code)")
                            if tr else "no ncu capture of the current kernel sources",
            "ncu_fp32": ({"fp32_ops_per_rkn_step": fc["fp32_ops_per_rkn_step"],
                          "fma_pipe_active_pct_240k_case": fc["fma_pipe_active_pct"],
                          "executed_tflops": executed, "executed_fp32_frac_of_peak": executed / peak["tflops"],
                          "note": "all executed FP32 work (FFMA = 2) per RKN step from ncu, times this launch's "
                                  "steps over its CUDA-event time"} if fc else None)}


def headline_batched(args, ws, rank, local, dist, g, fm, flush, sampler, peak):
    """The batched configuration as the benchmark's step: the whole call
    (staging, ten rounds with their top-K and zoom grids, classification of
    every event's best seed) in one CUDA graph, replayed once per step.  The
    library's kernel timer marks the scan launches inside the graph, so the
    coarse round's own CUDA-event time is read after every replay."""
    import torch
    import paper_1908_01949_gb300 as cdc
    n_ev = int(args.batched_events)
    evs, grids, S = make_batched_workload(n_ev, first=1000 * rank)
    counts = [int(np.prod(gr["n"])) for gr in grids]
    n = sum(counts)
    off, wid, dr = S.pack_events(evs)
    tr = cdc.Tracker(g, fm, device=local, max_events=n_ev, max_seeds=n, max_hits=int(wid.size))
    dev = tr.dev
    sp = cdc.scan_params(h=H, max_steps=MAX_STEPS, lam=LAM, max_partitions=MAX_PART, k=K, n_rounds=N_ROUNDS,
                         n_zoom=N_ZOOM, max_drift=MAX_DRIFT)
    off_h = torch.from_numpy(off.astype(np.int32)).pin_memory()
    wid_h = torch.from_numpy(wid.astype(np.int32)).pin_memory()
    dr_h = torch.from_numpy(dr.astype(np.float32)).pin_memory()
    gr_h = cdc.grids_to_tensor(grids, "cpu").pin_memory()
    off_t, wid_t, dr_t, gr_t = (x.to(dev) for x in (off_h, wid_h, dr_h, gr_h))
    n_tune = min(n_ev, 32)    # tune on the first 32 events (one coarse round per shape)
    if args.scan_shape:
        tuned, tune_ms = tuple(int(x) for x in args.scan_shape.split(",")), None
        tr.ctx.cdc_set_scan_config(*tuned)
    else:
        tuned, tune_ms = tr.tune(off_t[:n_tune + 1], wid_t, dr_t, gr_t[:n_tune], sp, reps=1)
    # capture: eager warm call, then the graph with the kernel timer's marks as graph nodes
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        tr.scan(off_t, wid_t, dr_t, gr_t, sp, want_hits=True, stream=side)
    side.synchronize()
    tr.ctx.cdc_kernel_timer(2)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        out = tr.scan(off_t, wid_t, dr_t, gr_t, sp, want_hits=True, stream=side)
    for _ in range(max(args.warmup, 3)):
        graph.replay()
    torch.cuda.synchronize()
    seeds_step = n + (N_ROUNDS - 1) * N_ZOOM * 243 * n_ev
    # launches of this repository's kernels per replay (ncu launch list): staging 2, block order 1; per round
    # prologue, scan, top-K partial and merge, best merge (5); a zoom-grid build per zoom round; assignment 1
    launches_per_step = 2 + 1 + 5 * N_ROUNDS + (N_ROUNDS - 1) + 1

    def run():
        times, coarse, steps = [], [], []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            graph.replay()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            try:
                _, nl, per = tr.ctx.cdc_kernel_time()
                coarse.append(float(per[0]) if nl else float("nan"))
            except cdc.CdcError:
                coarse.append(float("nan"))
            steps.append(out["steps"].cpu().numpy().astype(np.float64))
        return times, coarse, steps

    (times, coarse, steps), clocks = timed_region(run, sampler, torch.cuda.synchronize, dist, dev)
    ms = reduce_max(sum(times) / len(times), dist, dev)
    rkn_step = float(np.mean([s.sum() for s in steps]))
    coarse_steps = float(np.mean([s[0] for s in steps]))
    coarse_ms = float(np.mean(coarse))
    coarse_source = "event-record nodes around the coarse scan launch inside every timed replay"
    if not np.isfinite(coarse_ms):
        # the graph's timer nodes gave no time: the same call eager, marks around its coarse launch
        tr.ctx.cdc_kernel_timer(1)
        flush.zero_()
        tr.scan(off_t, wid_t, dr_t, gr_t, sp, want_hits=True)
        _, nl, per = tr.ctx.cdc_kernel_time()
        tr.ctx.cdc_kernel_timer(0)
        coarse_ms = float(per[0])
        coarse_source = "CUDA events around the coarse scan launch of one eager call of the same step"
    fl = out["flags"].cpu().numpy()
    # end to end: per step the events' hits and grids copied from pinned host memory into the graph's inputs,
    # the replay, and every event's best seeds and scores, hit classes and flags copied back; host wall clock
    k_e2e = max(1, min(args.steps, args.e2e_steps))
    res = {k: torch.empty(out[k].shape, dtype=out[k].dtype).pin_memory()
           for k in ("best_E", "best_seed", "hit_part", "flags")}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        for h, d in ((off_h, off_t), (wid_h, wid_t), (dr_h, dr_t), (gr_h, gr_t)):
            d.copy_(h, non_blocking=True)
        graph.replay()
        for k, h in res.items():
            h.copy_(out[k], non_blocking=True)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / k_e2e
    h2d = int(sum(x.numel() * x.element_size() for x in (off_h, wid_h, dr_h, gr_h)))
    d2h = int(sum(x.numel() * x.element_size() for x in res.values()))
    # classification quality (sec. 3.1, Eqs. 2-3): the grids are centred on the first turn, so scan partition k
    # is truth turn k
    truth = torch.as_tensor(np.concatenate([e.truth_part for e in evs]).astype(np.int8), device=dev)
    cls_counts = tr.classification_counts(off_t, out["hit_part"], truth, MAX_PART)
    eps, pur = (x.cpu().numpy() for x in tr.efficiency_purity(cls_counts))
    return {
        "ms": ms, "seeds_step": seeds_step, "rkn_step": rkn_step, "clocks": clocks, "n_events": n_ev,
        "launches_per_step": launches_per_step,
        "roofline": roofline("scan_kernel<map> (coarse round of the batched step, inside the graph)", coarse_steps,
                             coarse_ms, peak, "batched", tuned),
        "e2e": {"value": job_value(ws, seeds_step, e2e_ms), "unit": "seeds/s", "ms_per_step": e2e_ms,
                "steps": k_e2e, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "detail": {"events": n_ev, "coarse_seeds": n, "seeds_per_step": seeds_step,
                   "coarse_seeds_min_max": [min(counts), max(counts)], "hits": int(wid.size),
                   "events_per_s": job_value(ws, n_ev, ms), "coarse_launch_ms": coarse_ms,
                   "coarse_launch_timing": coarse_source,
                   "replay_ms": times, "graph": "one CUDA graph per step (all rounds, all events)",
                   "autotune": {"config": {"block": tuned[0], "chunk": tuned[1]}, "ms_by_shape": tune_ms,
                                "events": n_tune},
                   "flagged_events": int((fl != 0).sum()),
                   "classification": {"partition": list(range(MAX_PART)),
                                      "efficiency": [None if np.isnan(x) else float(x) for x in eps],
                                      "purity": [None if np.isnan(x) else float(x) for x in pur],
                                      "definition": "Eqs. 2-3 summed over the events; scan partition k = truth "
                                                    "turn k"}},
        "workload": {"evs": evs, "grids": grids, "counts": counts},
    }


def profile_batched(args, local, g, fm, flush):
    """One eager call of the batched step on its first N events, at a fixed
    launch shape (no autotuning): the call's first scan-kernel launch is its
    coarse round, the launch a profiler capture takes (-k scan_kernel -c 1)."""
    import torch
    import paper_1908_01949_gb300 as cdc
    n_ev = int(args.profile_batched)
    evs, grids, S = make_batched_workload(n_ev)
    n = int(sum(int(np.prod(gr["n"])) for gr in grids))
    off, wid, dr = S.pack_events(evs)
    tr = cdc.Tracker(g, fm, device=local, max_events=n_ev, max_seeds=n, max_hits=int(wid.size))
    tr.ctx.cdc_set_scan_config(*(tuple(int(x) for x in args.scan_shape.split(",")) if args.scan_shape else (128, 32)))
    sp = cdc.scan_params(h=H, max_steps=MAX_STEPS, lam=LAM, max_partitions=MAX_PART, k=K, n_rounds=N_ROUNDS,
                         n_zoom=N_ZOOM, max_drift=MAX_DRIFT)
    off_t, wid_t, dr_t = tr.events_to_device(off, wid, dr)
    gr_t = cdc.grids_to_tensor(grids, tr.dev)
    tr.ctx.cdc_kernel_timer(1)
    flush.zero_()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    out = tr.scan(off_t, wid_t, dr_t, gr_t, sp, want_hits=True)
    t1.record()
    torch.cuda.synchronize()
    _, nl, per = tr.ctx.cdc_kernel_time()
    tr.ctx.cdc_kernel_timer(0)
    ms = t0.elapsed_time(t1)
    seeds = n + (N_ROUNDS - 1) * N_ZOOM * 243 * n_ev
    steps = out["steps"].cpu().numpy()
    return {"events": n_ev, "coarse_seeds": n, "ms": ms, "seeds_per_s": seeds / (ms / 1e3),
            "coarse_launch_ms": float(per[0]) if nl else None, "coarse_rkn_steps": float(steps[0]),
            "rkn_steps": float(steps.sum())}


def multi_turn_leg(args, ws, rank, local, g, fm, flush, peak):
    """The single-event multi-turn configuration: circle Hough -> 10^6-seed grid
    -> ten rounds -> classification of the best seed per event.  Throughput:
    a stream of events with `inflight` of them in flight (one context and
    stream each, each slot its own distinct event); latency and the coarse
    round's roofline: one event at a time on one stream."""
    import torch
    import cdc_synth as S
    import paper_1908_01949_gb300 as cdc
    dev = torch.device("cuda", local)
    n_in = max(1, int(args.inflight))
    evs = [S.cfg2_case(1000 * rank + k, fm, occupancy=0.10)[2] for k in range(n_in)]
    tmpl = S.cfg2_grid_template()
    if args.profile_case == "reduced":
        tmpl["n"][0][4] = 6                       # 10 x 40 x 10 x 10 x 6 = 240000 coarse seeds
    seeds_coarse = int(np.prod(tmpl["n"][0]))
    seeds_per_step = seeds_coarse + (N_ROUNDS - 1) * N_ZOOM * 243
    hp = cdc.hough_params(grid_template=tmpl, **S.CFG2_HOUGH)
    sp = cdc.scan_params(h=H, max_steps=MAX_STEPS, lam=LAM, max_partitions=MAX_PART, k=K, n_rounds=N_ROUNDS,
                         n_zoom=N_ZOOM, max_drift=MAX_DRIFT)
    ne = 1

    def make_slot(k):
        """One event in flight: its own context (workspace), stream, event and buffers."""
        ev = evs[k]
        nh = int(ev.wire_id.size)
        t = cdc.Tracker(g, fm, device=local, max_events=1, max_seeds=seeds_coarse, max_hits=4096)
        d = dict(tr=t, ctx=t.ctx, stream=torch.cuda.current_stream() if k == 0 else torch.cuda.Stream(device=dev),
                 off_h=torch.tensor([0, nh], dtype=torch.int32).pin_memory(),
                 wid_h=torch.from_numpy(ev.wire_id.astype(np.int32)).pin_memory(),
                 dr_h=torch.from_numpy(ev.drift.astype(np.float32)).pin_memory(),
                 acc=torch.empty((ne, hp.n_bins, hp.n_bins), dtype=torch.int32, device=dev),
                 cand=torch.empty((ne, hp.max_cand, 28), dtype=torch.uint8, device=dev),
                 ncand=torch.empty(ne, dtype=torch.int32, device=dev),
                 grid=torch.empty((ne, cdc.GRID_BYTES), dtype=torch.uint8, device=dev),
                 hflags=torch.empty(ne, dtype=torch.int32, device=dev),
                 best_E=torch.empty((ne, K), dtype=torch.float32, device=dev),
                 best_seed=torch.empty((ne, K, 5), dtype=torch.float32, device=dev),
                 topk0=torch.empty((ne, K), dtype=torch.int64, device=dev),
                 hit_part=torch.empty(nh, dtype=torch.int8, device=dev),
                 sflags=torch.empty(ne, dtype=torch.int32, device=dev),
                 steps=torch.zeros(N_ROUNDS, dtype=torch.int64, device=dev),
                 out_E=torch.empty((ne, K), dtype=torch.float32).pin_memory(),
                 out_S=torch.empty((ne, K, 5), dtype=torch.float32).pin_memory(),
                 out_P=torch.empty(nh, dtype=torch.int8).pin_memory(),
                 out_F=torch.empty(ne, dtype=torch.int32).pin_memory())
        for a in ("off", "wid", "dr"):
            d[a] = d[a + "_h"].to(dev)
        return d

    slots = [make_slot(k) for k in range(n_in)]
    q0 = slots[0]
    tr, ctx, stream = q0["tr"], q0["ctx"], q0["stream"]

    def step(q, h2d=False, d2h=False):
        """One event through the hot path on slot q's stream; with h2d / d2h the
        inputs come from pinned host memory and the results go back to it."""
        st = q["stream"]
        with torch.cuda.stream(st):
            if h2d:
                for a in ("off", "wid", "dr"):
                    q[a].copy_(q[a + "_h"], non_blocking=True)
            q["ctx"].cdc_hough_seeds(ne, q["off"], q["wid"], hp, q["acc"], q["cand"], q["ncand"], q["grid"],
                                     q["hflags"], st)
            q["ctx"].cdc_scan_seeds(ne, q["off"], q["wid"], q["dr"], q["grid"], sp, None, q["topk0"], q["best_E"],
                                    q["best_seed"], q["hit_part"], None, None, q["sflags"], q["steps"], st)
            if d2h:
                q["out_E"].copy_(q["best_E"], non_blocking=True)
                q["out_S"].copy_(q["best_seed"], non_blocking=True)
                q["out_P"].copy_(q["hit_part"], non_blocking=True)
                q["out_F"].copy_(q["sflags"], non_blocking=True)

    grid_for_tuning(ctx, ne, q0["off"], q0["wid"], hp, q0["acc"], q0["cand"], q0["ncand"], q0["grid"], q0["hflags"],
                    stream)
    if args.scan_shape:
        tuned = tuple(int(x) for x in args.scan_shape.split(","))
        tune_ms = None
    else:
        tuned, tune_ms = tr.tune(q0["off"], q0["wid"], q0["dr"], q0["grid"], sp, reps=3, stream=stream)
    # zoom rounds (972 seeds per event): one event at a time, one warp per seed
    # shortens them (latency); with many events in flight one lane per seed
    # leaves the other events' coarse rounds the warp slots (throughput)
    lat_ws = args.warp_seeds if args.warp_seeds is not None else ctx.cdc_get_scan_config()[2]
    thr_ws = args.stream_warp_seeds
    for q in slots:
        q["ctx"].cdc_set_scan_config(*tuned, thr_ws)
    ctx.cdc_set_scan_config(*tuned, lat_ws)
    # Hough vote, maximum, slice peaks, merge; table clear + staging; block order of the coarse grid; per
    # round prologue, scan, top-K partial + merge, best merge; a zoom grid build per zoom round; hit assignment
    launches_per_step = 4 + 2 + 1 + 5 * N_ROUNDS + (N_ROUNDS - 1) + 1
    for i in range(args.warmup * n_in):
        step(slots[i % n_in])
    torch.cuda.synchronize()

    # latency and the roofline: one event at a time on one stream, the library's
    # CUDA events around every scan-kernel launch
    q0["steps"].zero_()
    ctx.cdc_kernel_timer(True)
    lat_ms = []
    for i in range(args.mt_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(q0)
        e1.record(stream)
        torch.cuda.synchronize()
        lat_ms.append(e0.elapsed_time(e1))
    _, _, kper = ctx.cdc_kernel_time()
    ctx.cdc_kernel_timer(False)
    ctx.cdc_set_scan_config(*tuned, thr_ws)
    rkn = q0["steps"].cpu().numpy().astype(np.float64)
    coarse_ms = [float(kper[i]) for i in range(0, len(kper), N_ROUNDS)]
    coarse_steps = float(rkn[0]) / args.mt_steps
    latency = statistics.median(lat_ms)

    # throughput: a stream of events, n_in of them in flight (one context and
    # stream each, round robin); every step is one event's whole hot path
    def run_stream(h2d=False, d2h=False):
        main = torch.cuda.current_stream()
        for q in slots:
            q["steps"].zero_()
            q["stream"].wait_stream(main)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(main)
        for i in range(args.mt_steps):
            q = slots[i % n_in]
            with torch.cuda.stream(q["stream"]):
                flush.zero_()
            step(q, h2d, d2h)
        for q in slots:
            main.wait_stream(q["stream"])
        e1.record(main)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3

    dev_ms, _ = run_stream()
    ms = dev_ms / args.mt_steps
    rkn_per_step = float(sum(q["steps"].sum().item() for q in slots)) / args.mt_steps
    _, e2e_wall = run_stream(h2d=True, d2h=True)
    e2e = e2e_wall / args.mt_steps
    h2d = int(np.mean([sum(q[a + "_h"].numel() * 4 for a in ("off", "wid", "dr")) for q in slots]))
    d2h = int(np.mean([q["out_E"].numel() * 4 + q["out_S"].numel() * 4 + q["out_P"].numel() + q["out_F"].numel() * 4
                       for q in slots]))
    # the Hough call of one event alone (vote and peak search), CUDA events on its stream
    hough_ms = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.cdc_hough_seeds(ne, q0["off"], q0["wid"], hp, q0["acc"], q0["cand"], q0["ncand"], q0["grid"],
                            q0["hflags"], stream)
        e1.record(stream)
        torch.cuda.synchronize()
        hough_ms.append(e0.elapsed_time(e1))
    # does the Hough grid (top candidate) of each in-flight event hold the signal's first turn
    held = held_any = 0
    half = 0.5 * np.asarray(tmpl["step"][0], np.float64) * np.asarray(tmpl["n"][0], np.float64)

    def holds(th, px, py, t):
        dth = (float(th) - t[0] + np.pi) % (2 * np.pi) - np.pi
        return abs(dth) <= half[0] and abs(px - t[2]) <= half[2] and abs(py - t[3]) <= half[3]

    for k, q in enumerate(slots):
        t = evs[k].truth_seeds[0]
        gr = cdc.tensor_to_grids(q["grid"])[0]
        held += int(gr["n"][0] > 0 and holds(gr["centre"][0], gr["centre"][2], gr["centre"][3], t))
        cd = cdc.decode_candidates(q["cand"]).reshape(-1)[:int(q["ncand"][0].item())]
        held_any += int(any(holds(c["theta0"], c["px0"], c["py0"], t) for c in cd))
    return {
        "workload": WORKLOAD_MULTI_TURN, "seeds_per_step": seeds_per_step, "ms_per_step": ms,
        "seeds_per_s": job_value(ws, seeds_per_step, ms), "rkn_steps_per_s": job_value(ws, rkn_per_step, ms),
        "events_in_flight": n_in, "distinct_events": n_in, "steps": args.mt_steps,
        "zoom_rounds": {"throughput_run": "warp per seed" if thr_ws >= N_ZOOM * 243 else "lane per seed",
                        "latency_run": "warp per seed" if lat_ws >= N_ZOOM * 243 else "lane per seed"},
        "latency_ms_per_event": latency,
        "roofline": roofline("scan_kernel<map> (coarse round of one event)", coarse_steps,
                             statistics.mean(coarse_ms), peak, "multi_turn", tuned) if coarse_ms else None,
        "autotune": {"config": {"block": tuned[0], "chunk": tuned[1]},
                     "shapes": [{"block": b, "chunk": c} for b, c in SCAN_SHAPES], "coarse_round_ms": tune_ms},
        "e2e": {"value": seeds_per_step / (e2e / 1e3), "unit": "seeds/s", "ms_per_step": e2e,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "launches_per_step": launches_per_step,
        "hough": {"radii_mm": [hp.r_min_um / 1000.0, (hp.r_min_um + (hp.n_r - 1) * hp.r_step_um) / 1000.0],
                  "angles": hp.n_phi, "candidates": hp.max_cand,
                  "ms_one_event": statistics.median(hough_ms),
                  "grid_holds_signal": held, "some_candidate_grid_holds_signal": held_any, "events": n_in,
                  "definition": "the (theta0, px0, py0) of the signal's first turn lies within the grid the top "
                                "Hough candidate centres (or one of the grids cdc_candidate_grids centres on the "
                                "candidates); the timed step scans the top candidate's grid"},
        "l2": "256 MiB flush before every step, issued on the step's stream inside the timed events "
              "(~40 us per step counted against the result)",
        "_cpu": (evs[0], q0["grid"]),
    }


def single_turn_leg(args, ws, rank, local, g, flush):
    """The uniform-field single-turn configuration: 4000 seeds around the
    truth of one event (40 uniform noise wires), ten rounds and the
    classification; one event per call (latency) and 64 distinct events in
    one call (throughput)."""
    import torch
    import cdc_synth as S
    import paper_1908_01949_gb300 as cdc
    cases = [S.cfg1_case(20_000 + 100 * rank + i) for i in range(64)]
    fu = cases[0][1]
    evs = [c[2] for c in cases]
    grids = np.concatenate([c[3] for c in cases])
    n1 = int(np.prod(grids[0]["n"]))
    off, wid, dr = S.pack_events(evs)
    tr = cdc.Tracker(g, fu, device=local, max_events=64, max_seeds=64 * n1, max_hits=int(wid.size))
    sp = cdc.scan_params(h=H, max_steps=1000, lam=LAM, max_partitions=1, k=K, n_rounds=N_ROUNDS, n_zoom=N_ZOOM,
                         max_drift=MAX_DRIFT)
    off_t, wid_t, dr_t = tr.events_to_device(off, wid, dr)
    gr_t = cdc.grids_to_tensor(grids, tr.dev)
    one = tr.events_to_device([0, evs[0].wire_id.size], evs[0].wire_id, evs[0].drift)
    tuned, _ = tr.tune(off_t, wid_t, dr_t, gr_t, sp, reps=1)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    lat = timed(lambda: tr.scan(*one, gr_t[:1], sp), 5)
    thr = timed(lambda: tr.scan(off_t, wid_t, dr_t, gr_t, sp), 3)
    per_event = n1 + (N_ROUNDS - 1) * N_ZOOM * 243
    return {"workload": "single-turn 104.97 MeV e-, uniform 1 T, 40 uniform noise wires; 8x4x5x5x5 = 4000-seed grid "
                        "around the truth; 10 rounds; classification", "seeds_per_event": per_event,
            "latency_ms_per_event": lat, "events_per_call": 64, "ms_per_call": thr,
            "seeds_per_s": 64 * per_event / (thr / 1e3), "events_per_s": 64 / (thr / 1e3),
            "autotune": {"block": tuned[0], "chunk": tuned[1]},
            "timing": "median CUDA-event time, L2 flushed before each call"}


def _gen_bidir(i):
    import cdc_synth as S
    return S.cfg2_case(20_000 + i, _GEN_FIELD, occupancy=0.10)[2]


BIDIR_SEEDS = 100_000


def bidirectional_leg(args, rank, local, g, fm, flush):
    """Bidirectional scan (sec. 2.2): the first turn of each multi-turn event
    scanned from its entrance (direction +1) and from its exit (direction -1),
    ten rounds each, all events of a direction in one call, then N_c (hits in
    partition 0 of both) per event and the N_c >= 20 cut.  Grids: the multi-turn
    grid scaled to 10^5 seeds around each truth seed (random sub-step offset)."""
    import multiprocessing as mp
    import torch
    import cdc_synth as S
    import paper_1908_01949_gb300 as cdc
    n_ev = int(args.bidir_events)
    with mp.get_context("spawn").Pool(min(os.cpu_count() or 1, 32), initializer=_gen_init) as pool:
        evs = pool.map(_gen_bidir, range(1000 * rank, 1000 * rank + n_ev), chunksize=1)
    rng = np.random.default_rng(11)
    ent = np.concatenate([S.scaled_grid(e.truth_seeds[0], BIDIR_SEEDS, rng) for e in evs])
    ext = np.concatenate([S.scaled_grid(e.exit_seeds[0], BIDIR_SEEDS, rng) for e in evs])
    for gr, e in zip(ext, evs):                      # the exit seed's (z0, pz0) is not at 0: centre them too
        gr["centre"][1], gr["centre"][4] = e.exit_seeds[0][1], e.exit_seeds[0][4]
    for gr, e in zip(ent, evs):
        gr["centre"][1], gr["centre"][4] = e.truth_seeds[0][1], e.truth_seeds[0][4]
    off, wid, dr = S.pack_events(evs)
    n_seeds = max(int(sum(np.prod(gr["n"]) for gr in ent)), int(sum(np.prod(gr["n"]) for gr in ext)))
    tr = cdc.Tracker(g, fm, device=local, max_events=n_ev, max_seeds=n_seeds, max_hits=int(wid.size))
    off_t, wid_t, dr_t = tr.events_to_device(off, wid, dr)
    ps = [cdc.scan_params(h=H, max_steps=MAX_STEPS, lam=LAM, max_partitions=1, direction=d, k=K, n_rounds=N_ROUNDS,
                          n_zoom=N_ZOOM, max_drift=MAX_DRIFT) for d in (1, -1)]
    gts = [cdc.grids_to_tensor(ent, tr.dev), cdc.grids_to_tensor(ext, tr.dev)]

    def run():
        outs = [tr.scan(off_t, wid_t, dr_t, gt, p) for gt, p in zip(gts, ps)]
        return outs, tr.common_hits(off_t, outs[0]["hit_part"], outs[1]["hit_part"])

    for _ in range(max(args.warmup, 1)):
        run()
    torch.cuda.synchronize()
    times = []
    for _ in range(3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        outs, nc = run()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    nc = nc.cpu().numpy()
    turn0 = np.array([int(np.sum(e.truth_part == 0)) for e in evs])
    # Eqs. 2-3 for the scanned turn (partition 0 of either direction = truth
    # turn 0) per event, averaged over the events that pass N_c >= 20; the
    # other truth turns count as signal partitions in the purity
    truth_t = torch.as_tensor(np.concatenate([e.truth_part for e in evs]).astype(np.int8), device=tr.dev)
    keep = np.flatnonzero(nc >= NC_CUT)
    quality = {}
    for name, o in zip(("entrance", "exit"), outs):
        C = tr.classification_counts(off_t, o["hit_part"], truth_t, 8)
        ep = np.array([[float(v[0]) for v in tr.efficiency_purity(C[e])] for e in keep]).reshape(-1, 2)
        quality[name] = {"efficiency_mean": float(np.nanmean(ep[:, 0])) if keep.size else None,
                         "purity_mean": float(np.nanmean(ep[:, 1])) if keep.size else None}
    return {"events": n_ev, "seeds_per_direction": n_seeds, "ms": ms, "events_per_s": n_ev / (ms / 1e3),
            "seeds_per_s": 2 * (n_seeds + (N_ROUNDS - 1) * N_ZOOM * 243 * n_ev) / (ms / 1e3),
            "n_common_mean": float(nc.mean()), "n_common_min": int(nc.min()),
            "pass_nc_ge_20": float(np.mean(nc >= NC_CUT)), "turn0_hits_mean": float(turn0.mean()),
            "classification_nc_ge_20": dict(quality, events=int(keep.size),
                                            definition="Eqs. 2-3 of the scanned turn per event, mean over the "
                                                       "events with N_c >= 20 (the paper: 76 % / 90 % for its "
                                                       "last turn partition on COMET simulation)"),
            "timing": "median of 3: both directions' ten-round scans and the N_c kernel"}


def event_loop_leg(args, rank, local, g, fm):
    """The event loop over turn partitions (sec. 2.3, Fig. 7) on multi-turn
    events: a scan around the first turn (10^5 seeds; the synthetic events have
    no trigger counter that would single out the last turn), then refine,
    extrapolation to the neighbouring turns and narrow scans until fewer than
    ten hits remain.
    Wall-clock per event (the loop waits for each step); efficiency and purity
    per truth turn (Eqs. 2-3) from the library's counting kernel."""
    import multiprocessing as mp
    import torch
    import cdc_synth as S
    import paper_1908_01949_gb300 as cdc
    from paper_1908_01949_gb300.event_loop import align_to_truth, event_loop, findable_truth
    n_ev = int(args.loop_events)
    with mp.get_context("spawn").Pool(min(os.cpu_count() or 1, 32), initializer=_gen_init) as pool:
        evs = pool.map(_gen_bidir, range(5000 + 1000 * rank, 5000 + 1000 * rank + n_ev), chunksize=1)
    tr = cdc.Tracker(g, fm, device=local, max_events=1, max_seeds=BIDIR_SEEDS, max_hits=4096)
    sp = cdc.scan_params(h=H, max_steps=MAX_STEPS, lam=LAM, max_partitions=1, k=K, n_rounds=N_ROUNDS,
                         n_zoom=N_ZOOM, max_drift=MAX_DRIFT)
    rp = cdc.refine_params(n_iter=REFINE_ITER, sigma=REFINE_SIGMA, checkpoint=REFINE_CKPT)
    rng = np.random.default_rng(13)
    grids = []
    for e in evs:
        gr = S.scaled_grid(e.truth_seeds[0], BIDIR_SEEDS, rng)
        gr["centre"][0][1], gr["centre"][0][4] = e.truth_seeds[0][1], e.truth_seeds[0][4]
        grids.append(gr)
    event_loop(tr, evs[0].wire_id, evs[0].drift, grids[0], sp, rp)          # warm-up
    torch.cuda.synchronize()
    n_turns = max(e.n_turns for e in evs)
    counts = np.zeros((n_turns + 1, n_turns + 1), np.int64)
    found = []
    t0 = time.perf_counter()
    for e, gr in zip(evs, grids):
        labels, seeds = event_loop(tr, e.wire_id, e.drift, gr, sp, rp)
        aligned = align_to_truth(labels, e.truth_part)
        dev = tr.dev
        c = tr.classification_counts(torch.tensor([0, e.wire_id.size], dtype=torch.int32, device=dev),
                                     torch.as_tensor(aligned, device=dev),
                                     torch.as_tensor(findable_truth(e.truth_part), device=dev), n_turns)
        counts += c[0].cpu().numpy()
        found.append(len(seeds))
    wall = time.perf_counter() - t0
    eps, pur = (x.cpu().numpy() for x in tr.efficiency_purity(torch.as_tensor(counts.astype(np.int32), device=tr.dev)))
    return {"events": n_ev, "ms_per_event": 1e3 * wall / n_ev, "events_per_s": n_ev / wall,
            "turns_found_mean": float(np.mean(found)), "truth_turns_mean": float(np.mean([e.n_turns for e in evs])),
            "efficiency_per_turn": [None if np.isnan(x) else float(x) for x in eps],
            "purity_per_turn": [None if np.isnan(x) else float(x) for x in pur],
            "truth": "turns of fewer than 10 hits (never taken as a turn by the loop) count as noise",
            "timing": "host wall clock over the events (each step waits for the GPU)"}


SPLIT_PZ, SPLIT_CHUNK = 4, 32768


def split_ab_leg(args, rank, local, g, fm, ev, grid_t, flush):
    """The coarse round of the multi-turn event on a reduced grid (4 pz0 values,
    160000 seeds) by the fused scan and by the paper's two-kernel organisation
    (states recorded by a thread per seed, then a block per seed and a thread
    per hit), timed with CUDA events; the scores agree to float rounding."""
    import torch
    import paper_1908_01949_gb300 as cdc
    gg = cdc.tensor_to_grids(grid_t).copy()
    gg["n"][0][4] = SPLIT_PZ
    n = int(np.prod(gg["n"][0]))
    tr = cdc.Tracker(g, fm, device=local, max_events=1, max_seeds=n, max_hits=4096)
    tr.ctx.cdc_reserve_split(args.split_chunk, MAX_STEPS)
    tr.ctx.cdc_set_scan_config(128, 32)
    off, wid, dr = tr.events_to_device([0, ev.wire_id.size], ev.wire_id, ev.drift)
    gt = cdc.grids_to_tensor(gg, tr.dev)
    sp = cdc.scan_params(h=H, max_steps=MAX_STEPS, lam=LAM, max_partitions=MAX_PART, k=K, n_rounds=1,
                         max_drift=MAX_DRIFT)
    E = torch.empty(n, dtype=torch.float32, device=tr.dev)
    flags = torch.empty(1, dtype=torch.int32, device=tr.dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), out

    ms_f, fused = timed(lambda: tr.scan(off, wid, dr, gt, sp, want_E=True, want_hits=False, n_seeds=n))
    ms_s, _ = timed(lambda: tr.ctx.cdc_scan_seeds_split(1, n, off, wid, dr, gt, sp, E, flags))
    Ef, Es = fused["E"].cpu().numpy(), E.cpu().numpy()
    return {"seeds": n, "fused_ms": ms_f, "split_ms": ms_s, "fused_seeds_per_s": n / (ms_f / 1e3),
            "split_seeds_per_s": n / (ms_s / 1e3), "speedup_fused_over_split": ms_s / ms_f,
            "max_rel_score_diff": float(np.max(np.abs(Es - Ef) / np.maximum(np.abs(Ef), 1e-30))),
            "split_chunk": args.split_chunk, "timing": "median of 3 single-round calls, L2 flushed before each"}


SWEEP_EVERY, SWEEP_REC, SWEEP_SEEDS = 250, 12, 10_000


def sweep_leg(args, rank, local, g, fm, flush):
    """Precision/scale sweep: scan throughput at 30 % occupancy (10^7 seeds
    over 64 events, one CUDA graph), the batched Hough of all events, and the
    position difference of the FP32 steppers from the FP64 GPU stepper against
    path length (0.5-6 m) on a 10^4-seed subsample of the events' grids."""
    import torch
    import cdc_synth as S
    import paper_1908_01949_gb300 as cdc
    n_ev = int(args.sweep_events)
    evs, grids, _ = make_batched_workload(n_ev, first=1000 * rank, gen=_gen_cfg5)
    counts = [int(np.prod(gr["n"])) for gr in grids]
    n = sum(counts)
    off, wid, dr = S.pack_events(evs)
    tr = cdc.Tracker(g, fm, device=local, max_events=n_ev, max_seeds=n, max_hits=int(wid.size))
    sp = cdc.scan_params(h=H, max_steps=MAX_STEPS, lam=LAM, max_partitions=MAX_PART, k=K, n_rounds=N_ROUNDS,
                         n_zoom=N_ZOOM, max_drift=MAX_DRIFT)
    off_t, wid_t, dr_t = tr.events_to_device(off, wid, dr)
    gr_t = cdc.grids_to_tensor(grids, tr.dev)
    graph, out = graph_scan(tr, off_t, wid_t, dr_t, gr_t, sp, args.warmup)
    ms, steps = time_graph(graph, out, flush, args.batched_steps)
    seeds_step = n + (N_ROUNDS - 1) * N_ZOOM * 243 * n_ev
    # batched Hough of all events
    hp = cdc.hough_params(grid_template=S.cfg2_grid_template())
    h = tr.hough(off_t, wid_t, hp)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    h = tr.hough(off_t, wid_t, hp)
    e1.record()
    torch.cuda.synchronize()
    hough_ms = e0.elapsed_time(e1)
    votes = int(h["acc"].sum(dtype=torch.int64))
    acc_bytes = 2 * int(h["acc"].numel()) * 4
    # FP32 steppers against the FP64 GPU stepper
    rng = np.random.default_rng(3)
    pick = np.sort(rng.choice(n, size=min(SWEEP_SEEDS, n), replace=False))
    base = np.concatenate([[0], np.cumsum(counts)])
    ev_of = np.searchsorted(base, pick, side="right") - 1
    seeds = np.stack([grid_value(grids[e], int(i - base[e])) for e, i in zip(ev_of, pick)]).astype(np.float32)
    gs = S.sweep_geometry(g)
    ts = cdc.Tracker(gs, fm, device=local, max_events=1, max_seeds=1, max_hits=1)
    pp = cdc.scan_params(h=H, max_steps=SWEEP_EVERY * SWEEP_REC, lam=LAM, max_partitions=16)
    ds = torch.as_tensor(seeds, device=ts.dev)
    pos = {prec: ts.propagate(ds, pp, every=SWEEP_EVERY, n_rec=SWEEP_REC, precision=prec)["pos"].cpu().numpy()
           for prec in (0, 2, 1)}
    curve = []
    for r in range(SWEEP_REC):
        path_m = SWEEP_EVERY * (r + 1) * H / 1000.0
        row = {"path_m": path_m}
        for prec, name in ((0, "scan_fp32"), (2, "refine_fp32")):
            d = np.linalg.norm(pos[prec][:, r] - pos[1][:, r], axis=1)
            d = d[np.isfinite(d)]
            row[name] = {"max_mm": float(d.max()) if d.size else None,
                         "median_mm": float(np.median(d)) if d.size else None,
                         "max_mm_per_m": float(d.max() / path_m) if d.size else None, "seeds": int(d.size)}
        curve.append(row)
    return {"events": n_ev, "occupancy": 0.30, "coarse_seeds": n, "seeds_per_step": seeds_step,
            "hits": int(wid.size), "ms_per_step": ms, "seeds_per_s": seeds_step / (ms / 1e3),
            "rkn_steps_per_s": steps / (ms / 1e3),
            "hough": {"events": n_ev, "ms": hough_ms, "votes": votes,
                      "votes_per_s": votes / (hough_ms / 1e3),
                      "accumulator_bytes": acc_bytes, "accumulator_gb_per_s": acc_bytes / (hough_ms / 1e3) / 1e9,
                      "bytes_note": "algorithmic: each event's int32 accumulator cleared once and read once by "
                                    "the peak search; the votes themselves are L2 atomics"},
            "position_vs_fp64_gpu": curve,
            "subsample": f"{seeds.shape[0]} seeds drawn from the events' grids, fixed-length propagation "
                         f"(no stop surfaces) to {SWEEP_EVERY * SWEEP_REC * H / 1000.0:.0f} m"}


def grid_value(gr, i):
    """Seed i (row-major) of one grid record, each value c + k s rounded once to FP32."""
    n = [int(x) for x in gr["n"]]
    k = []
    for a in range(4, -1, -1):
        k.append(i % n[a])
        i //= n[a]
    k = k[::-1]
    return np.array([np.float32(float(gr["centre"][a]) + (k[a] - (n[a] - 1) / 2.0) * float(gr["step"][a]))
                     for a in range(5)])



REFINE_K, REFINE_EVENTS, REFINE_ITER, REFINE_CKPT, REFINE_SIGMA = 64, 1024, 5, 128, 0.2
REFINE_SCAN_SEEDS = 20_000


def _gen_cfg4(i):
    import cdc_synth as S
    return S.cfg4_event(i, _GEN_FIELD, REFINE_SCAN_SEEDS)


def refine_leg(args, rank, local, g, fm, stream):
    """Throughput of cdc_refine_seeds on the differentiable-refine
    configuration: 1024 distinct events with 3-turn signals (10 % DIO-like
    occupancy), 64 seeds each (65536 seeds): the 64 best of one batched
    ten-round scan (k = 64) of a 2*10^4-seed grid around each event's first
    turn; five Gauss-Newton iterations, checkpointed adjoint gradient, FP64
    5x5 solves."""
    import torch
    import paper_1908_01949_gb300 as cdc
    n_ev = max(1, int(args.refine_events))
    evs, grids, S = make_batched_workload(n_ev, first=1000 * rank, gen=_gen_cfg4)
    off, wid, dr = S.pack_events(evs)
    n_scan = int(sum(int(np.prod(gr["n"])) for gr in grids))
    tr = cdc.Tracker(g, fm, device=local, max_events=n_ev, max_seeds=n_scan, max_hits=int(wid.size))
    dev = tr.dev
    sp = cdc.scan_params(h=H, max_steps=MAX_STEPS, lam=LAM, max_partitions=MAX_PART, k=REFINE_K,
                         n_rounds=N_ROUNDS, n_zoom=N_ZOOM, max_drift=MAX_DRIFT)
    off_t, wid_t, dr_t = tr.events_to_device(off, wid, dr)
    t0 = time.perf_counter()
    sc = tr.scan(off_t, wid_t, dr_t, cdc.grids_to_tensor(grids, dev), sp, want_hits=False, stream=stream)
    torch.cuda.synchronize()
    scan_s = time.perf_counter() - t0
    seeds = sc["best_seed"].reshape(-1, 5).contiguous()
    ok_seed = torch.isfinite(seeds).all(dim=1)
    seed_event = torch.arange(n_ev, dtype=torch.int32, device=dev).repeat_interleave(REFINE_K)
    rp = cdc.refine_params(n_iter=REFINE_ITER, sigma=REFINE_SIGMA, checkpoint=REFINE_CKPT)
    chi0 = tr.chi2_grad(seed_event, seeds, off_t, wid_t, dr_t, sp, rp, want_grad=False, stream=stream)["chi2"]
    for _ in range(max(1, min(args.warmup, 2))):
        out = tr.refine(seed_event, seeds, off_t, wid_t, dr_t, sp, rp, stream=stream)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.refine_reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = tr.refine(seed_event, seeds, off_t, wid_t, dr_t, sp, rp, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    c0 = chi0.cpu().numpy()
    c1 = out["chi2"].cpu().numpy()
    fl = out["flags"].cpu().numpy()
    ok = np.isfinite(c0) & np.isfinite(c1) & (c0 > 0)
    n = int(seeds.shape[0])
    return {"seeds": n, "events": n_ev, "distinct_events": n_ev, "seeds_per_event": REFINE_K,
            "turns": 3, "iterations": REFINE_ITER, "checkpoint": REFINE_CKPT, "ms": ms,
            "seeds_per_s": n / (ms / 1e3), "events_per_s": n_ev / (ms / 1e3),
            "finite_start_seeds": int(ok_seed.sum().item()),
            "median_chi2_ratio": float(np.median(c1[ok] / c0[ok])) if ok.any() else None,
            "flagged": int((fl != 0).sum()),
            "flagged_by_bit": {name.lower(): int(((fl & getattr(cdc, "FLAG_" + name)) != 0).sum())
                               for name in ("STEP_CAP", "FOUND_OVERFLOW", "NOT_SPD", "DOCA_ZERO", "LOST_HIT", "BAD_HIT")},
            "seed_selection": f"64 best of one batched ten-round scan (k = 64) of {REFINE_SCAN_SEEDS} seeds per "
                              f"event around its first turn ({scan_s:.2f} s, not timed)",
            "timing": f"median of {args.refine_reps} CUDA-event timed calls"}


# --------------------------------------------------------------- CUDA arm
def run_cuda(args, ws, rank, local):
    import torch
    import cdc_synth as S
    import paper_1908_01949_gb300 as cdc
    from paper_1908_01949_gb300 import build as B

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    g = S.make_geometry()
    fm = S.solenoid_map()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    sampler = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                           if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local)
    probe = cdc.Tracker(g, fm, device=local, max_events=1, max_seeds=1, max_hits=1)
    peak = fp32_peak(probe, sampler)
    stream = torch.cuda.current_stream()

    if args.profile_batched:
        pb = profile_batched(args, local, g, fm, flush)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": pb["seeds_per_s"], "unit": "seeds/s", "n_gpus": ws,
                              "steps": 1, "warmup": 0, "ms_per_step": pb["ms"], "higher_is_better": True,
                              "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                              "config": {"workload": WORKLOAD, "profile_case":
                                         f"one eager call on the first {pb['events']} events of the batched step "
                                         "for profiler captures, not a benchmark result"},
                              "profile_batched": pb, "fp32_peak": peak}))
        if dist:
            dist.destroy_process_group()
        return
    if args.profile_refine:
        args.refine_events = args.profile_refine
        rf = refine_leg(args, rank, local, g, fm, stream)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": rf["seeds_per_s"], "unit": "seeds/s", "n_gpus": ws,
                              "steps": args.refine_reps, "warmup": args.warmup, "ms_per_step": rf["ms"],
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                              "data": "synthetic",
                              "config": {"workload": "refine leg", "profile_case":
                                         f"the refine leg alone on {rf['events']} events for profiler captures, "
                                         "not a benchmark result"},
                              "refine": rf, "fp32_peak": peak}))
        if dist:
            dist.destroy_process_group()
        return
    if args.profile_case:
        mt = multi_turn_leg(args, ws, rank, local, g, fm, flush, peak)
        ev0, grid0 = mt.pop("_cpu")
        split = split_ab_leg(args, rank, local, g, fm, ev0, grid0, flush) if args.profile_split else None
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": mt["seeds_per_s"], "unit": "seeds/s", "n_gpus": ws,
                              "steps": args.mt_steps, "warmup": args.warmup, "ms_per_step": mt["ms_per_step"],
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                              "data": "synthetic",
                              "config": {"workload": WORKLOAD_MULTI_TURN, "profile_case":
                                         ("240000-seed" if args.profile_case == "reduced" else "10^6-seed")
                                         + " coarse grid for profiler captures, not a benchmark result"},
                              "coarse_scan": {"launch_ms": mt["roofline"]["launch_ms"],
                                              "rkn_steps": mt["roofline"]["rkn_steps"]},
                              "latency_ms_per_event": mt["latency_ms_per_event"], "multi_turn": mt,
                              "split_ab": split, "fp32_peak": peak}))
        if dist:
            dist.destroy_process_group()
        return

    head = headline_batched(args, ws, rank, local, dist, g, fm, flush, sampler, peak)
    work = head.pop("workload")
    legs = {}
    if not args.no_multi_turn:
        legs["multi_turn"] = guarded("multi_turn", lambda: multi_turn_leg(args, ws, rank, local, g, fm, flush, peak))
    if not args.no_single_turn:
        legs["single_turn"] = guarded("single_turn", lambda: single_turn_leg(args, ws, rank, local, g, flush))
    if not args.no_refine:
        legs["refine"] = guarded("refine", lambda: refine_leg(args, rank, local, g, fm, stream))
    if not args.no_sweep:
        legs["sweep"] = guarded("sweep", lambda: sweep_leg(args, rank, local, g, fm, flush))
    if not args.no_loop:
        legs["event_loop"] = guarded("loop", lambda: event_loop_leg(args, rank, local, g, fm))
    mt_cpu = legs.get("multi_turn", {}).pop("_cpu", None) if isinstance(legs.get("multi_turn"), dict) else None
    if not args.no_split and mt_cpu is not None:
        legs["split_ab"] = guarded("split_ab", lambda: split_ab_leg(args, rank, local, g, fm, mt_cpu[0], mt_cpu[1],
                                                                     flush))
    if not args.no_bidir:
        legs["bidirectional"] = guarded("bidir", lambda: bidirectional_leg(args, rank, local, g, fm, flush))
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = guarded("cpu_baseline", lambda: cpu_baseline(work, g, fm, target_s=args.cpu_seconds))
        if isinstance(legs.get("refine"), dict) and "seeds_per_s" in legs["refine"]:
            cpu["refine"] = guarded("cpu_refine", lambda: cpu_refine_baseline(g, fm, 16))
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    refine = legs.get("refine") or {}
    line = {
        "metric": METRIC, "value": job_value(ws, head["seeds_step"], head["ms"]), "unit": "seeds/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "events_per_step": head["n_events"], "seeds_per_step": head["seeds_step"],
                   "l2": "256 MiB flush before every replay, outside its timed events",
                   "parallelism": f"event-parallel x{ws} (each GPU its own 256 events, no collective)"},
        "rkn_steps_per_s": job_value(ws, head["rkn_step"], head["ms"]),
        "roofline": head["roofline"],
        "e2e": head["e2e"],
        "gpu_launches": head["launches_per_step"] * args.steps,
        "clocks": head["clocks"],
        "fp32_peak": peak,
        "batched": head["detail"],
        "refine_seeds_per_s": refine.get("seeds_per_s"),
        **legs,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def sample_workload_seeds(work, n, rng):
    """n seeds drawn uniformly from all coarse seeds of the batched workload:
    (event index, seed values) pairs."""
    counts = np.asarray(work["counts"], np.int64)
    base = np.concatenate([[0], np.cumsum(counts)])
    pick = np.sort(rng.choice(int(base[-1]), size=min(n, int(base[-1])), replace=False))
    ev_of = np.searchsorted(base, pick, side="right") - 1
    return [(int(e), grid_value(work["grids"][e], int(i - base[e]))) for e, i in zip(ev_of, pick)]


def oracle_on_sample(work, g, fm, sample, threads):
    """FP64 oracle scores of sampled seeds of the batched workload, events in
    parallel on `threads` host threads (one oracle call per event)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle as O
    P = O.scan_params(h=H, max_steps=MAX_STEPS, lam=LAM, max_partitions=MAX_PART)
    by_ev = {}
    for e, sd in sample:
        by_ev.setdefault(e, []).append(sd)

    def one(item):
        e, sds = item
        ev = work["evs"][e]
        r = O.scan(g, fm, ev.wire_id, ev.drift.astype(np.float64), np.asarray(sds, np.float64), P, threads=1)
        return int(r["n_steps"].sum())

    with ThreadPoolExecutor(threads) as ex:
        return sum(ex.map(one, sorted(by_ev.items())))


def cpu_baseline(work, g, fm, target_s=15.0):
    """FP64 oracle on a bounded random sample of the headline's coarse seeds,
    all host cores (events in parallel), and one core."""
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(0)
    n, t, done, steps = 2 * cores, 0.0, 0, 0
    while t < target_s:
        sample = sample_workload_seeds(work, n, rng)
        t0 = time.perf_counter()
        steps += oracle_on_sample(work, g, fm, sample, cores)
        t += time.perf_counter() - t0
        done += len(sample)
        n *= 2
    t1, done1, steps1, n1 = 0.0, 0, 0, 8
    while t1 < min(5.0, target_s / 3):
        sample = sample_workload_seeds(work, n1, rng)
        t0 = time.perf_counter()
        steps1 += oracle_on_sample(work, g, fm, sample, 1)
        t1 += time.perf_counter() - t0
        done1 += len(sample)
        n1 *= 2
    return {"value": done / t, "unit": "seeds/s", "cores": cores, "kind": "oracle", "rkn_steps_per_s": steps / t,
            "one_core": {"value": done1 / t1, "unit": "seeds/s", "rkn_steps_per_s": steps1 / t1,
                         "sample": f"{done1} seeds, {t1:.1f} s, one thread"},
            "sample": f"{done} seeds drawn at random from all coarse seeds of the step's "
                      f"{len(work['evs'])} events, same events and parameters, {t:.1f} s"}


def cpu_refine_baseline(g, fm, n_dist, target_s=3.0):
    """FP64 oracle refinement, one thread, on a bounded sample: seeds near
    the first-turn truth of the refine leg's first events (seeded noise),
    each classified at its start and refined with the leg's iterations."""
    import cdc_synth as S
    import oracle as O
    P = O.scan_params(h=H, max_steps=MAX_STEPS, lam=LAM, max_partitions=MAX_PART)
    evs = [S.cfg4_event(i, fm, REFINE_SCAN_SEEDS)[0] for i in range(max(1, n_dist))]
    rng = np.random.default_rng(4)
    sig = np.array([3e-4, 0.4, 0.15, 0.15, 0.1]) * 0.3
    t, done = 0.0, 0
    while t < target_s:
        ev = evs[done % len(evs)]
        sd = ev.truth_seeds[0] + rng.normal(0.0, 1.0, 5) * sig
        drift = ev.drift.astype(np.float64)
        t0 = time.perf_counter()
        part = O.scan(g, fm, ev.wire_id, drift, sd[None], P, per_hit=True, threads=1)["hit_part"][0]
        O.refine(g, fm, P, ev.wire_id, drift, part, sd, n_iter=REFINE_ITER, sigma=REFINE_SIGMA)
        t += time.perf_counter() - t0
        done += 1
    return {"value": done / t, "unit": "seeds/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} seeds near the first-turn truth of {len(evs)} of the refine leg's events, "
                      f"classification and {REFINE_ITER} Gauss-Newton iterations with the FP64 tangent gradient, "
                      f"{t:.1f} s, one thread"}


# --------------------------------------------------------- reference arm
def run_reference(args, ws, rank, local):
    """The FP64 oracle, as it stands, timed on the host cores on the headline's
    configuration: each step scores a bounded random sample of the batched
    workload's coarse seeds (events in parallel on all cores)."""
    if rank != 0:
        return
    import oracle as O
    import cdc_synth as S
    oracle_build = O.build()
    g, fm = S.make_geometry(), S.solenoid_map()
    evs, grids, _ = make_batched_workload(int(args.batched_events))
    work = {"evs": evs, "grids": grids, "counts": [int(np.prod(gr["n"])) for gr in grids]}
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(1)
    per_step = max(cores, int(args.ref_seeds))
    times, done, nsteps = [], 0, 0
    for i in range(args.warmup + args.steps):
        sample = sample_workload_seeds(work, per_step, rng)
        t0 = time.perf_counter()
        st = oracle_on_sample(work, g, fm, sample, cores)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            done += len(sample)
            nsteps += st
    tot = sum(times)
    v = done / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "seeds/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "seeds_per_step": per_step,
                       "sample": f"{per_step} seeds per step drawn at random from all coarse seeds of the "
                                 f"{len(evs)} events"},
            "rkn_steps_per_s": nsteps / tot,
            "cpu_baseline": {"value": v, "unit": "seeds/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} random coarse seeds of the batched workload per step "
                                       f"({os.path.relpath(oracle_build, ROOT)})"},
            "e2e": {"value": v, "unit": "seeds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10, help="timed graph replays of the batched step")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--e2e-steps", type=int, default=5, help="end-to-end steps (at most --steps)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="bound of the CPU-oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seeds", type=int, default=512, help="oracle seeds per step of the reference arm")
    ap.add_argument("--batched-events", type=int, default=256, help="events of the batched step")
    ap.add_argument("--no-multi-turn", action="store_true", help="skip the single-event multi-turn leg")
    ap.add_argument("--mt-steps", type=int, default=40, help="events per run of the multi-turn leg")
    ap.add_argument("--no-single-turn", action="store_true", help="skip the single-turn leg")
    ap.add_argument("--no-refine", action="store_true", help="skip the refine leg")
    ap.add_argument("--refine-events", type=int, default=REFINE_EVENTS, help="distinct events of the refine leg")
    ap.add_argument("--refine-reps", type=int, default=3, help="timed refine calls (median)")
    ap.add_argument("--batched-steps", type=int, default=3, help="timed graph replays of the sweep leg")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 30 %%-occupancy precision/scale leg")
    ap.add_argument("--sweep-events", type=int, default=64, help="events of the sweep leg")
    ap.add_argument("--no-bidir", action="store_true", help="skip the bidirectional-scan leg")
    ap.add_argument("--no-split", action="store_true", help="skip the two-kernel A/B leg")
    ap.add_argument("--no-loop", action="store_true", help="skip the event-loop leg")
    ap.add_argument("--loop-events", type=int, default=16, help="events of the event-loop leg")
    ap.add_argument("--split-chunk", type=int, default=SPLIT_CHUNK, help="seeds recorded at a time by the A/B leg")
    ap.add_argument("--bidir-events", type=int, default=32, help="events of the bidirectional leg")
    ap.add_argument("--scan-shape", default=None,
                    help="fixed scan-kernel shape 'block,chunk' instead of autotuning (profiler captures)")
    ap.add_argument("--warp-seeds", type=int, default=None,
                    help="multi-turn latency run: zoom rounds with at most this many seeds run one warp per seed "
                         "(0: never; default: the library's, 16 per SM)")
    ap.add_argument("--stream-warp-seeds", type=int, default=0,
                    help="the same for the multi-turn throughput and end-to-end runs (default 0: one lane per seed)")
    ap.add_argument("--inflight", type=int, default=8,
                    help="distinct events in flight (one context and stream each) in the multi-turn leg")
    ap.add_argument("--profile-batched", type=int, default=0, metavar="N",
                    help="one eager call of the batched step on its first N events (profiler captures; not a result)")
    ap.add_argument("--profile-refine", type=int, default=0, metavar="N",
                    help="only the refine leg on N events (profiler captures; not a result)")
    ap.add_argument("--profile-split", action="store_true",
                    help="with --profile-case, also the two-kernel A/B leg on the same event (profiler captures)")
    ap.add_argument("--profile-case", nargs="?", const="reduced", default=None, choices=["reduced", "full"],
                    help="only the multi-turn leg on a 240000-seed coarse grid, or ('full') its 10^6-seed grid "
                         "(profiler captures; not a result)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank, local)
    else:
        run_cuda(args, ws, rank, local)


if __name__ == "__main__":
    main()
