#!/usr/bin/env python
"""Benchmark of the MOLC high-order sweep (Sec. 3) on one or more GB300 GPUs.

One step = one call of molc_sweep_closure in FP32: the backward-Euler sweep of every direction, characteristic and
group, the cell moments and the Eddington factors, on the 512 x 512-cell, 17-group, 4 x 32-direction, h/2-spacing
synthetic Fleck-Cummings-shaped workload with three tanh fronts.  The intensity state (5.8 GB) is
far larger than L2, so no cache flush is needed between steps.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle instead (double precision, all host
cores, one group of the same workload per step).  Under torchrun the instance's groups are split into contiguous
ranges, one per rank (strong scaling; no collective on the data path; an all-gather of the results for a consumer
that needs all groups is timed separately).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from paper_2305_11998_gb300 import dist as pdist  # noqa: E402

WORKLOAD = "fc512_g17_d128"
METRIC = "segment×group updates/s"
# ncu dram bytes (read + write) per update of the dominant FP32 kernel, from an ncu capture of a smaller case of the
# same generators, scaled by the updates of the launch.  The figure is keyed to the SHA-256 of the kernel source it
# was taken on: once the source changes, the bench line reports traffic as null until a new capture is recorded.
SWEEP_FP32_TRAFFIC = {"kernel_source_sha256": "38366d64f88ca73ce5a36189f8a751ab0ff17c4fed866b8a71e82d1fd0ae8bde",
                      "dram_bytes_per_update": 8.4938}   # 384^2 x 17 groups, 4 x 32 directions, h/2
KERNEL_SOURCE = os.path.join(ROOT, "paper_2305_11998_gb300", "csrc", "molc_kernels.cu")


def traffic_per_update():
    """The recorded ncu bytes per update, or None when the kernel source differs from the captured one."""
    import hashlib
    rec = SWEEP_FP32_TRAFFIC
    if rec["kernel_source_sha256"] is None or rec["dram_bytes_per_update"] is None:
        return None
    try:
        with open(KERNEL_SOURCE, "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    return rec["dram_bytes_per_update"] if h == rec["kernel_source_sha256"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 100 for the GPU legs, 20 for --impl reference, whose steps each "
                         "take about a second of host time)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel-only", action="store_true",
                    help="only the sweeps (warmup + steps) in --precision, for profiler captures")
    ap.add_argument("--tiled", action="store_true",
                    help="--workload batch64 and --kernel-only: plans with the tiled FP32 sweep")
    ap.add_argument("--no-batch", action="store_true", help="leave the batched pattern out of the default line")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="precision of the --kernel-only sweeps (fp64: also the device's FP64 FMA rate)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 20 if args.impl == "reference" else 100
    return args


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms around the timed region; mark() brackets the
    region so that the summary keeps the samples taken inside it (one interval of slack on each side)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_S = 0.2

    def __init__(self):
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", str(int(self.PERIOD_S * 1000)), "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self, begin: bool):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            lines = open(self.path).read().splitlines()
        except Exception:
            lines = []
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        return summarize_clocks(lines, self.t0, self.t1, self.PERIOD_S)


def summarize_clocks(lines, t0=None, t1=None, period=0.2):
    """Median SM clock, max clock and active throttle reasons of nvidia-smi CSV rows (the FIELDS of
    ClockSampler); rows stamped within [t0 - period, t1 + period] (the timed region) when any are, else all."""
    import datetime
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            ts = None
        rows.append((ts, parts[1:]))
    if not rows:
        return None
    inside = [r for ts, r in rows
              if ts is not None and t0 is not None and t1 is not None and t0 - period <= ts <= t1 + period]
    use = inside if inside else [r for _, r in rows]

    def num(x):
        try:
            return float(x)
        except ValueError:
            return None

    sm = [v for v in (num(r[1]) for r in use) if v is not None]
    mx = [v for v in (num(p[2]) for _, p in rows) if v is not None]
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    reasons = sorted({n for r in use for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows), "samples_in_timed_region": len(inside)}


def cpu_oracle_sample(wl, d, max_seconds=12.0):
    """The double oracle, as it stands, on whole groups of the workload until about max_seconds."""
    import oracle
    geom = oracle.Geometry.from_workload(wl)
    _, nseg = oracle.counts(geom)
    cores = os.cpu_count() or 1
    done_updates = 0
    groups = []
    t0 = time.perf_counter()
    g = wl.G // 2
    while True:
        oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], groups=[g], precision="double",
                     want_I=False, threads=cores)
        done_updates += nseg
        groups.append(g)
        g = (g + 1) % wl.G
        if time.perf_counter() - t0 > max_seconds or len(groups) >= wl.G:
            break
    dt = time.perf_counter() - t0
    return {"value": done_updates / dt, "unit": "updates/s", "cores": cores, "kind": "oracle",
            "sample": f"double-precision oracle, {len(groups)} of {wl.G} groups of one step of {wl.name} "
                      f"({done_updates:.3e} updates, {dt:.1f} s, characteristic grid rebuilt per call)"}


def workload_name(wl):
    """The workload string both arms print in `config`."""
    fronts = {1: "one front", 3: "three fronts"}.get(wl.n_fronts, f"{wl.n_fronts} fronts")
    return (f"{wl.name}: {wl.nx}x{wl.ny} cells, {wl.G} groups, {wl.n_polar}x{wl.n_azim} directions, spacing "
            f"h/{wl.spacing_div}, {fronts}; one instance, its groups split over the GPUs")


def run_reference(args):
    ws, rank, _ = pdist.env()
    if rank != 0:
        return
    wl = synth.WORKLOADS[args.workload]
    d = wl.inputs(0)
    import oracle
    geom = oracle.Geometry.from_workload(wl)
    _, nseg = oracle.counts(geom)
    cores = os.cpu_count() or 1
    g = wl.G // 2

    def step(i):
        oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], groups=[(g + i) % wl.G],
                     precision="double", want_I=False, threads=cores)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i)
    dt = time.perf_counter() - t0
    value = nseg * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(wl), "sample_per_step": "one group of one sweep (groups rotate)"},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle",
                             "sample": f"one of {wl.G} groups per step, {nseg:.3e} updates per step"},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = pdist.env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_2305_11998_gb300 as molc

    wl = synth.WORKLOADS[args.workload]
    # one instance; with N > 1 ranks its groups are split into contiguous ranges, one per rank (no data exchange on
    # the path: every group is swept independently)
    groups = pdist.shard_groups(wl.G, ws, rank)
    d = pdist.shard_inputs(wl.inputs(seed=0), groups)
    P = molc.Plan.from_workload(wl, groups=groups if ws > 1 else None)
    info = P.info
    G, ncell = len(groups), wl.ncell
    updates_total = info.n_segments * wl.G     # every group costs the same updates
    k_h = torch.tensor(d["kappa"]).pin_memory()
    B_h = torch.tensor(d["B"]).pin_memory()
    bnd_h = torch.tensor(d["bnd"]).pin_memory()
    k_d, B_d, bnd_d = k_h.to(dev), B_h.to(dev), bnd_h.to(dev)
    I = P.new_intensity("fp32", dev)
    P.intensity_init("fp32", I, B_d)
    mom = P.new_moments(dev)

    fac = {k: torch.empty((G, ncell), dtype=torch.float64, device=dev) for k in ("fxx", "fxy", "fyy")}
    # kernels of one FP32 step: state scale, cell table, sweep, moment gather (+ the combine of split cells)
    launches_per_step = 4 + (1 if info.n_split_cells else 0)

    def step():
        return P.sweep_closure("fp32", k_d, B_d, wl.c, wl.dt, I, bnd_d, out=mom, f=fac)[1]

    def barrier():
        if ws > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    barrier()
    sampler = ClockSampler() if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    P.kernel_timing(True)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.mark(True)
    e0.record()
    for _ in range(args.steps):
        f = step()
    e1.record()
    torch.cuda.synchronize()
    if sampler:
        sampler.mark(False)
    barrier()
    ms = pdist.max_over_ranks(e0.elapsed_time(e1), dev)
    # a consumer that needs every group on every GPU (the grey closure of Eqs. 8-9) would all-gather the six moments
    # and three factors once per step: timed here separately, after the sweeps
    allgather = None
    if ws > 1:
        arrays = [mom[k] for k in ("E", "Fx", "Fy", "Nxx", "Nxy", "Nyy")] + [fac[k] for k in ("fxx", "fxy", "fyy")]
        for a in arrays:
            pdist.gather_groups(a, wl.G, groups, ws)
        torch.cuda.synchronize()
        barrier()
        e0.record()
        for _ in range(args.steps):
            for a in arrays:
                pdist.gather_groups(a, wl.G, groups, ws)
        e1.record()
        torch.cuda.synchronize()
        ag_ms = pdist.max_over_ranks(e0.elapsed_time(e1), dev) / args.steps
        allgather = {"ms_per_step": ag_ms, "bytes_per_rank": 9 * wl.G * ncell * 8,
                     "what": "NCCL all-gather of E, F, N and the Eddington factors of all groups, after the timed steps"}
    parts, kern_n = P.kernel_time_parts()
    kern_ms = parts["sweep"]
    P.kernel_timing(False)
    clocks = sampler.stop() if sampler else None
    status = P.device_status()
    ms_step = ms / args.steps
    value = updates_total * args.steps / (ms / 1e3)    # the whole instance's updates over the slowest rank's time

    # roofline of the dominant kernel (the FP32 sweep): algorithmic bytes per launch / average launch time
    gc = info.fp32_groups_per_warp
    n_chunks = -(-G // gc)
    alg_bytes = (8.0 * info.n_updates                       # deviation state: 4 B read + 4 B written per update
                 + 16.0 * info.n_track_segments * n_chunks  # segment records, once per group chunk
                 + 20.0 * ncell * G)                        # cell table {kappa~, r, B_hi, B_lo, dB}, read once
    # the cell-moment gather: the swept state read once more, the cell entry lists, B in, 6 moments + B_ref out,
    # and the 3 Eddington factors molc_sweep_closure forms there
    mom_bytes = (4.0 * info.n_updates + 16.0 * 2 * info.n_track_segments * n_chunks
                 + (8.0 + 56.0 + 24.0) * ncell * G)
    nk = max(kern_n, 1)
    kern_avg = kern_ms / nk
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (kern_avg / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (None if traffic_per_update() is None else traffic_per_update() * info.n_updates),
                "kernel": "sweep_fp32_kernel", "kernel_ms": kern_avg,
                "alg_bytes_per_launch": alg_bytes, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    kernels = {"prep_ms": parts["prep"] / nk, "sweep_ms": kern_avg, "moments_ms": parts["moments"] / nk,
               "moments_gbs": mom_bytes / (parts["moments"] / nk / 1e3) / 1e9 if parts["moments"] > 0 else None,
               "moments_alg_bytes": mom_bytes}
    # the whole step (every kernel of molc_sweep_closure) against the algorithmic bytes of the path: the FP32
    # state read and written (8 B per update), the segment records walked by both senses (8 B per track segment
    # per sense), kappa and B read once (16 B per cell-group), six FP64 moments and three Eddington factors
    # written once (72 B per cell-group)
    step_bytes = 8.0 * info.n_updates + 16.0 * info.n_track_segments + (16.0 + 72.0) * ncell * G
    step_gbs = step_bytes / (ms_step / 1e3) / 1e9
    roofline_step = {"bound": "hbm", "achieved": step_gbs, "peak": peak, "unit": "GB/s", "frac": step_gbs / peak,
                     "alg_bytes_per_step": step_bytes, "ms_per_step": ms_step,
                     "what": "all kernels of one molc_sweep_closure call (device events around the K steps)"}

    # end to end through the public API: every step copies its kappa, B and boundary in from pinned host
    # memory and its moments and Eddington factors out to pinned host memory.  The copies are pipelined
    # against the sweeps the way a caller would run them: inputs of step n+1 go in (one copy stream) while
    # step n sweeps, the results of step n come out (a second copy stream) while step n+1 sweeps; two device
    # and two host buffer sets alternate.  All copies of all K steps lie inside the timed region.
    e2e = None
    if not args.no_e2e:
        names = ("E", "Fx", "Fy", "Nxx", "Nxy", "Nyy", "fxx", "fxy", "fyy")
        ins_h = [(k_h, B_h, bnd_h), tuple(x.clone().pin_memory() for x in (k_h, B_h, bnd_h))]
        ins_d = [(k_d, B_d, bnd_d), tuple(torch.empty_like(x) for x in (k_d, B_d, bnd_d))]
        moms = [mom, P.new_moments(dev)]
        fes = [{k: torch.empty((G, ncell), dtype=torch.float64, device=dev) for k in ("fxx", "fxy", "fyy")}
               for _ in range(2)]
        outs_h = [{k: torch.empty((G, ncell), dtype=torch.float64).pin_memory() for k in names}
                  for _ in range(2)]
        h2d = sum(x.numel() for x in ins_h[0]) * 8
        d2h = sum(v.numel() for v in outs_h[0].values()) * 8
        cs = torch.cuda.current_stream()
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]     # slot's inputs are on the device
        ev_done = [torch.cuda.Event() for _ in range(2)]   # slot's step has run (inputs free, results ready)
        ev_out = [torch.cuda.Event() for _ in range(2)]    # slot's results are on the host (buffers free)

        def put_inputs(n):
            j = n % 2
            with torch.cuda.stream(s_in):
                if n >= 2:
                    s_in.wait_event(ev_done[j])
                for dst, src in zip(ins_d[j], ins_h[j]):
                    dst.copy_(src, non_blocking=True)
                ev_in[j].record(s_in)

        def run_e2e(K):
            s_in.wait_stream(cs)
            s_out.wait_stream(cs)
            put_inputs(0)
            for n in range(K):
                j = n % 2
                if n + 1 < K:
                    put_inputs(n + 1)
                cs.wait_event(ev_in[j])
                if n >= 2:
                    cs.wait_event(ev_out[j])
                k_, B_, bnd_ = ins_d[j]
                P.sweep_closure("fp32", k_, B_, wl.c, wl.dt, I, bnd_, out=moms[j], f=fes[j], stream=cs)
                ev_done[j].record(cs)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_done[j])
                    res = dict(moms[j], **fes[j])
                    for k in names:
                        outs_h[j][k].copy_(res[k], non_blocking=True)
                    ev_out[j].record(s_out)
            cs.wait_stream(s_in)
            cs.wait_stream(s_out)

        run_e2e(2)
        torch.cuda.synchronize()
        barrier()
        e0.record()
        run_e2e(args.steps)
        e1.record()
        torch.cuda.synchronize()
        barrier()
        ems = pdist.max_over_ranks(e0.elapsed_time(e1), dev)
        e2e = {"value": updates_total * args.steps / (ems / 1e3), "unit": "updates/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": ems / args.steps,
               "copies": "pinned host buffers, two copy streams pipelined against the sweeps (double-buffered)"}

    # the plain FP64 GPU sweep on the same workload (the speed-up denominator)
    fp64 = None
    if not args.no_fp64:
        I = None
        torch.cuda.empty_cache()
        I64 = P.new_intensity("fp64", dev)
        P.intensity_init("fp64", I64, B_d)
        P.sweep("fp64", k_d, B_d, wl.c, wl.dt, I64, bnd_d, out=mom)
        torch.cuda.synchronize()
        n64 = 2
        barrier()
        e0.record()
        for _ in range(n64):
            P.sweep_closure("fp64", k_d, B_d, wl.c, wl.dt, I64, bnd_d, out=mom, f=fac)
        e1.record()
        torch.cuda.synchronize()
        ms64 = pdist.max_over_ranks(e0.elapsed_time(e1), dev) / n64    # like `value`: the slowest rank's time
        fp64 = {"value": updates_total / (ms64 / 1e3), "unit": "updates/s", "ms_per_step": ms64,
                "speedup_fp32_over_fp64": ms64 / ms_step}
        del I64

    # the batched production pattern (64 uneven instances, one molc_batch_sweep per step, 5 steps in a CUDA graph)
    batch = None
    if ws == 1 and not args.no_batch:
        I = None     # the 512^2 state is no longer needed
        torch.cuda.empty_cache()
        _, bplans, _, bt, t_plan = batch_setup()
        bms = batch_graph_ms(bt, 5, 2)
        bupd = sum(Q.info.n_updates for Q in bplans)
        bbytes = batch_alg_bytes(bplans)
        batch = {"value": bupd * 5 / (bms / 1e3), "unit": "updates/s", "ms_per_step": bms / 5,
                 "updates_per_step": bupd, "steps": 5, "plans": t_plan,
                 "roofline": {"bound": "hbm", "achieved": bbytes * 5 / (bms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                              "frac": bbytes * 5 / (bms / 1e3) / 1e9 / peak},
                 "what": "64 seeded uneven instances (synth.batch_instances), molc_batch_sweep with factors, 5 steps "
                         "in one CUDA graph after 2 eager ones"}
        bt.close()
        for Q in bplans:
            Q.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(wl, d)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_name(wl),
                           "updates_per_step": updates_total,
                           "parallelism": f"groups over {ws} GPU(s): rank 0 sweeps groups {groups.start}-"
                                          f"{groups.stop - 1}",
                           "l2": "no flush: the 5.8 GB intensity state streamed each step is ~45x L2",
                           "step": "molc_sweep_closure (FP32 sweep, moments and Eddington factors in one call)"},
                "roofline": roofline, "roofline_step": roofline_step, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_step * args.steps, "clocks": clocks, "fp64_plain": fp64, "device_status": status,
                "allgather": allgather, "batch": batch}
        print(json.dumps(line), flush=True)
    P.close()
    if ws > 1:
        dist.destroy_process_group()


def run_kernel_only(args):
    """Sweeps only, in --precision (no closure, e2e or CPU legs): the command profiler captures use.  With
    fp64 it also reports the device's FP64 FMA rate (molc_fp64_fma_rate), the bound of the plain FP64 sweep."""
    import torch
    import paper_2305_11998_gb300 as molc
    wl = synth.WORKLOADS[args.workload]
    d = wl.inputs(seed=0)
    P = molc.Plan.from_workload(wl, tiled=args.tiled)
    dev = torch.device("cuda")
    prec = args.precision
    k, B, bnd = (torch.tensor(d[x], device=dev) for x in ("kappa", "B", "bnd"))
    I = P.new_intensity(prec, dev)
    P.intensity_init(prec, I, B)
    out = P.new_moments(dev)
    for _ in range(args.warmup):
        P.sweep(prec, k, B, wl.c, wl.dt, I, bnd, out=out)
    P.kernel_timing(True)
    for _ in range(args.steps):
        P.sweep(prec, k, B, wl.c, wl.dt, I, bnd, out=out)
    parts, n = P.kernel_time_parts()
    line = {"workload": wl.name, "precision": prec, "tiled": P.info.fp32_tile_items > 0, "launches": n,
            "kernel_ms": {k_: v / max(n, 1) for k_, v in parts.items()}, "updates": P.info.n_updates,
            "device_status": P.device_status()}
    if prec == "fp64":
        line["fp64_fma_flops"] = molc.fp64_fma_rate()
    print(json.dumps(line), flush=True)
    P.close()


def batch_setup(tiled=False, autotune=True):
    """The 64 seeded uneven instances of the batched pattern, their plans, bound arguments and the batch.  The
    plans are made twice with a fresh tuning cache: the first time every distinct signature is tuned (and
    recorded), the second time every configuration comes from the cache; both times are returned."""
    import shutil
    import tempfile
    import torch
    import paper_2305_11998_gb300 as molc
    dev = torch.device("cuda")
    wls = synth.batch_instances(64)
    tmp = tempfile.mkdtemp()
    molc.tune_cache(os.path.join(tmp, "tune.json"))
    try:
        t0 = time.perf_counter()
        plans = [molc.Plan.from_workload(wl, autotune=autotune, tiled=tiled) for wl in wls]
        t_cold = time.perf_counter() - t0
        t0 = time.perf_counter()
        again = [molc.Plan.from_workload(wl, autotune=autotune, tiled=tiled) for wl in wls]
        t_warm = time.perf_counter() - t0
    finally:
        molc.tune_cache(None)
        shutil.rmtree(tmp, ignore_errors=True)
    t_plan = {"plan_seconds_with_autotune": t_cold, "plan_seconds_from_tune_cache": t_warm,
              "tuned": sum(1 for P in plans if not P.info.tuned_from_cache),
              "from_cache_second_time": sum(1 for P in again if P.info.tuned_from_cache)}
    for P in again:
        P.close()
    args_list = []
    for wl, P in zip(wls, plans):
        d = wl.inputs(seed=wl.extra["seed"])
        k, B, bnd = (torch.tensor(d[x], device=dev) for x in ("kappa", "B", "bnd"))
        I = P.new_intensity("fp32", dev)
        P.intensity_init("fp32", I, B)
        f = {x: torch.empty((wl.G, wl.ncell), dtype=torch.float64, device=dev) for x in ("fxx", "fxy", "fyy")}
        args_list.append(dict(kappa=k, B=B, c=d["c"], dt=d["dt"], I=I, bnd=bnd, out=P.new_moments(dev), f=f))
    batch = molc.Batch(plans)
    batch.bind(args_list)
    return wls, plans, args_list, batch, t_plan


def batch_graph_ms(batch, steps, warmup, sampler=None):
    """CUDA-event time of `steps` batched steps captured in one CUDA graph and replayed once (after `warmup`
    eager steps)."""
    import torch
    for _ in range(max(warmup, 0)):
        batch.sweep()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(steps):
            batch.sweep()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.mark(True)
    e0.record()
    g.replay()
    e1.record()
    torch.cuda.synchronize()
    if sampler:
        sampler.mark(False)
    del g
    return e0.elapsed_time(e1)


def batch_alg_bytes(plans):
    """Algorithmic bytes of one batched step: every instance's FP32 state read and written (8 B per update), its
    segment records walked by both senses, kappa and B read once, six moments and three factors written."""
    return sum(8.0 * P.info.n_updates + 16.0 * P.info.n_track_segments + (16.0 + 72.0) * P.ncell * P.G
               for P in plans)


def run_batch(args):
    """The batched production pattern: 64 seeded uneven instances (cells per side 32-256, 8/17/32 groups, 2-4
    polar x 16-64 azimuthal directions, spacing h/2 or h/4), autotuned plans, all instances stepped by one
    molc_batch_sweep per step (sweep + Eddington factors), the K timed steps captured in one CUDA graph and
    replayed once.  Compared with looping the per-instance FP32 sweep and the plain FP64 sweep over the
    instances.  --tiled: the tiled sweep's one persistent launch over the items of every instance."""
    import torch
    dev = torch.device("cuda")
    wls, plans, args_list, batch, t_plan = batch_setup(tiled=args.tiled)
    n_upd = sum(P.info.n_updates for P in plans)
    sampler = ClockSampler()
    sampler.start()
    time.sleep(0.3)
    ms = batch_graph_ms(batch, args.steps, args.warmup, sampler)
    clocks = sampler.stop()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    status = max(P.device_status() for P in plans)
    # the same steps as per-instance calls (FP32 sweep + closure per plan, no batching, no graph)
    e0.record()
    for _ in range(2):
        for P, a in zip(plans, args_list):
            P.sweep("fp32", a["kappa"], a["B"], a["c"], a["dt"], a["I"], a["bnd"], out=a["out"])
            P.closure(a["out"], a["c"])
    e1.record()
    torch.cuda.synchronize()
    ms_loop32 = e0.elapsed_time(e1) / 2
    # the plain FP64 sweep looped over the instances (FP32 states released first)
    for a in args_list:
        a["I"] = None
    batch.close()
    torch.cuda.empty_cache()
    I64 = [P.new_intensity("fp64", dev) for P in plans]
    for P, a, I in zip(plans, args_list, I64):
        P.intensity_init("fp64", I, a["B"])
        P.sweep("fp64", a["kappa"], a["B"], a["c"], a["dt"], I, a["bnd"], out=a["out"])
    torch.cuda.synchronize()
    e0.record()
    for P, a, I in zip(plans, args_list, I64):
        P.sweep("fp64", a["kappa"], a["B"], a["c"], a["dt"], I, a["bnd"], out=a["out"])
        P.closure(a["out"], a["c"])
    e1.record()
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    depths = {}
    for P in plans:
        depths[P.info.fp32_sweep_depth] = depths.get(P.info.fp32_sweep_depth, 0) + 1
    line = {"metric": METRIC, "value": n_upd * args.steps / (ms / 1e3), "unit": "updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch64: 64 seeded uneven instances, cells per side 32-256, 8/17/32 groups, "
                                   "2-4 x 16-64 directions, spacing h/2 or h/4" + (", tiled sweep" if args.tiled else ""),
                       "updates_per_step": n_upd, "step": "molc_batch_sweep (FP32 sweep + Eddington factors), "
                                                          "K steps in one CUDA graph",
                       "state_gb": sum(P.intensity_bytes("fp32") for P in plans) / 1e9,
                       "plans": t_plan, "autotuned_depths": depths},
            "roofline": {"bound": "hbm", "achieved": batch_alg_bytes(plans) * args.steps / (ms / 1e3) / 1e9,
                         "peak": measured_peaks()[0], "unit": "GB/s",
                         "frac": batch_alg_bytes(plans) * args.steps / (ms / 1e3) / 1e9 / measured_peaks()[0]},
            "per_instance_fp32": {"value": n_upd / (ms_loop32 / 1e3), "ms_per_step": ms_loop32},
            "fp64_plain_loop": {"value": n_upd / (ms64 / 1e3), "ms_per_step": ms64,
                                "speedup_batch_over_fp64_loop": ms64 / (ms / args.steps)},
            "clocks": clocks, "device_status": status}
    print(json.dumps(line), flush=True)
    for P in plans:
        P.close()


def run_refine(args):
    """Refinement stress: 128x128 cells, 17 groups, 8 polar x 64 azimuthal directions, cold start with the left
    edge driven at 1 keV; the material grid is fixed while the ray spacing goes h/2, h/4, h/8, h/16.  T is
    advanced between steps by the host FP64 energy balance driven by the FP64 sweep at h/2; at every spacing the
    FP32 and FP64 sweeps step through that same T sequence.  Reports, per spacing, the FP32 and FP64 sweep
    throughput and the largest FP32 error against FP64 over the steps."""
    import torch
    import paper_2305_11998_gb300 as molc
    from paper_2305_11998_gb300 import multistep
    wl = synth.WORKLOADS["fc128_g17_d512"]
    steps = min(args.steps, wl.steps)
    t0 = time.perf_counter()
    Pref = molc.Plan.from_workload(wl)
    Ts = multistep.temperature_sequence(Pref, wl, wl.temperature(), steps)
    t_seq = time.perf_counter() - t0
    Pref.close()
    rows = []
    E_last = {"fp64": [], "fp32": []}   # grey E (sum over groups) after the last step, per spacing
    for div in (2, 4, 8, 16):
        P = molc.Plan.from_workload(wl, spacing=wl.h / div, autotune=True)
        n_upd = P.info.n_updates
        t32, t64 = [], []
        m64 = multistep.run_sequence(P, wl, Ts, "fp64", on_step=lambda n, m, ms: t64.append(ms))
        torch.cuda.empty_cache()
        m32 = multistep.run_sequence(P, wl, Ts, "fp32", on_step=lambda n, m, ms: t32.append(ms))
        E_last["fp64"].append(m64[-1]["E"].sum(axis=0))
        E_last["fp32"].append(m32[-1]["E"].sum(axis=0))
        worst = {}
        for a, b in zip(m32, m64):
            for k, v in multistep.precision_errors(a, b, wl.c).items():
                worst[k] = max(worst.get(k, 0.0), v)
        ms32 = float(np.median(t32[1:] if len(t32) > 1 else t32))
        ms64 = float(np.median(t64[1:] if len(t64) > 1 else t64))
        rows.append({"spacing": f"h/{div}", "updates_per_step": n_upd, "fp32_ms": ms32, "fp32_updates_per_s": n_upd / (ms32 / 1e3),
                     "fp64_ms": ms64, "fp64_updates_per_s": n_upd / (ms64 / 1e3), "speedup": ms64 / ms32,
                     "fp32_vs_fp64_max_error": worst, "fp32_sweep_depth": P.info.fp32_sweep_depth,
                     "device_status": P.device_status()})
        P.close()
        torch.cuda.empty_cache()
    # the paper's refinement norms of the grey E after the last step: ||dE_h|| = ||E_h - E_2h||_L2, rho_h
    vol = (wl.L / wl.nx) * (wl.L / wl.ny)
    for prec in ("fp64", "fp32"):
        for r, nr in zip(rows, multistep.refinement_norms(E_last[prec], vol)):
            r[f"refinement_E_{prec}"] = nr
    T = Ts[-1]
    print(json.dumps({"workload": f"{wl.name}: {wl.nx}x{wl.ny} cells, {wl.G} groups, {wl.n_polar}x{wl.n_azim} "
                                  f"directions, cold start, left edge at 1 keV, {steps} steps",
                      "temperature_sequence_seconds": t_seq, "T_range_keV": [float(T.min()), float(T.max())],
                      "per_spacing": rows}), flush=True)


def run_paper_layout(args):
    """The paper's characteristic grid at its production spacing: 40 x 40 cells on 6 cm (h_mat = 0.15 cm),
    h_moc = 1e-3 cm vertex bands, 17 groups, 4 x 36 = 144 directions; FP32 step (sweep + closure) timed over
    the steps, FP64 sweep beside it, FP32 moments compared with FP64 after one step."""
    import torch
    import paper_2305_11998_gb300 as molc
    from paper_2305_11998_gb300 import multistep
    dev = torch.device("cuda")
    wl = synth.Workload("fc40_paper", 40, 40, 6.0, 17, 0.001, 100.0, 4, 36, 150, 1, n_fronts=1)
    d = wl.inputs(0)
    q = wl.quadrature()
    P = molc.Plan(wl.nx, wl.ny, wl.L, wl.L, q.mu, q.cos_phi, q.sin_phi, q.w, wl.G, 1e-3, "paper", False,
                  autotune=True)
    k, B, bnd = (torch.tensor(d[x], device=dev) for x in ("kappa", "B", "bnd"))
    I = P.new_intensity("fp32", dev)
    P.intensity_init("fp32", I, B)
    mom = P.new_moments(dev)
    first = {kk: v.cpu().numpy() for kk, v in P.sweep("fp32", k, B, wl.c, wl.dt, I, bnd, out=mom).items()}
    for _ in range(max(args.warmup, 0)):
        P.sweep("fp32", k, B, wl.c, wl.dt, I, bnd, out=mom)
        P.closure(mom, wl.c)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    P.kernel_timing(True)
    e0.record()
    for _ in range(args.steps):
        P.sweep("fp32", k, B, wl.c, wl.dt, I, bnd, out=mom)
        P.closure(mom, wl.c)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    parts, n = P.kernel_time_parts()
    del I
    torch.cuda.empty_cache()
    I64 = P.new_intensity("fp64", dev)
    P.intensity_init("fp64", I64, B)
    e0.record()
    ref = {kk: v.cpu().numpy() for kk, v in P.sweep("fp64", k, B, wl.c, wl.dt, I64, bnd, out=mom).items()}
    e1.record()
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    info = P.info
    print(json.dumps({"workload": "fc40_paper: 40x40 cells on 6 cm, paper layout h_moc = 1e-3 cm, 17 groups, "
                                  "4x36 directions", "n_tracks": info.n_tracks, "updates_per_step": info.n_updates,
                      "fp32_ms_per_step": ms, "fp32_updates_per_s": info.n_updates / (ms / 1e3),
                      "kernels_ms": {kk: v / max(n, 1) for kk, v in parts.items()},
                      "fp64_sweep_ms": ms64, "fp64_updates_per_s": info.n_updates / (ms64 / 1e3),
                      "fp32_vs_fp64_first_step": multistep.precision_errors(first, ref, wl.c),
                      "fp32_sweep_depth": info.fp32_sweep_depth, "device_status": P.device_status()}), flush=True)
    P.close()


def main():
    args = parse()
    if args.kernel_only:
        run_kernel_only(args)
    elif args.workload == "paper40":
        run_paper_layout(args)
    elif args.workload == "refine":
        run_refine(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
