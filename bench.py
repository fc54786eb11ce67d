#!/usr/bin/env python
"""Benchmark: labelled Gvoxel/s on one GB300 (FP32 screening + exact rescoring,
next to the exact-only path), with the first-pass kernel's fraction of the HBM
label-write roofline and the arithmetic roofline beside it, an end-to-end
figure through host buffers, and the CPU oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...      # the CPU oracle alone

The default workload is Voronoi and Laguerre on periodic 1024^3 grids with
10^6 uniform sites each (one step = both grids); the clustered pair, the
Johnson-Mehl 1024^3 grid and the batch of 64 uneven grids are timed after it
as extra keys of the same line.  Prints one JSON line (rank 0).  Under
torchrun every rank labels its own copy of the workload (independent
problems: weak scaling, no collective on the data path; the only collectives
are the timing barrier and the max over ranks).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

METRIC = "labelled Gvoxel/s on 1 GB300, FP32+rescore vs exact path; % of HBM roofline"
L2_BYTES = 129 * 2 ** 20


def _workloads():
    return {
        # the metric's configuration: Voronoi and Laguerre on a periodic 1024^3
        # grid with 10^6 uniform sites each, one step = both grids
        "voronoi+laguerre-1024^3-uniform-1e6": lambda: [
            synthetic.precision_1024_1e6("voronoi", False),
            synthetic.precision_1024_1e6("laguerre", False)],
        # the same with Matern-clustered sites (uneven bins, voids)
        "voronoi+laguerre-1024^3-matern-1e6": lambda: [
            synthetic.precision_1024_1e6("voronoi", True),
            synthetic.precision_1024_1e6("laguerre", True)],
        "voronoi-1024^3-uniform-1e6": lambda: [synthetic.precision_1024_1e6("voronoi", False)],
        "laguerre-1024^3-uniform-1e6": lambda: [synthetic.precision_1024_1e6("laguerre", False)],
        "voronoi-1024^3-matern-1e6": lambda: [synthetic.precision_1024_1e6("voronoi", True)],
        "laguerre-1024^3-matern-1e6": lambda: [synthetic.precision_1024_1e6("laguerre", True)],
        "jm-1024^3-periodic-1e5": lambda: [synthetic.jm_1024_1e5()],
        # 64 uneven microstructures labelled by one persistent CUDA-graph launch
        "batch-64-uneven": lambda: synthetic.batch_64(),
        # the two open Laguerre grids of the 512^3 / 16384^2 configuration
        "laguerre-512^3+16384^2": lambda: [synthetic.laguerre_512_1e4(),
                                           synthetic.laguerre_16384sq_1e5()],
        "laguerre-512^3-open-1e4": lambda: [synthetic.laguerre_512_1e4()],
        # the 1024^3 / 10^6-site density (1074 voxels per site) on a grid small
        # enough for full ncu captures
        "voronoi-512^3-uniform-1.25e5": lambda: [synthetic.make_instance(
            "voronoi", (512, 512, 512), 125_000, seed=4, periodic=True,
            name="voronoi-3d-512^3-periodic-uniform-1.25e5")],
        "laguerre-512^3-uniform-1.25e5": lambda: [synthetic.make_instance(
            "laguerre", (512, 512, 512), 125_000, seed=4, periodic=True,
            name="laguerre-3d-512^3-periodic-uniform-1.25e5")],
        "jm-512^3-periodic-1.25e4": lambda: [synthetic.make_instance(
            "jm", (512, 512, 512), 12_500, seed=3, periodic=True,
            name="jm-3d-512^3-periodic-1.25e4")],
        # the Matern-clustered 1024^3 / 10^6-site density (10^4 parents of 100
        # sites in balls of radius 8) on a 512^3 grid
        "voronoi-512^3-matern-1.25e5": lambda: [_matern_512("voronoi")],
        "laguerre-512^3-matern-1.25e5": lambda: [_matern_512("laguerre")],
        "voronoi-64^3-periodic-100": lambda: [synthetic.voronoi_64_periodic_100()],
    }


def _matern_512(kind):
    sites = synthetic.matern_sites((512, 512, 512), 1_250, 100.0, 8.0, seed=5, periodic=True)
    return synthetic.make_instance(kind, (512, 512, 512), sites.shape[0], seed=5, periodic=True,
                                   sites=sites, name=f"{kind}-3d-512^3-periodic-matern-1.25e5")


DEFAULT_WORKLOAD = "voronoi+laguerre-1024^3-uniform-1e6"
# timed after the headline workload, in the same run, as extra keys of its line
EXTRAS = ("voronoi+laguerre-1024^3-matern-1e6", "jm-1024^3-periodic-1e5", "batch-64-uneven")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(dist, total_ms, device):
    """The slowest rank's timed region (every rank calls it; `dist` is
    torch.distributed, or None for one process)."""
    if dist is None:
        return total_ms
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(ws, nvox_per_rank, steps, total_ms):
    """Whole-job Gvoxel/s: every rank labels its own copy of the workload, so
    the voxels of all ranks over the slowest rank's time."""
    return ws * nvox_per_rank * steps / (total_ms * 1e-3) / 1e9


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "of measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "of fallback"


def _kernel_hash():
    h = hashlib.sha256()
    for name in sorted(os.listdir(os.path.join(ROOT, "paper_2201_13234_gb300", "csrc"))):
        with open(os.path.join(ROOT, "paper_2201_13234_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(workload):
    """DRAM bytes per first-pass launch from a committed ncu capture, if it was
    taken on the current kernel source (else null)."""
    path = os.path.join(ROOT, "profiles", "pass1_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    if rec.get("kernel_hash") != _kernel_hash():
        return None
    return rec.get("per_launch_bytes", {}).get(workload)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.p = None
        self.gpu = gpu_index
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "-i",
                                       str(gpu_index), "--format=csv,noheader,nounits",
                                       "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        rows = []
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        load = [r for r in rows if r[2] > 300.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i, v in enumerate(r[3]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(load),
                "power_w_max": max(r[2] for r in rows)}


def _cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine
    type); never raises."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine() or "unknown"


def _cpu_sample(insts, seconds: float, threads: int = 0):
    """Time the oracle's two-step algorithm (as it stands) on a z-slab of each
    grid with all of its sites; the slab is sized for about `seconds` in all.
    The cost-model threshold is computed once, outside the timing."""
    import oracle
    tot_vox, tot_t, desc = 0, 0.0, []
    per = seconds / len(insts)
    for inst in insts:
        thr = oracle.default_threshold(inst)
        if "void_radius_vox" in inst.meta:  # clustered sites: balls must reach the voids
            thr = oracle.ball_threshold(inst, inst.meta["void_radius_vox"])
        plane = inst.n_voxels // inst.dims[-1]
        t0 = time.perf_counter()
        oracle.twostep(inst, 0, 1, threads=threads, threshold=thr)
        t1 = max(time.perf_counter() - t0, 1e-4)
        nz = int(max(1, min(inst.dims[-1], per / t1)))
        reps, dt = 0, 0.0
        while reps == 0 or (dt < per and reps < 64):  # repeat small grids up to ~per seconds
            t0 = time.perf_counter()
            oracle.twostep(inst, 0, nz, threads=threads, threshold=thr)
            dt += time.perf_counter() - t0
            reps += 1
        tot_vox += plane * nz * reps
        tot_t += dt
        desc.append(f"{inst.name}: slab of {nz} of {inst.dims[-1]} layers x {reps}, "
                    f"all {inst.n_sites} sites")
    return tot_vox / tot_t / 1e9, tot_t, "; ".join(desc)


def run_reference(args, insts, ws, rank):
    if rank != 0:
        return
    cores = os.cpu_count()
    budget = 150.0 / max(1, args.steps + args.warmup)
    times, vox = [], 0
    desc = ""
    for i in range(args.warmup + args.steps):
        v, t, desc = _cpu_sample(insts, budget)
        if i >= args.warmup:
            times.append(t)
            vox += v * t * 1e9
    value = vox / sum(times) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gvoxel/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": args.workload,
                       "grids": [i.name for i in insts],
                       "reference": "the CPU oracle (paper's two-step algorithm, OpenMP)"},
            "cpu_baseline": {"value": value, "unit": "Gvoxel/s", "cores": cores,
                             "cpu_model": _cpu_model(),
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "Gvoxel/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)



class _Env:
    """Device, stream, optional process group and the L2 flush buffer."""

    def __init__(self, ws, local):
        import torch
        import paper_2201_13234_gb300 as vt

        torch.cuda.set_device(local)
        self.torch = torch
        self.vt = vt
        self.dev = torch.device("cuda", local)
        self.dist = None
        if ws > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=self.dev)
            self.dist = dist
        vt.load(build_if_missing=True)
        self.stream = torch.cuda.current_stream()
        self.flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=self.dev)
        self.gpu_index = local
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            try:
                self.gpu_index = int(vis.split(",")[local])
            except ValueError:
                pass
        self.sms = torch.cuda.get_device_properties(self.dev).multi_processor_count

    def T(self, a):
        return None if a is None else self.torch.from_numpy(np.ascontiguousarray(a)).to(self.dev)

    def pinned(self, a):
        return None if a is None else self.torch.from_numpy(np.ascontiguousarray(a)).pin_memory()

    def timed(self, fn, k, after=None, name="timed"):
        """k steps, each bracketed by CUDA events on the launching stream and
        preceded by an L2 flush (a 258 MB write); barrier + synchronize on
        both sides.  `after(i)` runs after step i's end event is recorded.
        The steps sit in an NVTX range `name` (profilers can select them)."""
        torch = self.torch
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(k)]
        if self.dist:
            self.dist.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(name)
        for i in range(k):
            self.flush.fill_(float(i))
            ev[i][0].record(self.stream)
            fn()
            ev[i][1].record(self.stream)
            if after is not None:
                after(i)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if self.dist:
            self.dist.barrier()
        return sum(a.elapsed_time(b) for a, b in ev)

    def busy(self, fn, seconds=1.5):
        """Keep the GPU busy before a timed region so the clock sampler sees it
        under load."""
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end:
            fn()
            self.torch.cuda.synchronize()


def measure_grids(E, insts, steps, warmup, exact_steps, autotune, e2e_steps, sampler=None,
                  brick_cfg=0, certify=0):
    """Single-grid path: every grid labelled through vt_voronoi / vt_laguerre /
    vt_johnson_mehl (binning, first pass and its culling re-run, second pass),
    autotuned; then the exact-only path and the end-to-end path."""
    vt, torch = E.vt, E.torch
    runs = []
    for inst in insts:
        runs.append(dict(inst=inst, sites=E.T(inst.sites), w=E.T(inst.w), t=E.T(inst.t),
                         v=E.T(inst.v),
                         labels=torch.empty(inst.dims[::-1], dtype=torch.int32, device=E.dev),
                         grid=vt.Grid(inst.dims, periodic=inst.periodic, timing=True,
                                      brick_cfg=brick_cfg, certify=certify),
                         exact=vt.Grid(inst.dims, periodic=inst.periodic, precision=vt.VT_EXACT,
                                       timing=True, brick_cfg=brick_cfg, certify=certify)))
    nvox = sum(r["inst"].n_voxels for r in runs)

    def step(key="grid"):
        for r in runs:
            r[key].label(r["inst"].kind, r["sites"], w=r["w"], t=r["t"], v=r["v"],
                         labels=r["labels"])

    if autotune:
        for r in runs:
            for key in ("grid", "exact"):
                r[key].autotune(r["inst"].kind, r["sites"], w=r["w"], t=r["t"], v=r["v"],
                                labels=r["labels"])
    for _ in range(max(3, warmup)):
        step()
    torch.cuda.synchronize()
    E.busy(step)

    def run_timed(key, k):
        p1, stats = [], []

        def after(i):  # the library's own stage events, read after the step's events
            for r in runs:
                st = r[key].sync()
                stats.append(st)
                p1.append(st["stage_ms"][1])
        total = E.timed(lambda: step(key), k, after, name="timed" if key == "grid" else "exact")
        return total, p1, stats

    total_ms, p1, stats = run_timed("grid", steps)
    clocks = sampler.stop() if sampler is not None else None
    total_ms = _max_over_ranks(E.dist, total_ms, E.dev)
    ex_ms, ex_p1, _ = run_timed("exact", exact_steps)
    out = {"runs": runs, "nvox": nvox, "total_ms": total_ms, "ms_step": total_ms / steps,
           "clocks": clocks,
           "p1_ms": sum(p1) / steps,
           "p1_ms_per_grid": [sum(p1[j::len(runs)]) / steps for j in range(len(runs))],
           # each grid's binning, first and second pass (the library's stage
           # events), averaged over the timed steps
           "stages_per_grid": [[sum(st["stage_ms"][i] for st in stats[j::len(runs)]) / steps
                                for i in range(3)] for j in range(len(runs))],
           "exact_ms_step": ex_ms / exact_steps, "exact_p1_ms": sum(ex_p1) / exact_steps}
    s0 = stats[-len(runs):]
    out["stats"] = {"rescored_fraction": sum(s["rescored"] for s in s0) / nvox,
                    "pass2_bricks": sum(s["pass2_bricks"] for s in s0),
                    "deferred_bricks": sum(s["deferred_bricks"] for s in s0),
                    "recull_bricks": sum(s["recull_bricks"] for s in s0),
                    "long_tiles": sum(s["long_tiles"] for s in s0),
                    "uniform_tiles": sum(s["uniform_tiles"] for s in s0),
                    "restaged_bricks": sum(s["restaged_bricks"] for s in s0),
                    "pruned_sites": sum(s["pruned_sites"] for s in s0),
                    "candidates_per_voxel": sum(s["candidates"] for s in s0) / nvox,
                    "stage_ms": [sum(s["stage_ms"][i] for s in s0) for i in range(3)]}
    if e2e_steps:
        host_in = [dict(sites=E.pinned(r["inst"].sites), w=E.pinned(r["inst"].w),
                        t=E.pinned(r["inst"].t), v=E.pinned(r["inst"].v)) for r in runs]
        host_out = [torch.empty(r["inst"].dims[::-1], dtype=torch.int32).pin_memory()
                    for r in runs]
        out["h2d"] = sum(sum(x.numel() * x.element_size() for x in h.values() if x is not None)
                         for h in host_in)
        out["d2h"] = sum(x.numel() * 4 for x in host_out)

        def e2e_step(direct):
            for r, h, o in zip(runs, host_in, host_out):
                if direct:  # vt_label_host: inputs copied in, labels stored into host memory
                    r["grid"].label_host(r["inst"].kind, h["sites"], w=h["w"], t=h["t"],
                                         v=h["v"], labels=o)
                    continue
                for key in ("sites", "w", "t", "v"):
                    if h[key] is not None:
                        r[key].copy_(h[key], non_blocking=True)
                r["grid"].label(r["inst"].kind, r["sites"], w=r["w"], t=r["t"], v=r["v"],
                                labels=r["labels"])
                o.copy_(r["labels"], non_blocking=True)

        def e2e_rate(direct):
            e2e_step(direct)  # warm (workspace)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(E.stream)
            for _ in range(e2e_steps):
                e2e_step(direct)
            e1.record(E.stream)
            torch.cuda.synchronize()
            return nvox * e2e_steps / (e0.elapsed_time(e1) * 1e-3) / 1e9

        out["e2e"] = e2e_rate(True)
        out["e2e_copy"] = e2e_rate(False)
        out["transfer"] = _transfer_rates(E, runs, host_out, e2e_steps)
        del host_in, host_out
    return out


def _transfer_rates(E, runs, host_out, k):
    """The CPU-GPU link alone at the label sizes: one cudaMemcpyAsync per grid
    (device labels to the pinned host buffers, and back), CUDA-event timed
    over k rounds.  The end-to-end rate cannot exceed labels / this time."""
    torch = E.torch
    nbytes = sum(o.numel() * 4 for o in host_out)
    out = {"bytes_per_round": nbytes, "rounds": k}
    for name, fn in (("d2h_gbs", lambda: [o.copy_(r["labels"], non_blocking=True)
                                           for r, o in zip(runs, host_out)]),
                     ("h2d_gbs", lambda: [r["labels"].copy_(o, non_blocking=True)
                                          for r, o in zip(runs, host_out)])):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(E.stream)
        for _ in range(k):
            fn()
        e1.record(E.stream)
        torch.cuda.synchronize()
        out[name] = nbytes * k / (e0.elapsed_time(e1) * 1e-3) / 1e9
    out["labels_gvoxel_s_at_d2h"] = out["d2h_gbs"] / 4.0
    return out


def measure_batch(E, insts, steps, warmup, autotune, e2e_steps, sampler=None):
    """Ensemble: every instance labelled by one replay of a CUDA graph (batched
    binning, one persistent first-pass kernel per class, the second pass), next
    to the same instances labelled one after another through the single-grid
    path (one launch sequence per instance)."""
    vt, torch = E.vt, E.torch
    items = [dict(kind=i.kind, dims=i.dims, periodic=i.periodic, sites=E.T(i.sites), w=E.T(i.w),
                  t=E.T(i.t), v=E.T(i.v),
                  labels=torch.empty(i.dims[::-1], dtype=torch.int32, device=E.dev))
             for i in insts]
    nvox = sum(i.n_voxels for i in insts)
    batch = vt.Batch(items)
    grids = [vt.Grid(i.dims, periodic=i.periodic) for i in insts]
    if autotune:
        batch.autotune()
        for g, it, inst in zip(grids, items, insts):
            g.autotune(inst.kind, it["sites"], w=it["w"], t=it["t"], v=it["v"],
                       labels=it["labels"])

    def step_graph():
        batch.run(use_graph=True)

    def step_single():
        for g, it, inst in zip(grids, items, insts):
            g.label(inst.kind, it["sites"], w=it["w"], t=it["t"], v=it["v"], labels=it["labels"])

    for _ in range(max(3, warmup)):
        step_graph()
        step_single()
    torch.cuda.synchronize()
    E.busy(step_graph)
    total_ms = E.timed(step_graph, steps)
    clocks = sampler.stop() if sampler is not None else None
    st = batch.sync()
    k1 = max(1, min(steps, 5))
    single_ms = E.timed(step_single, k1, name="per_instance") / k1
    total_ms = _max_over_ranks(E.dist, total_ms, E.dev)
    out = {"nvox": nvox, "total_ms": total_ms, "ms_step": total_ms / steps, "clocks": clocks,
           "single_ms": single_ms,
           "stats": {"rescored_fraction": st["rescored"] / nvox,
                     "pass2_bricks": st["pass2_bricks"], "uniform_tiles": st["uniform_tiles"],
                     "pruned_sites": st["pruned_sites"],
                     "candidates_per_voxel": st["candidates"] / nvox}}
    if e2e_steps:
        host_in = [dict(sites=E.pinned(i.sites), w=E.pinned(i.w), t=E.pinned(i.t),
                        v=E.pinned(i.v)) for i in insts]
        host_out = [torch.empty(i.dims[::-1], dtype=torch.int32).pin_memory() for i in insts]
        out["h2d"] = sum(sum(x.numel() * x.element_size() for x in h.values() if x is not None)
                         for h in host_in)
        out["d2h"] = sum(x.numel() * 4 for x in host_out)

        def e2e_rate(b, copy_back):
            b.run(use_graph=True)  # capture outside the timed region
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(E.stream)
            for _ in range(e2e_steps):
                for it, h in zip(items, host_in):
                    for key in ("sites", "w", "t", "v"):
                        if h[key] is not None:
                            it[key].copy_(h[key], non_blocking=True)
                b.run(use_graph=True)
                if copy_back:
                    for it, o in zip(items, host_out):
                        o.copy_(it["labels"], non_blocking=True)
            e1.record(E.stream)
            torch.cuda.synchronize()
            return nvox * e2e_steps / (e0.elapsed_time(e1) * 1e-3) / 1e9

        # labels stored by the kernels straight into the pinned host buffers
        # (the batch maps them), default plans; beside it, device labels
        # copied back after each replay
        host_batch = vt.Batch([dict(it, labels=o) for it, o in zip(items, host_out)])
        out["e2e"] = e2e_rate(host_batch, False)
        out["e2e_copy"] = e2e_rate(batch, True)
        del host_batch
    return out


def _alu_roofline(insts, value, clocks, sms, workload):
    """The arithmetic side of the roofline.  The paper's method evaluates
    ln N_s + 1 scores per voxel (Eq. dl); at 8 FP32 operations per 3D score
    (3 differences, 3 multiply-adds, a compare and a select; 6 in 2D) on
    128 FP32 lanes per SM that bounds the rate at SMs x 128 x clock / ops.
    The measured side comes from a committed ncu capture of the first pass
    (warp instructions per voxel, issue and pipe activity), used only while
    the kernel sources match the ones it was taken on."""
    import math
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    vox = sum(i.n_voxels for i in insts)
    ops = sum(i.n_voxels * (math.log(i.n_sites) + 1.0) * (8.0 if len(i.dims) == 3 else 6.0)
              for i in insts) / vox
    peak_ops = sms * 128 * mhz * 1e6
    roof = peak_ops / ops / 1e9
    out = {"bound": "alu", "algorithmic_ops_per_voxel": ops, "peak_ops_per_s": peak_ops,
           "roof_gvoxel_s": roof, "frac": value / roof, "clock_mhz": mhz, "sms": sms,
           "measured": None}
    rec = _counters(workload)
    if rec:
        ipv = rec["warp_instructions_per_voxel"]
        out["measured"] = dict(rec, issue_bound_gvoxel_s=sms * 4 * mhz * 1e6 / ipv / 1e9)
    return out


def _counters(workload):
    path = os.path.join(ROOT, "profiles", "pass1_counters.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    if rec.get("kernel_hash") != _kernel_hash():
        return None
    return rec.get("workloads", {}).get(workload)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="vt", choices=["vt", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(_workloads()))
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra workloads timed after the headline one")
    ap.add_argument("--exact-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--margin-scale", type=float, default=0.0,
                    help="with --profile: staging margin in mean cell radii (0: the default)")
    ap.add_argument("--certify", type=int, default=0, choices=[0, 1, 2, 3],
                    help="first-pass certification (1 after scoring, 2 before, 3 every brick "
                         "to the culling re-run; 0: the library's default, timed by the "
                         "autotuner)")
    ap.add_argument("--brick-cfg", type=int, default=0, choices=[0, 1],
                    help="initial warp-tile shape (0: 8x8x8, 1: compact 8x8x4); autotuning "
                         "may switch it")
    ap.add_argument("--profile", action="store_true",
                    help="only warm-up + timed FP32 steps with default plans (for ncu)")
    args = ap.parse_args()
    ws, rank, local = _dist()
    insts = _workloads()[args.workload]()
    if args.impl == "reference":
        run_reference(args, insts, ws, rank)
        return
    E = _Env(ws, local)
    is_batch = args.workload.startswith("batch")

    if args.profile:
        runs = [dict(inst=i, sites=E.T(i.sites), w=E.T(i.w), t=E.T(i.t), v=E.T(i.v),
                     grid=E.vt.Grid(i.dims, periodic=i.periodic, brick_cfg=args.brick_cfg,
                                    margin_scale=args.margin_scale, certify=args.certify),
                     labels=E.torch.empty(i.dims[::-1], dtype=E.torch.int32, device=E.dev))
                for i in insts]
        for _ in range(args.warmup + args.steps):
            for r in runs:
                r["grid"].label(r["inst"].kind, r["sites"], w=r["w"], t=r["t"], v=r["v"],
                                labels=r["labels"])
        E.torch.cuda.synchronize()
        st = [r["grid"].sync() for r in runs]
        keys = ("restaged_bricks", "deferred_bricks", "recull_bricks", "pass2_bricks", "long_tiles",
                "uniform_tiles", "rescored")
        print(json.dumps({"profile": args.workload, "steps": args.steps,
                          **{k: sum(x[k] for x in st) for k in keys},
                          "candidates_per_voxel": sum(x["candidates"] for x in st)
                          / sum(r["inst"].n_voxels for r in runs)}), flush=True)
        return

    e_steps = max(1, min(args.steps, 5))
    sampler = ClockSampler(E.gpu_index)
    if is_batch:
        m = measure_batch(E, insts, args.steps, args.warmup, not args.no_autotune, e_steps,
                          sampler)
    else:
        m = measure_grids(E, insts, args.steps, args.warmup, args.exact_steps,
                          not args.no_autotune, e_steps, sampler, brick_cfg=args.brick_cfg,
                          certify=args.certify)
    nvox = m["nvox"]
    value = _job_rate(ws, nvox, args.steps, m["total_ms"])
    peaks, which = _measured_peaks()
    peak = float(peaks["hbm_gbs"])
    label_bytes = 4.0 * nvox
    if is_batch:
        achieved = label_bytes / (m["ms_step"] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": None,
                    "kernel": "whole graph (binning, one k_pass1_group per class, k_pass2_batch)",
                    "peak_source": f"hbm_gbs {which}", "algorithmic_bytes_per_voxel": 4}
    else:
        achieved = label_bytes / (m["p1_ms"] * 1e-3) / 1e9 if m["p1_ms"] > 0 else None
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak if achieved else None,
                    "traffic": _traffic(args.workload),
                    "kernel": "first pass: k_stage + k_tiles (+ the culling re-run k_recull_warp)",
                    "timed_by": "CUDA events on the launching stream around the first pass",
                    "peak_source": f"hbm_gbs {which}", "algorithmic_bytes_per_voxel": 4,
                    "per_grid": [{"grid": r["inst"].name, "first_pass_ms": t,
                                  "frac": 4.0 * r["inst"].n_voxels / (t * 1e-3) / 1e9 / peak}
                                 for r, t in zip(m["runs"], m["p1_ms_per_grid"])],
                    "whole_step_frac": label_bytes / (m["ms_step"] * 1e-3) / 1e9 / peak}
    # drop the headline's buffers before the extras allocate theirs
    m.pop("runs", None)
    E.torch.cuda.empty_cache()

    extras = {}
    if ws == 1 and not args.no_extras and args.workload == DEFAULT_WORKLOAD:
        for name in EXTRAS:
            xi = _workloads()[name]()
            k = max(2, min(args.steps, 5))
            if name.startswith("batch"):
                x = measure_batch(E, xi, k, 3, not args.no_autotune, 0)
                extras[name] = {"value": x["nvox"] * k / (x["total_ms"] * 1e-3) / 1e9,
                                "unit": "Gvoxel/s", "ms_per_step": x["ms_step"],
                                "voxels": x["nvox"], "instances": len(xi),
                                "one_launch_per_instance_ms": x["single_ms"],
                                "speedup_graph_over_per_instance": x["single_ms"] / x["ms_step"],
                                "stats": x["stats"]}
            else:
                x = measure_grids(E, xi, k, 3, 2, not args.no_autotune, 0)
                xv = x["nvox"] * k / (x["total_ms"] * 1e-3) / 1e9
                extras[name] = {"value": xv, "unit": "Gvoxel/s", "ms_per_step": x["ms_step"],
                                "voxels": x["nvox"], "grids": [i.name for i in xi],
                                "first_pass_ms": x["p1_ms"],
                                "first_pass_frac": 4.0 * x["nvox"] / (x["p1_ms"] * 1e-3) / 1e9
                                / peak,
                                "exact": {"value": x["nvox"] / (x["exact_ms_step"] * 1e-3) / 1e9,
                                          "ms_per_step": x["exact_ms_step"]},
                                "speedup_fp32_over_exact": x["exact_ms_step"] / x["ms_step"],
                                "per_grid": [{"grid": i.name, "binning_ms": sg[0],
                                              "first_pass_ms": sg[1], "second_pass_ms": sg[2],
                                              "labelling_ms": sum(sg)}
                                             for i, sg in zip(xi, x["stages_per_grid"])],
                                "stats": x["stats"]}
                x.pop("runs", None)
            del x
            E.torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cv, ct, desc = _cpu_sample(insts, args.cpu_seconds)
        cpu = {"value": cv, "unit": "Gvoxel/s", "cores": os.cpu_count(),
               "cpu_model": _cpu_model(), "kind": "oracle",
               "sample": (desc if len(desc) < 600 else desc[:600] + " ...") + f" ({ct:.1f} s)"}
        try:  # the same oracle on one core, a smaller sample
            cv1, ct1, desc1 = _cpu_sample(insts, args.cpu_seconds / 4, threads=1)
            cpu["single_core"] = {"value": cv1, "unit": "Gvoxel/s",
                                  "sample": (desc1 if len(desc1) < 600 else desc1[:600] + " ...")
                                  + f" ({ct1:.1f} s)"}
        except Exception as e:  # reported, never fatal to the bench
            cpu["single_core"] = {"error": str(e)[:200]}

    if rank == 0:
        if is_batch:
            launches = (6 + (7 if any(i.kind == "jm" for i in insts) else 0)
                        + len({(len(i.dims), i.kind) for i in insts}) + 1) * args.steps
        else:
            # per grid: binning (6 kernels), the first pass and its culling
            # re-run, the second pass; Johnson-Mehl adds the site pruning and a
            # second binning
            launches = sum(9 + (7 if i.kind == "jm" else 0) for i in insts) * args.steps
        line = {
            "metric": METRIC, "value": value, "unit": "Gvoxel/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "grids": [i.name for i in insts][:8],
                       "instances": len(insts), "voxels_per_step_per_gpu": nvox,
                       "sites": sum(i.n_sites for i in insts),
                       "precision": "fp32 screen + exact rescore",
                       "l2": "L2 flushed (258 MB write) before every timed step; labels "
                             f"({label_bytes / 1e9:.2f} GB per step) exceed the 129 MB L2",
                       "parallelism": f"{ws} independent replica(s), one per GPU",
                       "autotune": not args.no_autotune},
            "roofline": roofline,
            "alu_roofline": _alu_roofline(insts, value / ws, m["clocks"], E.sms, args.workload),
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "clocks": m["clocks"],
            "stats": m["stats"],
        }
        if "e2e" in m:
            line["e2e"] = {"value": ws * m["e2e"], "unit": "Gvoxel/s",
                           "h2d_bytes_per_step": m["h2d"], "d2h_bytes_per_step": m["d2h"],
                           "copy_after": {"value": ws * m["e2e_copy"]}}
            if "transfer" in m:
                line["e2e"]["transfer"] = m["transfer"]
            line["e2e"]["how"] = (
                "inputs copied from pinned host memory; a batch whose labels are the pinned "
                "host buffers, stored into by the kernels (default plans)" if is_batch else
                "vt_label_host: pinned host sites copied in, labels stored by the kernels "
                "straight into pinned host memory")
        if is_batch:
            line["batch"] = {"graph_ms_per_step": m["ms_step"],
                             "one_launch_per_instance_ms": m["single_ms"],
                             "speedup_graph_over_per_instance": m["single_ms"] / m["ms_step"]}
        else:
            ex_value = nvox / (m["exact_ms_step"] * 1e-3) / 1e9
            line["exact"] = {"value": ex_value, "unit": "Gvoxel/s",
                             "ms_per_step": m["exact_ms_step"],
                             "first_pass_ms": m["exact_p1_ms"],
                             "speedup_fp32_over_exact": value / ws / ex_value}
        if extras:
            line["extra"] = extras
        print(json.dumps(line), flush=True)
    if E.dist:
        E.dist.destroy_process_group()


if __name__ == "__main__":
    main()
