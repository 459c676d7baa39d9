"""Throughput benchmark of the multiscale lattice Boltzmann step on GB300.

Workload (default): the force-driven Poiseuille channel, 1024 x 512 nodes, body force
1e-6 (lattice units), 32 high-order (D2Q36) rows per wall and D2Q9 in the core, Kn swept
over {0.02, 0.1, 0.5}: the three channels are advanced together, so one benchmark step
is one time step of all three lattices (1.57 M node updates, ~156 MB of populations
read and written, larger than the 126 MB L2). Populations are stored as FP32
deviations from w_i rho0 and collide in FP32. Inputs are synthetic (lbinputs).

Metric: MLUPS (million node updates per second, every node counted once per step) over
all GPUs; the JSON line also carries the HBM roofline of the step kernel, an
end-to-end figure through the C ABI with host-resident state, the FP64 CPU oracle
timed on the host cores, and the same workload with FP16 / BF16 / absolute-FP32
storage.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from lbinputs import config2, poiseuille  # noqa: E402

KN_SWEEP = (0.02, 0.1, 0.5)
STORE_BYTES = {"f64": 8, "f32": 4, "f32_dev": 4, "f16_dev": 2, "bf16_dev": 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--store", default="f32_dev")
    ap.add_argument("--no-forms", action="store_true", help="skip the other storage forms")
    ap.add_argument("--variant", type=int, default=-1, help="step-kernel layout (-1: autotune)")
    return ap.parse_args()


def workloads():
    return [config2(kn) for kn in KN_SWEEP]


ALU_OPS_PER_POP = 45   # FP32 operations per population update (Sec. 3.1 scheme)


def algorithmic_bytes(eff_map, sets, store):
    q = np.where(eff_map == 1, sets[1], sets[0])
    return 2 * STORE_BYTES[store] * int(q.sum())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def form_accuracy(lb, forms):
    """Relative velocity error (max over nodes, C18) of each storage form against the
    FP64 oracle on a steady force-driven channel (4 x 64, Kn 0.1, 32-row-per-wall
    equivalent band of 10 rows, 6000 steps): the accuracy behind each form's throughput."""
    import oracle
    from lbinputs import poiseuille
    w = poiseuille(nx=4, ny=64, rows=10, kn=0.1, g_lat=1e-5)
    steps = 6000
    out, ref = {}, None
    for name, (store, rnd) in forms.items():
        lat = lb.Lattice.from_workload(w, store=store, rounding=rnd, variant=0)
        if ref is None:
            o = oracle.Oracle(w.nx, w.ny, lat.effective_map(), kn_ref=w.kn_ref, gx=w.gx, walls=w.walls, dt=lat.dt,
                              h=lat.h)
            o.init_equilibrium(1.0, 0.0, 0.0)
            o.step(steps)
            ref = o.moments()
        lat.step(steps)
        m = lat.moments(mask=0b111)
        du = np.sqrt((m["ux"] - ref["ux"]) ** 2 + (m["uy"] - ref["uy"]) ** 2)
        out[name] = float(du.max() / np.sqrt(ref["ux"] ** 2 + ref["uy"] ** 2).max())
        lat.close()
    return out


def cpu_baseline(seconds=12.0):
    """The FP64 oracle on one full-size channel of the sweep (Kn = 0.1), all host cores."""
    import oracle
    w = config2(0.1)
    o = oracle.Oracle(w.nx, w.ny, w.region_map, kn_ref=w.kn_ref, gx=w.gx, walls=w.walls)
    o.init_equilibrium(1.0, 0.0, 0.0)
    o.step(1)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds or n < 2:
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    return {"value": w.cells * n / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"one 1024x512 channel (Kn 0.1) of the sweep, {n} steps, {dt:.1f} s, FP64, OpenMP"}


def max_over_ranks(torch, dist, ms, device):
    """The job's time: the slowest rank's (every rank gets it). Without a process group,
    this rank's own."""
    if dist is None:
        return ms
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world, cells_per_rank, steps, ms):
    """Whole-job throughput: every rank's cells (replicas of the same workload) over the
    job's time."""
    return world * cells_per_rank * steps / (ms / 1e3) / 1e6


def run_reference(args, rank):
    """The oracle as the reference arm: each step advances a 64-column slab of each of
    the three channels (the flow is x-invariant, so a slab is the same problem)."""
    if rank != 0:
        return
    import oracle
    labs = []
    for kn in KN_SWEEP:
        w = poiseuille(nx=64, ny=512, rows=32, kn=kn)
        o = oracle.Oracle(w.nx, w.ny, w.region_map, kn_ref=w.kn_ref, gx=w.gx, walls=w.walls)
        o.init_equilibrium(1.0, 0.0, 0.0)
        labs.append((w, o))
    for _ in range(args.warmup):
        for _, o in labs:
            o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _, o in labs:
            o.step(1)
    dt = time.perf_counter() - t0
    cells = sum(w.cells for w, _ in labs)
    value = cells * args.steps / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    line = {
        "impl": "reference", "metric": "coupled-LB MLUPS", "value": value, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "poiseuille 1024x512 x3 (Kn 0.02/0.1/0.5), D2Q9 core + D2Q36 32 rows/wall",
                   "sample": "64-column slab of each channel per step"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"64x512 slab of each of the 3 channels, {args.steps} steps"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def channel_lattices(lb, torch, store, variant=-1, rounding="nearest"):
    """The channels of the workload, each on its own CUDA stream (independent problems,
    as a user would run them: one channel's tail overlaps the next one's launch)."""
    streams = [torch.cuda.Stream() for _ in workloads()]
    lats = [lb.Lattice.from_workload(w, store=store, variant=variant, rounding=rounding, stream=s)
            for w, s in zip(workloads(), streams)]
    return lats, streams


def timed_steps(torch, lats, streams, steps):
    """CUDA events around `steps` steps of every channel: the start event on the current
    stream is waited for by every channel stream, and the stop event follows all of
    them. Returns milliseconds."""
    main = torch.cuda.current_stream()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(main)
    for s in streams:
        s.wait_event(start)
    for _ in range(steps):
        for lat in lats:
            lat.step(1)
    for s in streams:
        e = torch.cuda.Event()
        e.record(s)
        main.wait_event(e)
    stop.record(main)
    torch.cuda.synchronize()
    return start.elapsed_time(stop)


def launch_times(torch, lats, streams, reps):
    """Per-launch durations of the step kernel, one launch at a time: events on the
    launching stream, each launch ordered after the previous one's end event so that
    nothing overlaps and no host gap falls inside a measurement."""
    ev, prev = [], None
    for _ in range(reps):
        for i, (lat, s) in enumerate(zip(lats, streams)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if prev is not None:
                s.wait_event(prev)
            a.record(s)
            lat.step(1)
            b.record(s)
            ev.append((i, a, b))
            prev = b
    torch.cuda.synchronize()
    return [(i, a.elapsed_time(b)) for i, a, b in ev]


def time_form(lb, torch, store, steps, warmup, variant=-1, with_kernel_times=True, rounding="nearest"):
    lats, streams = channel_lattices(lb, torch, store, variant, rounding)
    for _ in range(warmup):
        for lat in lats:
            lat.step(1)
    torch.cuda.synchronize()
    total_ms = timed_steps(torch, lats, streams, steps)
    kern = [t for _, t in launch_times(torch, lats, streams, 20)] if with_kernel_times else []
    info = [lat.info() for lat in lats]
    eff = [lat.effective_map() for lat in lats]
    nbytes = [algorithmic_bytes(e, lat.sets, store) for e, lat in zip(eff, lats)]
    for lat in lats:
        lat.close()
    return total_ms, kern, nbytes, info


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import paper_1007_4895_gb300 as lb
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    cells = sum(w.cells for w in workloads())
    # main timed region: K steps of the three channels on this GPU, each channel on its
    # own stream
    lats, streams = channel_lattices(lb, torch, args.store, args.variant)
    for _ in range(args.warmup):
        for lat in lats:
            lat.step(1)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ms = timed_steps(torch, lats, streams, args.steps)
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(torch, dist, ms, "cuda")
    value = job_mlups(world, cells, args.steps, ms)
    variants = [lat.info()["variant"] for lat in lats]
    eff = [lat.effective_map() for lat in lats]
    nbytes = [algorithmic_bytes(e, lat.sets, args.store) for e, lat in zip(eff, lats)]

    # per-launch durations of the step kernel, on the stream it is launched on
    kt = launch_times(torch, lats, streams, max(3, min(60, args.steps // 50)))
    avg_ms = statistics.mean(t for _, t in kt)
    avg_bytes = statistics.mean(nbytes[i] for i, _ in kt)
    peak, peak_src = measured_peak_hbm()
    achieved = avg_bytes / (avg_ms / 1e3) / 1e9
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        try:
            tj = json.load(open(tp))
            if tj.get("store") == args.store and tj.get("kernel_sha") == kernel_sha():
                traffic = tj.get("bytes_per_launch")
        except Exception:
            traffic = None
    # the same launches against the FP32 ALU: 45 operations per population update (moments
    # 3, equilibrium and force 8, four limited fluxes 28, update 6), peak = SMs x 128 FP32
    # lanes x the SM clock sampled during the timed region
    pops = [algorithmic_bytes(e, lat.sets, args.store) // (2 * STORE_BYTES[args.store]) for e, lat in zip(eff, lats)]
    avg_pops = statistics.mean(pops[i] for i, _ in kt)
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    alu_peak = nsm * 128 * sm_mhz * 1e6 / 1e9
    alu_achieved = ALU_OPS_PER_POP * avg_pops / (avg_ms / 1e3) / 1e9
    roofline_alu = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "Gop/s",
                    "frac": alu_achieved / alu_peak, "ops_per_population": ALU_OPS_PER_POP,
                    "peak_source": f"derived: {nsm} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (sampled)"}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "lbk::step kernel (one launch per channel per step)",
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, copy burst)",
                "algorithmic_bytes_per_launch": avg_bytes, "launch_ms": avg_ms,
                "launches": "one at a time (isolated kernel durations)",
                "whole_job_frac": sum(nbytes) * args.steps / (ms / 1e3) / 1e9 / peak}

    # end to end through the C ABI with host-resident state: per step, each channel's
    # state comes in from pinned host memory and its mass / residual goes back
    e2e_steps = max(5, min(100, args.steps // 20))
    nbs = [lat.state_bytes() for lat in lats]
    host = [torch.empty(n, dtype=torch.uint8, pin_memory=True) for n in nbs]
    for lat, hbuf in zip(lats, host):
        lb.lb_state_store(lat.ctx, hbuf.data_ptr(), hbuf.numel())
    barrier()
    t0 = time.perf_counter()
    # each channel reads its previous step's result just before uploading its next
    # state, so one channel's upload overlaps the other channels' steps
    for k in range(e2e_steps):
        for lat, hbuf in zip(lats, host):
            if k > 0:
                lat.reductions()
            lb.lb_state_load(lat.ctx, hbuf.data_ptr(), hbuf.numel())
            lat.step(1)
    for lat in lats:
        lat.reductions()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * cells * e2e_steps / e2e_s / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": int(sum(nbs)), "d2h_bytes_per_step": (4 * 8 + 4) * len(lats),
           "steps": e2e_steps}
    for lat in lats:
        lat.close()

    forms = {}
    if not args.no_forms:
        variants_of_forms = {"f32": ("f32", "nearest"), "f16_dev": ("f16_dev", "nearest"),
                             "bf16_dev": ("bf16_dev", "nearest"), "f16_dev_sr": ("f16_dev", "stochastic"),
                             "bf16_dev_sr": ("bf16_dev", "stochastic")}
        for name, (store, rnd) in variants_of_forms.items():
            fs = max(50, min(args.steps, 1000))
            tot, kern, nb, info = time_form(lb, torch, store, fs, 5, args.variant, rounding=rnd)
            km = statistics.mean(kern)
            forms[name] = {"value": cells * fs / (tot / 1e3) / 1e6, "unit": "MLUPS",
                           "roofline_frac": (statistics.mean(nb) / (km / 1e3) / 1e9) / peak,
                           "variant": info[0]["variant"], "rounding": rnd}
        acc = form_accuracy(lb, dict({"f32_dev": ("f32_dev", "nearest")}, **variants_of_forms))
        for name, e in acc.items():
            forms.setdefault(name, {})["e_u_vs_fp64_oracle"] = e
        forms["accuracy_case"] = "steady Poiseuille 4x64, Kn 0.1, 6000 steps, max relative velocity error"

    line = {
        "metric": "coupled-LB MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "poiseuille 1024x512 x3 (Kn 0.02/0.1/0.5), D2Q9 core + D2Q36 32 rows/wall, "
                               "body force 1e-6 lattice, FP32 deviation storage",
                   "global_batch": 3 * world, "cells_per_gpu": cells, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (156 MB of populations touched per step)",
                   "kernel_variants": variants},
        "roofline": roofline,
        "roofline_alu": roofline_alu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": args.steps * sum(launches_per_step(v) for v in variants),
        "forms": forms,
    }
    if rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def launches_per_step(variant):
    """Kernels one lattice step launches on the benchmark workload (periodic x, no
    pressure columns, mode-B interfaces): the step kernel, plus the edge-list kernel of
    the split layouts (2, 3), whose list is never empty here (wall rows)."""
    return 2 if variant in (2, 3) else 1


def kernel_sha():
    import hashlib
    h = hashlib.sha1()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_1007_4895_gb300", "csrc"))):
        h.update(open(os.path.join(ROOT, "paper_1007_4895_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


if __name__ == "__main__":
    main()
