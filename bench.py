"""Throughput benchmark of the multiscale lattice Boltzmann step on GB300.

Headline workload: the pressure-driven long microchannel, 16384 x 128 nodes, inlet /
outlet density ratio 2, outlet Kn 0.2, region map fixed by the local-Kn threshold
(D2Q36 bands of 10 to 19 rows per wall, D2Q9 in the core), pressure columns at both
ends, populations stored as FP32 deviations from w_i rho0 and collided in FP32. One
step is one time step of the whole lattice: 2.1 M node updates, about 254 MB of
populations read and written (larger than the 126 MB L2, so no L2 flush is needed
between steps). Inputs are synthetic (lbinputs.config3).

Metric: MLUPS (million node updates per second, every node counted once per step) over
all GPUs. The JSON line also carries the HBM roofline of the step, the end-to-end rate
through the C ABI with the state resident in host memory (uploaded and read back every
step), the FP64 CPU oracle timed on the host cores, the other storage forms on the same
lattice with their error against the oracle, and, as a secondary key, the three
force-driven 1024 x 512 channels.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --profile long_channel|poiseuille|stream_box [--store S] [--variant V] [--steps N]

--profile only builds the named lattice and advances it N steps (for ncu).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from lbinputs import config2, config3, long_channel, long_channel_density, poiseuille  # noqa: E402

KN_SWEEP = (0.02, 0.1, 0.5)
STORE_BYTES = {"f64": 8, "f32": 4, "f32_dev": 4, "f16_dev": 2, "bf16_dev": 2}
ALU_OPS_PER_POP = 45   # FP32 operations per population update of the Sec. 3.1 scheme
HEADLINE = "long channel 16384x128 (rho_in/rho_out 2, Kn_out 0.2, local-Kn map), FP32 deviation storage"
PARITY_STEPS = 40      # steps of every storage form against the FP64 oracle on the headline lattice


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--store", default="f32_dev")
    ap.add_argument("--variant", type=int, default=-1, help="step-kernel layout (-1: autotune)")
    ap.add_argument("--no-forms", action="store_true", help="skip the other storage forms")
    ap.add_argument("--no-secondary", action="store_true", help="skip the three-channel secondary workload")
    ap.add_argument("--profile", default=None, choices=["long_channel", "poiseuille", "stream_box", "batched"],
                    help="build one lattice (or the 512-channel batch: a 20-step launch, then one of --steps "
                         "steps), advance it --steps steps, exit (for ncu)")
    return ap.parse_args()


def algorithmic_bytes(eff_map, sets, store):
    """2 Q s per node: every population read once and written once per step."""
    q = np.where(eff_map == 1, sets[1], sets[0])
    return 2 * STORE_BYTES[store] * int(q.sum())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 20 ms while the GPU is loaded."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.t0 = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.t0 = time.perf_counter()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def elapsed(self):
        return time.perf_counter() - self.t0

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
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


STEP_SOURCES = ("lb_internal.h", "lb_common.cuh", "lb_store.cuh", "lb_step_impl.cuh", "lb_step.cu", "lb_pair.cuh",
                "lb_ring.cuh", "lb_ring2.cuh", "lb_api.cu")


def kernel_sha():
    """Hash of the sources of the step's kernels (the step kernels of every layout and the
    pressure pass): DRAM counters taken on other sources are not reported."""
    import hashlib
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_1007_4895_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f in STEP_SOURCES or f.startswith(("lb_step_st_", "lb_pair_", "lb_ring_", "lb_ring2_")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:12]


def stored_traffic(workload, store, variant):
    """DRAM bytes per step from the committed ncu capture, when it was taken on the
    current kernel sources, this workload, storage and layout; else None."""
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        tj = json.load(open(tp))
    except Exception:
        return None
    for e in tj.get("captures", []):
        if (e.get("workload") == workload and e.get("store") == store and e.get("variant") == variant
                and e.get("kernel_sha") == kernel_sha()):
            return e.get("bytes_per_step")
    return None


# ------------------------------------------------------------- timing helpers

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


def timed_steps(torch, lats, streams, steps):
    """CUDA events around `steps` steps of every lattice: the start event on the current
    stream is waited for by every lattice's stream, and the stop event follows all of
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


def step_times(torch, lats, streams, reps):
    """Duration of one step of each lattice, one at a time: events on the lattice's own
    stream, each step ordered after the previous one's end event, so that nothing
    overlaps and no host gap falls inside a measurement."""
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


def launches_per_step(variant, pressure, force=False):
    """Kernels one lattice step launches: the step kernel, the edge-list kernel of the
    split layouts (2, 3; the list always holds the wall rows), and the pressure pass when
    the lattice has pressure columns (layout 10 does those inside its kernel unless the
    lattice has a body force)."""
    own_pressure = variant == 10 and not force
    return (2 if variant in (2, 3) else 1) + (1 if pressure and not own_pressure else 0)


# ------------------------------------------------------------- oracle parts

def cpu_baseline(seconds=12.0):
    """The FP64 oracle on the headline lattice, all host cores, for about `seconds`."""
    import oracle
    w = config3()
    o = oracle.Oracle(w.nx, w.ny, w.region_map, kn_ref=w.kn_ref, rho_ref=w.rho_ref, walls=w.walls, cfl=w.cfl)
    o.init_equilibrium(*w.init)
    o.step(1)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds or n < 2:
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    return {"value": w.cells * n / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"the 16384x128 long channel, {n} steps, {dt:.1f} s, FP64, OpenMP"}


def oracle_reference_fields(steps, lat):
    """The FP64 oracle's moments of the headline lattice after `steps` steps, on the map
    the GPU lattice runs (tile-quantised) with its time step and spacing."""
    import oracle
    w = config3()
    o = oracle.Oracle(w.nx, w.ny, lat.effective_map(), kn_ref=w.kn_ref, rho_ref=w.rho_ref, walls=w.walls,
                      dt=lat.dt, h=lat.h)
    o.init_equilibrium(*w.init)
    o.step(steps)
    return o.moments()


def field_error(got, ref):
    """Max relative errors: velocity (vector norm) by max |u_ref|, density by max rho."""
    du = np.sqrt((got["ux"] - ref["ux"]) ** 2 + (got["uy"] - ref["uy"]) ** 2)
    e_u = float(du.max() / np.sqrt(ref["ux"] ** 2 + ref["uy"] ** 2).max())
    e_rho = float(np.abs(got["rho"] - ref["rho"]).max() / np.abs(ref["rho"]).max())
    return e_u, e_rho


def steady_accuracy(lb, forms):
    """Relative velocity error (max over nodes) of each storage form against the FP64
    oracle on a steady force-driven channel (4 x 64, Kn 0.1, 10 high-order rows per wall,
    6000 steps): the long-run accuracy behind each form."""
    import oracle
    w = poiseuille(nx=4, ny=64, rows=10, kn=0.1, g_lat=1e-5)
    steps = 6000
    out, ref = {}, None
    for name, (store, rnd) in forms.items():
        lat = lb.Lattice.from_workload(w, store=store, rounding=rnd)
        if ref is None:
            o = oracle.Oracle(w.nx, w.ny, lat.effective_map(), kn_ref=w.kn_ref, gx=w.gx, walls=w.walls, dt=lat.dt,
                              h=lat.h)
            o.init_equilibrium(1.0, 0.0, 0.0)
            o.step(steps)
            ref = o.moments()
        lat.step(steps)
        out[name] = field_error(lat.moments(mask=0b111), ref)[0]
        lat.close()
    return out


def batched_sweep(lb, torch, store, steps=500):
    """The 512 seeded channels of the batched configuration (8 x 16..256 nodes, Couette
    and Poiseuille, Kn 0.01..1) advanced together by one persistent launch per call:
    MLUPS over `steps` steps (CUDA events on the batch's stream), with the algorithmic
    bytes of those steps against the measured HBM rate."""
    from lbinputs import batched_instances
    ws = batched_instances()
    b = lb.Batch(ws, store=store)
    b.step(20)
    b.sync()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    b.step(steps)
    e1.record(s)
    b.sync()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    nodes = sum(w.nx * w.ny for w in ws)
    nbytes = sum(algorithmic_bytes(b.lattice(i).effective_map(), b.lattice(i).sets, store) for i in range(len(ws)))
    peak, _ = measured_peak_hbm()
    out = {"value": nodes * steps / (ms / 1e3) / 1e6, "unit": "MLUPS", "lattices": len(ws), "nodes": nodes,
           "steps": steps, "ms": ms, "roofline_frac": nbytes * steps / (ms / 1e3) / 1e9 / peak,
           "kernel": b.info()}
    b.close()
    return out


def config5_study(lb, torch, nx=16384, ny=128, steps=2000, every=200, samples=100000, threshold=3e-4, epochs=20):
    """Learned interface placement on the long channel (the headline geometry at CFL 0.38,
    where an all-high-order map is stable): an all-D2Q36 run gives the features and the
    labels (beyond-second-order residual e3 > threshold) of `samples` nodes drawn with the
    same count from every wall distance; the network trains on the GPU; a run from the
    fixed local-Kn map then has its map updated by the network every `every` steps. The
    three maps (fixed, learned, all-D2Q36) are compared on velocity error against the
    all-D2Q36 run after `steps` steps, on their high-order fraction and on MLUPS (timed
    with their map updates), and the cost of one map update is timed."""
    from lbinputs import mlp_init, wall_stratified_sample
    w = long_channel(nx=nx, ny=ny, cfl=0.38)
    n = nx * ny
    allh = lb.Lattice(nx, ny, np.ones((ny, nx), np.uint8), sets=w.sets, kn_ref=w.kn_ref, rho_ref=w.rho_ref,
                      walls=w.walls, store="f32_dev", rho0=w.rho0, cfl=w.cfl)
    allh.init_equilibrium(*w.init)
    allh.step(steps)
    ref = allh.moments(mask=0b111)
    F = torch.empty((8, ny, nx), device="cuda")
    E = torch.empty((ny, nx), device="cuda")
    allh.features_into(F)
    allh.hermite_residual_into(E)
    idx = torch.tensor(wall_stratified_sample(ny, nx, samples), device="cuda", dtype=torch.long)
    X = F.reshape(8, n)[:, idx].contiguous()
    Y = (E.reshape(n)[idx] > threshold).float().contiguous()
    Xh = X.cpu().numpy()
    norm = np.concatenate([Xh.mean(1), Xh.std(1) + 1e-12]).astype(np.float32)
    net = lb.MLP(mlp_init(1007), norm)
    loss0 = net.grad(X, Y)[1]
    t0 = time.perf_counter()
    loss = net.train(X, Y, epochs=epochs, batch=256, lr=1e-3, seed=1007)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    pX = torch.empty(samples, device="cuda")
    net.infer(X, pX)
    acc = float(((pX > 0.5).float() == Y).float().mean())
    label_share = float(Y.mean())
    # inference over the whole lattice, CUDA events
    P = torch.empty(n, device="cuda")
    Fn = F.reshape(8, n)
    for _ in range(2):
        net.infer(Fn, P)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        net.infer(Fn, P)
    b.record()
    torch.cuda.synchronize()
    infer_ms = a.elapsed_time(b) / 5

    def run(map_kind):
        lat = lb.Lattice.from_workload(w, store="f32_dev") if map_kind != "all_high" else allh
        if map_kind == "learned":
            lat.set_mlp(net, every=every)
        if map_kind != "all_high":
            lat.step(steps)
        m = lat.moments(mask=0b111)
        du = np.sqrt((m["ux"] - ref["ux"]) ** 2 + (m["uy"] - ref["uy"]) ** 2)
        e_u = float(du.max() / np.sqrt(ref["ux"] ** 2 + ref["uy"] ** 2).max())
        phi = float((lat.effective_map() == 1).mean())
        stats = lat.map_stats() if map_kind == "learned" else None
        k = 2 * every
        torch.cuda.synchronize()
        t = time.perf_counter()
        lat.step(k)
        torch.cuda.synchronize()
        mlups = n * k / (time.perf_counter() - t) / 1e6
        out = {"e_u_vs_all_high": e_u, "phi_H": phi, "MLUPS": mlups, "variant": lat.info()["variant"]}
        if stats:
            out["map_updates"] = stats["updates"]
            out["fallbacks"] = stats["fallbacks"]
            t = time.perf_counter()
            lat.learned_map_now()
            torch.cuda.synchronize()
            out["map_update_ms"] = (time.perf_counter() - t) * 1e3
        return out

    res = {m: run(m) for m in ("fixed", "learned", "all_high")}
    return {"workload": f"long channel {nx}x{ny}, CFL 0.38, {steps} steps", "samples": samples,
            "label": f"e3 > {threshold:g} on the all-D2Q36 run", "label_share": label_share,
            "train": {"epochs": epochs, "seconds": train_s, "loss0": loss0, "loss": loss, "accuracy": acc},
            "infer_ms_whole_lattice": infer_ms, "update_every": every, "maps": res}


def run_reference(args, rank):
    """The oracle as the reference arm: each step advances a 512-column long channel of
    the headline's height, density ratio, Kn and map rule (a bounded sample of the
    headline lattice, with its per-node cost), on the host cores."""
    if rank != 0:
        return
    import oracle
    w = long_channel(nx=512, ny=128)
    o = oracle.Oracle(w.nx, w.ny, w.region_map, kn_ref=w.kn_ref, rho_ref=w.rho_ref, walls=w.walls, cfl=w.cfl)
    o.init_equilibrium(*w.init)
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    value = w.cells * args.steps / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    line = {
        "impl": "reference", "metric": "coupled-LB MLUPS", "value": value, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": HEADLINE, "sample": "512x128 long channel of the same density ratio, Kn and map rule per step"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"512x128 long channel, {args.steps} steps"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- profiling mode

def profile_only(args):
    import torch

    import paper_1007_4895_gb300 as lb
    if args.profile == "batched":
        from lbinputs import batched_instances
        b = lb.Batch(batched_instances(), store=args.store)
        b.step(20)
        b.step(args.steps)
        b.sync()
        torch.cuda.synchronize()
        print(args.profile, args.store, b.info())
        b.close()
        return
    if args.profile == "stream_box":
        periodic = {s: {"kind": "periodic"} for s in ("bottom", "top", "left", "right")}
        lat = lb.Lattice(2048, 1024, np.zeros((1024, 2048), np.uint8), kn_ref=0.002, rho_ref=1.0, walls=periodic,
                         store=args.store, scheme="stream")
    else:
        w = config3() if args.profile == "long_channel" else config2(0.1)
        lat = lb.Lattice.from_workload(w, store=args.store, variant=args.variant)
    lat.step(args.steps)
    torch.cuda.synchronize()
    print(args.profile, args.store, lat.info())


# ------------------------------------------------------------- the benchmark

def main():
    args = parse()
    if args.profile:
        profile_only(args)
        return
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

    # headline: K steps of the long channel on this GPU (one replica per rank)
    w = config3()
    stream = torch.cuda.Stream()
    lat = lb.Lattice.from_workload(w, store=args.store, variant=args.variant, stream=stream)
    for _ in range(args.warmup):
        lat.step(1)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ms = timed_steps(torch, [lat], [stream], args.steps)
    # keep the GPU loaded (untimed) until the clock sampler has seen a second of it
    while clocks.elapsed() < 1.0:
        for _ in range(200):
            lat.step(1)
        torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(torch, dist, ms, "cuda")
    value = job_mlups(world, w.cells, args.steps, ms)
    variant = lat.info()["variant"]
    nbytes = algorithmic_bytes(lat.effective_map(), lat.sets, args.store)

    # roofline of the step (step kernel + pressure pass), one step at a time
    st = [t for _, t in step_times(torch, [lat], [stream], 60)]
    step_ms = statistics.mean(st)
    peak, peak_src = measured_peak_hbm()
    achieved = nbytes / (step_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": stored_traffic("long_channel", args.store, variant),
                "kernel": "lbk step kernel + pressure pass (one step of the long channel)",
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, copy burst)",
                "algorithmic_bytes_per_launch": nbytes, "launch_ms": step_ms,
                "launches": "one step at a time (isolated)"}
    pops = nbytes // (2 * STORE_BYTES[args.store])
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    alu_peak = nsm * 128 * sm_mhz * 1e6 / 1e9
    alu_achieved = ALU_OPS_PER_POP * pops / (step_ms / 1e3) / 1e9
    roofline_alu = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "Gop/s",
                    "frac": alu_achieved / alu_peak, "ops_per_population": ALU_OPS_PER_POP,
                    "peak_source": f"derived: {nsm} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (sampled)"}

    # end to end through the C ABI with the state in host memory: every step uploads the
    # compact state from pinned host memory, steps, and reads the new state back
    e2e_steps = max(5, min(50, args.steps // 100))
    nb = lat.state_bytes()
    host = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    lb.lb_state_store(lat.ctx, host.data_ptr(), nb)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lb.lb_state_load(lat.ctx, host.data_ptr(), nb)
        lat.step(1)
        lb.lb_state_store(lat.ctx, host.data_ptr(), nb)   # synchronous: the host holds the new state
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * w.cells * e2e_steps / e2e_s / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": int(nb), "d2h_bytes_per_step": int(nb), "steps": e2e_steps,
           "what": "compact state (own-set populations) uploaded, one step, state read back"}
    lat.close()

    # the other storage forms on the headline lattice: rate, roofline, error against the
    # FP64 oracle after PARITY_STEPS steps from the same start
    forms = {}
    if not args.no_forms and rank == 0:
        specs = {"f32_dev": ("f32_dev", "nearest"), "f32": ("f32", "nearest"), "f16_dev": ("f16_dev", "nearest"),
                 "bf16_dev": ("bf16_dev", "nearest"), "f16_dev_sr": ("f16_dev", "stochastic"),
                 "bf16_dev_sr": ("bf16_dev", "stochastic")}
        # the same deviation formats with the per-column reference density (lb_opts.rho0_col:
        # the inlet-to-outlet density estimate), which takes the density offset out of the
        # stored values
        col = long_channel_density(w.nx, 2.0, 1.0)
        specs_col = {"f32_dev_col": ("f32_dev", "nearest"), "f16_dev_sr_col": ("f16_dev", "stochastic"),
                     "bf16_dev_sr_col": ("bf16_dev", "stochastic")}
        ref = None
        for name, (store, rnd) in list(specs.items()) + list(specs_col.items()):
            kw = {"rho0_col": col} if name.endswith("_col") else {}
            f = lb.Lattice.from_workload(w, store=store, rounding=rnd, **kw)
            if ref is None:
                ref = oracle_reference_fields(PARITY_STEPS, f)
            f.step(PARITY_STEPS)
            e_u, e_rho = field_error(f.moments(mask=0b111), ref)
            s2 = torch.cuda.current_stream()
            for _ in range(5):
                f.step(1)
            t = statistics.mean(x for _, x in step_times(torch, [f], [s2], 30))
            fb = algorithmic_bytes(f.effective_map(), f.sets, store)
            forms[name] = {"value": w.cells / (t / 1e3) / 1e6, "unit": "MLUPS",
                           "roofline_frac": fb / (t / 1e3) / 1e9 / peak, "variant": f.info()["variant"],
                           "rounding": rnd, f"e_u_vs_fp64_oracle_{PARITY_STEPS}_steps": e_u,
                           f"e_rho_vs_fp64_oracle_{PARITY_STEPS}_steps": e_rho}
            f.close()
        acc = steady_accuracy(lb, specs)
        for name, e in acc.items():
            forms[name]["e_u_steady_poiseuille_6000_steps"] = e
        forms["accuracy_cases"] = (f"the headline lattice after {PARITY_STEPS} steps against the FP64 oracle; "
                                   "steady Poiseuille 4x64, Kn 0.1, 6000 steps; max relative errors")
        forms["learned_placement"] = config5_study(lb, torch)
        forms["batched_512"] = batched_sweep(lb, torch, args.store)
        forms["batched_512_bf16_dev"] = batched_sweep(lb, torch, "bf16_dev")

    # secondary: three force-driven 1024 x 512 channels (Kn 0.02 / 0.1 / 0.5), one stream
    # each, stepped together
    secondary = None
    if not args.no_secondary:
        streams = [torch.cuda.Stream() for _ in KN_SWEEP]
        lats = [lb.Lattice.from_workload(config2(kn), store=args.store, variant=args.variant, stream=s)
                for kn, s in zip(KN_SWEEP, streams)]
        for _ in range(10):
            for x in lats:
                x.step(1)
        torch.cuda.synchronize()
        k2 = max(100, min(args.steps, 3000))
        ms2 = timed_steps(torch, lats, streams, k2)
        cells2 = sum(x.nx * x.ny for x in lats)
        nb2 = [algorithmic_bytes(x.effective_map(), x.sets, args.store) for x in lats]
        kt = step_times(torch, lats, streams, 20)
        one = statistics.mean(t for _, t in kt)
        secondary = {"workload": "poiseuille 1024x512 x3 (Kn 0.02/0.1/0.5), D2Q9 core + D2Q36 32 rows/wall, "
                                 "body force 1e-6 lattice",
                     "value": cells2 * k2 / (ms2 / 1e3) / 1e6, "unit": "MLUPS", "steps": k2,
                     "whole_job_frac": sum(nb2) * k2 / (ms2 / 1e3) / 1e9 / peak,
                     "one_channel_step_ms": one,
                     "one_channel_frac": statistics.mean(nb2) / (one / 1e3) / 1e9 / peak,
                     "variants": [x.info()["variant"] for x in lats],
                     "l2": "per channel launch 51.9 MB < L2: its writes stay in L2 within a launch"}
        for x in lats:
            x.close()

    line = {
        "metric": "coupled-LB MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": HEADLINE, "cells_per_gpu": w.cells, "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2 ({nbytes / 1e6:.0f} MB of populations read and written per step)",
                   "kernel_variant": variant},
        "roofline": roofline,
        "roofline_alu": roofline_alu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": args.steps * launches_per_step(variant, pressure=True),
        "forms": forms,
        "secondary": secondary,
    }
    if rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
