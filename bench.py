"""Benchmark of the fused D3Q27 central-Hermite MRT stream-collide step on GB300.

One "step" is one lattice time step over the whole workload (the fused
fluid kernel: pull gather, collision, bounce-back; and the inlet/outlet
nodes).  Default workload: the Re 6500 turbulent nozzle on a 144 x 144 x 1200
lattice (14 471 488 active cells), the largest of the nozzle workloads,
FP32 populations; FP16-shifted and FP64 storage are timed on the same
workload for the precision comparison.  Inputs are seeded and synthetic; the
population buffers (>= 0.9 GB each) exceed the 129 MB L2, so no flush is
needed between steps.

Timing: after W warm-up steps, regions of exactly K steps are timed with
CUDA events on the library's stream, each bracketed by a barrier and a
device synchronisation, repeated until at least --min-seconds of timed work
(and at least 5 regions); the median region gives ms_per_step.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (a bounded sample of the same workload per step).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fluid MLUPS & % HBM roofline (FP32/FP16 vs FP64); serving p50/p99 latency"
UNIT = "fluid MLUPS"
DEFAULT_WORKLOAD = "nozzle_re6500_144x144x1200"
STORAGE_BYTES = {"fp64": 8, "fp32": 4, "fp16s": 2}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16s": "f16 storage / f32 arithmetic"}
LINK_WORD_BYTES = 4


# FP64 flops per fluid-cell update of the step kernel (DADD + DMUL + 2 DFMA,
# counted by ncu on the Re 3500 nozzle).  The FP64 kernel keeps the FP64 pipe
# ~87 % busy, so its roofline is that pipe, not HBM.
FP64_FLOPS_PER_CELL = 541
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate


def algorithmic_bytes_per_cell(precision):
    """27 populations read + 27 written in the storage precision, plus the
    32-bit link word of the cell."""
    return 27 * 2 * STORAGE_BYTES[precision] + LINK_WORD_BYTES


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--precisions", default="fp32,fp16s,fp64",
                    help="first one is the headline; others are reported under by_precision")
    ap.add_argument("--min-seconds", type=float, default=3.0,
                    help="timed work per precision: K-step regions are repeated until this much (at least 5)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="oracle time of the whole --impl reference run (warm-up and timed steps)")
    ap.add_argument("--row-axis", choices=["auto", "x", "z"], default="auto",
                    help="axis of the storage rows (auto: z for the nozzles, the flow axis)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-walls", action="store_true",
                    help="skip the smooth-surface wall (interpolated bounce-back) timing")
    ap.add_argument("--serving-requests", type=int, default=64)
    ap.add_argument("--serving-stream", choices=["scaled", "full"], default="scaled",
                    help="full: the request mix at its full sizes (d 8-48, 2000-20000 steps; minutes)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


# The fluid kernel each precision runs by default (the roofline's dominant kernel).
FLUID_KERNEL = {"fp32": "k_step_tiles<fp32>", "fp16s": "k_step<fp16s>", "fp64": "k_step<fp64>"}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("lbm_device.cuh", "lbm_internal.h", "step_fp32.cu", "step_fp16s.cu", "step_fp64.cu"):
        with open(os.path.join(ROOT, "paper_2204_10566_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, precision):
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, or None when missing or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", "step_kernel_dram_traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        kv = dict(item.split("=", 1) for item in line.split())
        if kv.get("workload") == workload and kv.get("precision") == precision and kv.get("source") == src:
            return float(kv["dram_bytes_per_launch"])
    return None


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.25)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_setup(name):
    from paper_2204_10566_gb300 import inputs as I

    w = I.WORKLOADS[name]
    flags = I.workload_flags(name)
    if w["kind"] == "tgv":
        params = dict(nu=w["u0"] * (w["n"] / (2 * 3.141592653589793)) / w["Re"])
        periodic = 7
    else:
        params = I.workload_params(name)
        periodic = 0
    return w, flags, params, periodic


def aggregate_replicas(ms_local, cells_local, steps, dist=None, device="cpu"):
    """Whole-job numbers of N independent replicas (one lattice per rank):
    the job takes the slowest rank's time, and its work is the sum of all
    ranks' cell updates.  Returns (ms_max, total cells, MLUPS)."""
    import torch

    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    c = torch.tensor([float(cells_local)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    ms_max, cells = float(t.item()), float(c.item())
    return ms_max, cells, cells * steps / (ms_max * 1e-3) / 1e6


# --------------------------------------------------------------- our kernels

def timed_regions(torch, stream, run_region, steps, min_seconds, dist=None, device="cpu", min_repeats=5,
                  max_repeats=5000):
    """Time regions of exactly `steps` steps (run_region enqueues one) with
    CUDA events on `stream`, each bracketed by a barrier and a device
    synchronisation; the count of regions fills about min_seconds (at least
    min_repeats), agreed over ranks.  Returns the per-region milliseconds."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)  # probe region (not reported): sizes the repeat count
    run_region()
    e1.record(stream)
    torch.cuda.synchronize()
    probe_s = max(e0.elapsed_time(e1) * 1e-3, 1e-6)
    reps = int(min(max_repeats, max(min_repeats, -(-min_seconds // probe_s))))
    if dist is not None:
        t = torch.tensor([float(reps)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        reps = int(t.item())
    times = []
    for _ in range(reps):
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        run_region()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def time_precision(lbm, torch, flags, params, periodic, precision, steps, warmup, min_seconds, dist=None,
                   sampler=None, device="cpu", row_axis="auto", wall_q=None):
    """Median milliseconds of a K-step region of one precision (max over
    ranks is taken by the caller).  wall_q: (cells, q) of lbm_set_wall_q."""
    from paper_2204_10566_gb300 import inputs as I

    G = lbm.Lattice(flags, precision, periodic=periodic, row_axis=row_axis)
    G.set_params(**params)
    if wall_q is not None:
        G.set_wall_q(*wall_q)
    n = G.n_active
    G.init_fields(I.random_density_field(n, 0.001, 3), I.random_velocity_field(n, 0.01, 4))
    G.step(warmup).sync()
    if sampler:
        sampler.start()
    launched0 = G.kernel_launches()
    times = timed_regions(torch, G.stream, lambda: G.step(steps), steps, min_seconds, dist, device)
    clocks = sampler.stop() if sampler else None
    G.sync()
    info = G.layout_info()
    launched = G.kernel_launches() - launched0
    G.close()
    timing = {"regions": len(times), "steps_per_region": steps, "stat": "median",
              "ms_region_min": min(times), "ms_region_max": max(times),
              "launches_per_region": round(launched / (len(times) + 1))}  # the probe region and the timed ones
    return n, statistics.median(times), clocks, info, timing


def e2e_run(lbm, torch, flags, params, periodic, precision, steps):
    """The user's job through the public API with host buffers: upload the
    initial fields from pinned host memory, run the steps, read the moments
    back into pinned host memory; wall-clock timed."""
    from paper_2204_10566_gb300 import inputs as I

    G = lbm.Lattice(flags, precision, periodic=periodic)
    G.set_params(**params)
    n = G.n_active
    rho_h = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    u_h = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    rho_o = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    u_o = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    rho_h[:] = I.random_density_field(n, 0.001, 3)
    u_h[:] = I.random_velocity_field(n, 0.01, 4)
    G.init_fields(rho_h, u_h)
    G.step(10).sync()                      # warm the path once
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G.init_fields(rho_h, u_h)
    G.step(steps)
    G.moments(out=(rho_o, u_o))
    t1 = time.perf_counter()
    G.close()
    return dict(value=n * steps / (t1 - t0) / 1e6, unit=UNIT,
                h2d_bytes_per_step=n * 4 * 8 / steps, d2h_bytes_per_step=n * 4 * 8 / steps,
                seconds=t1 - t0, steps=steps)


# ------------------------------------------------------------ oracle sample

class OracleSample:
    """The FP64 CPU oracle on a sub-box of the workload (a z-slab from the
    middle of the lattice, cut in y when one plane is already too much),
    sized from a one-plane calibration to about target_seconds per step.
    The sample lattice is built and initialised once (uniform equilibrium,
    rho = 1, u = (0, 0, 0.01)); each timed sample continues from the state
    the previous one left."""

    U0 = (0.0, 0.0, 0.01)

    def __init__(self, flags, params, periodic, target_seconds):
        import numpy as np

        import oracle

        self.oracle = oracle
        self.np = np
        nz, ny, nx = flags.shape
        nu = params.get("nu") or params["u_char"] * params["L_char"] / params["Re"]
        self.omega = 1.0 / (3.0 * nu + 0.5)
        self.periodic = periodic & 3
        z0 = nz // 2
        plane = np.array(flags[z0:z0 + 1])
        dt, cells = self._time(self._lattice(plane), 1)
        per_cell = dt / max(cells, 1)
        want = max(1, int(target_seconds / per_cell))
        if want >= cells:
            planes, rows = min(nz - z0, max(1, want // max(cells, 1))), ny
        else:
            planes, rows = 1, max(2, int(ny * want / max(cells, 1)))
        self.flags = np.array(flags[z0:z0 + planes, :rows, :])
        self.cells = int((self.flags != 0).sum())
        self.L = self._lattice(self.flags)
        # a slab capped at the far end of the lattice takes several steps,
        # counted from one timed step of the slab itself
        self.steps = 1
        if planes == nz - z0 and rows == ny:
            dt1, _ = self._time(self.L, 1)
            self.steps = max(1, int(round(target_seconds / max(dt1, 1e-9))))
        self.threads = os.cpu_count() or 1
        self.desc = "%d oracle step%s on a %dx%dx%d sub-box (z from %d) of the workload, %d active cells" % (
            self.steps, "s" if self.steps > 1 else "", nx, rows, planes, z0, self.cells)

    def _lattice(self, f, nthreads=0):
        """An oracle lattice of flags f at the uniform equilibrium (the same
        populations init_equilibrium gives every active cell)."""
        np = self.np
        L = self.oracle.Lattice(f, self.omega, periodic=self.periodic, nthreads=nthreads)
        pop = np.zeros((f.size, 27))
        pop[f.reshape(-1) != 0] = self.oracle.equilibrium(1.0, np.array(self.U0))
        L.set_populations(pop)
        return L

    @staticmethod
    def _time(L, steps):
        t = time.perf_counter()
        L.step(steps)
        return time.perf_counter() - t, int((L.flags != 0).sum()) * steps

    def single_thread(self):
        """One oracle step on the first 16 z-planes of the slab with one
        thread: returns (MLUPS, cells)."""
        plane = self.np.array(self.flags[:16])
        dt, cells = self._time(self._lattice(plane, nthreads=1), 1)
        return cells / dt / 1e6, cells

    def step(self):
        """One timed sample; returns (MLUPS, seconds)."""
        dt, updates = self._time(self.L, self.steps)
        return updates / dt / 1e6, dt


# ----------------------------------------------------------------- serving

SERVING_STREAMS = {
    # scaled down from the full mix so that the default measurement takes seconds
    "scaled": dict(d=(8, 24), steps=(200, 2000)),
    # the request mix at its full sizes
    "full": dict(d=(8, 48), steps=(2000, 20000)),
}


def serving_measurement(capacity_mlups, n_requests, stream="scaled"):
    """Continuous batching on the seeded request stream (nozzle / pipe runs of
    throat diameter d, D = 3 d, L = 25 d, Re uniform in 500-6500, FP32 or
    FP16S with p = 1/2, Poisson arrivals at 1.2 x the measured single-stream
    FP32 capacity), against the same stream run back to back as plain FP32
    lattices, and again at 0.5 x the capacity (latency of an unsaturated
    server).  stream "full" is the request mix at its sizes (d 8-48,
    2000-20000 steps); "scaled" shrinks both so that it takes seconds."""
    import torch

    from paper_2204_10566_gb300 import inputs as I
    from paper_2204_10566_gb300 import serving

    d_range, steps_range = SERVING_STREAMS[stream]["d"], SERVING_STREAMS[stream]["steps"]
    probe = I.serving_requests(n=n_requests, seed=2204, rate=1.0, d_range=d_range, steps_range=steps_range)
    work = []
    for s in probe:
        f = serving.request_geometry(s)
        work.append(I.active_count(f) * s["steps"])
    rate = 1.2 * capacity_mlups * 1e6 / (sum(work) / len(work))
    specs = I.serving_requests(n=n_requests, seed=2204, rate=rate, d_range=d_range, steps_range=steps_range)
    free, _ = torch.cuda.mem_get_info()
    srv = serving.run_stream([dict(s) for s in specs], budget_bytes=int(0.5 * free), max_slots=32, steps_per_tick=32)
    b2b = serving.run_back_to_back([dict(s) for s in specs], "fp32")
    # the same arm with each request in its own storage precision (FP32 or FP16S, as served)
    b2b_own = serving.run_back_to_back([dict(s) for s in specs], None)
    # the same stream at 0.5x the capacity: latency when the server is not saturated
    low = I.serving_requests(n=n_requests, seed=2204, rate=rate * 0.5 / 1.2, d_range=d_range,
                             steps_range=steps_range)
    srv_low = serving.run_stream([dict(s) for s in low], budget_bytes=int(0.5 * free), max_slots=32,
                                 steps_per_tick=32)
    failed = [dict(d=specs[k]["d"], Re=round(specs[k]["Re"]), steps=specs[k]["steps"], kind=specs[k]["kind"],
                   precision=specs[k]["precision"], steps_done=r["steps_done"], error=str(r["error"]))
              for k, r in srv["results"].items() if r["state"] != 2]
    return {
        "low_load": {"offered_load": 0.5, "p50_s": srv_low["latency_p50_s"], "p99_s": srv_low["latency_p99_s"],
                     "aggregate_mlups": srv_low["mlups"]},
        "requests": n_requests, "arrival_rate_per_s": rate, "offered_load": 1.2, "failed_requests": failed,
        "stream": "%s: seed 2204; d uniform in %d-%d (D = 3d, L = 25d), Re 500-6500, %d-%d steps, FP32/FP16S, "
                  "nozzle/pipe" % ((stream,) + tuple(d_range) + tuple(steps_range)),
        "p50_s": srv["latency_p50_s"], "p99_s": srv["latency_p99_s"],
        "aggregate_mlups": srv["mlups"], "makespan_s": srv["makespan_s"],
        "back_to_back_fp32_mlups": b2b["mlups"], "back_to_back_s": b2b["seconds"],
        "back_to_back_setup_s": b2b["setup_seconds"],
        "speedup_vs_back_to_back": srv["mlups"] / b2b["mlups"],
        "back_to_back_own_precision_mlups": b2b_own["mlups"],
        "speedup_vs_back_to_back_own_precision": srv["mlups"] / b2b_own["mlups"],
        "steps_per_tick": 32, "graph_captures": srv["info"]["graph_captures"],
        "graph_launches": srv["info"]["graph_launches"],
    }


# ------------------------------------------------------------------ arms

def reference_arm(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    w, flags, params, periodic = workload_setup(args.workload)
    total = args.steps + args.warmup
    # each step a bounded sample, so that the whole run fits in ~150 s
    sample = OracleSample(flags, params, periodic, max(0.002, args.ref_seconds / max(total, 1)))
    vals = []
    t_all = 0.0
    for k in range(total):
        mlups, dt = sample.step()
        if k >= args.warmup:
            vals.append(mlups)
            t_all += dt
    threads, desc = sample.threads, sample.desc
    value = statistics.median(vals) if vals else 0.0
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / max(len(vals), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "precision": "fp64 (CPU oracle)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def ours_arm(args):
    import torch

    from paper_2204_10566_gb300 import build as lbuild

    lbuild.build()
    from paper_2204_10566_gb300 import lbm

    rank, world, local = env_rank()
    dist = None
    if world > 1:
        import torch.distributed as td

        torch.cuda.set_device(local)
        td.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = td
    else:
        torch.cuda.set_device(0)
    device = torch.cuda.current_device()
    w, flags, params, periodic = workload_setup(args.workload)
    precisions = args.precisions.split(",")
    head = precisions[0]
    peak, peak_kind = load_peaks()

    sampler = ClockSampler(device) if rank == 0 else None
    n, ms, clocks, info, timing = time_precision(lbm, torch, flags, params, periodic, head, args.steps, args.warmup,
                                                 args.min_seconds, dist, sampler, device="cuda",
                                                 row_axis=args.row_axis)
    ms_max, _, value = aggregate_replicas(ms, n, args.steps, dist, device="cuda")
    per_launch_s = ms * 1e-3 / max(args.steps, 1)
    alg_bytes = algorithmic_bytes_per_cell(head) * n
    achieved = alg_bytes / per_launch_s / 1e9
    traffic = recorded_traffic(args.workload, head)

    by_prec = {}
    for p in precisions[1:]:
        steps = args.steps
        n_p, ms_p, _, info_p, timing_p = time_precision(lbm, torch, flags, params, periodic, p, steps, args.warmup,
                                                        0.5 * args.min_seconds, dist, None, device="cuda",
                                                        row_axis=args.row_axis)
        ms_p = aggregate_replicas(ms_p, n_p, steps, dist, device="cuda")[0]
        ach_p = algorithmic_bytes_per_cell(p) * n_p / (ms_p * 1e-3 / steps) / 1e9
        if p == "fp64":
            tf = FP64_FLOPS_PER_CELL * n_p / (ms_p * 1e-3 / steps) / 1e12
            roof = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": tf / FP64_PEAK_TFLOPS, "peak_kind": "nominal FP64 rate", "flops_per_cell":
                    FP64_FLOPS_PER_CELL, "hbm_frac": ach_p / peak}
        else:
            roof = {"bound": "hbm", "achieved": ach_p, "peak": peak, "unit": "GB/s", "frac": ach_p / peak,
                    "peak_kind": peak_kind, "bytes_per_cell": algorithmic_bytes_per_cell(p)}
        roof["kernel"] = FLUID_KERNEL[p]
        if p != "fp64":
            roof["traffic"] = recorded_traffic(args.workload, p)
        by_prec[p] = {"value": world * n_p * steps / (ms_p * 1e-3) / 1e6, "unit": UNIT, "steps": steps,
                      "ms_per_step": ms_p / steps, "roofline": roof, "timing": timing_p}

    by_walls = None
    if not args.no_walls and w["kind"] == "nozzle":
        # the paper's wall treatment: Bouzidi interpolation on the smooth surface
        from paper_2204_10566_gb300 import inputs as I

        wq = I.nozzle_wall_q(w["D"], w["d"], w["L_total"], flags=flags)
        by_walls = {"walls": "interpolated bounce-back on the smooth nozzle surface (lbm_set_wall_q)",
                    "wall_cells": int(wq[0].size)}
        for p in [q for q in precisions if q != "fp64"]:
            n_w, ms_w, _, _, timing_w = time_precision(lbm, torch, flags, params, periodic, p, args.steps,
                                                       args.warmup, 0.5 * args.min_seconds, dist, None,
                                                       device="cuda", row_axis=args.row_axis, wall_q=wq)
            ms_w = aggregate_replicas(ms_w, n_w, args.steps, dist, device="cuda")[0]
            v_w = world * n_w * args.steps / (ms_w * 1e-3) / 1e6
            halfway = value if p == head else by_prec[p]["value"]
            by_walls[p] = {"value": v_w, "unit": UNIT, "ms_per_step": ms_w / args.steps,
                           "vs_halfway_walls": v_w / halfway, "timing": timing_w}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    e2e = e2e_run(lbm, torch, flags, params, periodic, head, args.steps)
    serve = None
    if world == 1 and not args.no_serving:
        serve = serving_measurement(value, args.serving_requests, args.serving_stream)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        sample = OracleSample(flags, params, periodic, args.cpu_seconds)
        mlups, dt = sample.step()
        st, st_cells = sample.single_thread()
        cpu = {"value": mlups, "unit": UNIT, "cores": sample.threads, "kind": "oracle", "sample": sample.desc,
               "seconds": dt, "single_thread": {"value": st, "unit": UNIT, "cores": 1,
                                                "sample": "1 oracle step on 16 z-planes of the slab, %d active cells" % st_cells}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[head], "data": "synthetic",
        "config": {"workload": args.workload, "precision": head, "active_cells": n, "box": list(flags.shape[::-1]),
                   "slots": info["slots"], "Re": w.get("Re"),
                   "row_axis": lbm.check_layout(flags, periodic, args.row_axis)["row_axis"],
                   "l2": "inputs larger than L2 (population buffers %.2f GB each)" % (info["buffer_bytes"] / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "frac_of_nominal_7900": achieved / 7900.0,
                     "kernel": FLUID_KERNEL[head],
                     "duration": "median K-step region / K: the fluid kernel with the inlet/outlet kernel "
                                 "beside it on the side stream",
                     "bytes_per_cell": algorithmic_bytes_per_cell(head)},
        "by_precision": by_prec,
        "by_walls": by_walls,
        "e2e": e2e,
        "gpu_launches": timing["launches_per_region"],
        "timing": dict(timing, note="gpu_launches counts the kernels of one timed K-step region"),
        "clocks": clocks,
        "cpu_baseline": cpu,
        "serving": serve,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours_arm(args)


if __name__ == "__main__":
    main()
