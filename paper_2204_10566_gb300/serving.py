"""Serving driver: replay a seeded request stream against the request server
(lbm_server_*), or run the same stream back to back as plain single-lattice
runs, and report time-to-result percentiles and aggregate throughput.

Each request is a nozzle (or straight pipe) flow: throat diameter d, pipe
diameter D = 3 d, length 25 d, Reynolds number Re on the throat (throat mean
velocity 0.05 lattice units), parabolic inlet with 1 % noise started smoothly
over a quarter of the run (at most 8000 steps), a step count
and a storage precision (FP32 or FP16-shifted).  The scheduling itself (slot
table, admission by device footprint, batched launches, CUDA graph) lives in
the C++ server; this module only submits requests when they arrive, ticks
the server, and records completions.
"""
import time

import numpy as np

from . import inputs as I
from . import lbm

U_THROAT = 0.05


def request_geometry(spec):
    if spec["kind"] == "nozzle":
        return I.nozzle_flags(spec["D"], spec["d"], spec["L_total"])
    return I.pipe_flags(spec["D"], spec["L_total"])


def request_params(spec):
    d, D = spec["d"], spec["D"]
    return dict(Re=spec["Re"], u_char=U_THROAT, L_char=float(d), u_in=U_THROAT * (d / D) ** 2, d_in=float(D),
                profile="parabolic", noise_amp=0.01, noise_seed=1000 + spec["id"],
                inlet_ramp=min(8000, spec["steps"] // 4))


def run_stream(specs, budget_bytes, max_slots=32, steps_per_tick=32, precision=None, time_scale=1.0):
    """Serve the stream: request k is submitted once the wall clock passes
    its arrival time (scaled by time_scale); the server is ticked until every
    request is finished.  Returns per-request results and summary numbers."""
    geoms = [request_geometry(s) for s in specs]
    srv = lbm.Server(budget_bytes, max_slots=max_slots, steps_per_tick=steps_per_tick)
    order = sorted(range(len(specs)), key=lambda k: specs[k]["arrival"])
    ids, done = {}, {}
    t0 = time.perf_counter()
    nxt = 0
    try:
        while len(done) < len(specs):
            now = time.perf_counter() - t0
            while nxt < len(order) and specs[order[nxt]]["arrival"] * time_scale <= now:
                k = order[nxt]
                s = specs[k]
                ids[k] = srv.submit(geoms[k], s["steps"], precision or s["precision"], **request_params(s))
                s["submitted"] = now
                nxt += 1
            running, queued = srv.tick()
            now = time.perf_counter() - t0
            for k, rid in ids.items():
                if k in done:
                    continue
                state, steps_done = srv.poll(rid)
                if state in (lbm.LBM_REQ_DONE, lbm.LBM_REQ_FAILED, lbm.LBM_REQ_CANCELLED):
                    cells = srv.cells(rid)
                    res, err = None, None
                    try:  # releases the request whatever its outcome
                        res = srv.result(rid)
                    except lbm.LbmError as e:
                        err = e
                    done[k] = dict(state=state, finish=now, cells=cells, steps_done=steps_done, result=res,
                                   error=err)
            if running == 0 and queued == 0 and nxt < len(order):
                time.sleep(max(0.0, specs[order[nxt]]["arrival"] * time_scale - (time.perf_counter() - t0)))
        info = srv.info()
    finally:
        srv.close()
    lat = np.array([done[k]["finish"] - specs[k]["arrival"] * time_scale for k in range(len(specs))])
    # cell updates the server actually ran (a failed request stops early)
    updates = sum(done[k]["cells"] * done[k]["steps_done"] for k in range(len(specs)))
    makespan = max(done[k]["finish"] for k in done) - min(s["arrival"] * time_scale for s in specs)
    return dict(results=done, latency_p50_s=float(np.percentile(lat, 50)), latency_p99_s=float(np.percentile(lat, 99)),
                cell_updates=float(updates), makespan_s=float(makespan), mlups=updates / makespan / 1e6, info=info)


def run_back_to_back(specs, precision="fp32"):
    """The same requests one after another as plain single-lattice runs
    (geometry set-up, steps, readback of rho and u), in arrival order.
    precision None runs each request in its own storage precision.  Also
    returns the seconds spent outside the steps and readback (index build,
    allocation, initialisation, release)."""
    import torch

    t0 = time.perf_counter()
    updates = 0.0
    run_s = 0.0
    for s in sorted(specs, key=lambda s: s["arrival"]):
        flags = request_geometry(s)
        with lbm.Lattice(flags, precision or s["precision"]) as G:
            G.set_params(**request_params(s))
            G.init_equilibrium(1.0, (0.0, 0.0, 0.0)).sync()
            t1 = time.perf_counter()
            G.step(s["steps"])
            G.moments()
            run_s += time.perf_counter() - t1
            updates += G.n_active * s["steps"]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return dict(cell_updates=updates, seconds=dt, mlups=updates / dt / 1e6, setup_seconds=dt - run_s)
