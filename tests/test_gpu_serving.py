"""Request server (continuous batching of many lattices, GPU required)."""
import numpy as np
import pytest

from paper_2204_10566_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2204_10566_gb300 import build

    build.build()
    from paper_2204_10566_gb300 import lbm, serving

    return lbm, serving


def tick_until(srv, done, timeout=120.0):
    """Tick the server until done() holds (indexes are built in a host worker
    thread, so a tick may find nothing to run yet)."""
    import time

    t0 = time.time()
    while not done():
        srv.tick()
        assert time.time() - t0 < timeout, "server made no progress"


def spec(k, kind, d, Re, steps, precision, L=10):
    return dict(id=k, arrival=0.0, kind=kind, d=d, D=3 * d, L_total=L * d, Re=Re, steps=steps, precision=precision)


MIX = [spec(0, "nozzle", 8, 800.0, 101, "fp32"), spec(1, "pipe", 6, 2000.0, 60, "fp16s"),
       spec(2, "nozzle", 10, 3000.0, 133, "fp32"), spec(3, "pipe", 8, 5000.0, 90, "fp16s"),
       spec(4, "nozzle", 6, 6500.0, 75, "fp16s")]


@pytest.mark.parametrize("kernel", ["tile", "pairs"])
def test_server_independent_of_the_contexts_fluid_kernel(mods, monkeypatch, kernel):
    """The server steps every lattice with its own multi-lattice kernels over
    all chunks and all inlet/outlet nodes, whatever fluid kernel the
    contexts would run alone (LBM_FLUID_KERNEL, read at context creation,
    changes a context's own chunk and node lists): the results are bitwise
    those of the default."""
    lbm, serving = mods
    ref = serving.run_stream([dict(s) for s in MIX], budget_bytes=4 << 30, steps_per_tick=16)
    monkeypatch.setenv("LBM_FLUID_KERNEL", kernel)
    got = serving.run_stream([dict(s) for s in MIX], budget_bytes=4 << 30, steps_per_tick=16)
    for k in range(len(MIX)):
        (ra, ua), (rb, ub) = ref["results"][k]["result"], got["results"][k]["result"]
        assert np.array_equal(ra, rb) and np.array_equal(ua, ub)
        assert np.abs(ua).max() > 0


def test_result_alone_equals_result_in_the_mix(mods):
    """Each lattice is updated by the same device code whatever else is
    resident: the result of a request served alone equals, bit for bit, its
    result in a mix of other nozzles and pipes of other sizes, Re, step
    counts and precisions; and it matches a plain lbm_step run of the same
    request within the storage precision's tolerance (the two kernels may
    contract floating-point operations differently)."""
    lbm, serving = mods
    mix = serving.run_stream([dict(s) for s in MIX], budget_bytes=4 << 30, steps_per_tick=16)
    for k in (0, 3):
        alone = serving.run_stream([dict(MIX[k])], budget_bytes=4 << 30, steps_per_tick=32)
        ra, ua = alone["results"][0]["result"]
        rm, um = mix["results"][k]["result"]
        assert np.array_equal(ra, rm) and np.array_equal(ua, um)
        s = MIX[k]
        with lbm.Lattice(serving.request_geometry(s), s["precision"]) as G:
            G.set_params(**serving.request_params(s))
            G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
            G.step(s["steps"])
            rp, up = G.moments()
        tol = 1e-5 if s["precision"] == "fp32" else 1e-3
        assert np.linalg.norm(up - um) / np.linalg.norm(up) < tol
        assert np.abs(rp - rm).max() < tol
        assert np.isfinite(um).all() and np.abs(um).max() > 0


def test_admission_respects_the_memory_budget(mods):
    lbm, serving = mods
    specs = [spec(k, "pipe" if k % 2 else "nozzle", 10, 1000.0 + 500 * k, 40 + 8 * k, "fp32") for k in range(6)]
    geom = serving.request_geometry(specs[0])
    info = lbm.check_layout(geom)
    one = 2 * 27 * 4 * info["slots"]
    budget = int(2.6 * one)              # room for about two lattices at a time
    out = serving.run_stream(specs, budget_bytes=budget, max_slots=8, steps_per_tick=8)
    assert all(r["state"] == lbm.LBM_REQ_DONE for r in out["results"].values())
    assert 0 < out["info"]["peak_bytes"] <= budget
    assert out["info"]["graph_captures"] == 1 and out["info"]["graph_launches"] == out["info"]["ticks"]


def test_submit_rejects_bad_requests(mods):
    lbm, serving = mods
    srv = lbm.Server(budget_bytes=1 << 20, max_slots=2, steps_per_tick=4)
    try:
        big = I.pipe_flags(30, 300)
        with pytest.raises(lbm.LbmError) as e:
            srv.submit(big, 10, "fp32", nu=0.01)
        assert e.value.status == lbm.LBM_ERR_OOM
        small = I.pipe_flags(6, 12)
        with pytest.raises(lbm.LbmError) as e:
            srv.submit(small, 10, "fp64", nu=0.01)
        assert e.value.status == lbm.LBM_ERR_ARG
        with pytest.raises(lbm.LbmError) as e:
            srv.submit(small, 10, "fp32", nu=0.01, ghost=(1.0, 1.2, 1.0, 1.0))
        assert e.value.status == lbm.LBM_ERR_ARG
        with pytest.raises(lbm.LbmError) as e:
            srv.submit(small, 10, "fp32", nu=-1.0)
        assert e.value.status == lbm.LBM_ERR_ARG
        with pytest.raises(lbm.LbmError) as e:
            srv.submit(small, 10, "fp16s", nu=0.01, fp16_scale=3000.0)
        assert e.value.status == lbm.LBM_ERR_ARG and "power of two" in str(e.value)
        with pytest.raises(lbm.LbmError) as e:
            srv.submit(small, 10, "fp32", nu=0.01, u_in=0.7)
        assert e.value.status == lbm.LBM_ERR_ARG and "sound speed" in str(e.value)
    finally:
        srv.close()


def test_cancel_queued_and_running(mods):
    lbm, serving = mods
    srv = lbm.Server(budget_bytes=2 << 30, max_slots=1, steps_per_tick=4)
    try:
        g = I.pipe_flags(12, 60)
        a = srv.submit(g, 400, "fp32", nu=0.02, u_in=0.01)
        b = srv.submit(g, 400, "fp32", nu=0.02, u_in=0.01)
        c = srv.submit(g, 8, "fp32", nu=0.02, u_in=0.01)
        tick_until(srv, lambda: srv.poll(a)[0] == lbm.LBM_REQ_RUNNING)
        assert srv.poll(a)[0] == lbm.LBM_REQ_RUNNING and srv.poll(b)[0] == lbm.LBM_REQ_QUEUED
        srv.cancel(a)
        srv.cancel(b)
        tick_until(srv, lambda: srv.poll(c)[0] == lbm.LBM_REQ_DONE)
        assert srv.poll(a)[0] == lbm.LBM_REQ_CANCELLED and srv.poll(b)[0] == lbm.LBM_REQ_CANCELLED
        assert srv.poll(c) == (lbm.LBM_REQ_DONE, 8)
        assert srv.info()["bytes_in_use"] == 0
    finally:
        srv.close()


def test_diverging_lattice_is_evicted_and_does_not_disturb_the_others(mods):
    """A lattice driven far beyond the low-Mach regime (host-side fault
    injection through its parameters) runs beside others.  The health check
    at the end of a tick finds its non-finite state: it is evicted and ends
    FAILED with LBM_ERR_UNSTABLE, its memory is freed, and the others'
    results are unchanged, bit for bit."""
    lbm, serving = mods
    base = [dict(MIX[0]), dict(MIX[1])]
    ref = serving.run_stream([dict(s) for s in base], budget_bytes=4 << 30, steps_per_tick=16)
    srv = lbm.Server(budget_bytes=4 << 30, max_slots=8, steps_per_tick=16)
    try:
        ids = [srv.submit(serving.request_geometry(s), s["steps"], s["precision"], **serving.request_params(s))
               for s in base]
        bad = srv.submit(I.pipe_flags(12, 40), 4000, "fp32", nu=1e-7, u_in=0.55, profile="plug")
        terminal = (lbm.LBM_REQ_DONE, lbm.LBM_REQ_FAILED)
        tick_until(srv, lambda: all(srv.poll(i)[0] in terminal for i in ids + [bad]))
        for k, i in enumerate(ids):
            assert srv.poll(i)[0] == lbm.LBM_REQ_DONE
            r, u = srv.result(i)
            rr, ur = ref["results"][k]["result"]
            assert np.array_equal(r, rr) and np.array_equal(u, ur)
        state, steps_done = srv.poll(bad)
        assert state == lbm.LBM_REQ_FAILED and 0 < steps_done < 4000
        with pytest.raises(lbm.LbmError) as e:
            srv.result(bad)
        assert e.value.status == lbm.LBM_ERR_UNSTABLE and "non-finite" in str(e.value)
        with pytest.raises(lbm.LbmError):  # released: the id is no longer known
            srv.poll(bad)
        tick_until(srv, lambda: srv.tick() == (0, 0))
        assert srv.info()["bytes_in_use"] == 0
    finally:
        srv.close()


def test_oversized_lattice_fails_without_running(mods):
    """A request whose index needs more slots than the server's 32-bit
    population offsets address passes submit's cheap checks (few active
    cells) and ends FAILED once its index is built; nothing is allocated for
    it and no kernel touches it.  Other requests are served normally."""
    lbm, serving = mods
    nx = (1 << 20) - 1
    f = np.zeros((11, 11, nx), dtype=np.uint8)
    f[:, :, 0] = 1
    f[:, :, -1] = 1
    srv = lbm.Server(budget_bytes=4 << 30, max_slots=4, steps_per_tick=8)
    try:
        big = srv.submit(f, 10, "fp32", nu=0.01)
        ok = srv.submit(I.pipe_flags(6, 12), 16, "fp32", nu=0.01, u_in=0.01)
        terminal = (lbm.LBM_REQ_DONE, lbm.LBM_REQ_FAILED)
        tick_until(srv, lambda: all(srv.poll(i)[0] in terminal for i in (big, ok)))
        assert srv.poll(big) == (lbm.LBM_REQ_FAILED, 0)
        with pytest.raises(lbm.LbmError) as e:
            srv.result(big)
        assert e.value.status == lbm.LBM_ERR_ARG and "storage slots" in str(e.value)
        assert srv.poll(ok)[0] == lbm.LBM_REQ_DONE
        assert srv.info()["peak_bytes"] < 1 << 24
    finally:
        srv.close()


def test_cancelled_requests_are_released(mods):
    lbm, serving = mods
    srv = lbm.Server(budget_bytes=1 << 30, max_slots=2, steps_per_tick=4)
    try:
        g = I.pipe_flags(8, 20)
        a = srv.submit(g, 100, "fp32", nu=0.02, u_in=0.01)
        srv.cancel(a)
        tick_until(srv, lambda: srv.poll(a)[0] == lbm.LBM_REQ_CANCELLED)
        with pytest.raises(lbm.LbmError) as e:
            srv.result(a)
        assert e.value.status == lbm.LBM_ERR_STATE and "cancelled" in str(e.value)
        with pytest.raises(lbm.LbmError) as e:
            srv.poll(a)
        assert e.value.status == lbm.LBM_ERR_ARG
    finally:
        srv.close()
