"""Device-allocation failures, injected on the host through the allocator
callback of lbm_desc / lbm_server_desc (no GPU fault is involved): the k-th
allocation returns NULL.  Every entry point that allocates must then return
LBM_ERR_OOM, free whatever it had allocated in that call, and leave the
context (or the server) usable."""
import numpy as np
import pytest

from paper_2204_10566_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_2204_10566_gb300 import build

    build.build()
    from paper_2204_10566_gb300 import lbm as m

    return m


def failing_allocator(lbm, fail_at=()):
    """PyTorch's caching allocator behind a counter: call k (1-based) in
    fail_at returns NULL; live maps each pointer handed out to its size."""

    class Counting(lbm.TorchAllocator):
        def __init__(self):
            super().__init__(0, torch.cuda.current_stream(0))
            self.calls = 0
            self.fail_at = set(fail_at)
            self.live = {}

        def _do_alloc(self, nbytes, user):
            self.calls += 1
            if self.calls in self.fail_at:
                return None
            p = super()._do_alloc(nbytes, user)
            if p:
                self.live[p] = nbytes
            return p

        def _do_free(self, ptr, user):
            assert ptr in self.live, "freed a pointer the allocator never handed out"
            del self.live[ptr]
            super()._do_free(ptr, user)

    return Counting()


FLAGS = I.nozzle_flags(12, 4, 40)


def test_every_geometry_allocation_failure_is_clean(lbm):
    probe = failing_allocator(lbm)
    with lbm.Lattice(FLAGS, "fp32", allocator=probe) as G:
        n_geom = probe.calls
        held = dict(probe.live)
        assert G.layout_info()["device_bytes"] == sum(held.values())
    assert n_geom >= 8 and probe.live == {}
    for k in range(1, n_geom + 1):
        a = failing_allocator(lbm, {k})
        with pytest.raises(lbm.LbmError) as e:
            lbm.Lattice(FLAGS, "fp16s", allocator=a)
        assert e.value.status == lbm.LBM_ERR_OOM, k
        assert a.live == {}, (k, a.live)


def test_failures_after_set_up_keep_the_context_usable(lbm):
    a = failing_allocator(lbm)
    G = lbm.Lattice(FLAGS, "fp32", allocator=a)
    try:
        G.set_params(nu=0.02, u_in=0.01)
        G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
        G.step(4).sync()
        held = dict(a.live)
        # statistics accumulators
        a.fail_at = {a.calls + 1}
        with pytest.raises(lbm.LbmError) as e:
            G.stats_begin(1)
        assert e.value.status == lbm.LBM_ERR_OOM and a.live == held
        # readback staging
        a.fail_at = {a.calls + 1}
        with pytest.raises(lbm.LbmError) as e:
            G.moments()
        assert e.value.status == lbm.LBM_ERR_OOM and a.live == held
        # host-side field upload staging
        a.fail_at = {a.calls + 1}
        with pytest.raises(lbm.LbmError) as e:
            G.init_fields(np.ones(G.n_active), np.zeros((G.n_active, 3)))
        assert e.value.status == lbm.LBM_ERR_OOM and a.live == held
        # the context still works: the same state as a run that saw no failure
        a.fail_at = set()
        G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
        G.step(4).sync()
        rho, u = G.moments()
        with lbm.Lattice(FLAGS, "fp32") as R:
            R.set_params(nu=0.02, u_in=0.01)
            R.init_equilibrium(1.0, (0.0, 0.0, 0.0))
            R.step(4).sync()
            rho_r, u_r = R.moments()
        assert np.array_equal(rho, rho_r) and np.array_equal(u, u_r) and np.abs(u).max() > 0
        G.stats_begin(1)
        G.step(2).sync()
        assert G.stats_get()[2] == 2
    finally:
        G.close()
    assert a.live == {}


def test_server_admission_failure(lbm):
    """An allocation failure while admitting a request ends that request
    FAILED with LBM_ERR_OOM, holding nothing; the next request is served."""
    a = failing_allocator(lbm, {3})
    srv = lbm.Server(budget_bytes=1 << 30, max_slots=2, steps_per_tick=4, allocator=a)
    try:
        g = I.pipe_flags(8, 24)
        r1 = srv.submit(g, 8, "fp32", nu=0.02, u_in=0.01)
        r2 = srv.submit(g, 8, "fp32", nu=0.02, u_in=0.01)
        terminal = (lbm.LBM_REQ_DONE, lbm.LBM_REQ_FAILED)
        import time

        t0 = time.time()
        while not all(srv.poll(r)[0] in terminal for r in (r1, r2)):
            srv.tick()
            assert time.time() - t0 < 60
        assert srv.poll(r1)[0] == lbm.LBM_REQ_FAILED
        with pytest.raises(lbm.LbmError) as e:
            srv.result(r1)
        assert e.value.status == lbm.LBM_ERR_OOM
        assert srv.poll(r2)[0] == lbm.LBM_REQ_DONE
        rho, u = srv.result(r2)
        assert np.isfinite(u).all()
        assert srv.info()["bytes_in_use"] == 0 and a.live == {}
    finally:
        srv.close()
    assert a.live == {}
