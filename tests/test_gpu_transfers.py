"""Host transfers of the fields (GPU required): lbm_init_fields and
lbm_get_moments in active order copy the caller's arrays as they are (one
copy per array, the moments split on the device), in box order through a
host repack.  Both orders give the same state and the same moments, and
pinned and pageable host arrays give the same results."""
import numpy as np
import pytest

from paper_2204_10566_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOX, ACTIVE = 1, 0


@pytest.fixture(scope="module")
def lbm():
    from paper_2204_10566_gb300 import build

    build.build()
    from paper_2204_10566_gb300 import lbm as m

    assert torch.cuda.is_available()
    return m


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_active_and_box_orders_agree(lbm, precision):
    flags = I.nozzle_flags(12, 4, 40)
    act = flags.reshape(-1) != 0
    n = int(act.sum())
    rho = I.random_density_field(n, 0.01, 5)
    u = I.random_velocity_field(n, 0.02, 6)
    rho_box = np.zeros(flags.size)
    u_box = np.zeros((flags.size, 3))
    rho_box[act], u_box[act] = rho, u
    out = []
    for layout, (r, v) in ((ACTIVE, (rho, u)), (BOX, (rho_box, u_box))):
        G = lbm.Lattice(flags, precision)
        G.set_params(nu=0.02, u_in=0.01, d_in=12.0)
        G.init_fields(r, v, layout=layout)
        G.step(3).sync()
        out.append((G.get_populations(ACTIVE), G.moments(ACTIVE), G.moments(BOX)))
        G.close()
    (fa, (ra, ua), (rab, uab)), (fb, (rb, ub), (rbb, ubb)) = out
    assert np.array_equal(fa, fb)
    assert np.array_equal(ra, rb) and np.array_equal(ua, ub)
    assert np.array_equal(ra, rab[act]) and np.array_equal(ua, uab[act])
    assert np.array_equal(rbb, rab) and not rab[~act].any() and not uab[~act].any()


def test_pinned_host_arrays(lbm):
    """The benchmark's end-to-end path: fields from pinned host memory in,
    moments into pinned host memory out, equal to the pageable-array run."""
    flags = I.nozzle_flags(12, 4, 40)
    n = int((flags != 0).sum())
    rho = I.random_density_field(n, 0.01, 7)
    u = I.random_velocity_field(n, 0.02, 8)
    rho_p = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    u_p = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    rho_p[:], u_p[:] = rho, u
    ro = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    uo = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    G = lbm.Lattice(flags, "fp32")
    G.set_params(nu=0.02, u_in=0.01, d_in=12.0)
    G.init_fields(rho_p, u_p).step(4)
    G.moments(out=(ro, uo))
    H = lbm.Lattice(flags, "fp32")
    H.set_params(nu=0.02, u_in=0.01, d_in=12.0)
    H.init_fields(rho, u).step(4)
    rh, uh = H.moments()
    assert np.array_equal(ro, rh) and np.array_equal(uo, uh)
    G.close()
    H.close()
