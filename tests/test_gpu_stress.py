"""Full time-average statistics of the CUDA path (GPU required): mean
velocity, velocity products (Reynolds stress), viscous stress and density,
sampled inside the step kernel, against the oracle's per-step definitions
on the same seeded input; the mode switch, the checkpoint round trip and a
physical check of the viscous stress (a decaying shear wave).

Tolerances: FP64 storage reproduces the oracle to rounding (1e-12 relative
to each field's scale).  FP32 and FP16-shifted storage round every stored
population (relative 6e-8, resp. absolute 2^-11 / s per unit of deviation,
s = 4096); the stress is a difference of second moments of order
nu |grad u|, so its bound is set relative to the field's largest value:
1e-4 (FP32) and 5e-2 (FP16S) in relative L2.
"""
import numpy as np
import pytest

from paper_2204_10566_gb300 import inputs as I

from gpu_util import gpu_lattice, omega_of_nu, oracle_lattice, random_state, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOX = 1
FIELDS = ("u", "uu", "sigma", "rho")
TOL = {"fp64": 1e-12, "fp32": 1e-4, "fp16s": 5e-2}


@pytest.fixture(scope="module")
def lbm():
    from paper_2204_10566_gb300 import build

    build.build()
    from paper_2204_10566_gb300 import lbm as m

    assert torch.cuda.is_available()
    return m


def small_nozzle():
    """Inlet pipe, cone, throat and sudden expansion at 12 x 12 x 40 with the
    velocity inlet and pressure outlet (walls, ragged rows, boundary nodes)."""
    flags = I.nozzle_flags(12, 4, 40)
    bc = dict(profile="parabolic", u_in=0.01, d_in=12.0, noise_amp=0.05, seed=9)
    return flags, 0.02, bc


def run_full_stats(orc, lbm, flags, nu, precision, warm, steps, ghost=(1.0, 1.0, 1.0, 1.0), periodic=0, **bc):
    O = oracle_lattice(orc, flags, nu, periodic=periodic, ghost=ghost, **bc)
    f0 = random_state(orc, flags, 21, u_amp=0.02)
    O.set_populations(f0)
    G = gpu_lattice(lbm, flags, precision, nu, periodic=periodic, ghost=ghost, **bc)
    G.set_populations(f0, layout=BOX)
    O.step(warm)
    ref = O.step_sampled(steps)
    G.step(warm)
    G.stats_begin(1, full=True)
    G.step(steps).sync()
    got = G.stats_get_full(BOX)
    return ref, got, flags.reshape(-1) != 0


def compare(ref, got, act, tol, fields=FIELDS):
    for k in fields:
        a, b = got[k][act], ref[k][act]
        if tol <= 1e-10:
            err = np.abs(a - b).max() / np.abs(b).max()
        else:
            err = rel_l2(a, b)
        assert err < tol, (k, err)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_full_statistics_match_oracle(orc, lbm, precision):
    flags, nu, bc = small_nozzle()
    ref, got, act = run_full_stats(orc, lbm, flags, nu, precision, 3, 6, **bc)
    assert got["samples"] == 6
    tol = TOL[precision]
    compare(ref, got, act, tol, ("sigma",))
    compare(ref, got, act, 1e-12 if precision == "fp64" else (1e-5 if precision == "fp32" else 2e-3), ("u", "uu"))
    assert np.abs(got["rho"][act] - ref["rho"][act]).max() < (1e-13 if precision == "fp64" else 1e-5)
    r = got["reynolds"]
    u = got["u"]
    assert np.allclose(r[:, 3], got["rho"] * (got["uu"][:, 3] - u[:, 0] * u[:, 1]))
    assert np.all(got["sigma"][~act] == 0.0)


def test_full_statistics_general_ghost_rates(orc, lbm):
    """The general-rate collision (27-moment cascade) records the same
    stress definition."""
    flags, nu, bc = small_nozzle()
    ref, got, act = run_full_stats(orc, lbm, flags, nu, "fp64", 2, 4, ghost=(0.8, 1.2, 1.5, 0.6), **bc)
    compare(ref, got, act, 1e-12)


def test_statistics_mode_switch_and_errors(orc, lbm):
    flags, nu, bc = small_nozzle()
    G = gpu_lattice(lbm, flags, "fp32", nu, **bc)
    G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    G.stats_begin(1)                       # axial
    G.step(3)
    with pytest.raises(lbm.LbmError) as e:
        G.stats_get_full()
    assert e.value.status == lbm.LBM_ERR_STATE
    with pytest.raises(lbm.LbmError) as e:
        G.stats_begin(1, full=True)        # mode change while sampling
    assert e.value.status == lbm.LBM_ERR_STATE
    G.stats_end()
    G.stats_begin(1, full=True)            # new mode: samples restart
    G.step(2).sync()
    assert G.stats_get_full()["samples"] == 2
    m1, _, n = G.stats_get()               # the axial means stay readable
    assert n == 2 and np.allclose(m1, G.stats_get_full()["u"][:, 2])


def test_full_statistics_checkpoint_round_trip(lbm):
    flags, nu, bc = small_nozzle()
    A = gpu_lattice(lbm, flags, "fp32", nu, **bc)
    A.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    A.stats_begin(1, full=True)
    A.step(10)
    img = A.checkpoint()
    A.step(10).sync()
    B = gpu_lattice(lbm, flags, "fp32", nu, **bc)
    B.restore(img)
    B.step(10).sync()
    a, b = A.stats_get_full(), B.stats_get_full()
    assert a["samples"] == b["samples"] == 20
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_shear_wave_stress_on_gpu(lbm, precision):
    """Decaying shear wave u_x = U sin(k y) e^{-nu k^2 t} on a periodic
    64-cell box: the time-averaged sigma_xy equals rho nu d_y <u_x> within the
    second-order discretisation error (0.1 % at 64 cells)."""
    n, nu, U = 64, 0.02, 0.01
    k = 2 * np.pi / n
    c = np.arange(n) + 0.5
    flags = np.ones((2, n, 4), dtype=np.uint8)
    G = gpu_lattice(lbm, flags, precision, nu, periodic=7)
    u = np.zeros((2, n, 4, 3))
    u[..., 0] = (U * np.sin(k * c))[None, :, None]
    G.init_fields(np.ones(flags.size), u.reshape(-1, 3), layout=BOX)
    G.step(50)
    G.stats_begin(1, full=True)
    G.step(20).sync()
    s = G.stats_get_full(BOX)
    ux = s["u"][:, 0].reshape(2, n, 4)[0, :, 0]
    sxy = s["sigma"][:, 3].reshape(2, n, 4)[0, :, 0]
    A = (ux * np.sin(k * c)).sum() / (np.sin(k * c) ** 2).sum()
    B = (sxy * np.cos(k * c)).sum() / (np.cos(k * c) ** 2).sum()
    assert abs(B / (nu * A * k) - 1.0) < 2e-3
    assert np.abs(s["sigma"][:, [0, 1, 2, 4, 5]]).max() < 1e-3 * abs(B)
