"""CUDA path vs the FP64 oracle, through the C ABI (GPU required).

Tolerances (stated for the method): FP64 storage <= 1e-12 relative per
population after 100 steps; FP32 <= 1e-5 relative L2 on the velocity after
100 laminar steps; FP16-shifted <= 1e-3 relative L2 on the velocity.
Integer work (geometry, index, noise draws) must match exactly.
"""
import numpy as np
import pytest

from paper_2204_10566_gb300 import inputs as I

from gpu_util import (gpu_lattice, max_rel, omega_of_nu, oracle_cell_update, oracle_lattice, random_state,
                      rel_l2)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOX = 1  # LBM_LAYOUT_BOX


@pytest.fixture(scope="module")
def lbm():
    from paper_2204_10566_gb300 import build

    build.build()
    from paper_2204_10566_gb300 import lbm as m

    assert torch.cuda.is_available()
    return m


def run_both(orc, lbm, flags, precision, steps, nu=0.02, periodic=0, seed=0, ghost=(1.0, 1.0, 1.0, 1.0),
             rows="auto", **bc):
    O = oracle_lattice(orc, flags, nu, periodic=periodic, ghost=ghost, **bc)
    f0 = random_state(orc, flags, seed)
    O.set_populations(f0)
    G = gpu_lattice(lbm, flags, precision, nu, periodic=periodic, ghost=ghost, rows=rows, **bc)
    G.set_populations(f0, layout=BOX)
    O.step(steps)
    G.step(steps).sync()
    act = flags.reshape(-1) != 0
    return O, G, act


def ragged_flags():
    """Rows of odd lengths and offsets, an interior hole and a bump: several
    chunks per row, ragged tails, padding slots inside row spans."""
    g = np.random.default_rng(12)
    f = np.ones((9, 11, 37), dtype=np.uint8)
    f[:, :, :3] = 0
    f[:, 4:7, 15:18] = 0          # a hole inside the row spans
    f[2:4, 1, 30:] = 0            # ragged row ends
    f[5, 9, 5:11] = 0
    f[g.random(f.shape) < 0.03] = 0
    return f


@pytest.mark.parametrize("rows", ["x", "z"])
@pytest.mark.parametrize("ghost", [(1.0, 1.0, 1.0, 1.0), (0.8, 1.2, 1.5, 0.6)])
def test_periodic_fp64_elementwise(orc, lbm, ghost, rows):
    flags = np.ones((5, 6, 13), dtype=np.uint8)
    O, G, act = run_both(orc, lbm, flags, "fp64", 3, periodic=7, ghost=ghost, rows=rows)
    fg = G.get_populations(BOX)
    assert max_rel(fg[act], O.f[act]) < 1e-13


@pytest.mark.parametrize("rows", ["x", "z"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 2e-6), ("fp16s", 3e-3)])
def test_walls_ragged_rows(orc, lbm, precision, tol, rows):
    flags = ragged_flags()
    O, G, act = run_both(orc, lbm, flags, precision, 4, nu=0.05, rows=rows)
    fg = G.get_populations(BOX)
    assert max_rel(fg[act], O.f[act]) < tol
    rho, u = G.moments(BOX)
    mo = O.moments()
    if precision == "fp64":
        assert np.abs(rho[act] - mo[act, 0]).max() < 1e-14
        assert np.abs(u[act] - mo[act, 1:]).max() < 1e-14


@pytest.mark.parametrize("rows", ["x", "z"])
@pytest.mark.parametrize("precision,ramp", [("fp64", 0), ("fp32", 0), ("fp16s", 0), ("fp64", 4), ("fp32", 4)])
def test_nee_duct_parabolic_noise(orc, lbm, precision, ramp, rows):
    """Velocity inlet (parabolic profile + seeded noise, impulsive or ramped
    start) and pressure outlet by non-equilibrium extrapolation, periodic
    cross-section."""
    flags = np.ones((12, 8, 8), dtype=np.uint8)
    flags[0] = 2
    flags[-1] = 3
    bc = dict(profile="parabolic", u_in=0.03, d_in=8.0, noise_amp=0.02, seed=77, rho_out=1.001, ramp=ramp)
    O, G, act = run_both(orc, lbm, flags, precision, 6, nu=0.03, periodic=3, rows=rows, **bc)
    fg = G.get_populations(BOX)
    rho, u = G.moments(BOX)
    mo = O.moments()
    if precision == "fp64":
        assert max_rel(fg[act], O.f[act]) < 1e-13
    else:
        tol = 1e-5 if precision == "fp32" else 1e-3
        assert rel_l2(u[act], mo[act, 1:]) < tol


@pytest.mark.parametrize("rows", ["x", "z"])
def test_noise_draws_bit_exact(orc, lbm, rows):
    """The inlet perturbation is integer work: the boundary velocity the GPU
    imposes equals the oracle's prescribed value to FP64 rounding at every
    inlet node, for several steps (a single wrong bit of the hash would
    show as an O(noise) difference)."""
    flags = np.ones((6, 5, 7), dtype=np.uint8)
    flags[0] = 2
    flags[-1] = 3
    bc = dict(profile="plug", u_in=0.02, noise_amp=0.5, seed=123456789)
    O, G, act = run_both(orc, lbm, flags, "fp64", 3, nu=0.05, periodic=3, rows=rows, **bc)
    rho, u = G.moments(BOX)
    inlet = flags.reshape(-1) == 2
    assert np.abs(u[inlet] - O.moments()[inlet, 1:]).max() < 1e-15


def nozzle_re500_setup():
    w = I.WORKLOADS["nozzle_re500_24x24x160"]
    nu = w["u_throat"] * w["d"] / w["Re"]
    bc = dict(profile="plug", u_in=I.inlet_mean_velocity(w))
    return I.workload_flags("nozzle_re500_24x24x160"), nu, bc


@pytest.fixture(scope="module")
def re500_oracle(orc):
    """The Re 500 laminar nozzle, 100 steps from rest, on the oracle."""
    flags, nu, bc = nozzle_re500_setup()
    O = oracle_lattice(orc, flags, nu, **bc)
    O.init_equilibrium(1.0, [0.0, 0.0, 0.0])
    O.step(100)
    return flags, O


@pytest.mark.parametrize("rows", ["x", "z"])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_nozzle_re500_100_steps(lbm, re500_oracle, precision, rows):
    flags, O = re500_oracle
    _, nu, bc = nozzle_re500_setup()
    G = gpu_lattice(lbm, flags, precision, nu, rows=rows, **bc)
    G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    G.step(100).sync()
    act = flags.reshape(-1) != 0
    rho, u = G.moments(BOX)
    mo = O.moments()
    e_u = rel_l2(u[act], mo[act, 1:])
    if precision == "fp64":
        assert max_rel(G.get_populations(BOX)[act], O.f[act]) < 1e-12
    elif precision == "fp32":
        assert e_u < 1e-5
    else:
        assert e_u < 1e-3
    assert np.isfinite(rho).all()


def test_totals_and_health(orc, lbm):
    flags = ragged_flags()
    O, G, act = run_both(orc, lbm, flags, "fp64", 2, nu=0.05)
    m, mom = G.totals()
    ref = O.totals()
    assert abs(m - ref[0]) < 1e-11 * abs(ref[0])
    assert np.abs(mom - ref[1:]).max() < 1e-12 * abs(ref[0])
    h = G.health()
    assert h[5] == 0.0 and h[4] > 0.0
    # closed box with walls: mass is conserved by the step (to rounding)
    G.step(5).sync()
    assert abs(G.totals()[0] - m) < 1e-11 * m


def test_fused_health_check(orc, lbm):
    flags = ragged_flags()
    O, G, act = run_both(orc, lbm, flags, "fp32", 1, nu=0.05)
    G.set_check_every(2)
    G.step(4).sync()
    h = G.health()
    m, mom = G.totals()
    assert abs(h[0] - m) < 1e-6 * m and h[5] == 0.0


def test_unstable_state_is_reported(orc, lbm):
    flags = np.ones((4, 4, 8), dtype=np.uint8)
    f = random_state(orc, flags, 3)
    f[17, 5] = np.nan
    G = gpu_lattice(lbm, flags, "fp32", 0.05, periodic=7)
    G.set_populations(f, layout=BOX)
    G.set_check_every(1)
    G.step(2)
    with pytest.raises(lbm.LbmError) as e:
        G.sync()
    assert e.value.status == lbm.LBM_ERR_UNSTABLE


def test_statistics_match_oracle_samples(orc, lbm):
    flags = np.ones((10, 6, 6), dtype=np.uint8)
    flags[0] = 2
    flags[-1] = 3
    bc = dict(profile="parabolic", u_in=0.02, d_in=6.0, noise_amp=0.05, seed=4)
    O, G, act = run_both(orc, lbm, flags, "fp64", 2, nu=0.04, periodic=3, **bc)
    G.stats_begin(2)
    s1 = np.zeros(flags.size)
    s2 = np.zeros(flags.size)
    k = 0
    for step in range(1, 9):
        O.step(1)
        if (step - 1) % 2 == 0:
            uz = O.moments()[:, 3]
            s1 += uz
            s2 += uz * uz
            k += 1
    G.step(8).sync()
    m1, m2, n = G.stats_get(BOX)
    assert n == k == 4
    assert np.abs(m1[act] - s1[act] / k).max() < 1e-15
    assert np.abs(m2[act] - s2[act] / k).max() < 1e-16


@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
def test_checkpoint_restore_bitwise(orc, lbm, precision):
    flags, nu, bc = nozzle_re500_setup()
    A = gpu_lattice(lbm, flags, precision, nu, **bc)
    A.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    A.stats_begin(1)
    A.step(20)
    img = A.checkpoint()
    A.step(20).sync()
    B = gpu_lattice(lbm, flags, precision, nu, **bc)
    B.restore(img)
    assert B.step_count() == 20
    B.step(20).sync()
    assert np.array_equal(A.get_populations(), B.get_populations())
    assert np.array_equal(A.stats_get()[0], B.stats_get()[0])


def test_fp16s_rest_state_exact(lbm):
    flags = I.nozzle_flags(12, 4, 40, inlet=False, outlet=False)
    G = gpu_lattice(lbm, flags, "fp16s", 0.01, fp16_scale=1024.0)
    G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    f0 = G.get_populations()
    G.step(10).sync()
    assert np.array_equal(G.get_populations(), f0)


def test_geometry_errors(lbm):
    bad = np.ones((4, 4, 4), dtype=np.uint8)
    bad[0, 0, 0] = 2    # inlet whose axis neighbours are all fluid: ambiguous partner
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(bad, "fp32")
    assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(np.zeros((3, 3, 3), dtype=np.uint8), "fp32")
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(np.full((3, 3, 3), 9, dtype=np.uint8), "fp32")
    G = lbm.Lattice(np.ones((3, 3, 8), dtype=np.uint8), "fp32", periodic=7)
    with pytest.raises(lbm.LbmError) as e:
        G.step(1)
    assert e.value.status == lbm.LBM_ERR_STATE
    with pytest.raises(lbm.LbmError) as e:
        G.set_params(nu=-1.0, Re=0.0)
    assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError) as e:
        G.set_params(nu=0.01, u_in=0.7)   # faster than the lattice sound speed
    assert e.value.status == lbm.LBM_ERR_ARG
    G.set_params(nu=0.01)
    G.init_equilibrium()
    G.step(0).sync()
    assert G.step_count() == 0


# --------------------------------------------------- full-size sampled parity

@pytest.mark.parametrize("name,precision", [("nozzle_re3500_96x96x800", "fp32"),
                                            ("nozzle_re6500_144x144x1200", "fp32"),
                                            ("nozzle_re6500_144x144x1200", "fp16s")])
def test_full_size_sampled_cells(orc, lbm, name, precision):
    """Full-size nozzle in the launch configuration the benchmark times:
    random rho, u fields, two steps; the second step's output at sampled
    cells (interior, wall-adjacent, inlet, outlet) against the oracle's
    single-cell update of the GPU's own first-step state."""
    w = I.WORKLOADS[name]
    flags = I.workload_flags(name)
    nu = w["u_throat"] * w["d"] / w["Re"]
    bc = dict(profile=w["profile"], u_in=I.inlet_mean_velocity(w), d_in=float(w["D"]), noise_amp=w["noise"],
              seed=w["seed"], rho_out=1.0, ramp=w.get("ramp", 0))
    G = gpu_lattice(lbm, flags, precision, nu, **bc)
    n = G.n_active
    G.init_fields(I.random_density_field(n, 0.01, 5), I.random_velocity_field(n, 0.02, 6))
    G.step(1).sync()
    f1 = G.get_populations(BOX)
    G.step(1).sync()
    act_idx = np.nonzero(flags.reshape(-1) != 0)[0]
    g = np.random.default_rng(9)
    pick = list(g.choice(act_idx, 200, replace=False))
    pick += list(np.nonzero(flags.reshape(-1) == 2)[0][:20]) + list(np.nonzero(flags.reshape(-1) == 3)[0][:20])
    nz, ny, nx = flags.shape
    inlet = dict(profile=w["profile"], u_in=bc["u_in"], d_in=float(w["D"]), axis=(nx / 2, ny / 2),
                 noise_amp=w["noise"], seed=w["seed"], rho_out=1.0, ramp=bc["ramp"])
    f2 = G.get_populations(BOX)
    errs = []
    for b in pick:
        z, y, x = b // (nx * ny), (b // nx) % ny, b % nx
        ref, mom = oracle_cell_update(orc, f1, flags, x, y, z, 0, omega_of_nu(nu), inlet=inlet, t_new=2)
        errs.append(np.abs(f2[b] - ref).max() / np.abs(ref).max())
    tol = 2e-6 if precision == "fp32" else 2e-3
    assert max(errs) < tol
