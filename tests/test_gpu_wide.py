"""The 64-bit element-offset kernels (GPU required).

Lattices of 2^32 / 27 slots (~159 M) or more index their population arrays
with 64-bit offsets, through separate instantiations of the step kernels.
Such a lattice needs tens of gigabytes, so these tests switch the small
parity cases onto that path with LBM_WIDE_OFFSETS=1 (read when a context is
created) and hold them to the same tolerances as the 32-bit path.
"""
import numpy as np
import pytest

from paper_2204_10566_gb300 import inputs as I

from gpu_util import gpu_lattice, max_rel, oracle_lattice, random_state, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOX = 1
Q = 27


@pytest.fixture(scope="module")
def lbm():
    from paper_2204_10566_gb300 import build

    build.build()
    from paper_2204_10566_gb300 import lbm as m

    assert torch.cuda.is_available()
    return m


@pytest.fixture
def wide(monkeypatch):
    monkeypatch.setenv("LBM_WIDE_OFFSETS", "1")


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_wide_offsets_nee_duct(orc, lbm, wide, precision):
    flags = np.ones((12, 8, 8), dtype=np.uint8)
    flags[0] = 2
    flags[-1] = 3
    bc = dict(profile="parabolic", u_in=0.03, d_in=8.0, noise_amp=0.02, seed=77, rho_out=1.001)
    O = oracle_lattice(orc, flags, 0.03, periodic=3, **bc)
    G = gpu_lattice(lbm, flags, precision, 0.03, periodic=3, **bc)
    f0 = random_state(orc, flags, 3)
    O.set_populations(f0)
    G.set_populations(f0, layout=BOX)
    O.step(6)
    G.step(6).sync()
    act = flags.reshape(-1) != 0
    if precision == "fp64":
        assert max_rel(G.get_populations(BOX)[act], O.f[act]) < 1e-13
    else:
        tol = 1e-5 if precision == "fp32" else 1e-3
        assert rel_l2(G.moments(BOX)[1][act], O.moments()[act, 1:]) < tol


@pytest.mark.parametrize("ghost", [(1.0, 1.0, 1.0, 1.0), (0.8, 1.2, 1.5, 0.6)])
def test_wide_offsets_walls_and_ghost_rates(orc, lbm, wide, ghost):
    """Nozzle walls with interpolated links, and the general-rate collision."""
    D, d, L = 12, 4, 40
    flags = I.nozzle_flags(D, d, L)
    cells, q = I.nozzle_wall_q(D, d, L)
    wq = np.full((flags.size, Q), 128, dtype=np.uint8)
    wq[cells] = q
    bc = dict(profile="parabolic", u_in=0.01, d_in=float(D), noise_amp=0.02, seed=5)
    O = oracle_lattice(orc, flags, 0.02, ghost=ghost, wall_q=wq, **bc)
    G = gpu_lattice(lbm, flags, "fp64", 0.02, ghost=ghost, **bc)
    G.set_wall_q(cells, q)
    f0 = random_state(orc, flags, 19)
    O.set_populations(f0)
    G.set_populations(f0, layout=BOX)
    O.step(4)
    G.step(4).sync()
    act = flags.reshape(-1) != 0
    assert max_rel(G.get_populations(BOX)[act], O.f[act]) < 1e-12
