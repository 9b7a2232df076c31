"""Grid convergence and collision stability (GPU required).

Resolution ladder (the paper's grid study, Sec. 3, Table 2): the Re 6500
nozzle at the four levels R1-R4 of Table 2, throat diameters d = 18, 24, 36
and 52 cells (the table's 17.4, 23.2, 34.8 and 51.5 cells over a 4 mm
throat), each at its Table 2 throat velocity (the lattice speed its grid
spacing and time step give, half its CFL number: 0.124 at R1-R3, 0.118 at
R4), in the 60 d long domain of Sec. 2.2 (0.24 m over a 4 mm throat; R4 is
a 156 x 156 x 3120 box), walls interpolated on the smooth surface as in the
paper, and the same smooth inlet start in throat flow-through units.  The
time-averaged centreline velocity upstream of the sudden expansion, as a
function of z / d, converges towards R4 level by level; the paper reports
~3 % between its levels.

Ghost rates (Appendix A): relaxing every moment of order 3-6 to equilibrium
(rate 1, the paper's choice) keeps an under-resolved Taylor-Green vortex
stable where relaxing them at omega (lattice BGK with the same full Hermite
equilibrium) diverges.
"""
import os

import numpy as np
import pytest

from paper_2204_10566_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOX = 1
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
# Fluid and throat of Sec. 2.2 (SI): density, dynamic viscosity, throat diameter.
RHO, MU, D_THR = 1056.0, 3.5e-3, 0.004


@pytest.fixture(scope="module")
def lbm():
    from paper_2204_10566_gb300 import build

    build.build()
    from paper_2204_10566_gb300 import lbm as m

    assert torch.cuda.is_available()
    return m


def table2_re6500():
    """(delta_r, delta_t) in SI of Table 2's Re 6500 rows R1-R4 (tests/golden)."""
    rows = []
    with open(os.path.join(GOLDEN, "table2_resolutions.txt")) as fh:
        for ln in fh:
            if ln.strip() and not ln.lstrip().startswith("#"):
                lv, re_, dr, dt = ln.split()
                if float(re_) == 6500.0:
                    rows.append((float(dr) * 1e-4, float(dt) * 1e-6))
    return rows


def ladder_level(lbm, d, dr, dt, flow_units=30.0, Re=6500.0):
    """One level: the throat velocity of Table 2's (delta_r, delta_t) through
    lbm_params_from_physical, Re on the voxelised throat diameter d, 60 d long
    domain.  Returns z / d, the time-averaged centreline u_z / u_thr, and the
    expansion's z / d."""
    _, lu = lbm.params_from_physical(Re, dr, RHO, MU, D_THR, delta_t=dt)
    u = lu["u_char"]
    D, L = 3 * d, 60 * d
    flags = I.nozzle_flags(D, d, L)
    steps = int(flow_units * d / u)
    G = lbm.Lattice(flags, "fp32")
    G.set_params(Re=Re, u_char=u, L_char=float(d), u_in=u * (d / D) ** 2, d_in=float(D), profile="parabolic",
                 noise_amp=0.0, inlet_ramp=steps * 2 // 5)
    G.set_wall_q(*I.nozzle_wall_q(D, d, L, flags=flags))
    G.set_check_every(500)
    G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    G.step(steps // 2)
    G.stats_begin(1)
    G.step(steps - steps // 2).sync()
    m1, _, _ = G.stats_get(BOX)
    G.close()
    # the axis runs along the corner of the four middle cells
    line = m1.reshape(L, D, D)[:, D // 2 - 1:D // 2 + 1, D // 2 - 1:D // 2 + 1].mean(axis=(1, 2))
    z = (np.arange(L) + 0.5) / d
    return z, line / u, (D + I.cone_length(D, d) + 4 * d) / d, u


def test_resolution_ladder_table2(lbm):
    rows = table2_re6500()
    levels = [ladder_level(lbm, d, dr, dt) for d, (dr, dt) in zip(I.LADDER_THROAT_CELLS, rows)]
    z_exp = min(lv[2] for lv in levels)
    zq = np.linspace(0.5, z_exp - 0.5, 300)
    prof = [np.interp(zq, z, u) for z, u, _, _ in levels]
    assert np.isfinite(prof).all()
    err = [float(np.linalg.norm(p - prof[-1]) / np.linalg.norm(prof[-1])) for p in prof[:-1]]
    print("Table 2 ladder, Re 6500, u_thr %s: |Rk - R4| upstream of the expansion %s"
          % ([round(lv[3], 4) for lv in levels], [round(e, 4) for e in err]))
    for zz in (1.0, 4.0, 8.0, 11.0, z_exp - 0.5, z_exp + 2.0, z_exp + 5.0, z_exp + 10.0):
        print("  z/d %.1f: %s" % (zz, [round(float(np.interp(zz, z, u)), 4) for z, u, _, _ in levels]))
    assert err[0] > err[1] > err[2]  # converging towards the finest level
    assert err[2] < 0.03


def tgv_energy(lbm, n, Re, ghost, steps, u0=0.05):
    nu = u0 * n / (2 * np.pi) / Re
    k = 2 * np.pi / n
    c = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    u = np.stack([u0 * np.sin(k * X) * np.cos(k * Y) * np.cos(k * Z),
                  -u0 * np.cos(k * X) * np.sin(k * Y) * np.cos(k * Z), np.zeros_like(X)], axis=-1)
    G = lbm.Lattice(np.ones((n, n, n), dtype=np.uint8), "fp32", periodic=7)
    omega = 1.0 / (3.0 * nu + 0.5)
    G.set_params(nu=nu, ghost=ghost if ghost is not None else (omega,) * 4)
    G.init_fields(np.ones(n ** 3), u.reshape(-1, 3), layout=BOX)
    G.step(steps).sync()
    e = float((G.moments(BOX)[1] ** 2).sum()) / n ** 3
    G.close()
    return e


def test_unit_ghost_rates_stabilise_under_resolved_flow(lbm):
    n, steps = 64, 4000
    e0 = 0.05 ** 2 / 4  # mean u^2 of the initial field
    for Re in (1600.0, 20000.0, 200000.0):
        e_chm = tgv_energy(lbm, n, Re, (1.0, 1.0, 1.0, 1.0), steps)
        e_bgk = tgv_energy(lbm, n, Re, None, steps)
        print("TGV 64^3 Re %g: energy CHM ghost 1 %.4g, all rates omega %.4g" % (Re, e_chm, e_bgk))
        assert np.isfinite(e_chm) and 0.0 < e_chm < e0
    assert not (np.isfinite(e_bgk) and e_bgk < e0)  # all rates omega: diverged at Re 200 000
