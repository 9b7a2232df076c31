"""Flow-level checks of the CUDA path (GPU required): periodic Taylor-Green
vortices against the oracle and the exact decay, and the time-averaged axial
velocity of the transitional / turbulent nozzles across storage precisions.
Pointwise agreement is lost to chaos there; the averaged radial profiles of
FP32 and FP16S must agree with the FP64 GPU run within 2 % where the
averages converge within the window (upstream of the sudden expansion and
the jet's near field), and within the run-to-run variability further
downstream."""
import numpy as np
import pytest

from paper_2204_10566_gb300 import inputs as I

from gpu_util import gpu_lattice, max_rel, omega_of_nu, oracle_cell_update, oracle_lattice, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOX = 1


@pytest.fixture(scope="module")
def lbm():
    from paper_2204_10566_gb300 import build

    build.build()
    from paper_2204_10566_gb300 import lbm as m

    return m


def tgv3d_fields(n, u0):
    """3-D Taylor-Green vortex initial field on an n^3 periodic box (cell
    centres), with the pressure of the incompressible solution."""
    k = 2 * np.pi / n
    c = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    u = np.stack([u0 * np.sin(k * X) * np.cos(k * Y) * np.cos(k * Z),
                  -u0 * np.cos(k * X) * np.sin(k * Y) * np.cos(k * Z),
                  np.zeros_like(X)], axis=-1).reshape(-1, 3)
    p = u0 ** 2 / 16.0 * (np.cos(2 * k * X) + np.cos(2 * k * Y)) * (np.cos(2 * k * Z) + 2.0)
    rho = (1.0 + 3.0 * p).reshape(-1)
    return rho, u


@pytest.fixture(scope="module")
def tgv64_oracle(orc):
    n, u0, Re = 64, 0.04, 400.0
    nu = u0 * n / (2 * np.pi) / Re
    flags = np.ones((n, n, n), dtype=np.uint8)
    rho, u = tgv3d_fields(n, u0)
    O = oracle_lattice(orc, flags, nu, periodic=7)
    O.init_equilibrium(rho, u)
    f0 = O.f.copy()
    O.step(4)
    return flags, nu, rho, u, f0, O


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_tgv64_against_oracle(lbm, tgv64_oracle, precision):
    """Taylor-Green vortex at 64^3, Re 400, four steps from the same initial
    populations: FP64 elementwise, FP32 / FP16S on the velocity."""
    flags, nu, rho, u, f0, O = tgv64_oracle
    G = gpu_lattice(lbm, flags, precision, nu, periodic=7)
    G.set_populations(f0, layout=BOX)
    G.step(4).sync()
    if precision == "fp64":
        assert max_rel(G.get_populations(BOX), O.f) < 1e-12
    else:
        _, ug = G.moments(BOX)
        tol = 1e-5 if precision == "fp32" else 1e-3
        assert rel_l2(ug, O.moments()[:, 1:]) < tol


TGV_N, TGV_U0 = 256, 0.04


@pytest.fixture(scope="module")
def tgv256_fields():
    return tgv3d_fields(TGV_N, TGV_U0)


def tgv256_nu(Re):
    """nu of the 256^3 vortex at Re = u0 / (k nu)."""
    return TGV_U0 / (2 * np.pi / TGV_N * Re)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_tgv256_sampled_cells(orc, lbm, tgv256_fields, precision):
    """Taylor-Green vortex at the full 256^3 size (u0 = 0.04, Re 1600), in
    the launch configuration of a plain step: the second step's output at 200
    sampled cells against the oracle's single-cell update of the GPU's own
    first-step state."""
    n, nu = TGV_N, tgv256_nu(1600.0)
    flags = np.ones((n, n, n), dtype=np.uint8)
    G = gpu_lattice(lbm, flags, precision, nu, periodic=7)
    G.init_fields(*tgv256_fields, layout=BOX)
    G.step(1).sync()
    f1 = G.get_populations(BOX)
    G.step(1).sync()
    f2 = G.get_populations(BOX)
    G.close()
    pick = np.random.default_rng(11).choice(flags.size, 200, replace=False)
    errs = []
    for b in pick:
        z, y, x = b // (n * n), (b // n) % n, b % n
        ref, _ = oracle_cell_update(orc, f1, flags, x, y, z, 7, omega_of_nu(nu))
        errs.append(np.abs(f2[b] - ref).max() / np.abs(ref).max())
    tol = {"fp64": 1e-13, "fp32": 2e-6, "fp16s": 2e-3}[precision]
    print("TGV 256^3 sampled cells %s: max rel %.3g" % (precision, max(errs)))
    assert max(errs) < tol


def tgv256_run(lbm, fields, precision, Re, s0, s1):
    """Mean kinetic energy <|u|^2> at steps s0 and s1 and the velocity at s1."""
    n = TGV_N
    G = gpu_lattice(lbm, np.ones((n, n, n), dtype=np.uint8), precision, tgv256_nu(Re), periodic=7)
    G.init_fields(*fields, layout=BOX)
    G.step(s0).sync()
    e0 = float(np.mean(np.einsum("ij,ij->i", *(2 * (G.moments(BOX)[1],)))))
    G.step(s1 - s0).sync()
    u1 = G.moments(BOX)[1]
    G.close()
    return e0, float(np.mean(np.einsum("ij,ij->i", u1, u1))), u1


@pytest.mark.parametrize("Re", [100.0, 400.0, 1600.0])
def test_tgv256_precision_sweep_and_initial_decay(lbm, tgv256_fields, Re):
    """Taylor-Green vortex, 256^3, u0 = 0.04, Re 100 / 400 / 1600, in FP64,
    FP32 and FP16S storage.

    Precision sweep: the FP32 and FP16S velocities at step 120 against the
    FP64 run (measured 7.5e-6 and 6-7e-4 rel. L2 at all three Re).

    Exact decay: at t = 0 the vortex has no enstrophy production, so its
    kinetic energy first decays at d ln E / dt = -6 nu k^2, the viscous
    dissipation of the initial field.  At Re 100 the rate over steps 20-120
    (under 0.12 of the eddy time 1/(u0 k)) matches it: measured 1.0005 (FP64)
    and 0.998 (FP32).  The run starts from f^eq, without the non-equilibrium
    part, and that initial layer of the second-order moments decays as
    |1 - omega|^t.  At Re 400 and 1600 (omega = 1.95 and 1.99) it outlasts
    the window while the viscous loss over it is only 1.5e-3 and 3.7e-4 of
    E, so the rate there reads 1.07 and 1.45 and is reported, not checked.
    FP16S storage noise adds energy and lowers its measured rate (0.90)."""
    s0, s1 = 20, 120
    k = 2 * np.pi / TGV_N
    exact = 6.0 * tgv256_nu(Re) * k * k
    res = {p: tgv256_run(lbm, tgv256_fields, p, Re, s0, s1) for p in ("fp64", "fp32", "fp16s")}
    rate = {p: -np.log(r[1] / r[0]) / (s1 - s0) / exact for p, r in res.items()}
    d32 = rel_l2(res["fp32"][2], res["fp64"][2])
    d16 = rel_l2(res["fp16s"][2], res["fp64"][2])
    print("TGV 256^3 Re %g: decay rate / exact FP64 %.5f FP32 %.5f FP16S %.5f; |u32-u64| %.3g |u16-u64| %.3g"
          % (Re, rate["fp64"], rate["fp32"], rate["fp16s"], d32, d16))
    assert d32 < 3e-5
    assert d16 < 3e-3
    if Re == 100.0:
        assert abs(rate["fp64"] - 1.0) < 0.01
        assert abs(rate["fp32"] - 1.0) < 0.01


@pytest.mark.parametrize("n", [64, 128])
def test_tgv2d_decay_rate(lbm, n):
    """2-D Taylor-Green vortex (uniform in z; an exact Navier-Stokes
    solution): kinetic energy decays as exp(-4 nu k^2 t).  FP32 on the GPU."""
    u0 = 0.02
    nu = 0.01 * n / 64.0
    k = 2 * np.pi / n
    c = np.arange(n) + 0.5
    Y, X = np.meshgrid(c, c, indexing="ij")
    ux = u0 * np.sin(k * X) * np.cos(k * Y)
    uy = -u0 * np.cos(k * X) * np.sin(k * Y)
    rho = 1.0 - 3.0 * u0 ** 2 / 4.0 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    nz = 4
    flags = np.ones((nz, n, n), dtype=np.uint8)
    u = np.zeros((nz, n, n, 3))
    u[..., 0] = ux
    u[..., 1] = uy
    G = gpu_lattice(lbm, flags, "fp32", nu, periodic=7)
    G.init_fields(np.broadcast_to(rho, (nz, n, n)).reshape(-1), u.reshape(-1, 3), layout=BOX)
    steps = int(0.5 / (nu * k * k))
    G.step(steps // 4).sync()
    e0 = (G.moments(BOX)[1] ** 2).sum()
    G.step(steps - steps // 4).sync()
    e1 = (G.moments(BOX)[1] ** 2).sum()
    rate = -np.log(e1 / e0) / (4 * (steps - steps // 4)) / (nu * k * k)
    assert abs(rate - 1.0) < 5e-3


def duct_exact_shape(n, terms=40):
    """Fourier-series solution for laminar flow in a square duct of side n,
    walls at the cell faces, at the cell centres (up to a factor)."""
    c = np.arange(n) + 0.5 - n / 2.0
    Y, X = np.meshgrid(c, c, indexing="ij")
    u = np.zeros_like(X)
    for k in range(terms):
        m = 2 * k + 1
        u += (-1) ** k / m ** 3 * (1 - np.cosh(m * np.pi * Y / n) / np.cosh(m * np.pi / 2)) * np.cos(m * np.pi * X / n)
    return u


def duct_shape_error(lbm, n, nu, precision):
    nz = 4 * n
    flags = np.ones((nz, n, n), dtype=np.uint8)
    flags[0] = 2
    flags[-1] = 3
    G = gpu_lattice(lbm, flags, precision, nu, u_in=0.01)
    G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    steps = int(40 * n * n)
    G.step(steps).sync()
    uz = G.moments(BOX)[1][:, 2].reshape(nz, n, n)[nz // 2]
    G.close()
    ex = duct_exact_shape(n)
    return rel_l2(uz / uz.mean(), ex / ex.mean())


def test_square_duct_poiseuille_convergence(lbm):
    """Laminar square-duct flow behind a plug velocity inlet: the mid-plane
    profile converges to the analytic Fourier-series solution at second
    order in the resolution (fixed tau = 1, walls by halfway bounce-back)."""
    e8, e16, e32 = (duct_shape_error(lbm, n, 1.0 / 6.0, "fp64") for n in (8, 16, 32))
    assert e8 < 1e-2 and e32 < 1e-3
    assert e8 / e16 > 3.0 and e16 / e32 > 3.0


def radial_profiles(m1, flags):
    """Azimuthal means of a box field m1 (nz, ny, nx) over the fluid cells of
    each plane, in unit-width radial bins about the nozzle axis: (nz, bins)."""
    nz, ny, nx = flags.shape
    yy, xx = np.mgrid[0:ny, 0:nx]
    rb = np.floor(np.hypot(xx + 0.5 - nx / 2.0, yy + 0.5 - ny / 2.0)).astype(int).ravel()
    nbins = rb.max() + 1
    out = np.zeros((nz, nbins))
    for z in range(nz):
        w = (flags[z] != 0).ravel().astype(float)
        cnt = np.bincount(rb, weights=w, minlength=nbins)
        out[z] = np.bincount(rb, weights=w * m1[z].ravel(), minlength=nbins) / np.maximum(cnt, 1.0)
    return out


def nozzle_stats_run(lbm, name, precision, steps, avg_from, seed=None):
    """<u_z> time-averaged over steps avg_from+1 .. steps (FP64 accumulators)
    as radial profiles on every plane, and the sample count."""
    flags = I.workload_flags(name)
    params = dict(I.workload_params(name))
    if seed is not None:
        params["noise_seed"] = seed
    G = lbm.Lattice(flags, precision)
    G.set_params(**params)
    G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    G.step(avg_from)
    G.stats_begin(1)
    G.step(steps - avg_from).sync()
    m1, m2, n = G.stats_get(BOX)
    G.close()
    assert np.isfinite(m1).all() and np.isfinite(m2).all()
    return radial_profiles(m1.reshape(flags.shape), flags), n


def expansion_start(name):
    w = I.WORKLOADS[name]
    return w["D"] + I.cone_length(w["D"], w["d"]) + 4 * w["d"]


def statistics_regions(name):
    """Plane ranges of the statistics check: upstream of the sudden
    expansion (inlet pipe, cone, throat), the near field of the jet (the first
    two throat diameters after the expansion) and the far field (the rest,
    short of the outlet planes)."""
    w = I.WORKLOADS[name]
    z_exp, d, nz = expansion_start(name), w["d"], w["L_total"]
    return {"upstream": np.arange(4, z_exp), "near field": np.arange(z_exp, z_exp + 2 * d),
            "far field": np.arange(z_exp + 2 * d, nz - 4)}


def check_statistics(name, ref, runs, floor_run):
    """Time-averaged axial velocity of each run in runs against the FP64 run
    ref, as the relative L2 difference of the radial profiles over the planes
    of each region: within 2 % upstream of the expansion and in the near field
    of the jet, where the averages converge within the window; in the far
    field, where the jet breaks down and two realizations differ by more than
    2 % over any affordable window, within the run-to-run variability: twice
    the difference between ref and floor_run (the same flow with another
    inlet-noise seed) plus 1 % (the ratio of two such differences scatters
    about 1)."""
    regions = statistics_regions(name)
    rel = lambda a, b, zs: float(np.linalg.norm(a[zs] - b[zs]) / np.linalg.norm(b[zs]))
    floor = rel(floor_run, ref, regions["far field"])
    report = {"far-field noise floor": floor}
    for label, prof in runs.items():
        for region, zs in regions.items():
            e = rel(prof, ref, zs)
            report["%s %s" % (label, region)] = e
            bound = 0.02 if region != "far field" else 2.0 * floor + 0.01
            assert e < bound, (label, region, e, bound)
    print(name, {k: round(v, 4) for k, v in report.items()})
    return report


def test_transitional_nozzle_time_averaged_profiles(lbm):
    """Re 3500 nozzle (96x96x800, parabolic inlet + 1 % noise), 30 000 steps
    averaged over steps 10 001-30 000: FP32 and FP16-shifted <u_z> against the
    FP64 GPU run, region by region (check_statistics)."""
    name = "nozzle_re3500_96x96x800"
    ref, n = nozzle_stats_run(lbm, name, "fp64", 30000, 10000)
    assert n == 20000
    floor = nozzle_stats_run(lbm, name, "fp32", 30000, 10000, seed=3)[0]
    runs = {p: nozzle_stats_run(lbm, name, p, 30000, 10000)[0] for p in ("fp32", "fp16s")}
    check_statistics(name, ref, runs, floor)


def test_turbulent_nozzle_time_averaged_profiles(lbm):
    """Re 6500 nozzle (144x144x1200, parabolic inlet + 2 % noise, smooth start
    over 8000 steps), 40 000 steps averaged over steps 15 001-40 000: FP32 and
    FP16-shifted <u_z> against the FP64 GPU run, region by region
    (check_statistics); FP64 statistics accumulators throughout."""
    name = "nozzle_re6500_144x144x1200"
    ref, n = nozzle_stats_run(lbm, name, "fp64", 40000, 15000)
    assert n == 25000
    floor = nozzle_stats_run(lbm, name, "fp32", 40000, 15000, seed=3)[0]
    runs = {p: nozzle_stats_run(lbm, name, p, 40000, 15000)[0] for p in ("fp32", "fp16s")}
    check_statistics(name, ref, runs, floor)
