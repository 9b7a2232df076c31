"""The FP32 / FP16S fluid kernel variants against the FP64 oracle (GPU
required).

With the default ghost rates and 32-bit offsets, FP32 lattices run the tile
fluid kernel (one warp per tile of up to 32 consecutive cells of a row; tiles
of 32 fluid cells without wall links store through shared memory) and FP16S
lattices the chunk kernel (one thread per cell, a warp-uniform fast path for
warps of plain fluid cells).  LBM_FLUID_KERNEL, read when a context is
created, selects another variant: "chunk" (the chunk kernel in FP32 too,
with the inlet/outlet nodes in trailing blocks), "tile" (the tile kernel in
FP16S too) or "pairs" (FP16S: pairs of consecutive fast tiles on the pair
kernel, two adjacent cells per thread on the packed FP32 pipe, and the chunks
of every other tile on the chunk kernel, in two launches).  The wall-cell
and inlet/outlet kernels run on a second stream beside the fluid kernel.
Every variant must meet the method's tolerances on geometries that exercise
every path: walls in every direction and ragged rows (general tiles), long
wall-free rows (fast tiles), inlet/outlet nodes with noise, periodic rows,
both row axes, and the fused statistics and health check, whose partial sums
follow one another across the launches of a step.
"""
import numpy as np
import pytest

from paper_2204_10566_gb300 import inputs as I

from gpu_util import gpu_lattice, max_rel, oracle_lattice, random_state, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOX = 1
TOL_U = {"fp32": 1e-5, "fp16s": 1e-3}


@pytest.fixture(scope="module")
def lbm():
    from paper_2204_10566_gb300 import build

    build.build()
    from paper_2204_10566_gb300 import lbm as m

    assert torch.cuda.is_available()
    return m


@pytest.fixture(params=["default", "tile", "chunk", "pairs"])
def kernel(request, monkeypatch):
    if request.param == "default":  # FP32: tile kernel, FP16S: chunk kernel
        monkeypatch.delenv("LBM_FLUID_KERNEL", raising=False)
    else:
        monkeypatch.setenv("LBM_FLUID_KERNEL", request.param)
    return request.param


def long_channel():
    """A channel 120 cells long in z with an obstacle: long wall-free rows
    (fast tiles) beside rows along the walls and around the obstacle."""
    f = np.ones((120, 10, 9), dtype=np.uint8)
    f[:, 0, :] = 0
    f[:, -1, :] = 0
    f[40:52, 3:6, 3:6] = 0
    f[0, 1:-1, :] = 2
    f[-1, 1:-1, :] = 3
    return f


def run(orc, lbm, flags, precision, steps, rows, periodic=0, nu=0.03, **bc):
    O = oracle_lattice(orc, flags, nu, periodic=periodic, **bc)
    f0 = random_state(orc, flags, 21)
    O.set_populations(f0)
    G = gpu_lattice(lbm, flags, precision, nu, periodic=periodic, rows=rows, **bc)
    G.set_populations(f0, layout=BOX)
    O.step(steps)
    G.step(steps).sync()
    act = flags.reshape(-1) != 0
    _, u = G.moments(BOX)
    return rel_l2(u[act], O.moments()[act, 1:]), G, O, act


@pytest.mark.parametrize("rows", ["x", "z"])
@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
def test_channel_with_obstacle(orc, lbm, kernel, precision, rows):
    flags = long_channel()
    bc = dict(profile="parabolic", u_in=0.03, d_in=9.0, noise_amp=0.02, seed=5)
    err, G, O, act = run(orc, lbm, flags, precision, 6, rows, periodic=1, **bc)
    assert err < TOL_U[precision], err
    if precision == "fp32":
        assert max_rel(G.get_populations(BOX)[act], O.f[act]) < 2e-6


@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
def test_periodic_box_rows_wrap(orc, lbm, kernel, precision):
    """Rows along x of a fully periodic box 40 cells long: tiles at the row
    ends write the wrap-around copies, the others run fast."""
    flags = np.ones((5, 4, 40), dtype=np.uint8)
    err, G, O, act = run(orc, lbm, flags, precision, 5, "x", periodic=7)
    assert err < TOL_U[precision], err


@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
def test_statistics_and_health_check(orc, lbm, kernel, precision):
    """Fused statistics sampling and the health reduction on every fluid
    kernel variant: sums of u_z against the oracle's per-step moments, the
    health record (partial sums of all launches of a step) against
    lbm_get_totals."""
    flags = long_channel()
    bc = dict(profile="plug", u_in=0.02, d_in=9.0)
    O = oracle_lattice(orc, flags, 0.03, periodic=1, **bc)
    f0 = random_state(orc, flags, 8)
    O.set_populations(f0)
    G = gpu_lattice(lbm, flags, precision, 0.03, periodic=1, **bc)
    G.set_populations(f0, layout=BOX)
    G.set_check_every(2)
    G.stats_begin(1)
    s1 = np.zeros(flags.size)
    for _ in range(4):
        O.step(1)
        s1 += O.moments()[:, 3]
    G.step(4).sync()
    act = flags.reshape(-1) != 0
    m1, _, n = G.stats_get(BOX)
    assert n == 4
    assert np.abs(m1[act] - s1[act] / 4).max() < (2e-6 if precision == "fp32" else 2e-4)
    h = G.health()
    mass, mom = G.totals()
    assert abs(h[0] - mass) < (1e-6 if precision == "fp32" else 1e-5) * mass and h[5] == 0.0


@pytest.mark.parametrize("precision", ["fp32", "fp16s", "fp64"])
def test_kernel_launch_count(lbm, kernel, precision):
    """lbm_kernel_launches counts what each variant launches per step: the
    fluid kernel(s), the inlet/outlet kernel (fused into the FP32 chunk
    kernel) and the final pass of a health check."""
    flags = long_channel()
    G = gpu_lattice(lbm, flags, precision, 0.03, periodic=1, u_in=0.02, d_in=9.0)
    G.init_equilibrium()
    n0 = G.kernel_launches()
    G.step(3).sync()
    if precision == "fp32" and kernel == "chunk":
        per_step = 1
    elif precision == "fp16s" and kernel == "pairs":
        per_step = 3
    else:
        per_step = 2
    assert G.kernel_launches() - n0 == 3 * per_step
    G.set_check_every(2)
    n1 = G.kernel_launches()
    G.step(4).sync()
    assert G.kernel_launches() - n1 == 4 * per_step + 2
