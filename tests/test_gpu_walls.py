"""Interpolated bounce-back on the CUDA path (GPU required): wall distances
of the smooth nozzle surface (Sec. 2.2), set through lbm_set_wall_q, against
the oracle on the same seeded input; the plates of a channel placed where
their link fractions say; a round pipe closer to Hagen-Poiseuille flow than
with voxelised (halfway) walls.

Tolerances as in the other parity tests: FP64 1e-12 relative per
population, FP32 1e-5 and FP16S 1e-3 relative L2 on the velocity.
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


def dense_q(flags, cells, q):
    out = np.full((flags.size, Q), 128, dtype=np.uint8)
    out[cells] = q
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_nozzle_wall_q_against_oracle(orc, lbm, precision):
    """Small nozzle (walls of the cone, throat and expansion, inlet and
    outlet nodes whose partners sit next to the wall), random state, five
    steps."""
    D, d, L = 12, 4, 40
    flags = I.nozzle_flags(D, d, L)
    cells, q = I.nozzle_wall_q(D, d, L)
    assert cells.size > 0 and (q != 128).any() and (q < 128).any() and (q > 128).any()
    bc = dict(profile="parabolic", u_in=0.01, d_in=float(D), noise_amp=0.02, seed=5)
    nu = 0.02
    O = oracle_lattice(orc, flags, nu, wall_q=dense_q(flags, cells, q), **bc)
    f0 = random_state(orc, flags, 17)
    O.set_populations(f0)
    G = gpu_lattice(lbm, flags, precision, nu, **bc)
    G.set_wall_q(cells, q)
    G.set_populations(f0, layout=BOX)
    O.step(5)
    G.step(5).sync()
    act = flags.reshape(-1) != 0
    if precision == "fp64":
        assert max_rel(G.get_populations(BOX)[act], O.f[act]) < 1e-12
    else:
        _, u = G.moments(BOX)
        tol = 1e-5 if precision == "fp32" else 1e-3
        assert rel_l2(u[act], O.moments()[act, 1:]) < tol
    # the halfway default is restored by an empty list
    G.set_wall_q(np.zeros(0, dtype=np.int64), np.zeros((0, Q), dtype=np.uint8))


def test_wall_q_rejects_bad_input(lbm):
    flags = I.nozzle_flags(12, 4, 40)
    G = gpu_lattice(lbm, flags, "fp32", 0.02)
    solid = int(np.nonzero(flags.reshape(-1) == 0)[0][0])
    with pytest.raises(lbm.LbmError):
        G.set_wall_q([solid], np.full((1, Q), 100, dtype=np.uint8))
    fluid = int(np.nonzero(flags.reshape(-1) == 1)[0][0])
    with pytest.raises(lbm.LbmError):
        G.set_wall_q([fluid, fluid], np.full((2, Q), 100, dtype=np.uint8))
    with pytest.raises(lbm.LbmError):
        G.set_wall_q([fluid], np.zeros((1, Q), dtype=np.uint8))


def channel_walls(lbm, precision, n, ylo, yhi, nu=0.125, nz=None):
    nz = nz or 3 * n
    flags = np.ones((nz, n, 1), dtype=np.uint8)
    flags[0] = 2
    flags[-1] = 3
    cells, rows = [], []
    for z in range(1, nz - 1):
        for j, qv, cy in ((0, 0.5 - ylo, 1), (n - 1, yhi - (n - 0.5), -1)):
            r = np.full(Q, 128, dtype=np.uint8)
            for i in range(Q):
                if (i // 3) % 3 - 1 == cy:
                    r[i] = int(round(qv * 256))
            cells.append(z * n + j)
            rows.append(r)
    G = gpu_lattice(lbm, flags, precision, nu, periodic=1, u_in=0.01)
    G.set_wall_q(np.array(cells), np.array(rows))
    G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    G.step(int(60 * n * n)).sync()
    uz = G.moments(BOX)[1][:, 2].reshape(nz, n)[nz // 2]
    y = np.arange(n) + 0.5
    return np.sort(np.roots(np.polyfit(y, uz, 2)).real)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_channel_plates_where_the_wall_distances_put_them(lbm, precision):
    w = channel_walls(lbm, precision, 16, 0.3, 15.8)
    assert np.abs(w - [0.3, 15.8]).max() < 0.06
    w = channel_walls(lbm, precision, 16, -0.3, 16.25)
    assert np.abs(w - [-0.3, 16.25]).max() < 0.04


def pipe_shape_error(lbm, D, wall_q, nu=1.0 / 6.0):
    L = 4 * D
    flags = I.pipe_flags(D, L)
    G = gpu_lattice(lbm, flags, "fp64", nu, u_in=0.01)
    if wall_q:
        cells, q = I.nozzle_wall_q(D, D, L, L_in=L, L_cone=1, L_throat=0)
        G.set_wall_q(cells, q)
    G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    G.step(int(30 * D * D)).sync()
    uz = G.moments(BOX)[1][:, 2].reshape(L, D, D)[L // 2]
    c = np.arange(D) + 0.5 - D / 2.0
    r2 = c[None, :] ** 2 + c[:, None] ** 2
    inside = flags[L // 2] != 0
    ex = 1.0 - r2 / (D / 2.0) ** 2
    return rel_l2(uz[inside] / uz[inside].mean(), ex[inside] / ex[inside].mean())


def test_round_pipe_closer_to_hagen_poiseuille(lbm):
    """A round pipe of diameter 16 behind a plug inlet: with the circle's
    wall distances the developed profile is at least twice as close to the
    paraboloid of Hagen-Poiseuille flow as with the voxelised wall."""
    e_stair = pipe_shape_error(lbm, 16, False)
    e_q = pipe_shape_error(lbm, 16, True)
    print("pipe shape error: halfway %.4g, interpolated %.4g" % (e_stair, e_q))
    assert e_q < 0.5 * e_stair


def test_wall_cells_enter_health_and_statistics(lbm):
    """The cells with interpolated walls run in their own kernel; the fused
    health check and the statistics still cover every active cell."""
    D, d, L = 12, 4, 40
    flags = I.nozzle_flags(D, d, L)
    cells, q = I.nozzle_wall_q(D, d, L)
    G = gpu_lattice(lbm, flags, "fp64", 0.02, profile="parabolic", u_in=0.01, d_in=float(D))
    G.set_wall_q(cells, q)
    G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    G.step(60)
    G.set_check_every(2)
    G.stats_begin(1)
    acc = np.zeros(G.n_active)
    for _ in range(6):
        G.step(1)
        acc += G.moments()[1][:, 2]
    G.sync()
    h = G.health()
    rho, u = G.moments()
    assert abs(h[0] - rho.sum()) < 1e-10 * rho.sum()
    assert np.abs(h[1:4] - (rho[:, None] * u).sum(axis=0)).max() < 1e-12 * rho.sum()
    m1, _, n = G.stats_get()
    assert n == 6 and np.abs(m1 - acc / 6).max() < 1e-15


@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
def test_side_stream_changes_no_bit(lbm, precision, monkeypatch):
    """The wall-cell and inlet/outlet kernels run on a second stream beside
    the fluid kernel; with them in sequence on one stream (LBM_SIDE_STREAM=0)
    the populations, the health record and the statistics are bitwise the
    same."""
    D, d, L = 12, 4, 40
    flags = I.nozzle_flags(D, d, L)
    cells, q = I.nozzle_wall_q(D, d, L)
    out = []
    for side in ("1", "0"):
        monkeypatch.setenv("LBM_SIDE_STREAM", side)
        G = gpu_lattice(lbm, flags, precision, 0.02, profile="parabolic", u_in=0.02, d_in=float(D),
                        noise_amp=0.02, seed=3)
        G.set_wall_q(cells, q)
        G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
        G.set_check_every(3)
        G.stats_begin(1)
        G.step(40).sync()
        out.append((G.get_populations(BOX), G.health(), G.stats_get(BOX)[0]))
        G.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
def test_steps_captured_in_a_cuda_graph(lbm, precision):
    """lbm_step inside a stream capture: the fork onto the side stream and the
    join back are captured with the kernels, and two replays of a captured
    run of four steps give bitwise the populations of the same steps run
    without a graph (no noise and no ramp, so the steps do not depend on t)."""
    D, d, L = 12, 4, 40
    flags = I.nozzle_flags(D, d, L)
    cells, q = I.nozzle_wall_q(D, d, L)

    def make(stream):
        G = lbm.Lattice(flags, precision, stream=stream)
        G.set_params(nu=0.02, u_in=0.02, d_in=float(D), profile="parabolic", noise_amp=0.0, inlet_ramp=0)
        G.set_wall_q(cells, q)
        G.init_equilibrium(1.0, (0.0, 0.0, 0.0))
        return G

    s = torch.cuda.Stream()
    G = make(s)
    G.step(2).sync()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        G.step(4)  # an even count: the two buffers end where they started
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    E = make(torch.cuda.current_stream())
    E.step(10).sync()
    assert np.array_equal(G.get_populations(BOX), E.get_populations(BOX))
    G.close()
    E.close()
