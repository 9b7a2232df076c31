"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check compares the oracle with something other than itself: closed
forms, invariants, printed formulas of Appendix A, library routines, an
independent brute-force restatement, or published reference outputs.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2204_10566_gb300 import inputs as I

TH = 1.0 / 3.0
Q = 27


def vel():
    return np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(Q)], dtype=float)


def midx(m):
    return (m % 3, (m // 3) % 3, m // 9)


# ------------------------------------------------------------- stencil, weights

def test_weights_quadrature_moments(orc):
    """Appendix A: third-order Gauss-Hermite quadrature.  The weights must
    reproduce the Maxwellian moments at u = 0 up to fifth order:
    sum w = 1, sum w c_a c_b = theta0 delta_ab,
    sum w c_a c_b c_c c_d = theta0^2 (d_ab d_cd + d_ac d_bd + d_ad d_bc), odd ones 0."""
    c = orc.velocities().astype(float)
    w = orc.weights()
    assert np.allclose(c, vel())
    assert abs(w.sum() - 1.0) < 1e-15
    d = np.eye(3)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), TH * d, atol=1e-16)
    four = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = TH ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                     + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(four, iso, atol=1e-16)
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-16)
    # 1-D weights printed in Appendix A: 2/3 at c = 0 and 1/6 at c = +-1.
    assert abs(w[13] - (2 / 3) ** 3) < 1e-16 and abs(w[0] - (1 / 6) ** 3) < 1e-16


# ---------------------------------------------------------- Hermite polynomials

def printed_hermite(idx, xi):
    """Appendix A's explicit 'cyc' forms for orders 0..4, written for the
    dimensional polynomials (each delta carries theta0)."""
    n = len(idx)
    x = [xi[a] for a in idx]
    dl = lambda a, b: TH if idx[a] == idx[b] else 0.0
    if n == 0:
        return 1.0
    if n == 1:
        return x[0]
    if n == 2:
        return x[0] * x[1] - dl(0, 1)
    if n == 3:
        return x[0] * x[1] * x[2] - (dl(0, 1) * x[2] + dl(0, 2) * x[1] + dl(1, 2) * x[0])
    if n == 4:
        pairs = [((0, 1), (2, 3)), ((0, 2), (1, 3)), ((0, 3), (1, 2))]
        single = sum(dl(*p) * x[q[0]] * x[q[1]] + dl(*q) * x[p[0]] * x[p[1]] for p, q in pairs)
        double = sum(dl(*p) * dl(*q) for p, q in pairs)
        return x[0] * x[1] * x[2] * x[3] - single + double
    raise ValueError


def test_hermite_matches_printed_forms(orc):
    g = np.random.default_rng(7)
    for n in range(5):
        for idx in itertools.product(range(3), repeat=n):
            xi = g.normal(size=3)
            assert abs(orc.hermite(list(idx), xi) - printed_hermite(idx, xi)) < 1e-13


def test_hermite_orthogonality_on_stencil(orc):
    """sum_i w_i H_m(c_i) H_m'(c_i) = delta_mm' mx! my! mz! theta0^|m| for the 27
    stencil-supported polynomials (orthogonality of the quadrature)."""
    c = vel()
    w = orc.weights()
    H = np.array([[orc.hermite_m(m, c[i]) for i in range(Q)] for m in range(Q)])
    G = (H * w) @ H.T
    ref = np.diag([math.prod(math.factorial(k) for k in midx(m)) * TH ** sum(midx(m)) for m in range(Q)])
    assert np.allclose(G, ref, atol=1e-15)


def test_hermite_sixth_order_aliasing(orc):
    """On the D3Q27 nodes H_xxx vanishes identically (c^3 = c): the reason the
    expansion keeps only per-axis degree <= 2."""
    for i in range(Q):
        assert abs(orc.hermite([0, 0, 0], vel()[i])) < 1e-15


# ----------------------------------------------------------------- equilibrium

def product_form_equilibrium(rho, u):
    """Independent closed form: the 1-D populations g(c; u) fixed by the three
    1-D moments 1, u, theta0 + u^2 (solved with numpy), multiplied over axes."""
    cs = np.array([-1.0, 0.0, 1.0])
    V = np.vstack([np.ones(3), cs, cs ** 2])
    g = [np.linalg.solve(V, [1.0, ua, TH + ua * ua]) for ua in u]
    return np.array([rho * g[0][i % 3] * g[1][(i // 3) % 3] * g[2][i // 9] for i in range(Q)])


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_closed_forms(orc, seed):
    g = np.random.default_rng(seed)
    rho = 1.0 + 0.1 * g.uniform(-1, 1)
    u = 0.15 * g.uniform(-1, 1, size=3)
    feq = orc.equilibrium(rho, u)
    assert np.allclose(feq, orc.equilibrium_tuples(rho, u), atol=1e-16)
    assert np.allclose(feq, product_form_equilibrium(rho, u), rtol=1e-13, atol=1e-16)
    c = vel()
    assert abs(feq.sum() - rho) < 1e-14
    assert np.allclose(c.T @ feq, rho * u, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib->ab", feq, c, c), rho * (np.outer(u, u) + TH * np.eye(3)), atol=1e-15)


def central_moment(f, u, m):
    """Direct definition of one central Hermite moment from Sec. 2.1:
    sum_i prod_a h_{m_a}(c_ia - u_a) f_i with h0 = 1, h1 = x, h2 = x^2 - theta0."""
    c = vel()
    out = 0.0
    for i in range(Q):
        p = 1.0
        for a, k in enumerate(midx(m)):
            x = c[i, a] - u[a]
            p *= (1.0, x, x * x - TH)[k]
        out += p * f[i]
    return out


@pytest.mark.parametrize("seed", range(4))
def test_central_equilibrium_moments_vanish(orc, seed):
    """Appendix A: T f^eq = (rho, 0, ..., 0) with the full expansion."""
    g = np.random.default_rng(100 + seed)
    rho = 1.0 + 0.05 * g.uniform(-1, 1)
    u = 0.2 * g.uniform(-1, 1, size=3)
    T = orc.transform(u)
    a = T @ orc.equilibrium(rho, u)
    assert abs(a[0] - rho) < 1e-15
    assert np.abs(a[1:]).max() < 2e-16 * 27
    for m in range(Q):   # rows of T against the definition
        e = np.zeros(Q)
        for i in range(Q):
            e[:] = 0.0
            e[i] = 1.0
            assert abs(T[m, i] - central_moment(e, u, m)) < 1e-15


# ------------------------------------------------------------------- collision

def near_eq(orc, seed, amp=0.02):
    g = np.random.default_rng(seed)
    rho = 1.0 + 0.03 * g.uniform(-1, 1)
    u = 0.08 * g.uniform(-1, 1, size=3)
    feq = orc.equilibrium(rho, u)
    return feq * (1.0 + amp * g.uniform(-1, 1, size=Q))


@pytest.mark.parametrize("seed", range(6))
def test_collision_conserves_mass_momentum(orc, seed):
    f = near_eq(orc, seed)
    fp, mom = orc.collide(f, 1.7, ghost=(0.9, 1.1, 1.3, 0.7))
    c = vel()
    assert abs(fp.sum() - f.sum()) < 1e-15
    assert np.allclose(c.T @ fp, c.T @ f, atol=1e-16)
    assert abs(mom[0] - f.sum()) < 1e-15


def test_equilibrium_is_fixed_point(orc):
    feq = orc.equilibrium(1.01, [0.04, -0.02, 0.07])
    fp, _ = orc.collide(feq, 1.9)
    assert np.allclose(fp, feq, atol=1e-17, rtol=0)


@pytest.mark.parametrize("omega", [0.6, 1.0, 1.95])
def test_collision_reduces_to_bgk(orc, omega):
    """All rates equal omega: T^-1 S T = omega I and the MRT step is the LBGK
    equation of Sec. 2.1, f* = f + omega (f^eq - f)."""
    f = near_eq(orc, 11)
    fp, mom = orc.collide(f, omega, ghost=(omega,) * 4, omega_cons=omega)
    feq = product_form_equilibrium(f.sum(), vel().T @ f / f.sum())
    assert np.allclose(fp, f + omega * (feq - f), atol=1e-16, rtol=1e-14)


@pytest.mark.parametrize("ghost", [(1.0, 1.0, 1.0, 1.0), (0.8, 1.2, 1.5, 0.5)])
def test_collision_relaxes_each_central_moment(orc, ghost):
    """S acts diagonally on central Hermite moments: order-2 moments scale by
    (1 - omega), order-n ghosts by (1 - omega_n) (their equilibria are 0,
    Appendix A), orders 0 and 1 are unchanged."""
    omega = 1.37
    f = near_eq(orc, 21, amp=0.05)
    fp, mom = orc.collide(f, omega, ghost=ghost)
    u = mom[1:]
    for m in range(Q):
        n = sum(midx(m))
        a0 = central_moment(f, u, m)
        a1 = central_moment(fp, u, m)
        rate = {0: 0.0, 1: 0.0, 2: omega}.get(n, ghost[n - 3] if n >= 3 else 0.0)
        if n == 0:
            assert abs(a1 - a0) < 1e-15
        elif n == 1:
            assert abs(a1) < 1e-16 and abs(a0) < 1e-16
        else:
            assert abs(a1 - (1.0 - rate) * a0) < 1e-15


def test_conserved_rate_is_immaterial(orc):
    f = near_eq(orc, 5)
    a, _ = orc.collide(f, 1.3, omega_cons=1.0)
    b, _ = orc.collide(f, 1.3, omega_cons=0.3)
    assert np.allclose(a, b, atol=1e-17, rtol=1e-15)


def test_gaussian_elimination_matches_lapack(orc):
    g = np.random.default_rng(3)
    for _ in range(5):
        A = g.normal(size=(27, 27)) + 5 * np.eye(27)
        b = g.normal(size=27)
        assert np.allclose(orc.solve(A, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-13)
    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    assert np.allclose(orc.solve(A, [2.0, 3.0]), [3.0, 2.0])   # needs the pivot


# ------------------------------------------------------------------- streaming

def np_stream(f, flags, periodic):
    """Brute-force pull streaming with halfway bounce-back on a dense box
    (test restatement, written with numpy shifts)."""
    nz, ny, nx = flags.shape
    c = vel().astype(int)
    F = f.reshape(nz, ny, nx, Q)
    out = np.zeros_like(F)
    solid = flags == 0
    for i in range(Q):
        cx, cy, cz = c[i]
        src = np.roll(F[..., i], shift=(cz, cy, cx), axis=(0, 1, 2))
        ssolid = np.roll(solid, shift=(cz, cy, cx), axis=(0, 1, 2))
        # leaving a non-periodic box counts as solid
        zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        outside = np.zeros_like(solid)
        if not periodic & 1:
            outside |= (xx - cx < 0) | (xx - cx >= nx)
        if not periodic & 2:
            outside |= (yy - cy < 0) | (yy - cy >= ny)
        if not periodic & 4:
            outside |= (zz - cz < 0) | (zz - cz >= nz)
        bb = ssolid | outside
        out[..., i] = np.where(bb, F[..., Q - 1 - i], src)
    out[solid] = 0.0
    return out.reshape(-1, Q)


@pytest.mark.parametrize("periodic", [7, 0, 2])
def test_streaming_pull_and_bounce_back(orc, periodic):
    """With every rate 0 the collision is the identity, so a step is pure pull
    streaming: f_i(x) <- f_i(x - c_i), or f_opp(i)(x) when x - c_i is a wall."""
    flags = np.ones((5, 4, 6), dtype=np.uint8)
    flags[2, 1, 3] = 0
    flags[4, 0, 0] = 0
    g = np.random.default_rng(periodic)
    f = g.uniform(0.01, 0.05, size=(flags.size, Q))
    f[flags.reshape(-1) == 0] = 0.0
    L = orc.Lattice(flags, omega=0.0, ghost=(0, 0, 0, 0), periodic=periodic)
    L.set_populations(f)
    L.step(1)
    assert np.abs(L.f - np_stream(f, flags, periodic)).max() < 5e-16


def test_periodic_streaming_returns_impulse(orc):
    flags = np.ones((4, 5, 6), dtype=np.uint8)
    f = np.tile(orc.weights(), (flags.size, 1))
    f[7, 5] += 0.01   # cell 7, direction 5 = (+1, 0, -1)
    L = orc.Lattice(flags, omega=0.0, ghost=(0, 0, 0, 0), periodic=7)
    L.set_populations(f)
    L.step(12)       # lcm of the x and z periods 6 and 4
    assert np.abs(L.f - f).max() < 1e-15


def test_closed_box_conserves_mass(orc):
    flags = np.ones((6, 5, 4), dtype=np.uint8)
    flags[3, 2, 1] = 0
    g = np.random.default_rng(9)
    L = orc.Lattice(flags, omega=1.4)
    n = flags.size
    L.init_equilibrium(1.0 + 0.01 * g.uniform(-1, 1, n), 0.03 * g.uniform(-1, 1, (n, 3)))
    m0 = L.totals()[0]
    L.step(5)
    assert abs(L.totals()[0] - m0) < 1e-12


def test_rest_state_with_walls_is_fixed_point(orc):
    flags = I.nozzle_flags(12, 4, 40, inlet=False, outlet=False)
    L = orc.Lattice(flags, omega=1.2)
    L.init_equilibrium(1.0, [0.0, 0.0, 0.0])
    f0 = L.f.copy()
    L.step(3)
    assert np.abs(L.f - f0).max() < 5e-16


# ------------------------------------------------------------------ brute force

def brute_force_step(f, flags, omega, ghost):
    """Independent restatement: numpy streaming, T(u) as the tensor product of
    1-D Hermite polynomials h0 = 1, h1 = x, h2 = x^2 - theta0, product-form
    equilibrium, LAPACK solve."""
    fs = np_stream(f, flags, 7)
    c = vel()
    out = np.zeros_like(fs)
    rates = []
    for m in range(Q):
        n = sum(midx(m))
        rates.append(1.0 if n <= 1 else (omega if n == 2 else ghost[n - 3]))
    S = np.diag(rates)
    for b in range(fs.shape[0]):
        fb = fs[b]
        rho = fb.sum()
        u = c.T @ fb / rho
        T = np.zeros((Q, Q))
        for m in range(Q):
            for i in range(Q):
                p = 1.0
                for a, k in enumerate(midx(m)):
                    x = c[i, a] - u[a]
                    p *= (1.0, x, x * x - TH)[k]
                T[m, i] = p
        feq = product_form_equilibrium(rho, u)
        out[b] = fb + np.linalg.solve(T, S @ T @ (feq - fb))
    return out


def test_brute_force_4cubed_periodic(orc):
    flags = np.ones((4, 4, 4), dtype=np.uint8)
    g = np.random.default_rng(44)
    n = flags.size
    L = orc.Lattice(flags, omega=1.6, ghost=(1.0, 0.9, 1.1, 1.2), periodic=7)
    L.init_equilibrium(1.0 + 0.02 * g.uniform(-1, 1, n), 0.05 * g.uniform(-1, 1, (n, 3)))
    L.f *= 1.0 + 0.01 * g.uniform(-1, 1, L.f.shape)
    f0 = L.f.copy()
    L.step(1)
    ref = brute_force_step(f0, flags, 1.6, (1.0, 0.9, 1.1, 1.2))
    assert np.abs(L.f - ref).max() < 1e-15


# ------------------------------------------------------------- flow solutions

def omega_of_nu(nu):
    """Sec. 2.1: tau = mu/(rho theta0) + dt/2, i.e. omega = 1/(3 nu + 1/2)."""
    return 1.0 / (3.0 * nu + 0.5)


def tgv2d_rate(orc, N, nu, steps):
    k = 2 * np.pi / N
    u0 = 0.01
    x = (np.arange(N) + 0.0)
    X, Y = np.meshgrid(x, x, indexing="xy")            # [y, x]
    ux = u0 * np.sin(k * X) * np.cos(k * Y)
    uy = -u0 * np.cos(k * X) * np.sin(k * Y)
    rho = 1.0 - 3.0 * u0 ** 2 / 4.0 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    flags = np.ones((1, N, N), dtype=np.uint8)
    L = orc.Lattice(flags, omega=omega_of_nu(nu), periodic=7)
    u = np.stack([ux.ravel(), uy.ravel(), np.zeros(N * N)], axis=1)
    L.init_equilibrium(rho.ravel(), u)
    # skip the start-up layer of an equilibrium initialisation, then fit
    # the kinetic energy decay exp(-4 nu k^2 t) over the remaining steps
    L.step(steps // 4)
    e0 = (L.moments()[:, 1:3] ** 2).sum()
    L.step(steps - steps // 4)
    e1 = (L.moments()[:, 1:3] ** 2).sum()
    measured = -np.log(e1 / e0) / (4 * (steps - steps // 4))
    return measured / (nu * k * k)


def test_taylor_green_2d_decay(orc):
    """2-D Taylor-Green vortex (exact Navier-Stokes solution) in a periodic
    box: velocity decays as exp(-2 nu k^2 t), nu tied to omega by the
    relaxation-time relation of Sec. 2.1."""
    r16 = tgv2d_rate(orc, 16, 0.02, 120)
    r32 = tgv2d_rate(orc, 32, 0.02, 240)
    assert abs(r16 - 1.0) < 5e-3
    assert abs(r32 - 1.0) < 1e-3


def shear_wave_rate(orc, H, nu, steps):
    """u_x = U sin(pi (y + 1/2) / H) between halfway bounce-back walls at
    y = -1/2 and y = H - 1/2 decays as exp(-nu (pi/H)^2 t)."""
    y = np.arange(H)
    U = 0.01
    prof = U * np.sin(np.pi * (y + 0.5) / H)
    flags = np.ones((1, H, 2), dtype=np.uint8)
    L = orc.Lattice(flags, omega=omega_of_nu(nu), periodic=1 | 4)
    u = np.zeros((2 * H, 3))
    u[:, 0] = np.repeat(prof, 2)
    L.init_equilibrium(1.0, u)
    L.step(steps)
    amp = (L.moments()[:, 1].reshape(H, 2)[:, 0] * prof).sum() / (prof * prof).sum()
    return -np.log(amp) / steps / (nu * (np.pi / H) ** 2)


def test_shear_wave_between_walls(orc):
    r8 = shear_wave_rate(orc, 8, 0.05, 100)
    r16 = shear_wave_rate(orc, 16, 0.05, 400)
    assert abs(r16 - 1.0) < 0.01
    # second order in the resolution: the error falls about 4x per doubling
    assert 3.0 < abs(r8 - 1.0) / abs(r16 - 1.0) < 5.0


# ------------------------------------------------------------ viscous stress

def test_viscous_stress_of_equilibrium_is_zero(orc):
    """The equilibrium has no non-equilibrium second moment: sigma = 0 for
    any rho, u (a dropped theta0 term or a raw instead of central moment
    fails on the diagonal)."""
    rng = np.random.default_rng(7)
    for _ in range(5):
        rho = 1.0 + 0.1 * rng.standard_normal()
        u = 0.08 * rng.standard_normal(3)
        assert np.abs(orc.viscous_stress(orc.equilibrium(rho, u), 1.6)).max() < 1e-15


def stress_wave(orc, n, nu, steps, longitudinal):
    """Periodic sine wave of u_x along y (shear) or x (longitudinal), one
    box cell thick otherwise.  Returns the ratio of the sampled stress
    amplitude (sigma_xy resp. sigma_xx on cos) to the Navier-Stokes value
    rho nu (d_b u_a + d_a u_b) from the velocity amplitude of the same
    state, and the largest other component relative to it."""
    k = 2 * np.pi / n
    c = np.arange(n) + 0.5
    shape = (1, 2, n) if longitudinal else (1, n, 2)
    L = orc.Lattice(np.ones(shape, dtype=np.uint8), omega=omega_of_nu(nu), periodic=7)
    u = np.zeros(shape + (3,))
    if longitudinal:
        u[0, :, :, 0] = 0.005 * np.sin(k * c)[None, :]
    else:
        u[0, :, :, 0] = 0.01 * np.sin(k * c)[:, None]
    L.init_equilibrium(1.0, u.reshape(-1, 3))
    L.step(steps)
    sig = L.field_stress().reshape(shape + (6,))[0]
    L.step(1)                                   # the velocity of the same (pre-collision) state
    m = L.last_moments.reshape(shape + (4,))[0]
    line = (lambda a: a[0, :]) if longitudinal else (lambda a: a[:, 0])
    ux, rho = line(m[..., 1]), line(m[..., 0])
    A = (ux * np.sin(k * c)).sum() / (np.sin(k * c) ** 2).sum()
    comp = 0 if longitudinal else 3
    B = (line(sig[..., comp]) * np.cos(k * c)).sum() / (np.cos(k * c) ** 2).sum()
    expect = (2.0 if longitudinal else 1.0) * rho.mean() * nu * A * k
    others = [q for q in range(6) if q != comp and not (longitudinal and q in (1, 2))]
    rest = max(np.abs(line(sig[..., q])).max() for q in others)
    return B / expect, rest / abs(B)


def test_viscous_stress_shear_wave(orc):
    """Sec. 2.2: sigma_xy = rho nu d_y u_x for a decaying shear wave
    u_x = U sin(k y), second-order convergent in the resolution; the other
    components vanish.  A wrong sign, the post- instead of the pre-collision
    moment (factor 1 - omega) or a missing (1 - omega/2) all fail."""
    r16, o16 = stress_wave(orc, 16, 0.02, 50, False)
    r32, o32 = stress_wave(orc, 32, 0.02, 50, False)
    assert abs(r32 - 1.0) < 5e-3
    assert 3.0 < abs(r16 - 1.0) / abs(r32 - 1.0) < 5.0
    assert o16 < 1e-3 and o32 < 1e-3


def test_viscous_stress_longitudinal_wave(orc):
    """Longitudinal (acoustic) wave u_x = U(t) sin(k x): sigma_xx =
    2 rho nu d_x u_x, the full strain rate of the relation in Appendix A
    (all six second-order moments relax at omega); off-diagonal terms 0."""
    r, o = stress_wave(orc, 64, 0.02, 60, True)
    assert abs(r - 1.0) < 1e-2
    assert o < 1e-6


def test_sampled_time_averages_of_a_decaying_wave(orc):
    """Per-step sampled time averages (Sec. 2.2 mean / fluctuation
    decomposition) of a decaying shear wave u_x = A sin(k y) lambda^t,
    lambda = exp(-nu k^2): over n steps the mean of u is A times the mean
    of lambda^t for t = 1..n (sampled after each step), the mean of u_x^2
    the same with lambda^2t, and the mean stress sigma_xy that of the
    pre-step states, t = 0..n-1; rho averages to 1 and every other
    component to 0 (the diagonal stresses to second order in u)."""
    n, nu, steps = 32, 0.02, 20
    k = 2 * np.pi / n
    c = np.arange(n) + 0.5
    s, co = np.sin(k * c), np.cos(k * c)
    L = orc.Lattice(np.ones((1, n, 2), dtype=np.uint8), omega=omega_of_nu(nu), periodic=7)
    u = np.zeros((1, n, 2, 3))
    u[0, :, :, 0] = 0.01 * s[:, None]
    L.init_equilibrium(1.0, u.reshape(-1, 3))
    L.step(50)
    A0 = (L.moments().reshape(n, 2, 4)[:, 0, 1] * s).sum() / (s * s).sum()
    S0 = (L.field_stress().reshape(n, 2, 6)[:, 0, 3] * co).sum() / (co * co).sum()
    lam = np.exp(-nu * k * k)
    t = np.arange(1, steps + 1)
    avg = L.step_sampled(steps)
    um = avg["u"].reshape(n, 2, 3)[:, 0]
    uu = avg["uu"].reshape(n, 2, 6)[:, 0]
    sg = avg["sigma"].reshape(n, 2, 6)[:, 0]
    assert abs((um[:, 0] * s).sum() / (s * s).sum() / (A0 * np.mean(lam ** t)) - 1.0) < 1e-4
    assert abs((uu[:, 0] * s * s).sum() / (s ** 4).sum() / (A0 ** 2 * np.mean(lam ** (2 * t))) - 1.0) < 2e-4
    assert abs((sg[:, 3] * co).sum() / (co * co).sum() / (S0 * np.mean(lam ** (t - 1))) - 1.0) < 1e-4
    assert np.abs(avg["rho"] - 1.0).max() < 1e-6
    assert np.abs(um[:, 1:]).max() < 1e-9 and np.abs(uu[:, 1:]).max() < 1e-9
    assert np.abs(sg[:, [0, 1, 2, 4, 5]]).max() < 1e-3 * abs(S0)


# --------------------------------------------------------------- inlet/outlet

def duct_flags(n, nz):
    f = np.ones((nz, n, n), dtype=np.uint8)
    f[0] = 2
    f[-1] = 3
    return f


def duct_exact_shape(n, terms=40):
    """Fully developed laminar flow in a square duct of side n (walls at the
    cell faces -1/2 and n - 1/2): the Fourier-series solution of
    nu Laplacian(u) = -G on the cross-section, sampled at the cell centres
    (up to a constant factor)."""
    c = np.arange(n) + 0.5 - n / 2.0
    Y, X = np.meshgrid(c, c, indexing="ij")
    u = np.zeros_like(X)
    for k in range(terms):
        m = 2 * k + 1
        u += (-1) ** k / m ** 3 * (1 - np.cosh(m * np.pi * Y / n) / np.cosh(m * np.pi / 2)) * np.cos(m * np.pi * X / n)
    return u


def test_square_duct_poiseuille_profile(orc):
    """Velocity inlet (plug) and pressure outlet on a 6 x 6 duct with halfway
    bounce-back walls: the mid-plane profile develops into the analytic
    duct solution, and so does its viscous shear stress.  At tau = 7/8 (the magic-parameter value of halfway
    bounce-back with unit ghost rates) the shape error is 0.24 %; walls
    half a cell further out (full-way bounce-back) change the shape by 19 %."""
    n, nz, nu = 6, 24, 0.125
    L = orc.Lattice(duct_flags(n, nz), omega=omega_of_nu(nu), u_in=0.01)
    L.init_equilibrium(1.0, [0.0, 0.0, 0.0])
    L.step(1250)
    prev = L.moments()[:, 3].reshape(nz, n, n)[nz // 2].copy()
    L.step(250)
    m = L.moments().reshape(nz, n, n, 4)
    uz = m[nz // 2, :, :, 3]
    assert np.abs(uz - prev).max() < 1e-6 * np.abs(uz).max()      # steady
    shape, ex = uz / uz.mean(), duct_exact_shape(n)
    ex = ex / ex.mean()
    assert np.linalg.norm(shape - ex) / np.linalg.norm(ex) < 5e-3
    # steady and mass-conserving: the same axial mass flux through every
    # interior plane (the inlet node plane itself carries the imposed
    # velocity, not the streamed flux)
    flux = (m[1:-1, ..., 0] * m[1:-1, ..., 3]).sum(axis=(1, 2))
    assert np.ptp(flux) < 1e-6 * flux.mean()
    # the wall shear of the developed flow: sigma_xz = rho nu d_x u_z of the
    # Fourier-series solution (scaled to the measured mean velocity) within
    # 3 % on the mid-plane and 4 % in the wall-adjacent column (measured 2.0
    # and 2.4 %, falling to 0.75 and 1.3 % at twice the resolution), where
    # the gather takes the bounced-back populations
    c = np.arange(n) + 0.5 - n / 2.0
    Yc, Xc = np.meshgrid(c, c, indexing="ij")
    dudx = np.zeros_like(Xc)
    for kk in range(60):
        mm = 2 * kk + 1
        dudx -= ((-1) ** kk / mm ** 3 * (1 - np.cosh(mm * np.pi * Yc / n) / np.cosh(mm * np.pi / 2))
                 * np.sin(mm * np.pi * Xc / n) * mm * np.pi / n)
    sig_mid = L.field_stress().reshape(nz, n, n, 6)[nz // 2, ..., 4]
    expect = m[nz // 2, ..., 0] * nu * (uz.mean() / duct_exact_shape(n).mean()) * dudx
    assert np.linalg.norm(sig_mid - expect) / np.linalg.norm(expect) < 0.03
    assert np.abs(sig_mid[:, 0] - expect[:, 0]).max() < 0.04 * np.abs(expect[:, 0]).max()
    # the outlet nodes carry the stress of the developed flow: the wall shear
    # sigma_xz, sigma_yz on the outlet plane matches that two planes upstream
    # (measured 7.6e-4 of its maximum; the outlet condition bends it slightly)
    sig = L.field_stress().reshape(nz, n, n, 6)
    shear_out, shear_up = sig[-1, ..., 4:6], sig[-3, ..., 4:6]
    assert np.abs(shear_up).max() > 0.0
    assert np.abs(shear_out - shear_up).max() < 3e-3 * np.abs(shear_up).max()


def channel_wall_fit(orc, n, nz, nu, ylo, yhi, use_q=True, steps=3000):
    """Developed flow between two plates behind a plug inlet, one cell deep
    (x periodic), with the plates at y = ylo and y = yhi (cell faces at 0 and
    n; cell centres at j + 1/2).  Every link that leaves the box through a
    plate is cut at q = 0.5 - ylo (bottom) or yhi - (n - 0.5) (top).  Returns
    the plate positions read off a parabola fitted to the mid-plane u_z."""
    flags = duct_flags(1, nz)[:, :1, :1].repeat(n, axis=1)
    wq = np.full((flags.size, Q), 128, dtype=np.uint8)
    c = vel()
    for z in range(nz):
        for j, qv, cy in ((0, 0.5 - ylo, 1), (n - 1, yhi - (n - 0.5), -1)):
            for i in range(Q):
                if c[i, 1] == cy:
                    wq[z * n + j, i] = int(round(qv * 256))
    L = orc.Lattice(flags, omega=omega_of_nu(nu), periodic=1, u_in=0.01, wall_q=wq if use_q else None)
    L.init_equilibrium(1.0, [0.0, 0.0, 0.0])
    L.step(steps)
    uz = L.moments()[:, 3].reshape(nz, n)[nz // 2]
    y = np.arange(n) + 0.5
    return np.sort(np.roots(np.polyfit(y, uz, 2)).real)


def test_interpolated_bounce_back_places_the_walls(orc):
    """Sec. 2.2 walls: Bouzidi's interpolated bounce-back puts a plane wall
    where its link fractions q say, for both of its branches (q < 1/2 and
    q >= 1/2): the developed channel profile vanishes within 0.06 cells of
    the true plates (halfway bounce-back would leave them at the box faces,
    0.2-0.3 cells off).  Links at q = 1/2 reproduce halfway bounce-back."""
    w = channel_wall_fit(orc, 8, 24, 0.125, 0.3, 7.8)
    assert np.abs(w - [0.3, 7.8]).max() < 0.06
    w = channel_wall_fit(orc, 8, 24, 0.125, -0.3, 8.25)
    assert np.abs(w - [-0.3, 8.25]).max() < 0.04
    halfway = channel_wall_fit(orc, 8, 24, 0.125, 0.3, 7.8, use_q=False)
    assert np.abs(halfway - [0.0, 8.0]).max() < 1e-3
    flags = I.nozzle_flags(12, 4, 30)
    A = orc.Lattice(flags, omega=1.4, u_in=0.01)
    B = orc.Lattice(flags, omega=1.4, u_in=0.01, wall_q=np.full((flags.size, Q), 128, dtype=np.uint8))
    for L in (A, B):
        L.init_equilibrium(1.0, [0.0, 0.0, 0.0])
        L.step(5)
    assert np.array_equal(A.f, B.f)


def test_plug_flow_is_fixed_point(orc):
    """Uniform flow through a periodic duct with a plug velocity inlet and a
    rho = 1 outlet is an exact steady state of the scheme."""
    u0 = 0.03
    flags = duct_flags(3, 10)
    L = orc.Lattice(flags, omega=1.3, periodic=3, u_in=u0)
    L.init_equilibrium(1.0, [0.0, 0.0, u0])
    f0 = L.f.copy()
    L.step(4)
    assert np.abs(L.f - f0).max() < 1e-16


def test_inlet_start_up_ramp(orc):
    """Smooth start of the velocity inlet over T steps (a reading: the paper
    gives no start-up): the imposed velocity rises monotonically from 0 to
    the target, is symmetric about T/2 (r(s) + r(1 - s) = 1), has zero slope
    at both ends, and T = 0 is the impulsive start."""
    u0, T = 0.02, 16
    flags = duct_flags(3, 8)

    def inlet_speeds(ramp, steps):
        L = orc.Lattice(flags, omega=1.3, periodic=3, u_in=u0, ramp=ramp)
        L.init_equilibrium(1.0, [0.0, 0.0, 0.0])
        inlet = flags.reshape(-1) == 2
        out = []
        for _ in range(steps):
            L.step(1)
            ub = L.last_moments[inlet, 1:]
            assert np.abs(ub[:, :2]).max() == 0.0 and np.ptp(ub[:, 2]) == 0.0
            out.append(ub[0, 2] / u0)
        return np.array(out)

    r = inlet_speeds(T, T + 3)                 # r[t - 1] = r(t / T)
    assert np.all(np.diff(r[:T]) > 0) and np.all(r[T - 1:] == 1.0)
    for t in range(1, T):
        assert abs(r[t - 1] + r[T - t - 1] - 1.0) < 1e-15
    assert r[0] < 3.0 / T ** 2 and 1.0 - r[T - 2] < 3.0 / T ** 2
    assert np.all(inlet_speeds(0, 3) == 1.0)


def test_nee_boundary_nodes(orc):
    """Non-equilibrium extrapolation: the boundary node carries the imposed
    macroscopic state (inlet: u prescribed, rho of the interior neighbour;
    outlet: rho_out, u of the neighbour) plus the neighbour's non-equilibrium
    part, checked with the independent product-form equilibrium."""
    flags = duct_flags(4, 8)
    n = flags.size
    g = np.random.default_rng(8)
    L = orc.Lattice(flags, omega=1.5, periodic=3, u_in=0.02, rho_out=1.001,
                    profile=orc.PARABOLIC, d_in=4.0, axis=(2.0, 2.0), noise_amp=0.01, seed=5)
    L.init_equilibrium(1.0 + 0.01 * g.uniform(-1, 1, n), 0.03 * g.uniform(-1, 1, (n, 3)))
    L.f *= 1.0 + 0.02 * g.uniform(-1, 1, L.f.shape)
    L.step(1)
    mom = L.last_moments          # recorded by the step (the statistics use these)
    field = L.moments()           # read back from the populations
    nx = ny = 4
    for y in range(ny):
        for x in range(nx):
            for z, kind in ((0, 2), (7, 3)):
                b = x + nx * (y + ny * z)
                bf, nrm = L.nee_neighbour(x, y, z)
                assert bf == x + nx * (y + ny * (1 if z == 0 else 6))
                rf, uf = mom[bf, 0], mom[bf, 1:]
                if kind == 2:
                    r2 = (x + 0.5 - 2.0) ** 2 + (y + 0.5 - 2.0) ** 2
                    ub = np.array([0.0, 0.0, 2 * 0.02 * (1 - 4 * r2 / 16.0)])
                    ub += np.array([0.01 * 0.02 * orc.noise(5, 1, b, a) for a in range(3)])
                    rb = rf
                else:
                    ub, rb = uf, 1.001
                neq_f = L.f[bf] - product_form_equilibrium(rf, uf)
                expect = product_form_equilibrium(rb, ub) + neq_f
                assert np.allclose(L.f[b], expect, atol=1e-15)
                got = orc.moments(L.f[b])
                assert abs(got[0] - rb) < 1e-14 and np.allclose(got[1:], ub, atol=1e-14)
                for m in (mom[b], field[b]):
                    assert abs(m[0] - rb) < 1e-14 and np.allclose(m[1:], ub, atol=1e-14)


def test_nee_partner_must_be_unique(orc):
    """An inlet node's interior partner is its one FLUID axis neighbour: a
    node with two or with none has no partner, and the step refuses the flag
    field."""
    flags = np.ones((4, 3, 3), dtype=np.uint8)
    flags[0, 1, 1] = 2          # inlet whose +x, -x, +y, -y and +z neighbours are all fluid
    L = orc.Lattice(flags, omega=1.0, periodic=3)
    assert L.nee_neighbour(1, 1, 0)[0] == -1
    L.init_equilibrium(1.0, [0.0, 0.0, 0.0])
    with pytest.raises(RuntimeError):
        L.step(1)
    flags = np.zeros((4, 3, 3), dtype=np.uint8)
    flags[0, 1, 1] = 2          # inlet without any fluid neighbour
    flags[2:, 1, 1] = 1
    L = orc.Lattice(flags, omega=1.0)
    assert L.nee_neighbour(1, 1, 0)[0] == -1
    duct = duct_flags(4, 8)     # every inlet node of a duct has exactly one
    L = orc.Lattice(duct, omega=1.0, periodic=3)
    assert all(L.nee_neighbour(x, y, 0)[0] == x + 4 * (y + 4) for x in range(4) for y in range(4))


# -------------------------------------------------------------- noise, totals

def test_splitmix64_reference_outputs(orc):
    """SplitMix64 (Steele, Lea, Flood 2014), generator state 0: the first two
    outputs of the public reference implementation."""
    assert orc.splitmix64(0) == 0xE220A8397B1DCDAF
    assert orc.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_noise_uniform(orc):
    vals = np.array([orc.noise(3, s, node, c) for s in range(20) for node in range(200) for c in range(3)])
    assert vals.min() >= -1.0 and vals.max() < 1.0
    assert np.all(((vals + 1.0) * 2 ** 23) == np.round((vals + 1.0) * 2 ** 23))   # 24-bit grid
    hist, _ = np.histogram(vals, bins=10, range=(-1, 1))
    expected = len(vals) / 10
    chi2 = ((hist - expected) ** 2 / expected).sum()
    assert chi2 < 30.0          # 9 dof, p ~ 4e-4
    assert abs(vals.mean()) < 0.02
    assert orc.noise(3, 4, 5, 1) == orc.noise(3, 4, 5, 1)
    assert orc.noise(3, 4, 5, 1) != orc.noise(3, 4, 5, 2)


def test_noise_depends_on_every_counter(orc):
    """The draw for (seed, step, node, component) changes with each of the
    four: streams that differ in one counter are uncorrelated and share no
    value (24-bit draws coincide with probability 2^-24)."""
    base = dict(seed=3, step=7, node=0, comp=0)
    for key, other in (("seed", 4), ("step", 8), ("node", None), ("comp", 2)):
        a, b = [], []
        for k in range(600):
            p = dict(base, node=k)
            q = dict(p, **{key: other}) if other is not None else dict(p, node=k + 600)
            a.append(orc.noise(p["seed"], p["step"], p["node"], p["comp"]))
            b.append(orc.noise(q["seed"], q["step"], q["node"], q["comp"]))
        a, b = np.array(a), np.array(b)
        assert np.count_nonzero(a == b) <= 1, key
        assert abs(np.corrcoef(a, b)[0, 1]) < 0.15, key
    # distinct (node, component) pairs give independent draws: among 3000
    # 24-bit draws about 0.27 coincide by chance (birthday bound), while two
    # pairs that share a counter value would repeat a draw every time
    repeats = 0
    for seed, step in ((1, 1), (2, 5), (11, 7)):
        grid = np.array([orc.noise(seed, step, node, comp) for node in range(1000) for comp in range(3)])
        repeats += grid.size - np.unique(grid).size
    assert repeats <= 6


def test_totals_compensated_on_an_ill_conditioned_sum(orc):
    """Totals of 57 unit masses between +1e16 and -1e16: a plain running sum
    loses every unit (half an ulp of 1e16 is 1), a compensated one stays
    within Kahan's bound 2 eps sum|x| (about 4.4) of the exact 57."""
    flags = np.ones((3, 4, 5), dtype=np.uint8)
    flags[1, 1, 1] = 0
    act = np.nonzero(flags.reshape(-1) != 0)[0]
    f = np.zeros((flags.size, Q))
    f[act, 13] = 1.0
    f[act[0], 13], f[act[-1], 13] = 1e16, -1e16
    L = orc.Lattice(flags, omega=1.0)
    L.set_populations(f)
    exact = math.fsum(f[act, 13])
    bound = 2.0 * np.finfo(float).eps * np.abs(f[act, 13]).sum()
    plain = 0.0
    for v in f[act, 13]:
        plain += v
    assert exact == 57.0 and abs(plain - exact) > bound
    assert abs(L.totals()[0] - exact) <= bound


def test_totals_compensated(orc):
    flags = np.ones((3, 4, 5), dtype=np.uint8)
    flags[1, 1, 1] = 0
    g = np.random.default_rng(1)
    f = g.uniform(0, 0.1, size=(flags.size, Q))
    L = orc.Lattice(flags, omega=1.0)
    L.set_populations(f)
    act = flags.reshape(-1) != 0
    c = vel()
    exp = [math.fsum(f[act].ravel())] + [math.fsum((f[act] * c[:, a]).ravel()) for a in range(3)]
    assert np.allclose(L.totals(), exp, rtol=1e-15, atol=1e-15)


# ------------------------------------------------------------------- geometry

def test_nozzle_voxel_counts():
    """Active-cell counts of the three synthetic nozzles (geometry recipe of the
    workload definitions: D = 3 d, 10-degree cone, 4 d throat)."""
    assert I.active_count(I.workload_flags("nozzle_re500_24x24x160")) == 48716
    assert I.active_count(I.workload_flags("nozzle_re3500_96x96x800")) == 4286996
    f = I.workload_flags("nozzle_re500_24x24x160")
    assert (f[0] == 2).sum() == (f[1] != 0).sum() and (f[-1] == 3).sum() == (f[-2] != 0).sum()


def test_wall_distances_of_a_round_pipe():
    """inputs.nozzle_wall_q on a straight pipe of radius R: every wall link's
    q is the root of |p_xy - s c_xy - centre| = R along the link, found in
    closed form (quadratic), to within the 1/256 quantisation; links that
    stay inside keep 128."""
    D, L = 16, 6
    cells, q = I.nozzle_wall_q(D, D, L, L_in=L, L_cone=1, L_throat=0)
    flags = I.pipe_flags(D, L)
    nz, ny, nx = flags.shape
    c = np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)], dtype=float)
    R = D / 2.0
    checked = 0
    for b, row in zip(cells, q):
        x, y, z = b % nx, (b // nx) % ny, b // (nx * ny)
        assert flags[z, y, x] == 1
        px, py = x + 0.5 - R, y + 0.5 - R
        for i in range(27):
            sx, sy, sz = x - int(c[i, 0]), y - int(c[i, 1]), z - int(c[i, 2])
            inside_box = 0 <= sx < nx and 0 <= sy < ny and 0 <= sz < nz
            solid = not inside_box or flags[sz, sy, sx] == 0
            if not solid:
                assert row[i] == 128
                continue
            # |(px - s cx, py - s cy)| = R, smallest root in (0, 1]
            a = c[i, 0] ** 2 + c[i, 1] ** 2
            bq = -2.0 * (px * c[i, 0] + py * c[i, 1])
            cq = px * px + py * py - R * R
            s = (-bq + math.sqrt(bq * bq - 4 * a * cq)) / (2 * a)
            assert abs(row[i] / 256.0 - s) <= 0.5 / 256 + 1e-9, (b, i, row[i], s)
            checked += 1
    assert checked > 1000
