"""Helpers shared by the GPU tests: build both sides from the same seeded
inputs, and compute single-cell oracle updates for sampled parity checks."""
import numpy as np

from paper_2204_10566_gb300 import inputs as I

Q = 27
VEL = np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(Q)], dtype=np.int64)


def omega_of_nu(nu):
    """Sec. 2.1 relaxation-time relation in lattice units (oracle side)."""
    return 1.0 / (3.0 * nu + 0.5)


def oracle_lattice(orc, flags, nu, periodic=0, ghost=(1.0, 1.0, 1.0, 1.0), profile="plug", u_in=0.0, d_in=None,
                   noise_amp=0.0, seed=0, rho_out=1.0, ramp=0, wall_q=None):
    nz, ny, nx = flags.shape
    return orc.Lattice(flags, omega_of_nu(nu), ghost=ghost, periodic=periodic,
                       profile=orc.PLUG if profile == "plug" else orc.PARABOLIC, u_in=u_in,
                       d_in=d_in if d_in else nx, axis=(nx / 2.0, ny / 2.0), noise_amp=noise_amp, seed=seed,
                       rho_out=rho_out, ramp=ramp, wall_q=wall_q)


def gpu_lattice(lbm, flags, precision, nu, periodic=0, ghost=(1.0, 1.0, 1.0, 1.0), profile="plug", u_in=0.0,
                d_in=None, noise_amp=0.0, seed=0, rho_out=1.0, fp16_scale=0.0, ramp=0, rows="auto"):
    nz, ny, nx = flags.shape
    G = lbm.Lattice(flags, precision, periodic=periodic, fp16_scale=fp16_scale, row_axis=rows)
    G.set_params(nu=nu, ghost=ghost, u_in=u_in, d_in=d_in if d_in else nx, profile=profile,
                 noise_amp=noise_amp, noise_seed=seed, rho_out=rho_out, inlet_ramp=ramp)
    return G


def random_state(orc, flags, seed, rho_amp=0.01, u_amp=0.03, neq_amp=0.01):
    """Near-equilibrium populations on the box (solid cells 0): equilibrium of
    seeded random rho, u (oracle) times a seeded random relative perturbation."""
    n = flags.size
    rho = I.random_density_field(n, rho_amp, seed)
    u = I.random_velocity_field(n, u_amp, seed + 1)
    act = flags.reshape(-1) != 0
    f = np.zeros((n, Q))
    for b in np.nonzero(act)[0]:
        f[b] = orc.equilibrium(rho[b], u[b])
    f *= 1.0 + I.random_uniform((n, Q), neq_amp, seed + 2)
    return f


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


# ------------------------------------------------------- single-cell oracle

def _flag(flags, x, y, z, periodic):
    nz, ny, nx = flags.shape
    for v, n, bit in ((x, nx, 1), (y, ny, 2), (z, nz, 4)):
        if (v < 0 or v >= n) and not periodic & bit:
            return 0, None
    x, y, z = x % nx, y % ny, z % nz
    return flags[z, y, x], (z * ny + y) * nx + x


def gather_cell(f, flags, x, y, z, periodic):
    """Pull-stream gather with halfway bounce-back for one cell from a dense
    box state f[b, i] (restated from Sec. 2.1/2.2 for sampling)."""
    nz, ny, nx = flags.shape
    b = (z * ny + y) * nx + x
    out = np.empty(Q)
    for i in range(Q):
        cx, cy, cz = VEL[i]
        fl, src = _flag(flags, x - cx, y - cy, z - cz, periodic)
        out[i] = f[b, Q - 1 - i] if fl == 0 else f[src, i]
    return out


def oracle_cell_update(orc, f, flags, x, y, z, periodic, omega, ghost=(1.0, 1.0, 1.0, 1.0), inlet=None, t_new=1):
    """Post-collision populations of one active cell after one step, from the
    oracle's collision and equilibrium.  inlet: dict(profile, u_in, d_in,
    axis, noise_amp, seed, rho_out) for boundary nodes."""
    nz, ny, nx = flags.shape
    kind = flags[z, y, x]
    if kind == 1:
        return orc.collide(gather_cell(f, flags, x, y, z, periodic), omega, ghost)
    dirs = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    part = [d for d in dirs if _flag(flags, x + d[0], y + d[1], z + d[2], periodic)[0] == 1]
    assert len(part) == 1
    n = part[0]
    xf, yf, zf = (x + n[0]) % nx, (y + n[1]) % ny, (z + n[2]) % nz
    ff, mf = orc.collide(gather_cell(f, flags, xf, yf, zf, periodic), omega, ghost)
    rf, uf = mf[0], mf[1:]
    if kind == 2:
        speed = inlet["u_in"]
        if inlet["profile"] == "parabolic":
            r2 = (x + 0.5 - inlet["axis"][0]) ** 2 + (y + 0.5 - inlet["axis"][1]) ** 2
            speed = 2.0 * inlet["u_in"] * (1.0 - 4.0 * r2 / inlet["d_in"] ** 2)
        ub = np.array(n, dtype=float) * speed
        node = (z * ny + y) * nx + x
        if inlet["noise_amp"]:
            ub = ub + np.array([inlet["noise_amp"] * inlet["u_in"] * orc.noise(inlet["seed"], t_new, node, a)
                                for a in range(3)])
        if t_new < inlet.get("ramp", 0):
            s = t_new / inlet["ramp"]
            ub = ub * (s * s * (3.0 - 2.0 * s))
        rb = rf
    else:
        ub, rb = uf, inlet["rho_out"]
    fb = orc.equilibrium(rb, ub) + (ff - orc.equilibrium(rf, uf))
    return fb, np.concatenate([[rb], ub])
