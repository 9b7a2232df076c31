"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds no lattice Boltzmann arithmetic: only geometry (flag
fields), workload descriptions, and seeded random numbers.  Both sides of a
parity test take their inputs from here and compute everything else on their
own.

Geometry: the FDA benchmark nozzle of Sec. 2.2 (axisymmetric: inlet pipe,
conical contraction, throat, sudden expansion) voxelised on a box whose axis
is z.  The real FDA CAD lengths are in a figure the text does not carry, so the
lengths follow the workload definitions below: inlet pipe diameter D = 3 d
(the inlet/throat Reynolds ratio of 3 quoted in Sec. 3), inlet pipe length D,
a 10-degree half-angle cone, a 4 d throat, and the expansion pipe for the rest.
Voxel (x, y, z) is inside iff (x+1/2-D/2)^2 + (y+1/2-D/2)^2 <= r(z+1/2)^2.

Flag values: 0 SOLID, 1 FLUID, 2 INLET (plane z = 0), 3 OUTLET (plane z = nz-1).
"""
import math

import numpy as np

SOLID, FLUID, INLET, OUTLET = 0, 1, 2, 3


def cone_length(D, d, half_angle_deg=10.0):
    """Axial length of a cone from radius D/2 to d/2 at the given half-angle."""
    return int(round((D - d) / 2.0 / math.tan(math.radians(half_angle_deg))))


def nozzle_radius(z_centre, D, d, L_in, L_cone, L_throat, half_angle_deg=10.0):
    """Wall radius r(z) of the nozzle at axial position z_centre (cells).  In
    the cone the wall keeps the true half-angle, r = D/2 - (z - L_in) tan(angle),
    never below d/2 (L_cone is rounded to whole cells)."""
    if z_centre < L_in:
        return D / 2.0
    if z_centre < L_in + L_cone:
        r = D / 2.0 - (z_centre - L_in) * math.tan(math.radians(half_angle_deg))
        return max(r, d / 2.0)
    if z_centre < L_in + L_cone + L_throat:
        return d / 2.0
    return D / 2.0


def nozzle_flags(D, d, L_total, L_in=None, L_cone=None, L_throat=None, half_angle_deg=10.0,
                 inlet=True, outlet=True):
    """Flag field (nz, ny, nx) = (L_total, D, D) of the voxelised nozzle."""
    L_in = D if L_in is None else L_in
    L_cone = cone_length(D, d, half_angle_deg) if L_cone is None else L_cone
    L_throat = 4 * d if L_throat is None else L_throat
    c = np.arange(D) + 0.5 - D / 2.0
    r2 = c[None, :] ** 2 + c[:, None] ** 2          # [y, x]
    flags = np.zeros((L_total, D, D), dtype=np.uint8)
    for z in range(L_total):
        r = nozzle_radius(z + 0.5, D, d, L_in, L_cone, L_throat, half_angle_deg)
        flags[z][r2 <= r * r] = FLUID
    if inlet:
        flags[0][flags[0] == FLUID] = INLET
    if outlet:
        flags[-1][flags[-1] == FLUID] = OUTLET
    return flags


def nozzle_radius_array(z, D, d, L_in, L_cone, L_throat, half_angle_deg=10.0):
    """nozzle_radius for an array of axial positions."""
    z = np.asarray(z, dtype=np.float64)
    t = math.tan(math.radians(half_angle_deg))
    cone = np.maximum(D / 2.0 - (z - L_in) * t, d / 2.0)
    r = np.where(z < L_in, D / 2.0, np.where(z < L_in + L_cone, cone,
                                              np.where(z < L_in + L_cone + L_throat, d / 2.0, D / 2.0)))
    return r


def nozzle_wall_q(D, d, L_total, L_in=None, L_cone=None, L_throat=None, half_angle_deg=10.0, flags=None,
                  iterations=40):
    """Wall distances of the smooth nozzle surface for the interpolated
    bounce-back: for every FLUID cell of the voxelised nozzle and every link i
    whose pull source x - c_i is solid (or outside the box), the fraction q of
    the link, from the cell centre towards x - c_i, at which the segment
    first leaves the nozzle (bisection on the signed radius distance).
    Returns (cells, q): box indices (n,) and q quantised to uint8 in 1/256
    (1..255) as an (n, 27) array, 128 on the other links."""
    L_in = D if L_in is None else L_in
    L_cone = cone_length(D, d, half_angle_deg) if L_cone is None else L_cone
    L_throat = 4 * d if L_throat is None else L_throat
    if flags is None:
        flags = nozzle_flags(D, d, L_total, L_in, L_cone, L_throat, half_angle_deg)
    nz, ny, nx = flags.shape
    c = np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)])
    # candidates: FLUID cells with a solid (or outside) cell among their 26
    # neighbours, in box order; the others have no wall link
    solid = np.pad(flags == SOLID, 1, constant_values=True)
    near = np.zeros(flags.shape, dtype=bool)
    for i in range(27):
        near |= solid[1 - c[i, 2]:1 - c[i, 2] + nz, 1 - c[i, 1]:1 - c[i, 1] + ny, 1 - c[i, 0]:1 - c[i, 0] + nx]
    fz, fy, fx = np.nonzero((flags == FLUID) & near)
    del solid, near
    solid_src = np.zeros((fz.size, 27), dtype=bool)
    for i in range(27):
        sx, sy, sz = fx - c[i, 0], fy - c[i, 1], fz - c[i, 2]
        inside = (sx >= 0) & (sx < nx) & (sy >= 0) & (sy < ny) & (sz >= 0) & (sz < nz)
        fl = np.zeros(fz.size, dtype=np.uint8)
        fl[inside] = flags[sz[inside], sy[inside], sx[inside]]
        solid_src[:, i] = fl == SOLID
    rows = np.nonzero(solid_src.any(axis=1))[0]
    q = np.full((rows.size, 27), 128, dtype=np.uint8)
    px, py, pz = fx[rows] + 0.5, fy[rows] + 0.5, fz[rows] + 0.5

    def outside(s, i, sel):  # points at fraction s of link i from the centres of cells sel
        x, y, z = px[sel] - s * c[i, 0], py[sel] - s * c[i, 1], pz[sel] - s * c[i, 2]
        r = np.hypot(x - D / 2.0, y - D / 2.0)
        return r > nozzle_radius_array(z, D, d, L_in, L_cone, L_throat, half_angle_deg)

    for i in range(27):
        sel = solid_src[rows, i]
        if not sel.any():
            continue
        lo = np.zeros(int(sel.sum()))
        hi = np.ones(lo.size)
        for _ in range(iterations):
            mid = 0.5 * (lo + hi)
            out = outside(mid, i, sel)
            hi = np.where(out, mid, hi)
            lo = np.where(out, lo, mid)
        q[sel, i] = np.clip(np.rint(hi * 256.0), 1, 255).astype(np.uint8)
    cells = (fx[rows].astype(np.int64) + nx * (fy[rows].astype(np.int64) + ny * fz[rows].astype(np.int64)))
    return cells, q


def pipe_flags(D, L_total, inlet=True, outlet=True):
    """Straight circular pipe of diameter D (cells) along z."""
    return nozzle_flags(D, D, L_total, L_in=L_total, L_cone=1, L_throat=0, inlet=inlet, outlet=outlet)


def box_flags(nx, ny, nz):
    """All-fluid box (use with periodic boundaries)."""
    return np.full((nz, ny, nx), FLUID, dtype=np.uint8)


def channel_flags(nx, ny, nz):
    """All-fluid box whose y faces are walls when y is not periodic."""
    return box_flags(nx, ny, nz)


def active_count(flags):
    return int(np.count_nonzero(flags != SOLID))


# ------------------------------------------------------------------ workloads

WORKLOADS = {
    # Re 500 laminar nozzle: D = 24, d = 8, lengths 24/45/32/59, plug inlet.
    "nozzle_re500_24x24x160": dict(kind="nozzle", D=24, d=8, L_total=160, Re=500.0, u_throat=0.05,
                                   profile="plug", noise=0.0, seed=0, steps=200),
    # Re 3500 transitional nozzle: D = 96, d = 32, parabolic inlet + 1 % noise.
    # The two jet workloads start the inlet smoothly over `ramp` steps: an
    # impulsive start sends a pressure pulse through the nozzle that, with
    # almost no bulk damping at tau -> 1/2, blew up most Re 6500 runs near
    # the cone-throat junction around step 6000.
    "nozzle_re3500_96x96x800": dict(kind="nozzle", D=96, d=32, L_total=800, Re=3500.0, u_throat=0.05,
                                    profile="parabolic", noise=0.01, seed=1, steps=20000, ramp=8000),
    # Re 6500 under-resolved turbulent nozzle: D = 144, d = 48, parabolic + 2 % noise.
    "nozzle_re6500_144x144x1200": dict(kind="nozzle", D=144, d=48, L_total=1200, Re=6500.0,
                                       u_throat=0.05, profile="parabolic", noise=0.02, seed=2,
                                       steps=50000, ramp=8000),
    # Periodic Taylor-Green vortex, 256^3, u0 = 0.04.
    "tgv_256": dict(kind="tgv", n=256, u0=0.04, Re=1600.0, steps=1000),
}


# Throat diameters (cells) of the resolution ladder R1-R3 (Sec. 3).  The
# grid spacings of Table 2, 2.3, 1.725 and 1.15 (x 1e-4 m), on the 4 mm
# throat give 17.4, 23.2 and 34.8 cells; these are rounded up to multiples
# of 6, which keeps the table's spacing ratios 1 : 4/3 : 2 exactly.
# Throat diameters (cells) of the resolution ladder: Table 2's R1-R4 grid
# spacings (Re 6500) over a 4 mm throat are 17.4, 23.2, 34.8 and 51.5 cells;
# R1-R3 keep the table's spacing ratios 1 : 4/3 : 2 exactly, R4 is rounded up.
LADDER_THROAT_CELLS = (18, 24, 36, 52)


def workload_flags(name):
    w = WORKLOADS[name]
    if w["kind"] == "nozzle":
        return nozzle_flags(w["D"], w["d"], w["L_total"])
    if w["kind"] == "pipe":
        return pipe_flags(w["D"], w["L_total"])
    if w["kind"] == "tgv":
        return box_flags(w["n"], w["n"], w["n"])
    raise KeyError(name)


def inlet_mean_velocity(w):
    """Mean inlet velocity u0 = u_throat (d/D)^2 (Sec. 2.2 throat-velocity relation)."""
    return w["u_throat"] * (w["d"] / w["D"]) ** 2


def workload_params(name):
    """Flow parameters of a nozzle or pipe workload, as keyword arguments of
    the library's parameter set (Re on the throat, throat mean velocity and
    diameter as the characteristic scales)."""
    w = WORKLOADS[name]
    return dict(Re=w["Re"], u_char=w["u_throat"], L_char=float(w["d"]), u_in=inlet_mean_velocity(w),
                d_in=float(w["D"]), profile=w["profile"], noise_amp=w["noise"], noise_seed=w["seed"],
                inlet_ramp=w.get("ramp", 0))


# ------------------------------------------------------------- random fields

def rng(seed):
    return np.random.default_rng(seed)


def random_uniform(shape, amplitude, seed):
    """Uniform numbers in [-amplitude, amplitude) with a fixed seed."""
    return amplitude * (2.0 * rng(seed).random(shape) - 1.0)


def random_velocity_field(n, amplitude, seed):
    """(n, 3) velocities, uniform in [-amplitude, amplitude)."""
    return random_uniform((n, 3), amplitude, seed)


def random_density_field(n, amplitude, seed):
    """(n,) densities 1 + uniform in [-amplitude, amplitude)."""
    return 1.0 + random_uniform((n,), amplitude, seed)


def serving_requests(n=64, seed=2204, rate=None, d_range=(8, 48), re_range=(500.0, 6500.0),
                     steps_range=(2000, 20000), scale=1.0):
    """Seeded request stream for the serving loop: Poisson arrivals, nozzle or
    pipe geometries of throat diameter d (D = 3 d, L = 25 d, each scaled by
    ``scale``), Re uniform in re_range, step counts uniform in steps_range,
    storage FP32 or FP16-shifted with probability 1/2."""
    g = rng(seed)
    rate = 1.0 if rate is None else rate
    t = 0.0
    out = []
    for k in range(n):
        t += g.exponential(1.0 / rate)
        d = int(g.integers(d_range[0], d_range[1] + 1))
        d = max(4, int(round(d * scale)))
        out.append(dict(
            id=k,
            arrival=t,
            kind="nozzle" if g.random() < 0.5 else "pipe",
            d=d, D=3 * d, L_total=25 * d,
            Re=float(g.uniform(*re_range)),
            steps=int(g.integers(steps_range[0], steps_range[1] + 1)),
            precision="fp32" if g.random() < 0.5 else "fp16s",
        ))
    return out
