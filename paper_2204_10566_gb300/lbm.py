"""Thin Python binding of the C ABI in include/lbm.h.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``liblbm.so``.  PyTorch supplies device memory (through the
library's allocator callback) and the CUDA stream.  There is no CPU fallback:
if the library is missing, importing ``capi()`` raises.

``capi()`` returns the raw ctypes library with the C signatures declared, so
every C call is available under its own name.  ``Lattice`` wraps one context
with numpy in/out arrays; its methods call the C functions of the same names.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_STATE, LBM_ERR_UNSTABLE, LBM_ERR_TIMEOUT = range(7)
LBM_FP64, LBM_FP32, LBM_FP16S = 0, 1, 2
LBM_SOLID, LBM_FLUID, LBM_INLET, LBM_OUTLET = 0, 1, 2, 3
LBM_PROFILE_PLUG, LBM_PROFILE_PARABOLIC = 0, 1
LBM_LAYOUT_ACTIVE, LBM_LAYOUT_BOX = 0, 1
LBM_PERIODIC_X, LBM_PERIODIC_Y, LBM_PERIODIC_Z = 1, 2, 4
LBM_ROWS_AUTO, LBM_ROWS_X, LBM_ROWS_Z = 0, 1, 2
ROW_AXES = {"auto": LBM_ROWS_AUTO, "x": LBM_ROWS_X, "z": LBM_ROWS_Z}
LBM_STATS_AXIAL, LBM_STATS_FULL = 0, 1
LBM_STATS_FULL_COMPONENTS = 16

PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16s": LBM_FP16S}
PROFILES = {"plug": LBM_PROFILE_PLUG, "parabolic": LBM_PROFILE_PARABOLIC}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class lbm_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class lbm_desc(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("periodic", C.c_int32), ("precision", C.c_int32),
        ("fp16_scale", C.c_float), ("device", C.c_int32), ("row_axis", C.c_int32),
        ("stream", C.c_void_p),
        ("allocator", lbm_allocator),
    ]


class lbm_params(C.Structure):
    _fields_ = [
        ("nu", C.c_double), ("Re", C.c_double), ("u_char", C.c_double), ("L_char", C.c_double),
        ("omega3", C.c_double), ("omega4", C.c_double), ("omega5", C.c_double), ("omega6", C.c_double),
        ("u_in", C.c_double), ("d_in", C.c_double), ("axis_x", C.c_double), ("axis_y", C.c_double),
        ("noise_amp", C.c_double), ("rho_out", C.c_double),
        ("noise_seed", C.c_uint64),
        ("inlet_profile", C.c_int32), ("inlet_ramp", C.c_int32),
    ]


class lbm_physical(C.Structure):
    _fields_ = [
        ("Re", C.c_double), ("d_thr", C.c_double), ("rho", C.c_double), ("mu", C.c_double),
        ("delta_r", C.c_double), ("delta_t", C.c_double), ("CFL", C.c_double),
    ]


class lbm_server_desc(C.Structure):
    _fields_ = [
        ("device", C.c_int32), ("stream", C.c_void_p), ("allocator", lbm_allocator),
        ("budget_bytes", C.c_int64), ("max_slots", C.c_int32), ("steps_per_tick", C.c_int32),
    ]


class lbm_request(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("periodic", C.c_int32),
        ("precision", C.c_int32), ("fp16_scale", C.c_float), ("flags", C.c_void_p),
        ("params", lbm_params), ("steps", C.c_int64),
    ]


LBM_REQ_QUEUED, LBM_REQ_RUNNING, LBM_REQ_DONE, LBM_REQ_CANCELLED, LBM_REQ_FAILED = range(5)


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (_STATUS.get(status, "?"), status, msg))
        self.status = status


_STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error", 4: "call out of order",
           5: "non-finite state", 6: "device wait timed out"}

_lib = None

_dp = C.POINTER(C.c_double)
_SIGS = {
    "lbm_status_string": (C.c_char_p, [C.c_int]),
    "lbm_params_default": (None, [C.POINTER(lbm_params)]),
    "lbm_create": (C.c_int, [C.POINTER(lbm_desc), C.POINTER(C.c_void_p)]),
    "lbm_destroy": (C.c_int, [C.c_void_p]),
    "lbm_last_error": (C.c_char_p, [C.c_void_p]),
    "lbm_make_nozzle": (C.c_int, [C.c_int32] * 6 + [C.c_double, C.c_void_p]),
    "lbm_check_layout": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                   C.POINTER(C.c_int64)]),
    "lbm_set_geometry": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_fluid_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "lbm_set_wall_q": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "lbm_set_params": (C.c_int, [C.c_void_p, C.POINTER(lbm_params)]),
    "lbm_params_check": (C.c_int, [C.POINTER(lbm_params), _dp, _dp, C.POINTER(C.c_char_p)]),
    "lbm_params_from_physical": (C.c_int, [C.POINTER(lbm_physical), C.POINTER(lbm_params), _dp,
                                           C.POINTER(C.c_char_p)]),
    "lbm_get_omega": (C.c_int, [C.c_void_p, _dp]),
    "lbm_init_equilibrium": (C.c_int, [C.c_void_p, C.c_double, _dp]),
    "lbm_init_fields": (C.c_int, [C.c_void_p, _dp, _dp, C.c_int32]),
    "lbm_set_populations": (C.c_int, [C.c_void_p, _dp, C.c_int32]),
    "lbm_get_populations": (C.c_int, [C.c_void_p, _dp, C.c_int32]),
    "lbm_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "lbm_sync": (C.c_int, [C.c_void_p]),
    "lbm_step_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "lbm_set_check_every": (C.c_int, [C.c_void_p, C.c_int64]),
    "lbm_get_moments": (C.c_int, [C.c_void_p, _dp, _dp, C.c_int32]),
    "lbm_get_totals": (C.c_int, [C.c_void_p, _dp, _dp]),
    "lbm_get_health": (C.c_int, [C.c_void_p, _dp]),
    "lbm_stats_begin": (C.c_int, [C.c_void_p, C.c_int64]),
    "lbm_stats_end": (C.c_int, [C.c_void_p]),
    "lbm_stats_reset": (C.c_int, [C.c_void_p]),
    "lbm_stats_get": (C.c_int, [C.c_void_p, _dp, _dp, C.POINTER(C.c_int64), C.c_int32]),
    "lbm_stats_set_mode": (C.c_int, [C.c_void_p, C.c_int32]),
    "lbm_stats_get_full": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_int64), C.c_int32]),
    "lbm_checkpoint_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "lbm_checkpoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "lbm_restore": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "lbm_layout_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "lbm_kernel_launches": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "lbm_totals_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_float, C.c_int64, C.c_int64, C.c_void_p,
                                     C.c_void_p]),
    "lbm_server_create": (C.c_int, [C.POINTER(lbm_server_desc), C.POINTER(C.c_void_p)]),
    "lbm_server_destroy": (C.c_int, [C.c_void_p]),
    "lbm_server_last_error": (C.c_char_p, [C.c_void_p]),
    "lbm_server_submit": (C.c_int, [C.c_void_p, C.POINTER(lbm_request), C.POINTER(C.c_int64)]),
    "lbm_server_tick": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lbm_server_poll": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "lbm_server_cells": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "lbm_server_result": (C.c_int, [C.c_void_p, C.c_int64, _dp, _dp]),
    "lbm_server_cancel": (C.c_int, [C.c_void_p, C.c_int64]),
    "lbm_server_info": (C.c_int, [C.c_void_p, _dp]),
    "lbm_server_check_request": (C.c_int, [C.POINTER(lbm_request), C.c_int64, C.POINTER(C.c_int64),
                                           C.POINTER(C.c_char_p)]),
}


def declared_functions():
    """Names of the C functions this binding declares (all of include/lbm.h)."""
    return sorted(_SIGS)


def capi():
    """The loaded ``liblbm.so`` with argument/return types declared."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblbm.so is not built (run __graft_entry__.build()); there is no fallback")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


def make_params(nu=0.0, Re=0.0, u_char=0.0, L_char=0.0, ghost=(1.0, 1.0, 1.0, 1.0), u_in=0.0, d_in=0.0,
                axis=(-1.0, -1.0), noise_amp=0.0, noise_seed=0, rho_out=1.0, profile="plug", inlet_ramp=0):
    """An lbm_params filled from lbm_params_default and the given values."""
    p = lbm_params()
    capi().lbm_params_default(C.byref(p))
    p.nu, p.Re, p.u_char, p.L_char = nu, Re, u_char, L_char
    p.omega3, p.omega4, p.omega5, p.omega6 = (float(g) for g in ghost)
    p.u_in, p.d_in = u_in, d_in
    p.axis_x, p.axis_y = axis
    p.noise_amp, p.noise_seed, p.rho_out = noise_amp, int(noise_seed), rho_out
    p.inlet_profile = PROFILES[profile] if isinstance(profile, str) else int(profile)
    p.inlet_ramp = int(inlet_ramp)
    return p


def params_check(p):
    """lbm_params_check: (nu, omega) of a parameter set, on the host; raises
    LbmError naming the failed check."""
    nu, omega, why = C.c_double(), C.c_double(), C.c_char_p()
    st = capi().lbm_params_check(C.byref(p), C.byref(nu), C.byref(omega), C.byref(why))
    if st != LBM_OK:
        raise LbmError(st, "lbm_params_check: " + why.value.decode())
    return nu.value, omega.value


def params_from_physical(Re, delta_r, rho, mu, d_thr, delta_t=0.0, CFL=0.0, **kw):
    """lbm_params_from_physical: (lbm_params, dict) of a run given in
    physical units (SI).  The params hold Re, u_char and L_char (plus any
    make_params keywords); the dict holds Re, L_char, u_char, nu, CFL and
    delta_t.  Give delta_t, or CFL for the time step of the CFL rule."""
    ph = lbm_physical(Re=float(Re), d_thr=float(d_thr), rho=float(rho), mu=float(mu), delta_r=float(delta_r),
                      delta_t=float(delta_t), CFL=float(CFL))
    p = make_params(**kw)
    out = (C.c_double * 5)()
    why = C.c_char_p()
    st = capi().lbm_params_from_physical(C.byref(ph), C.byref(p), out, C.byref(why))
    if st != LBM_OK:
        raise LbmError(st, "lbm_params_from_physical: " + why.value.decode())
    lu = dict(zip(["L_char", "u_char", "nu", "CFL", "delta_t"], list(out)))
    lu["Re"] = float(Re)
    return p, lu


def lattice_units(Re, delta_r, delta_t, rho, mu, d_thr):
    """Lattice units of a physical run with a given time step
    (lbm_params_from_physical): dict with Re, L_char, u_char, nu, CFL and
    delta_t."""
    return params_from_physical(Re, delta_r, rho, mu, d_thr, delta_t=delta_t)[1]


def cfl_time_step(Re, delta_r, CFL, rho, mu, d_thr):
    """Time step (s) of the CFL rule for a physical run
    (lbm_params_from_physical with a CFL number instead of a time step)."""
    return params_from_physical(Re, delta_r, rho, mu, d_thr, CFL=CFL)[1]["delta_t"]


def make_nozzle(D, d, L_total, L_in=None, L_cone=-1, L_throat=None, half_angle_deg=10.0):
    """lbm_make_nozzle: flag field (L_total, D, D) uint8."""
    out = np.zeros((L_total, D, D), dtype=np.uint8)
    L_in = D if L_in is None else L_in
    L_throat = 4 * d if L_throat is None else L_throat
    st = capi().lbm_make_nozzle(D, d, L_in, L_cone, L_throat, L_total, half_angle_deg, out.ctypes.data)
    if st != LBM_OK:
        raise LbmError(st, "lbm_make_nozzle")
    return out


def check_layout(flags, periodic=0, row_axis="auto"):
    """lbm_check_layout: host-only index build + invariant check, rows along
    row_axis ("auto", "x" or "z").  Returns a dict of counts (row_axis is the
    axis used, "x" or "z"); raises LbmError on an inconsistent field or
    index."""
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    nz, ny, nx = flags.shape
    out = (C.c_int64 * 8)()
    st = capi().lbm_check_layout(flags.ctypes.data, nx, ny, nz, int(periodic), ROW_AXES[row_axis], out)
    if st != LBM_OK:
        raise LbmError(st, "lbm_check_layout")
    keys = ["active", "slots", "row_records", "chunks", "boundary_nodes", "wall_links", "rows"]
    info = dict(zip(keys, list(out)[:7]))
    info["row_axis"] = "z" if out[7] == LBM_ROWS_Z else "x"
    return info


class TorchAllocator:
    """Device memory from PyTorch's caching allocator, handed to the library
    through its allocator callback (called only at set-up / transfers)."""

    def __init__(self, device, stream):
        import torch

        self.torch = torch
        self.device = device
        self.stream = stream
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)

    def _do_alloc(self, nbytes, user):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:  # report failure as NULL: the library returns LBM_ERR_OOM
            return None

    def _do_free(self, ptr, user):
        self.torch.cuda.caching_allocator_delete(ptr)

    def struct(self):
        return lbm_allocator(self._alloc, self._free, None)


class Lattice:
    """One solver context (lbm_create .. lbm_destroy) with numpy marshalling.

    flags: uint8 array (nz, ny, nx) of LBM_SOLID/FLUID/INLET/OUTLET.
    precision: "fp64", "fp32" or "fp16s"; fp16_scale: FP16S scale s (0 selects
    the library default 4096).  stream: a torch.cuda.Stream (default: the
    current stream of the device).
    """

    def __init__(self, flags, precision="fp32", periodic=0, fp16_scale=0.0, device=0, stream=None,
                 torch_allocator=True, allocator=None, row_axis="auto"):
        import torch

        self.lib = capi()
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        if flags.ndim != 3:
            raise ValueError("flags must be (nz, ny, nx)")
        self.flags = flags
        self.shape = flags.shape
        nz, ny, nx = flags.shape
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        if allocator is not None:  # any object with struct() -> lbm_allocator
            self.allocator = allocator
        else:
            self.allocator = TorchAllocator(device, self.stream) if torch_allocator else None
        d = lbm_desc()
        d.nx, d.ny, d.nz = nx, ny, nz
        d.periodic = int(periodic)
        d.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        d.fp16_scale = float(fp16_scale)
        d.device = device
        d.row_axis = ROW_AXES[row_axis]
        d.stream = C.c_void_p(self.stream.cuda_stream)
        if self.allocator is not None:
            d.allocator = self.allocator.struct()
        self._desc = d
        ctx = C.c_void_p()
        st = self.lib.lbm_create(C.byref(d), C.byref(ctx))
        if st != LBM_OK:
            raise LbmError(st, "lbm_create")
        self.ctx = ctx
        self.precision = precision
        try:
            self._check(self.lib.lbm_set_geometry(self.ctx, flags.ctypes.data))
        except LbmError:
            self.close()
            raise
        n = C.c_int64()
        self._check(self.lib.lbm_fluid_count(self.ctx, C.byref(n)))
        self.n_active = n.value

    # -- plumbing
    def _check(self, st):
        if st != LBM_OK:
            msg = self.lib.lbm_last_error(self.ctx).decode() if getattr(self, "ctx", None) else ""
            raise LbmError(st, msg)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _count(self, layout):
        return self.n_active if layout == LBM_LAYOUT_ACTIVE else int(np.prod(self.shape))

    # -- parameters and state
    def set_wall_q(self, cells, q):
        """lbm_set_wall_q: cells (n,) box indices, q (n, 27) uint8 wall
        distances in 1/256 of a link (128 = halfway); empty clears them."""
        cells = np.ascontiguousarray(cells, dtype=np.int64).reshape(-1)
        q = np.ascontiguousarray(q, dtype=np.uint8).reshape(-1, 27)
        if q.shape[0] != cells.size:
            raise ValueError("cells and q disagree in length")
        self._check(self.lib.lbm_set_wall_q(self.ctx, cells.ctypes.data if cells.size else None,
                                            q.ctypes.data if cells.size else None, cells.size))
        return self

    def set_params(self, **kw):
        """lbm_set_params; keywords as make_params."""
        p = make_params(**kw)
        self._check(self.lib.lbm_set_params(self.ctx, C.byref(p)))
        return self

    def omega(self):
        w = C.c_double()
        self._check(self.lib.lbm_get_omega(self.ctx, C.byref(w)))
        return w.value

    def init_equilibrium(self, rho=1.0, u=(0.0, 0.0, 0.0)):
        uu = np.ascontiguousarray(u, dtype=np.float64)
        self._check(self.lib.lbm_init_equilibrium(self.ctx, float(rho), _ptr(uu)))
        return self

    def init_fields(self, rho, u, layout=LBM_LAYOUT_ACTIVE):
        n = self._count(layout)
        rho = np.ascontiguousarray(np.broadcast_to(rho, (n,)), dtype=np.float64)
        u = np.ascontiguousarray(np.broadcast_to(u, (n, 3)), dtype=np.float64)
        self._check(self.lib.lbm_init_fields(self.ctx, _ptr(rho), _ptr(u), layout))
        return self

    def set_populations(self, f, layout=LBM_LAYOUT_ACTIVE):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self._count(layout), 27)
        self._check(self.lib.lbm_set_populations(self.ctx, _ptr(f), layout))
        return self

    def get_populations(self, layout=LBM_LAYOUT_ACTIVE):
        f = np.zeros((self._count(layout), 27))
        self._check(self.lib.lbm_get_populations(self.ctx, _ptr(f), layout))
        return f

    def step(self, n=1):
        self._check(self.lib.lbm_step(self.ctx, int(n)))
        return self

    def sync(self):
        self._check(self.lib.lbm_sync(self.ctx))
        return self

    def step_count(self):
        t = C.c_int64()
        self._check(self.lib.lbm_step_count(self.ctx, C.byref(t)))
        return t.value

    def set_check_every(self, k):
        self._check(self.lib.lbm_set_check_every(self.ctx, int(k)))
        return self

    def moments(self, layout=LBM_LAYOUT_ACTIVE, out=None):
        """lbm_get_moments -> (rho[n], u[n, 3]); ``out`` may supply both arrays
        (e.g. views of pinned host memory)."""
        n = self._count(layout)
        rho, u = out if out is not None else (np.zeros(n), np.zeros((n, 3)))
        assert rho.dtype == np.float64 and u.dtype == np.float64 and rho.size == n and u.size == 3 * n
        self._check(self.lib.lbm_get_moments(self.ctx, _ptr(rho), _ptr(u), layout))
        return rho, u

    def totals(self):
        m = C.c_double()
        mom = np.zeros(3)
        self._check(self.lib.lbm_get_totals(self.ctx, C.byref(m), _ptr(mom)))
        return m.value, mom

    def health(self):
        out = np.zeros(6)
        self._check(self.lib.lbm_get_health(self.ctx, _ptr(out)))
        return out

    def stats_begin(self, stride=1, full=None):
        """Start sampling every stride-th step.  full=True selects the full
        statistics (u, u u, viscous stress, rho), full=False the axial ones;
        None keeps the current mode."""
        if full is not None:
            self._check(self.lib.lbm_stats_set_mode(self.ctx, LBM_STATS_FULL if full else LBM_STATS_AXIAL))
        self._check(self.lib.lbm_stats_begin(self.ctx, int(stride)))
        return self

    def stats_end(self):
        self._check(self.lib.lbm_stats_end(self.ctx))
        return self

    def stats_reset(self):
        self._check(self.lib.lbm_stats_reset(self.ctx))
        return self

    def stats_get(self, layout=LBM_LAYOUT_ACTIVE):
        n = self._count(layout)
        m1 = np.zeros(n)
        m2 = np.zeros(n)
        k = C.c_int64()
        self._check(self.lib.lbm_stats_get(self.ctx, _ptr(m1), _ptr(m2), C.byref(k), layout))
        return m1, m2, k.value

    def stats_get_full(self, layout=LBM_LAYOUT_ACTIVE):
        """Full-mode time averages as a dict of arrays: u (n, 3), uu (n, 6),
        sigma (n, 6) (components xx, yy, zz, xy, xz, yz), rho (n,), the
        Reynolds stress reynolds = <rho> (<u_a u_b> - <u_a><u_b>) (n, 6), and
        the sample count."""
        n = self._count(layout)
        m = np.zeros((n, LBM_STATS_FULL_COMPONENTS))
        k = C.c_int64()
        self._check(self.lib.lbm_stats_get_full(self.ctx, _ptr(m), C.byref(k), layout))
        u, uu, sigma, rho = m[:, 0:3], m[:, 3:9], m[:, 9:15], m[:, 15]
        pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
        reynolds = rho[:, None] * (uu - np.stack([u[:, a] * u[:, b] for a, b in pairs], axis=1))
        return dict(u=u, uu=uu, sigma=sigma, rho=rho, reynolds=reynolds, samples=k.value)

    def checkpoint(self):
        n = C.c_size_t()
        self._check(self.lib.lbm_checkpoint_size(self.ctx, C.byref(n)))
        buf = np.zeros(n.value, dtype=np.uint8)
        self._check(self.lib.lbm_checkpoint(self.ctx, buf.ctypes.data, n.value))
        return buf

    def restore(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(self.lib.lbm_restore(self.ctx, buf.ctypes.data, buf.size))
        return self

    def layout_info(self):
        s, b, d = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self.lib.lbm_layout_info(self.ctx, C.byref(s), C.byref(b), C.byref(d)))
        return dict(slots=s.value, buffer_bytes=b.value, device_bytes=d.value)

    def kernel_launches(self):
        """Kernels lbm_step has launched on this lattice so far."""
        n = C.c_int64()
        self._check(self.lib.lbm_kernel_launches(self.ctx, C.byref(n)))
        return n.value


def make_request(flags, steps, precision="fp32", periodic=0, fp16_scale=0.0, **params):
    """An lbm_request over a C-contiguous uint8 flag array (nz, ny, nx), which
    the caller keeps alive while the request is in use."""
    nz, ny, nx = flags.shape
    r = lbm_request()
    r.nx, r.ny, r.nz, r.periodic = nx, ny, nz, int(periodic)
    r.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    r.fp16_scale = float(fp16_scale)
    r.flags = flags.ctypes.data
    r.params = make_params(**params)
    r.steps = int(steps)
    return r


def check_request(flags, steps, precision="fp32", budget_bytes=1 << 40, periodic=0, fp16_scale=0.0, **params):
    """lbm_server_check_request (host only): the checks a request server
    applies to a request, with its index build.  Returns a dict of counts;
    raises LbmError with the reason of a refusal."""
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    r = make_request(flags, steps, precision, periodic, fp16_scale, **params)
    out = (C.c_int64 * 4)()
    why = C.c_char_p()
    st = capi().lbm_server_check_request(C.byref(r), int(budget_bytes), out, C.byref(why))
    if st != LBM_OK:
        raise LbmError(st, "lbm_server_check_request: " + why.value.decode())
    return dict(zip(["active", "slots", "footprint", "boundary_nodes"], list(out)))


class Server:
    """A request server (lbm_server_create .. lbm_server_destroy): continuous
    batching of many lattices on one GPU.  Memory comes from PyTorch's
    caching allocator; work runs on a dedicated torch stream."""

    def __init__(self, budget_bytes, max_slots=32, steps_per_tick=32, device=0, stream=None, torch_allocator=True,
                 allocator=None):
        import torch

        self.lib = capi()
        self.stream = stream if stream is not None else torch.cuda.Stream(device)
        if allocator is not None:  # any object with struct() -> lbm_allocator
            self.allocator = allocator
        else:
            self.allocator = TorchAllocator(device, self.stream) if torch_allocator else None
        d = lbm_server_desc()
        d.device = device
        d.stream = C.c_void_p(self.stream.cuda_stream)
        if self.allocator is not None:
            d.allocator = self.allocator.struct()
        d.budget_bytes = int(budget_bytes)
        d.max_slots = int(max_slots)
        d.steps_per_tick = int(steps_per_tick)
        self._desc = d
        h = C.c_void_p()
        st = self.lib.lbm_server_create(C.byref(d), C.byref(h))
        if st != LBM_OK:
            raise LbmError(st, "lbm_server_create")
        self.h = h
        self._keep = {}

    def _check(self, st):
        if st != LBM_OK:
            raise LbmError(st, self.lib.lbm_server_last_error(self.h).decode())

    def submit(self, flags, steps, precision="fp32", periodic=0, fp16_scale=0.0, **params):
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        r = make_request(flags, steps, precision, periodic, fp16_scale, **params)
        rid = C.c_int64()
        self._check(self.lib.lbm_server_submit(self.h, C.byref(r), C.byref(rid)))
        return rid.value

    def tick(self):
        run, q = C.c_int32(), C.c_int32()
        self._check(self.lib.lbm_server_tick(self.h, C.byref(run), C.byref(q)))
        return run.value, q.value

    def poll(self, rid):
        st, n = C.c_int32(), C.c_int64()
        self._check(self.lib.lbm_server_poll(self.h, int(rid), C.byref(st), C.byref(n)))
        return st.value, n.value

    def cells(self, rid):
        n = C.c_int64()
        self._check(self.lib.lbm_server_cells(self.h, int(rid), C.byref(n)))
        return n.value

    def result(self, rid):
        n = self.cells(rid)
        rho, u = np.zeros(n), np.zeros((n, 3))
        self._check(self.lib.lbm_server_result(self.h, int(rid), _ptr(rho), _ptr(u)))
        return rho, u

    def cancel(self, rid):
        self._check(self.lib.lbm_server_cancel(self.h, int(rid)))

    def info(self):
        out = np.zeros(8)
        self._check(self.lib.lbm_server_info(self.h, _ptr(out)))
        keys = ["cell_updates", "ticks", "bytes_in_use", "peak_bytes", "graph_launches", "graph_captures",
                "finished", "queued"]
        return dict(zip(keys, out.tolist()))

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
