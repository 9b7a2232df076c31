"""C-ABI library checks that need no GPU: it builds, loads, exports every
function include/lbm.h declares, and its host-only entry points behave."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2204_10566_gb300 import build as lbuild
from paper_2204_10566_gb300 import inputs as I
from paper_2204_10566_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    lbuild.build()
    return lbm.capi()


def header_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported(lib):
    names = header_functions()
    assert len(names) >= 29
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(lbm.declared_functions()) == names


def test_status_strings(lib):
    assert lib.lbm_status_string(0) == b"ok"
    assert lib.lbm_status_string(5) == b"non-finite state"


def test_params_default(lib):
    p = lbm.lbm_params()
    lib.lbm_params_default(C.byref(p))
    assert (p.omega3, p.omega4, p.omega5, p.omega6) == (1.0, 1.0, 1.0, 1.0)
    assert p.rho_out == 1.0 and p.inlet_profile == lbm.LBM_PROFILE_PLUG and p.axis_x < 0


def test_struct_sizes_match_header():
    # lbm_desc: 7 int32 + float, pointer, 3 pointers; lbm_params: 14 doubles + u64 + 2 int32
    assert C.sizeof(lbm.lbm_desc) == 32 + 8 + 24
    assert C.sizeof(lbm.lbm_params) == 14 * 8 + 8 + 8


@pytest.mark.parametrize("name", ["nozzle_re500_24x24x160", "nozzle_re3500_96x96x800"])
def test_make_nozzle_matches_input_generator(lib, name):
    w = I.WORKLOADS[name]
    got = lbm.make_nozzle(w["D"], w["d"], w["L_total"])
    assert np.array_equal(got, I.workload_flags(name))


def test_make_nozzle_rejects_bad_sizes(lib):
    out = np.zeros(10, dtype=np.uint8)
    assert lib.lbm_make_nozzle(8, 12, 8, -1, 4, 10, 10.0, out.ctypes.data) == lbm.LBM_ERR_ARG
    assert lib.lbm_make_nozzle(8, 4, 8, -1, 4, 10, 95.0, out.ctypes.data) == lbm.LBM_ERR_ARG


def test_create_rejects_bad_descriptors(lib):
    ctx = C.c_void_p()
    d = lbm.lbm_desc()
    d.nx, d.ny, d.nz, d.precision = 0, 4, 4, 1
    assert lib.lbm_create(C.byref(d), C.byref(ctx)) == lbm.LBM_ERR_ARG
    d.nx, d.precision = 4, 7
    assert lib.lbm_create(C.byref(d), C.byref(ctx)) == lbm.LBM_ERR_ARG
    d.precision, d.fp16_scale = 2, 3.0   # not a power of two
    assert lib.lbm_create(C.byref(d), C.byref(ctx)) == lbm.LBM_ERR_ARG
    assert lib.lbm_destroy(None) == lbm.LBM_OK


def _ragged():
    g = np.random.default_rng(12)
    f = np.ones((9, 11, 37), dtype=np.uint8)
    f[:, :, :3] = 0
    f[:, 4:7, 15:18] = 0
    f[2:4, 1, 30:] = 0
    f[g.random(f.shape) < 0.03] = 0
    return f


def _duct(n, nz, nx=None):
    f = np.ones((nz, n, nx or n), dtype=np.uint8)
    f[0] = 2
    f[-1] = 3
    return f


@pytest.mark.parametrize("rows", ["x", "z"])
@pytest.mark.parametrize("case", ["nozzle", "ragged", "box13", "box70", "duct", "pipe", "long_rows"])
@pytest.mark.parametrize("periodic", [0, 7, 3, 4])
def test_layout_invariants(lib, case, periodic, rows):
    """The sparse index the kernels use: every staged copy aligned and in
    bounds, every fluid cell in exactly one work unit, every pull stored
    (checked on the host, independently of how the index was built)."""
    if case == "nozzle":
        f = I.workload_flags("nozzle_re500_24x24x160")
    elif case == "ragged":
        f = _ragged()
    elif case == "box13":
        f = np.ones((5, 6, 13), dtype=np.uint8)
    elif case == "box70":
        f = np.ones((3, 4, 70), dtype=np.uint8)
    elif case == "duct":
        f = _duct(8, 12)
    elif case == "pipe":
        f = I.pipe_flags(18, 30)
    else:
        f = np.ones((2, 3, 300), dtype=np.uint8)
        f[:, :, 131:140] = 0
    if periodic and case in ("nozzle", "pipe"):
        pytest.skip("walls of the nozzle need no periodic faces")
    if case == "duct" and periodic & 4:
        pytest.skip("inlet/outlet planes need a non-periodic z")
    info = lbm.check_layout(f, periodic, rows)
    assert info["active"] == int((f != 0).sum())
    assert info["boundary_nodes"] == int(((f == 2) | (f == 3)).sum())
    assert info["row_records"] >= 1 and info["slots"] % 64 == 0 and info["row_axis"] == rows


def test_row_axis_choice(lib):
    """AUTO stores rows along z when the box is longer in z than in x.  On the
    Re 3500 nozzle that leaves far fewer chunk lanes idle than rows along x."""
    f = I.workload_flags("nozzle_re3500_96x96x800")
    assert lbm.check_layout(np.ones((4, 4, 9), dtype=np.uint8))["row_axis"] == "x"
    assert lbm.check_layout(np.ones((9, 4, 4), dtype=np.uint8))["row_axis"] == "z"
    assert lbm.check_layout(np.ones((9, 4, 9), dtype=np.uint8))["row_axis"] == "x"
    auto = lbm.check_layout(f)
    xr = lbm.check_layout(f, 0, "x")
    assert auto["row_axis"] == "z"
    assert auto["active"] == xr["active"] == 4286996
    idle_z = 1.0 - auto["active"] / (8.0 * auto["chunks"])
    idle_x = 1.0 - xr["active"] / (8.0 * xr["chunks"])
    assert idle_z < 0.5 * idle_x, (idle_z, idle_x)


def test_layout_rejects_inconsistent_fields(lib):
    bad = np.ones((4, 4, 4), dtype=np.uint8)
    bad[0, 0, 0] = 2
    with pytest.raises(lbm.LbmError) as e:
        lbm.check_layout(bad)
    assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError):
        lbm.check_layout(np.zeros((2, 2, 2), dtype=np.uint8))
