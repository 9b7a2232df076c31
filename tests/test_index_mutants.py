"""The library's own index check rejects plausible index-building mistakes
(CPU only).

Each case plants one mistake in a copy of the host index builder
(paper_2204_10566_gb300/csrc/geometry.cpp), compiles that file alone into a
library, and runs lbm_check_layout, which builds the index and checks it
with the independent validator, on a set of flag fields.  At least one
field must be refused (or give wrong counts).  The unmodified builder
passes all of them.  Each case runs in a child process, so that a broken
builder cannot disturb the test run.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2204_10566_gb300", "csrc")

# name: (text in geometry.cpp, planted text)
MUTANTS = {
    "ghost_marks_wrong_array": (
        "out.mask[(size_t)(base[row_of(ys, zs)] + x - cx)] |= 1u << i;",
        "out.mask[(size_t)(base[row_of(ys, zs)] + x - cx)] |= 1u << (26 - i);"),
    "neighbour_row_direction": ("int yy = y - cy, zz = z - cz;", "int yy = y + cy, zz = z - cz;"),
    "neighbour_rows_y_z_swapped": (
        "out.row_nb[(size_t)r * ROW_RECORD_INTS + j] = base[row_of(yy, zz)];",
        "out.row_nb[(size_t)r * ROW_RECORD_INTS + j] = base[row_of(zz % ny, yy % nz)];"),
    "boundary_nodes_in_chunk_lanes": (
        "if (x < nx && flags[box_index(x, y, z, nx, ny)] == LBM_FLUID) lanes |= 1u << l;",
        "if (x < nx && flags[box_index(x, y, z, nx, ny)] != LBM_SOLID) lanes |= 1u << l;"),
    "row_range_one_short": (
        "const int hi = ((need_hi[r] + 1 + CHUNK - 1) / CHUNK) * CHUNK;",
        "const int hi = ((need_hi[r] + CHUNK - 1) / CHUNK) * CHUNK;"),
    "periodic_copy_wrong_arrays": (
        "for (int i = 2; i < 27; i += 3) out.mask[(size_t)(base[r] - 1)] |= 1u << i;",
        "for (int i = 0; i < 27; i += 3) out.mask[(size_t)(base[r] - 1)] |= 1u << i;"),
    "boundary_node_slot": (
        "out.bnodes.push_back(make_int4(x, (int)row_of(y, z), slot, (int)out.mask[(size_t)slot]));",
        "out.bnodes.push_back(make_int4(x, (int)row_of(y, z), slot + 1, (int)out.mask[(size_t)slot]));"),
    "active_slot_shifted": ("const int32_t slot = base[row_of(y, z)] + x;", "const int32_t slot = base[row_of(y, z)] + x + 1;"),
    "ghost_row_not_wrapped": ("        ys = py ? yw : y;", "        ys = y;"),
    "neighbour_row_not_wrapped": ("                if (py) yy = (yy + ny) % ny;\n", ""),
    "chunk_start_unaligned": (
        "for (int x0 = (int)std::floor(act_lo[r] / (double)CHUNK) * CHUNK; x0 <= act_hi[r]; x0 += CHUNK) {",
        "for (int x0 = act_lo[r]; x0 <= act_hi[r]; x0 += CHUNK) {"),
}

# the flag fields each case is checked on: (name, shape, recipe, periodic)
CHILD = r'''
import ctypes as C, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2204_10566_gb300 import inputs as I

def ragged():
    g = np.random.default_rng(12)
    f = np.ones((9, 11, 37), dtype=np.uint8)
    f[:, :, :3] = 0; f[:, 4:7, 15:18] = 0; f[2:4, 1, 30:] = 0; f[g.random(f.shape) < 0.03] = 0
    return f

def duct():
    f = np.ones((12, 8, 8), dtype=np.uint8); f[0] = 2; f[-1] = 3
    return f

def side_inlet():
    f = np.zeros((6, 6, 10), dtype=np.uint8); f[1:5, 1:5, :] = 1; f[1:5, 1:5, 0] = 2; f[1:5, 1:5, -1] = 3
    return f

cases = [(I.workload_flags("nozzle_re500_24x24x160"), 0), (ragged(), 0), (ragged(), 7), (ragged(), 3),
         (np.ones((5, 6, 13), dtype=np.uint8), 7), (duct(), 0), (duct(), 3), (I.pipe_flags(18, 30), 0),
         (side_inlet(), 0)]
L = C.CDLL(LIB)
L.lbm_check_layout.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int64)]
refused = 0
for f, p in cases:
    f = np.ascontiguousarray(f, dtype=np.uint8)
    nz, ny, nx = f.shape
    out = (C.c_int64 * 8)()
    st = L.lbm_check_layout(f.ctypes.data, nx, ny, nz, p, out)
    ok = st == 0 and out[0] == int((f != 0).sum()) and out[4] == int(((f == 2) | (f == 3)).sum())
    refused += not ok
print(refused)
'''


def cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    if not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        pytest.skip("CUDA headers not found")
    return inc


def build(directory, name, text):
    src = os.path.join(str(directory), name + ".cpp")
    lib = os.path.join(str(directory), name + ".so")
    with open(src, "w") as fh:
        fh.write(text.replace('#include "lbm_internal.h"', '#include "%s"' % os.path.join(CSRC, "lbm_internal.h")))
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-I" + cuda_include(), src, "-o", lib],
                   check=True, capture_output=True)
    return lib


def refused_fields(lib):
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\nLIB = %r\n" % (ROOT, lib) + CHILD],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return int(r.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def source():
    with open(os.path.join(CSRC, "geometry.cpp")) as fh:
        return fh.read()


def test_unmodified_builder_passes(tmp_path, source):
    assert refused_fields(build(tmp_path, "unmodified", source)) == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_layout_check_refuses_planted_mistake(tmp_path, source, name):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, "the builder text of %s is no longer unique" % name
    assert refused_fields(build(tmp_path, name, source.replace(old, new))) > 0
