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
        "out.mask[(size_t)(base[row_of(as, bs)] + p - cp)] |= 1u << i;",
        "out.mask[(size_t)(base[row_of(as, bs)] + p - cp)] |= 1u << (26 - i);"),
    "neighbour_row_direction": ("int aa = a - ca, bb = b - cb;", "int aa = a + ca, bb = b - cb;"),
    "neighbour_rows_cross_axes_swapped": (
        "out.row_nb[(size_t)r * ROW_RECORD_INTS + j] = base[row_of(aa, bb)];",
        "out.row_nb[(size_t)r * ROW_RECORD_INTS + j] = base[row_of(bb % F.na, aa % F.nb)];"),
    "boundary_nodes_in_chunk_lanes": (
        "if (p < F.np && flags[F.box(p, a, b)] == LBM_FLUID) lanes |= 1u << l;",
        "if (p < F.np && flags[F.box(p, a, b)] != LBM_SOLID) lanes |= 1u << l;"),
    "row_range_one_short": (
        "const int hi = ((need_hi[r] + 1 + CHUNK - 1) / CHUNK) * CHUNK;",
        "const int hi = ((need_hi[r] + CHUNK - 1) / CHUNK) * CHUNK;"),
    "periodic_copy_wrong_arrays": (
        "if (F.pp && p == F.np - 1 && cp == 1) out.mask[(size_t)(base[r] - 1)] |= 1u << i;",
        "if (F.pp && p == F.np - 1 && cp == -1) out.mask[(size_t)(base[r] - 1)] |= 1u << i;"),
    "boundary_node_slot": (
        "out.bnodes.push_back(make_int4(p, (int)row_of(a, b), slot, (int)out.mask[(size_t)slot]));",
        "out.bnodes.push_back(make_int4(p, (int)row_of(a, b), slot + 1, (int)out.mask[(size_t)slot]));"),
    "active_slot_shifted": ("const int32_t slot = base[row_of(a, b)] + p;", "const int32_t slot = base[row_of(a, b)] + p + 1;"),
    "ghost_row_not_wrapped": ("        as = F.pa ? aw : a;", "        as = a;"),
    "neighbour_row_not_wrapped": ("                if (F.pa) aa = (aa + F.na) % F.na;\n", ""),
    "chunk_start_unaligned": (
        "for (int p0 = (int)std::floor(act_lo[r] / (double)CHUNK) * CHUNK; p0 <= act_hi[r]; p0 += CHUNK) {",
        "for (int p0 = act_lo[r]; p0 <= act_hi[r]; p0 += CHUNK) {"),
    "z_rows_cross_directions_swapped": ("            cp = cz, ca = cx, cb = cy;", "            cp = cz, ca = cy, cb = cx;"),
    "pair_items_overlap": ("            t += 2;\n", "            t += 1;\n"),
    "rest_chunks_counted_from_fluid_lanes": ("(uint32_t)tiles[(size_t)t * TILE_INTS + 2]) / CHUNK",
                                             "(uint32_t)tiles[(size_t)t * TILE_INTS + 1]) / CHUNK"),
    "z_rows_storage_order": ("        return ax == 0 ? box_index(p, a, b, nx, ny) : box_index(a, b, p, nx, ny);",
                             "        return ax == 0 ? box_index(p, a, b, nx, ny) : box_index(b, a, p, nx, ny);"),
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
         (ragged(), 5), (np.ones((5, 6, 13), dtype=np.uint8), 7), (np.ones((13, 6, 5), dtype=np.uint8), 7),
         (duct(), 0), (duct(), 3), (I.pipe_flags(18, 30), 0), (side_inlet(), 0)]
L = C.CDLL(LIB)
L.lbm_check_layout.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                               C.POINTER(C.c_int64)]
refused = 0
for f, p in cases:
    f = np.ascontiguousarray(f, dtype=np.uint8)
    nz, ny, nx = f.shape
    for rows in (1, 2):  # rows along x, rows along z
        out = (C.c_int64 * 8)()
        st = L.lbm_check_layout(f.ctypes.data, nx, ny, nz, p, rows, out)
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
