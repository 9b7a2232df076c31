"""lbm_totals_noalloc: totals of a caller-owned population array with no
device allocation.

Callers whose device memory belongs to their own pool (with a fixed budget),
or whose loop cannot afford the device-wide synchronisation of cudaMalloc /
cudaFree, use this entry point: it takes the populations and the output
buffer from the caller and keeps its only scratch (per-block partial sums)
in a static device array.  The test compares it, through the C ABI, with the
context-based lbm_get_totals on the same state, twice in a row (the static
scratch keeps the previous call's contents, which must not leak into the
next result).  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_util import gpu_lattice, random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-9, "fp16s": 1e-9}


@pytest.fixture(scope="module")
def lbm():
    from paper_2204_10566_gb300 import build

    build.build()
    from paper_2204_10566_gb300 import lbm as m

    assert torch.cuda.is_available()
    return m


def storage_tensor(orc, f_active, precision, scale):
    """The library's storage form [27][n] of populations f (n, 27)."""
    dev = f_active - orc.weights()[None, :]
    if precision == "fp64":
        t = torch.tensor(dev.T.copy(), dtype=torch.float64)
    elif precision == "fp32":
        t = torch.tensor(dev.T.copy(), dtype=torch.float32)
    else:
        t = torch.tensor((dev * scale).T.copy(), dtype=torch.float32).to(torch.float16)
    return t.contiguous().cuda()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_noalloc_totals_match_context_totals(orc, lbm, precision):
    flags = np.ones((6, 7, 19), dtype=np.uint8)
    flags[2, 3, 5:9] = 0
    f0 = random_state(orc, flags, 31)
    G = gpu_lattice(lbm, flags, precision, 0.05, periodic=7)
    G.set_populations(f0, layout=1)
    G.step(3).sync()
    f_act = G.get_populations()              # storage values, converted back to f
    n = f_act.shape[0]
    scale = 4096.0
    data = storage_tensor(orc, f_act, precision, scale)
    prec = {"fp64": lbm.LBM_FP64, "fp32": lbm.LBM_FP32, "fp16s": lbm.LBM_FP16S}[precision]
    stream = torch.cuda.current_stream()
    lib = lbm.capi()
    for call in range(2):
        mass, mom = G.totals()                # the existing entry point
        out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.lbm_totals_noalloc(C.c_void_p(data.data_ptr()), prec, scale, n, n, C.c_void_p(out.data_ptr()),
                                    C.c_void_p(stream.cuda_stream))
        assert st == lbm.LBM_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - mass) <= TOL[precision] * abs(mass), (call, got[0], mass)
        assert np.abs(got[1:4] - mom).max() <= TOL[precision] * abs(mass), (call, got[1:4], mom)
        assert got[5] == 0.0 and got[4] > 0.0
        G.step(1).sync()                      # a different state for the second call
        f_act = G.get_populations()
        data = storage_tensor(orc, f_act, precision, scale)


PREC = {"fp64": 0, "fp32": 1, "fp16s": 2}
STORE = {"fp64": torch.float64, "fp32": torch.float32, "fp16s": torch.float16}


def call_noalloc(lbm, data, precision, n, stride, scale=4096.0, stream=None):
    out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    stream = stream or torch.cuda.current_stream()
    st = lbm.capi().lbm_totals_noalloc(C.c_void_p(data.data_ptr()), PREC[precision], scale, n, stride,
                                       C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return st, out.cpu().numpy()


def random_storage(orc, n, stride, precision, seed, scale=4096.0):
    """Caller-owned storage [27][stride] of n near-rest cells (the pad
    columns hold garbage that must not be read), and the populations its
    values decode to, (n, 27), in FP64."""
    g = np.random.default_rng(seed)
    w = orc.weights()
    dev = w[None, :] * g.uniform(-0.02, 0.02, (n, 27))
    host = np.full((27, stride), 7.0)
    if precision == "fp16s":
        host[:, :n] = (dev * scale).T
        t = torch.tensor(host, dtype=torch.float32).to(torch.float16)
        decoded = t[:, :n].to(torch.float64).numpy().T / scale
    else:
        host[:, :n] = dev.T
        t = torch.tensor(host, dtype=STORE[precision])
        decoded = t[:, :n].to(torch.float64).numpy().T
    return t.contiguous().cuda(), w[None, :] + decoded


def oracle_totals(orc, f):
    """Kahan-summed FP64 mass and momentum of populations f (n, 27)."""
    n = f.shape[0]
    L = orc.Lattice(np.ones((1, 1, n), dtype=np.uint8), 1.0, periodic=7)
    L.set_populations(f)
    return L.totals()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_noalloc_many_blocks_against_the_oracle(orc, lbm, precision):
    """About a million cells (245 blocks of partial sums, a ragged last
    block) in an array whose stride exceeds n, against the oracle's
    compensated totals of the same decoded populations; then a call with far
    fewer blocks on another array, which must not see the stale partials of
    the first call, and the first array again."""
    n, stride = 1_000_003, 1_000_003 + 61
    big, f_big = random_storage(orc, n, stride, precision, 5)
    small_n = 5_000
    small, f_small = random_storage(orc, small_n, small_n + 3, precision, 6)
    for data, f, m, s in ((big, f_big, n, stride), (small, f_small, small_n, small_n + 3), (big, f_big, n, stride)):
        st, got = call_noalloc(lbm, data, precision, m, s)
        assert st == lbm.LBM_OK
        ref = oracle_totals(orc, f)
        assert abs(got[0] - ref[0]) <= 1e-12 * ref[0], (m, got[0], ref[0])
        assert np.abs(got[1:4] - ref[1:4]).max() <= 1e-12 * ref[0], (m, got[1:4], ref[1:4])
        assert got[5] == 0.0 and 0.0 < got[4] < 0.2


def test_noalloc_at_the_size_limit(lbm):
    """n = LBM_NOALLOC_MAX_CELLS (every partial of the static scratch in
    use), FP16S: every cell holds the same dyadic deviations, so the totals
    have a closed form (the mass sum is exact in FP64).  A small call after
    it reads only its own partials."""
    n = 16777216
    stride = n + 8
    k = np.array([(i % 5) - 2 for i in range(27)], dtype=np.float64)  # stored values (f - w) s
    scale = 4096.0
    data = torch.tensor(k, dtype=torch.float16, device="cuda")[:, None].expand(27, stride).contiguous()
    st, got = call_noalloc(lbm, data, "fp16s", n, stride, scale)
    assert st == lbm.LBM_OK
    c = np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)], dtype=np.float64)
    rho = 1.0 + k.sum() / scale
    j = (c * k[:, None]).sum(0) / scale
    assert got[0] == n * rho
    assert np.abs(got[1:4] - n * j).max() <= 1e-13 * n
    st, got2 = call_noalloc(lbm, data, "fp16s", 1000, stride, scale)
    assert st == lbm.LBM_OK and got2[0] == 1000 * rho
    st, _ = call_noalloc(lbm, data, "fp16s", n + 1, stride, scale)
    assert st == lbm.LBM_ERR_ARG


FIRST_CALL_IN_CAPTURE = r"""
import ctypes as C, sys
import torch
sys.path.insert(0, sys.argv[1])
from paper_2204_10566_gb300 import lbm
lib = lbm.capi()
data = torch.zeros((27, 64), dtype=torch.float32, device="cuda")
out = torch.zeros(6, dtype=torch.float64, device="cuda")
s = torch.cuda.Stream()
g = torch.cuda.CUDAGraph()
with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
    out.add_(1.0)
    st = lib.lbm_totals_noalloc(C.c_void_p(data.data_ptr()), 1, 0.0, 64, 64, C.c_void_p(out.data_ptr()),
                                C.c_void_p(s.cuda_stream))
torch.cuda.synchronize()
st2 = lib.lbm_totals_noalloc(C.c_void_p(data.data_ptr()), 1, 0.0, 64, 64, C.c_void_p(out.data_ptr()),
                             C.c_void_p(s.cuda_stream))
torch.cuda.synchronize()
print(st, st2, out[0].item())
"""


def test_noalloc_first_call_inside_a_capture(lbm):
    """The first call in a context looks up the scratch address, which is
    refused inside a stream capture: a fresh process makes its first call in
    a relaxed-mode capture and gets LBM_ERR_STATE with nothing enqueued; the
    next call, outside the capture, works."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", FIRST_CALL_IN_CAPTURE, root], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    st, st2, mass = r.stdout.split()[-3:]
    assert int(st) == lbm.LBM_ERR_STATE and int(st2) == lbm.LBM_OK
    assert float(mass) == 64.0  # 64 cells at rest: rho = 1 each


def test_noalloc_rejects_sizes_beyond_its_scratch(lbm):
    lib = lbm.capi()
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    too_many = C.c_int64(16777216 + 1)
    st = lib.lbm_totals_noalloc(C.c_void_p(dummy.data_ptr()), lbm.LBM_FP32, 0.0, too_many, too_many,
                                C.c_void_p(out.data_ptr()), None)
    assert st == lbm.LBM_ERR_ARG
    st = lib.lbm_totals_noalloc(C.c_void_p(dummy.data_ptr()), lbm.LBM_FP32, 0.0, 8, 4,
                                C.c_void_p(out.data_ptr()), None)
    assert st == lbm.LBM_ERR_ARG
