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
