"""Host-side checks of the request server that need no GPU
(lbm_server_check_request): the checks lbm_server_submit applies, the index
build the server's worker threads run, and the 32-bit population offsets of
the multi-lattice kernels, which bound a served lattice at 2^32 / 27 storage
slots.  Oversized requests are refused on the host, before any allocation
or launch (no lattice of that size is ever run)."""
import numpy as np
import pytest

from paper_2204_10566_gb300 import build as lbuild
from paper_2204_10566_gb300 import inputs as I
from paper_2204_10566_gb300 import lbm

# 32-bit element offsets: i * slots + slot < 2^32 for the 27 arrays, less the
# kernels' margin of 64 slots
MAX_SLOTS_32 = 0xFFFFFFFF // 27 - 64


@pytest.fixture(scope="module", autouse=True)
def lib():
    lbuild.build()
    return lbm.capi()


def test_small_request_passes_with_its_counts():
    f = I.pipe_flags(6, 12)
    info = lbm.check_request(f, 100, "fp32", nu=0.01)
    assert info["active"] == int((f != 0).sum())
    assert info["boundary_nodes"] == int(((f == 2) | (f == 3)).sum())
    assert info["slots"] >= info["active"] and info["slots"] % 64 == 0
    # two population buffers of 27 arrays, plus the index
    assert info["footprint"] > 2 * 27 * 4 * info["slots"]
    info16 = lbm.check_request(f, 100, "fp16s", nu=0.01)
    assert info16["slots"] == info["slots"] and info16["footprint"] < info["footprint"]


def test_budget_refusals():
    f = I.pipe_flags(6, 12)
    info = lbm.check_request(f, 100, "fp32", nu=0.01)
    # below the population buffers alone: can never fit
    with pytest.raises(lbm.LbmError) as e:
        lbm.check_request(f, 100, "fp32", budget_bytes=2 * 27 * 4 * info["active"] - 1, nu=0.01)
    assert e.value.status == lbm.LBM_ERR_OOM and "never fit" in str(e.value)
    # above that bound but below the exact footprint: refused once the index is known
    with pytest.raises(lbm.LbmError) as e:
        lbm.check_request(f, 100, "fp32", budget_bytes=info["footprint"] - 1, nu=0.01)
    assert e.value.status == lbm.LBM_ERR_OOM and "footprint" in str(e.value)
    assert lbm.check_request(f, 100, "fp32", budget_bytes=info["footprint"], nu=0.01) == info


@pytest.mark.parametrize("kw, word", [
    (dict(precision="fp64", nu=0.01), "FP32 and FP16S"),
    (dict(precision="fp32", nu=0.01, ghost=(1.0, 1.5, 1.0, 1.0)), "ghost rates"),
    (dict(precision="fp32", nu=-1.0), "give nu"),
    (dict(precision="fp16s", nu=0.01, fp16_scale=3000.0), "power of two"),
])
def test_bad_requests(kw, word):
    with pytest.raises(lbm.LbmError) as e:
        lbm.check_request(I.pipe_flags(6, 12), 100, **kw)
    assert e.value.status == lbm.LBM_ERR_ARG and word in str(e.value)
    with pytest.raises(lbm.LbmError) as e:
        lbm.check_request(I.pipe_flags(6, 12), 0, "fp32", nu=0.01)
    assert e.value.status == lbm.LBM_ERR_ARG


def test_too_many_active_cells_for_32_bit_offsets():
    """Every active cell has a slot, so a lattice with more active cells than
    the limit is refused by the cheap checks of submit (no index build)."""
    f = np.ones((160, 1000, 1000), dtype=np.uint8)  # 1.6e8 periodic fluid cells
    assert int(f.sum()) > MAX_SLOTS_32
    with pytest.raises(lbm.LbmError) as e:
        lbm.check_request(f, 10, "fp16s", periodic=7, nu=0.01)
    assert e.value.status == lbm.LBM_ERR_ARG and "32-bit" in str(e.value)


def test_too_many_slots_for_32_bit_offsets():
    """A sparse lattice whose rows still span ~10^6 slots each: 242 active
    cells (both ends of every x-row of an 11 x 11 cross-section) but
    169 rows x ~1.05 M slots (the rows and their ghost neighbours store every
    position between the two ends).  Submit's cheap checks pass; the index
    build refuses it before allocating its per-slot arrays."""
    nx = (1 << 20) - 1
    f = np.zeros((11, 11, nx), dtype=np.uint8)
    f[:, :, 0] = 1
    f[:, :, -1] = 1
    with pytest.raises(lbm.LbmError) as e:
        lbm.check_request(f, 10, "fp32", nu=0.01)
    assert e.value.status == lbm.LBM_ERR_ARG
    msg = str(e.value)
    assert "storage slots" in msg and str(MAX_SLOTS_32) in msg
    # the same rows at half the length fit
    g = np.ascontiguousarray(f[:, :, : nx // 2 + 1])
    g[:, :, -1] = 1
    info = lbm.check_request(g, 10, "fp32", nu=0.01)
    assert info["active"] == 242 and MAX_SLOTS_32 // 2 < info["slots"] <= MAX_SLOTS_32
