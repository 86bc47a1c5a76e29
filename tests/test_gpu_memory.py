"""The library's device memory pool, through the C ABI: handles created and
destroyed repeatedly (and on a side stream) give the oracle's results every
time; memory freed by hb_destroy stays in the pool and hb_trim_memory gives
it back to the device."""
import numpy as np
import pytest
import torch

from paper_1308_2144_gb300 import graphs
from paper_1308_2144_gb300 import hyperball as hbl
from tests.test_gpu_parity import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_2144_gb300 import build
    build.build()
    hbl.load()


def test_repeated_handles_and_trim(orc):
    off, tgt = graphs.rmat_graph(scale=16, edge_factor=16, seed=3).numpy()
    n = off.size - 1
    ref = orc.run(off, tgt, 7, 11)
    d_off, d_tgt = to_dev(off, tgt)
    hbl.hb_trim_memory()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    device_bytes = 0
    for k in range(3):
        stream = side if k == 1 else None
        hb = hbl.HyperBall(d_off, d_tgt, log2m=7, seed=11, n=n, stream=stream)
        assert hb.run() == ref.steps
        assert np.array_equal(hb.registers(device="cpu").numpy(), ref.regs)
        device_bytes = hb.info()["device_bytes"]
        hb.close()
    torch.cuda.synchronize()
    kept = torch.cuda.mem_get_info()[0]
    hbl.hb_trim_memory()
    torch.cuda.synchronize()
    freed = torch.cuda.mem_get_info()[0] - kept
    # the pool held at least the handle's own allocations until the trim
    assert device_bytes > 0 and freed >= device_bytes // 2, (freed, device_bytes)


def test_state_beyond_device_memory_is_refused(orc):
    """A handle whose counters alone (2 x n x 4096 bytes at log2m 12) exceed
    the device: hb_create returns HB_ERR_OOM and the library keeps working."""
    free_b, total_b = torch.cuda.mem_get_info()
    n = min(2**31 - 2, int(total_b // (2 * 4096)) + (1 << 20))
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    tgt = torch.zeros(0, dtype=torch.int32, device="cuda")
    with pytest.raises(hbl.HBError) as e:
        hbl.hb_create(off, tgt, n, 0, 12, 1)
    assert e.value.status == hbl.HB_ERR_OOM
    del off
    hbl.hb_trim_memory()
    g_off, g_tgt = graphs.plain_graph(n=2000, seed=2).numpy()
    hb = hbl.HyperBall(*to_dev(g_off, g_tgt), log2m=5, seed=3, n=g_off.size - 1)
    assert hb.run() == orc.run(g_off, g_tgt, 5, 3).steps
    hb.close()


def test_l2_fetch_granularity_is_set_read_and_restored():
    """hb_set_l2_fetch_bytes: a limit of this process's context; set, read
    back, refused outside 32/64/128, and put back."""
    prev = hbl.hb_set_l2_fetch_bytes(0)
    assert prev in (0, 32, 64, 128)
    try:
        hbl.hb_set_l2_fetch_bytes(128)
        assert hbl.hb_set_l2_fetch_bytes(0) == 128
        hbl.hb_set_l2_fetch_bytes(32)
        assert hbl.hb_set_l2_fetch_bytes(0) == 32
        with pytest.raises(hbl.HBError) as e:
            hbl.hb_set_l2_fetch_bytes(48)
        assert e.value.status == hbl.HB_ERR_INVALID
        assert hbl.hb_set_l2_fetch_bytes(0) == 32
    finally:
        if prev:
            hbl.hb_set_l2_fetch_bytes(prev)
    assert hbl.hb_set_l2_fetch_bytes(0) == prev
