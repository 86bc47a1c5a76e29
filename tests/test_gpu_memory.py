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
