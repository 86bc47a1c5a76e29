"""The debug build (libhyperball_debug.so: every arc target range-checked in
the gather before its counter is read), through the C ABI in a child
process that loads it: results equal the oracle's bit for bit on valid
graphs, and a target made invalid after creation is reported as
HB_ERR_STATE with the check's message instead of being read.

The invalid target reaches only the checked gather: the handle borrows the
caller's device arrays, keeps the caller's node order (no relabelled copy)
and runs without a frontier (no reverse CSR, no marking kernels), and the
test reads nothing else that follows the targets."""
import os
import subprocess
import sys
import textwrap

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import numpy as np, torch
    import oracle
    from paper_1308_2144_gb300 import graphs, hyperball as hbl
    assert hbl.LIB_PATH.endswith("libhyperball_debug.so"), hbl.LIB_PATH
    # valid graphs: bit-exact with the oracle
    for b, seed in ((4, 42), (6, 7)):
        off, tgt = graphs.plain_graph(n=3000, seed=seed).numpy()
        ref = oracle.run(off, tgt, b, seed)
        hb = hbl.HyperBall(torch.from_numpy(off).cuda(), torch.from_numpy(tgt).cuda(), log2m=b, seed=seed,
                           n=off.size - 1)
        assert hb.run() == ref.steps
        assert np.array_equal(hb.registers(device="cpu").numpy(), ref.regs)
        hb.close()
    # a target made invalid after creation: reported, not read
    off, tgt = graphs.plain_graph(n=3000, seed=5).numpy()
    n = off.size - 1
    d_off = torch.from_numpy(off).cuda()
    d_tgt = torch.from_numpy(tgt).cuda()
    hb = hbl.HyperBall(d_off, d_tgt, log2m=4, seed=1, n=n, borrow=True, relabel=False, frontier="off")
    d_tgt[d_tgt.numel() // 2] = n + 1000
    torch.cuda.synchronize()
    try:
        hb.step()
    except hbl.HBError as e:
        assert e.status == hbl.HB_ERR_STATE, e.status
        assert "outside [0, n)" in str(e), str(e)
    else:
        raise AssertionError("the invalid target was not reported")
    print("debug build ok")
""")


def test_debug_build_checks_targets():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_2144_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, HYPERBALL_LIB=lib, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "debug build ok" in r.stdout
