"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/hyperball.h declares; argument errors are caught on the host before
any device work (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1308_2144_gb300 import build, hyperball as hbl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return hbl.load()


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hb_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared("hyperball.h")
    assert "hb_create" in names and "hb_run_to_fixpoint" in names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(hbl.EXPORTS) == sorted(n for n in names if n in hbl.EXPORTS)


def test_library_is_built_for_sm103a(tmp_path):
    """One translation unit compiled with the library's own arch and flags:
    ptxas reports every kernel it assembles for sm_103a and none for any
    other target."""
    import subprocess
    src = os.path.join(os.path.dirname(build.__file__), "csrc", "hb_noalloc.cu")
    r = subprocess.run([build.nvcc(), *build.ARCH, *build.FLAGS, "-Xptxas", "-v", "-c", src,
                        "-o", str(tmp_path / "x.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    targets = re.findall(r"for '(sm_\w+)'", r.stderr)
    assert targets and set(targets) == {"sm_103a"}, set(targets)


def test_version_string(lib):
    assert "sm_103a" in hbl.hb_version()


def test_default_options(lib):
    o = hbl.Options()
    lib.hb_default_options(ctypes.byref(o))
    assert o.flags == 0 and o.frontier == 0 and o.max_steps == 1 << 20 and not o.stream
    assert o.arcs_per_slot == 0


STRUCTS = {"hb_options": hbl.Options, "hb_info": hbl.Info, "hb_graph_desc": hbl.GraphDesc,
           "hb_server_options": hbl.ServerOptions, "hb_request_info": hbl.RequestInfo}


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field
    offsets (a C program built against include/hyperball.h prints them)."""
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hyperball.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.splitlines())
    for cname, cls in STRUCTS.items():
        assert int(got[f"{cname} size"]) == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert int(got[f"{cname} {field}"]) == getattr(cls, field).offset, (cname, field)


@pytest.mark.parametrize("log2m", [0, 3, 13, 20])
def test_log2m_out_of_range_is_rejected_on_host(lib, log2m):
    off = np.array([0, 1, 1], dtype=np.int64)
    tgt = np.array([1], dtype=np.int32)
    with pytest.raises(hbl.HBError) as e:
        hbl.hb_create(off, tgt, 2, 1, log2m, 42)
    assert e.value.status == hbl.HB_ERR_INVALID
    assert "log2m" in str(e.value)


def test_bad_sizes_are_rejected_on_host(lib):
    off = np.array([0, 1], dtype=np.int64)
    tgt = np.array([0], dtype=np.int32)
    for n, m in ((-1, 1), (2**31, 1), (1, -5)):
        with pytest.raises(hbl.HBError) as e:
            hbl.hb_create(off, tgt, n, m, 4, 1)
        assert e.value.status == hbl.HB_ERR_INVALID
    off32 = off.astype(np.int32)
    with pytest.raises(hbl.HBError):
        hbl.hb_create(off32, tgt, 1, 2**31, 4, 1)
    with pytest.raises(hbl.HBError):
        hbl.hb_create(off, tgt, 1, 1, 4, 1, hbl.make_options(frontier=7))


def test_null_handle_is_rejected(lib):
    assert lib.hb_step(None, None) == hbl.HB_ERR_INVALID
    assert lib.hb_get_registers(None, None) == hbl.HB_ERR_INVALID
    lib.hb_destroy(None)


def test_binding_constants_match_the_header(tmp_path):
    """The status codes, flags, frontier policies and request states the
    binding defines have the header's values."""
    import subprocess
    names = sorted(k for k, v in vars(hbl).items() if k.startswith("HB_") and isinstance(v, int))
    names += [f"HB_FRONTIER_{k.upper()}" for k in hbl.FRONTIER]
    src = tmp_path / "consts.c"
    src.write_text("\n".join(['#include <stdio.h>', '#include "hyperball.h"', "int main(void) {"]
                             + [f'printf("{nm} %lld\\n", (long long)({nm}));' for nm in names]
                             + ["return 0;", "}"]))
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    assert len(names) >= 20
    for nm in names:
        want = hbl.FRONTIER[nm[len("HB_FRONTIER_"):].lower()] if nm.startswith("HB_FRONTIER_") else getattr(hbl, nm)
        assert int(got[nm]) == want, nm
