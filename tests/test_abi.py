"""The C-ABI library builds, loads and exports every symbol include/mhs.h
declares.  No compute call is made here (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    with open(os.path.join(ROOT, "include", header)) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mhs_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2109_06042_gb300 import build
    try:
        return build.build()
    except RuntimeError as e:  # pragma: no cover - toolkit missing
        pytest.skip(str(e))


def test_header_declares_the_boundary():
    names = _declared("mhs.h")
    for must in ("mhs_load", "mhs_reduce_round", "mhs_kernelize", "mhs_result", "mhs_free",
                 "mhs_load_batch", "mhs_load_device", "mhs_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(mhs_\w+)", out))
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        for name in _declared(hdr):
            assert name in exported, f"{name} declared in {hdr} but not exported"


def test_binding_covers_the_header(libpath):
    from paper_2109_06042_gb300 import mhs
    declared = set(_declared("mhs.h"))
    assert declared == set(mhs.exported_names())


def test_library_loads_without_gpu(libpath):
    from paper_2109_06042_gb300 import mhs
    L = mhs.lib()
    assert mhs.version().startswith("mhs-gb300")
    o = mhs.make_options("popcount", 3, False)
    assert (o.contraction, o.max_rounds, o.use_graphs) == (2, 3, 0)
    assert L.mhs_count(None) == 0


def test_bad_options_rejected_on_host(libpath):
    """Option validation runs before any device call."""
    import ctypes

    import numpy as np

    from paper_2109_06042_gb300 import mhs
    o = mhs.make_options()
    o.reserved[0] = 1
    ptr = np.zeros(1, np.int32)
    h = ctypes.c_void_p()
    st = mhs.lib().mhs_load(0, 0, ptr.ctypes.data_as(mhs._P32), ptr.ctypes.data_as(mhs._P32),
                            ptr.ctypes.data_as(mhs._P32), 0, ctypes.byref(o), None,
                            ctypes.byref(h))
    assert st == mhs.MHS_EINVAL
