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


def test_noalloc_argument_errors_on_host(libpath):
    """mhs_kernelize_noalloc maps bad sizes and missing arrays to MHS_EINVAL
    with a message in the caller's buffer, before any CUDA call (so this runs
    without a GPU)."""
    import ctypes

    from paper_2109_06042_gb300 import mhs
    L = mhs.lib()
    buf = ctypes.create_string_buffer(128)
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size checks come first
    cases = [((-1, 4, 8), b">= 0"), ((4, -2, 8), b">= 0"), ((4, 4, -1), b">= 0"),
             ((4097, 4, 8), b"too large"), ((4, 4097, 8), b"too large"),
             ((4, 4, 65537), b"too large")]
    for (n, m, nnz), msg in cases:
        st = L.mhs_kernelize_noalloc(n, m, dummy, dummy, dummy, nnz, dummy, dummy, None, None,
                                     buf, 128)
        assert st == mhs.MHS_EINVAL and msg in buf.value, (n, m, nnz, buf.value)
    st = L.mhs_kernelize_noalloc(4, 4, None, dummy, dummy, 8, dummy, dummy, None, None, buf, 128)
    assert st == mhs.MHS_EINVAL and b"NULL" in buf.value
    # a one-byte buffer still gets a terminated (empty) message
    small = ctypes.create_string_buffer(1)
    assert L.mhs_kernelize_noalloc(-1, 0, dummy, dummy, dummy, 0, dummy, dummy, None, None,
                                   small, 1) == mhs.MHS_EINVAL
    assert small.value == b""


def test_batch_host_validation_names_the_lowest_bad_instance(libpath):
    """mhs_load_batch validates a large batch on several host threads before
    any CUDA call; the error names the lowest malformed instance, with the
    same message a single-threaded check gives."""
    import numpy as np

    from paper_2109_06042_gb300 import instances as I
    from paper_2109_06042_gb300 import mhs

    insts = [I.tiny_random(9000 + i, nmax=24, mmax=16) for i in range(100)]

    def first_pair_edge(inst):  # a hyperedge of at least two vertices
        for e in range(inst.m):
            if inst.edge_ptr[e + 1] - inst.edge_ptr[e] >= 2:
                return e
        raise AssertionError("no hyperedge of two vertices")

    def expect(fragments):
        with pytest.raises(mhs.MhsError) as ei:
            mhs.Instance.load_batch(insts)
        assert ei.value.status == mhs.MHS_EINVAL
        for frag in fragments:
            assert frag in str(ei.value), str(ei.value)

    e70 = first_pair_edge(insts[70])
    p = int(insts[70].edge_ptr[e70])
    kept = insts[70].edge_vtx.copy()
    insts[70].edge_vtx[p + 1] = insts[70].edge_vtx[p]  # a vertex listed twice
    insts[90].edge_vtx[0] = insts[90].n  # a vertex id out of range
    expect(["instance 70:", "twice"])
    insts[70].edge_vtx[:] = kept
    expect(["instance 90:", "outside"])
    insts[5].demand[0] = 0
    expect(["instance 5:", "demand"])
    assert np.all(insts[5].demand[1:] >= 1)
