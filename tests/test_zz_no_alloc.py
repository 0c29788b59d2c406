"""mhs_kernelize_noalloc: the kernelization entry point that allocates no
memory (its working set is a fixed device array inside the library), for
callers that may not call cudaMalloc while they run.

Its results must equal those of the allocating path (mhs_load_device +
mhs_kernelize + mhs_result_device) exactly, on two calls in a row (the
second call reuses the array the first one left behind).  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_2109_06042_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2109_06042_gb300 import build
    build.build()
    from paper_2109_06042_gb300 import mhs
    return torch, mhs


def _dev(torch, inst):
    d = torch.device("cuda:0")
    vtx = inst.edge_vtx if inst.nnz else np.zeros(1, np.int32)
    dem = inst.demand if inst.m else np.zeros(1, np.int32)
    return (torch.from_numpy(np.ascontiguousarray(inst.edge_ptr, np.int32)).to(d),
            torch.from_numpy(np.ascontiguousarray(vtx, np.int32)).to(d),
            torch.from_numpy(np.ascontiguousarray(dem, np.int32)).to(d))


def _allocating(torch, mhs, inst, ptr, vtx, dem):
    d = torch.device("cuda:0")
    av = torch.zeros(max(inst.n, 1), dtype=torch.uint8, device=d)
    ae = torch.zeros(max(inst.m, 1), dtype=torch.uint8, device=d)
    with mhs.Instance.load_device(inst.n, inst.m, ptr, vtx, dem, inst.k,
                                  contraction="popcount") as h:
        h.kernelize()
        h.result_device(av, ae)
        rounds = h.result()["rounds"]
    torch.cuda.synchronize()
    return av.cpu().numpy()[:inst.n], ae.cpu().numpy()[:inst.m], rounds


def _noalloc(torch, mhs, inst, ptr, vtx, dem):
    d = torch.device("cuda:0")
    # poison the outputs so stale values cannot pass
    av = torch.full((max(inst.n, 1),), 7, dtype=torch.uint8, device=d)
    ae = torch.full((max(inst.m, 1),), 7, dtype=torch.uint8, device=d)
    rounds = mhs.kernelize_noalloc(inst.n, inst.m, ptr, vtx, dem, inst.nnz, av, ae)
    torch.cuda.synchronize()
    return av.cpu().numpy()[:inst.n], ae.cpu().numpy()[:inst.m], rounds


def test_noalloc_matches_allocating_path_twice(env):
    torch, mhs = env
    cases = [I.config_uniform(0), I.config_batch_one(4007),
             I.uniform_random(4096, 4096, 2, 16, 3, 0, 99), I.config_uniform(1)]
    for inst in cases:
        assert inst.nnz <= 65536
        ptr, vtx, dem = _dev(torch, inst)
        ref = _allocating(torch, mhs, inst, ptr, vtx, dem)
        for call in range(2):
            got = _noalloc(torch, mhs, inst, ptr, vtx, dem)
            assert np.array_equal(got[0], ref[0]), (inst.name, call)
            assert np.array_equal(got[1], ref[1]), (inst.name, call)
            assert got[2] == ref[2], (inst.name, call)


def test_noalloc_rejects_oversize(env):
    torch, mhs = env
    inst = I.uniform_random(5000, 100, 2, 4, 1, 0, 3)
    ptr, vtx, dem = _dev(torch, inst)
    av = torch.zeros(inst.n, dtype=torch.uint8, device="cuda:0")
    ae = torch.zeros(inst.m, dtype=torch.uint8, device="cuda:0")
    with pytest.raises(mhs.MhsError) as ei:
        mhs.kernelize_noalloc(inst.n, inst.m, ptr, vtx, dem, inst.nnz, av, ae)
    assert ei.value.status == mhs.MHS_EINVAL
    assert "too large" in str(ei.value)


def test_noalloc_malformed_then_valid(env):
    """A vertex id out of range is caught by the device-side validation
    (MHS_EINVAL); the next valid call still matches the allocating path."""
    torch, mhs = env
    inst = I.config_uniform(2)
    ptr, vtx, dem = _dev(torch, inst)
    bad = vtx.clone()
    bad[5] = inst.n + 3
    av = torch.zeros(inst.n, dtype=torch.uint8, device="cuda:0")
    ae = torch.zeros(inst.m, dtype=torch.uint8, device="cuda:0")
    with pytest.raises(mhs.MhsError) as ei:
        mhs.kernelize_noalloc(inst.n, inst.m, ptr, bad, dem, inst.nnz, av, ae)
    assert ei.value.status == mhs.MHS_EINVAL
    ref = _allocating(torch, mhs, inst, ptr, vtx, dem)
    got = _noalloc(torch, mhs, inst, ptr, vtx, dem)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    assert got[2] == ref[2]


def test_noalloc_on_a_side_stream(env):
    """The call runs on the stream it is given (a non-default torch stream)."""
    torch, mhs = env
    inst = I.config_batch_one(4011)
    ptr, vtx, dem = _dev(torch, inst)
    ref = _allocating(torch, mhs, inst, ptr, vtx, dem)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        av = torch.full((inst.n,), 7, dtype=torch.uint8, device="cuda:0")
        ae = torch.full((inst.m,), 7, dtype=torch.uint8, device="cuda:0")
    for _ in range(2):
        rounds = mhs.kernelize_noalloc(inst.n, inst.m, ptr, vtx, dem, inst.nnz, av, ae,
                                       stream=side)
        side.synchronize()
        assert np.array_equal(av.cpu().numpy(), ref[0])
        assert np.array_equal(ae.cpu().numpy(), ref[1])
        assert rounds == ref[2]


def test_noalloc_empty_instances(env):
    """No hyperedges (every vertex isolated, so deleted) and no vertices at
    all: masks and round counts equal the allocating path's."""
    torch, mhs = env
    for inst in (I.from_edges(0, [], []), I.from_edges(6, [], [])):
        ptr, vtx, dem = _dev(torch, inst)
        ref = _allocating(torch, mhs, inst, ptr, vtx, dem)
        for _ in range(2):
            got = _noalloc(torch, mhs, inst, ptr, vtx, dem)
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
            assert got[2] == ref[2]


def test_noalloc_rejects_host_memory(env):
    """A CPU tensor is refused before any kernel runs (the binding checks,
    and so does the library itself for a pointer it is handed directly)."""
    torch, mhs = env
    import ctypes
    inst = I.config_uniform(3)
    ptr, vtx, dem = _dev(torch, inst)
    av_host = torch.zeros(inst.n, dtype=torch.uint8)
    ae = torch.zeros(inst.m, dtype=torch.uint8, device="cuda:0")
    with pytest.raises(mhs.MhsError) as ei:
        mhs.kernelize_noalloc(inst.n, inst.m, ptr, vtx, dem, inst.nnz, av_host, ae)
    assert ei.value.status == mhs.MHS_EINVAL
    buf = ctypes.create_string_buffer(256)
    st = mhs.lib().mhs_kernelize_noalloc(
        inst.n, inst.m, ctypes.c_void_p(ptr.data_ptr()), ctypes.c_void_p(vtx.data_ptr()),
        ctypes.c_void_p(dem.data_ptr()), inst.nnz, ctypes.c_void_p(av_host.data_ptr()),
        ctypes.c_void_p(ae.data_ptr()), None, None, buf, 256)
    assert st == mhs.MHS_EINVAL and b"device memory" in buf.value
    # the context is unharmed: a valid call still matches
    ref = _allocating(torch, mhs, inst, ptr, vtx, dem)
    got = _noalloc(torch, mhs, inst, ptr, vtx, dem)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
