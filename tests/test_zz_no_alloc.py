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
