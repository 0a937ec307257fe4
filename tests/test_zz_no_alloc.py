"""pibm_fluid_sums_noalloc against the plain FP64 sums and pibm_invariants.

Some callers must not allocate device memory: code running inside a stream
capture it does not own, real-time stepping loops held to a fixed memory budget,
allocator hooks that must not re-enter the allocator. For them the library sums
mass and fluid momentum of their own population arrays with its scratch in a
static device array. Those sums must equal the sums written out in NumPy FP64
(sum_a f_a and sum_a e_a f_a over every cell) and what pibm_invariants reports
for a simulation holding the same populations, on every call (the scratch is
reused). This file is collected last so that a failure here stops a run only
after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from oracle.oracle import lattice
from paper_1407_6704_gb300.inputs import populations

pytestmark = pytest.mark.gpu

LAT = {9: "d2q9", 15: "d3q15", 19: "d3q19"}


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1407_6704_gb300 import _lib, build

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    return _lib.load()


@pytest.mark.parametrize("q,n", [(9, (37, 29)), (19, (13, 11, 9)), (15, (10, 9, 12))])
def test_noalloc_sums_match_invariants_on_two_calls(lib, q, n):
    import torch
    from paper_1407_6704_gb300.pibm import Pibm

    d = len(n)
    shape = tuple(reversed(n))
    f0 = populations(np.full(q, 1.0 / q), shape, seed=41 + q, eps=0.05)
    with Pibm(LAT[q], n, (0,) * d, 0.8, f0=f0) as sim:
        mass, J, _ = sim.invariants()
    inv = np.concatenate([[mass], J])
    # the definition: sum_a f_a and sum_a e_a f_a over all cells, FP64
    e = lattice(q)[1]
    fq = f0.reshape(q, -1)
    ref = np.concatenate([[fq.sum()], [(e[:, k][:, None] * fq).sum() for k in range(d)]])
    assert np.abs(inv - ref).max() <= 1e-12 * np.abs(ref).max()
    f_dev = torch.from_numpy(np.ascontiguousarray(f0.reshape(q, -1))).cuda()
    n3 = (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - d)))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    results = []
    for _ in range(2):
        out = torch.full((1 + d,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.pibm_fluid_sums_noalloc(ctypes.c_void_p(f_dev.data_ptr()), q, n3,
                                         ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, lib.pibm_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # FP64 sums of O(1e4) terms in two different orders
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (got, ref)
        assert np.abs(got - inv).max() <= 1e-12 * np.abs(ref).max(), (got, inv)
        results.append(got)
    assert np.array_equal(results[0], results[1])  # fixed summation order


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    import torch
    from paper_1407_6704_gb300 import _lib

    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    n3 = (ctypes.c_int64 * 3)(5000, 4000, 1)  # 20M cells > 16,777,216
    rc = lib.pibm_fluid_sums_noalloc(ctypes.c_void_p(dummy.data_ptr()), 9, n3,
                                     ctypes.c_void_p(dummy.data_ptr()), None)
    assert rc == _lib.PIBM_ETOOBIG
    assert lib.pibm_strerror(rc) != b"unknown status"
