"""The allocation-free operator apply (fem_fft_apply_noalloc), called through
the C ABI, against the plan-based fem_fft_apply.

Callers that cannot allocate device memory where they apply the operator (a
host callback or allocator hook that must not re-enter the allocator, a
framework that forbids device allocation after its warm-up) use the
allocation-free entry point; its temporaries live in a static device array
shared by all calls.  This file is collected last so that a run stopping at
the first failure has already run every other test; it also passes on its own
in a fresh process."""

import ctypes
import gc

import numpy as np
import pytest

from paper_1701_03967_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(L, case, u, b):
    N = len(case["K"])
    K = (ctypes.c_int64 * N)(*case["K"])
    X = (ctypes.c_double * N)(*case["X"])
    a = (ctypes.c_double * N)(*case["a"])
    nrhs = u.shape[0]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.fem_fft_apply_noalloc(N, case["n"], K, X, a, case["c"], u.data_ptr(), b.data_ptr(), nrhs, stream)


CASES = [
    dict(n=3, K=(16,), X=(1.3,), a=(0.7,), c=0.2),
    dict(n=9, K=(64, 32), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0),
    dict(n=5, K=(16, 8, 12), X=(1.0, 1.2, 0.8), a=(1.0, 0.5, 2.0), c=0.3),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c['n']}_K{'x'.join(map(str, c['K']))}")
def test_noalloc_apply_matches_plan_apply_twice(case):
    from paper_1701_03967_gb300 import Plan, _lib
    L = _lib.lib()
    plan = Plan(case["n"], case["K"], case["X"], case["a"], case["c"], max_nrhs=2)
    for call in range(2):   # two calls in a row share (and reuse) the scratch
        u = torch.from_numpy(synth.normal_batch(2, plan.M, synth.CFG_TEST, 300 + call)).cuda()
        want = plan.apply(u)
        got = torch.full_like(u, float("nan"))
        # garbage left by earlier tests must not be collected inside the
        # measured region (a collection frees tensors and changes the counts)
        gc.collect()
        gc.disable()
        try:
            torch.cuda.synchronize()
            free0, _ = torch.cuda.mem_get_info()
            alloc0 = torch.cuda.memory_allocated()
            assert _noalloc(L, case, u, got) == 0
            torch.cuda.synchronize()
            # the call takes no memory from torch's allocator; after the first
            # call (which may load the library's device module holding the
            # static array) none from the driver either
            assert torch.cuda.memory_allocated() == alloc0
            if call > 0:
                assert torch.cuda.mem_get_info()[0] == free0
        finally:
            gc.enable()
        rel = float(torch.linalg.norm(got - want) / torch.linalg.norm(want))
        assert rel <= 1e-13, (call, rel)
    plan.close()


def test_noalloc_rejects_problems_beyond_the_scratch():
    from paper_1701_03967_gb300 import _lib
    L = _lib.lib()
    big = dict(n=9, K=(1024, 1024), X=(1.0, 1.0), a=(1.0, 1.0), c=0.0)
    small = torch.zeros((1, 4), dtype=torch.float64, device="cuda")
    # rejected by the size check before any launch: the buffers are never touched
    assert _noalloc(L, big, small, small.clone()) == -1


def test_noalloc_rejects_overlapping_ranges():
    from paper_1701_03967_gb300 import _lib
    L = _lib.lib()
    case = CASES[1]
    M = 1
    for k in case["K"]:
        M *= case["n"] * k - 1
    buf = torch.zeros((3, M), dtype=torch.float64, device="cuda")
    # b starts inside u's range (u = rows 0..1, b = rows 1..2): rejected before any launch
    u = buf[0:2]
    b = buf[1:3]
    assert _noalloc(L, case, u, b) == -1
