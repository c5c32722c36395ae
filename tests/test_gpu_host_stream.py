"""Pipelined host-to-host solves through the C ABI (fem_fft_solve_host,
fem_fft_host_wait; HostSolveStream wraps them): several distinct right-hand
sides from pinned host memory, one and several per call, results identical to
the device solve of the same plan (the pipeline only moves data; it must not
change a bit), and the mixed path against the oracle."""

import numpy as np
import pytest

from oracle import solve as osolve
from paper_1701_03967_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASE = dict(n=3, K=(12, 16), X=(1.0, 2.0), a=(1.0, 2.5), c=0.5)


@pytest.mark.parametrize("max_nrhs", [1, 2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_host_stream_matches_device_solve(max_nrhs, precision):
    from paper_1701_03967_gb300 import HostSolveStream, Plan
    pl = Plan(CASE["n"], CASE["K"], CASE["X"], CASE["a"], CASE["c"], precision, max_nrhs=max_nrhs)
    M = pl.M
    nsub = 7
    bs = [torch.from_numpy(synth.normal_field(M, synth.CFG_TEST, k)).pin_memory() for k in range(nsub)]
    us = [torch.empty_like(b).pin_memory() for b in bs]
    pipe = HostSolveStream(pl)
    for b, u in zip(bs, us):
        pipe.submit(b, u)
    pipe.synchronize()
    # several right-hand sides in one call (groups of max_nrhs through the slots)
    b3 = torch.from_numpy(synth.normal_batch(3, M, synth.CFG_TEST, 40)).pin_memory()
    u3 = torch.empty_like(b3).pin_memory()
    pl.solve_host(b3, u3)
    pl.host_wait()
    torch.cuda.synchronize()
    assert torch.equal(u3, pl.solve(b3.cuda()).cpu())
    prob = osolve.Problem(CASE["n"], CASE["K"], CASE["X"], CASE["a"], CASE["c"])
    for k, (b, u) in enumerate(zip(bs, us)):
        ref = pl.solve(b.cuda()).cpu()
        assert torch.equal(u, ref), k
        if k < 2:
            want = osolve.solve(prob, b.numpy())
            tol = 1e-12 if precision == "fp64" else 1e-10
            assert np.linalg.norm(u.numpy() - want) / np.linalg.norm(want) <= tol
    pl.close()


def test_host_stream_rejects_wrong_shapes():
    from paper_1701_03967_gb300 import HostSolveStream, Plan
    pl = Plan(CASE["n"], CASE["K"], CASE["X"], CASE["a"], CASE["c"], "fp64")
    pipe = HostSolveStream(pl)
    with pytest.raises(ValueError):
        pipe.submit(torch.zeros(5, dtype=torch.float64).pin_memory(), torch.zeros(5, dtype=torch.float64))
    with pytest.raises(TypeError):
        pl.solve_host(torch.zeros(pl.M, dtype=torch.float64).cuda(), torch.zeros(pl.M, dtype=torch.float64))
    pl.close()
