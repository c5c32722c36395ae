"""Pencils too long for one CTA's shared memory (contiguous axis): the
global four-step path of the transforms and the 1D solve, against the
oracle's dense eigenbasis where it fits in host memory, and by the mass
round trip (the direct FC_n transform expands calC^-1 y, Theorem 2) and the
float64 solve at the paper's sizes (Section 5 uses K up to 2^20)."""

import numpy as np
import pytest

from oracle import solve as osolve
from paper_1701_03967_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def _relmax(x, y):
    return float(np.max(np.abs(x - y)) / np.max(np.abs(y)))


# float64 pencils beyond the shared-memory kernels: n=2 K=4096, n=1 K=8192, n=1 K=6144 (radix 3)
ORACLE_CASES = [dict(n=2, K=4096, c=0.5), dict(n=1, K=8192, c=0.0), dict(n=1, K=6144, c=2.0)]


@pytest.mark.parametrize("case", ORACLE_CASES, ids=lambda c: f"n{c['n']}_K{c['K']}")
def test_long_transforms_and_solve_match_oracle(case):
    from paper_1701_03967_gb300 import Plan
    n, K = case["n"], case["K"]
    prob = osolve.Problem(n, (K,), None, None, case["c"])
    plan = Plan(n, (K,), None, None, case["c"], "fp64", max_nrhs=2)
    y = synth.normal_batch(2, prob.M, synth.CFG_TEST, 600)
    yt = torch.from_numpy(y).cuda()
    # forward against the oracle, up to the free signs of the bubble vectors
    got = plan.forward(yt).cpu().numpy()
    want = osolve.forward_coefficients(prob, y)
    lam, cn, p = plan.axis_tables(0)
    _, S, _ = prob.basis1d(0)
    sg = np.ones(prob.M[0])
    for l in range(n - 1):
        sg[l] = np.sign(p[0, l] @ S[0:n - 1, l])
    assert _rel(got * sg, want) <= 1e-12
    assert _relmax(got * sg, want) <= 1e-12
    w = synth.normal_batch(2, prob.M, synth.CFG_TEST, 601)
    gw = plan.inverse(torch.from_numpy(w * sg).cuda()).cpu().numpy()
    assert _rel(gw, osolve.inverse_expansion(prob, w)) <= 1e-12
    # the 1D solve (fused forward / divide / inverse pass on the long path)
    u = plan.solve(yt).cpu().numpy()
    want_u = osolve.solve(prob, y)
    assert _rel(u, want_u) <= 1e-12
    assert _relmax(u, want_u) <= 1e-12
    plan.close()


@pytest.mark.parametrize("n,K", [(5, 1 << 16), (9, 1 << 14), (2, 3 << 14), (5, 1 << 20)])
def test_long_mass_round_trip(n, K):
    """inverse F_n(forward FC_n(calC y)) = y for K up to 2^20 (float64)."""
    from paper_1701_03967_gb300 import Plan
    M = n * K - 1
    nrhs = 2 if K <= (1 << 16) else 1
    plan = Plan(n, (K,), None, None, 0.0, "fp64", max_nrhs=nrhs)
    y = torch.from_numpy(synth.normal_batch(nrhs, (M,), synth.CFG_TEST, 602)).cuda()
    w = plan.inverse(plan.forward(plan.apply_mass(y)))
    rel = float(torch.linalg.vector_norm(w - y) / torch.linalg.vector_norm(y))
    assert rel <= 1e-12, rel
    # the direct F_n transform folds the mass product into the same passes
    w2 = plan.inverse(plan.forward_fn(y))
    assert float(torch.linalg.vector_norm(w2 - y) / torch.linalg.vector_norm(y)) <= 1e-12
    plan.close()


def test_long_mixed_solve_matches_fp64():
    """n=5 K=8192: the float32 pencil exceeds one CTA's shared memory; the
    refined mixed solve matches the float64 solve (long path both) to the
    mixed bar."""
    from paper_1701_03967_gb300 import Plan
    n, K = 5, 8192
    M = n * K - 1
    b = torch.from_numpy(synth.normal_batch(2, (M,), synth.CFG_TEST, 603)).cuda()
    p64 = Plan(n, (K,), None, None, 1.0, "fp64", max_nrhs=2)
    pmx = Plan(n, (K,), None, None, 1.0, "mixed", max_nrhs=2)
    u64 = p64.solve(b)
    umx = pmx.solve(b)
    rel = float(torch.linalg.vector_norm(umx - u64) / torch.linalg.vector_norm(u64))
    assert rel <= 1e-10, rel
    p64.close()
    pmx.close()
