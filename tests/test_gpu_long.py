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


# Strided long pencils: an earlier axis of a 2D/3D field too long for one
# CTA (pencil-fastest workspace, group padded to 16 pencils).  Axis 0 long:
# the fused forward/divide/inverse pass on the long path, its divisor taking
# the later axes' eigenvalues (one or two of them); a middle axis long: the
# forward and inverse passes with pencils strided by the last axis.
STRIDED_CASES = [
    dict(n=(1, 2), K=(8192, 4), a=(1.0, 2.0), c=0.5),       # fused pass long, 7 pencils per outer index
    dict(n=(1, 1, 2), K=(6144, 2, 2), a=(1.0, 1.5, 0.7), c=0.0),   # fused long, two later axes, K = 3 * 2^11
    dict(n=(2, 1, 2), K=(2, 6144, 2), a=(0.8, 1.0, 1.3), c=1.0),   # middle axis long
]


def _bubble_signs(plan, prob):
    """Signs of the oracle's bubble vectors relative to the plan's, as one
    array over the field (the free signs of Theorem 1's element modes)."""
    sgs = []
    for i in range(prob.N):
        n = prob.ns[i]
        sg = np.ones(prob.M[i])
        if n >= 2:
            _, _, p = plan.axis_tables(i)
            _, S, _ = prob.basis1d(i)
            for l in range(n - 1):
                sg[l] = np.sign(p[0, l] @ S[0:n - 1, l])
        sgs.append(sg)
    out = sgs[0]
    for sg in sgs[1:]:
        out = np.multiply.outer(out, sg)
    return out


@pytest.mark.parametrize("case", STRIDED_CASES, ids=lambda c: "n" + "x".join(map(str, c["n"])) + "_K" +
                         "x".join(map(str, c["K"])))
def test_strided_long_pencils_match_oracle(case):
    from paper_1701_03967_gb300 import Plan
    prob = osolve.Problem(case["n"], case["K"], None, case["a"], case["c"])
    p64 = Plan(case["n"], case["K"], None, case["a"], case["c"], "fp64", max_nrhs=2)
    y = synth.normal_batch(2, prob.M, synth.CFG_TEST, 610)
    yt = torch.from_numpy(y).cuda()
    sg = _bubble_signs(p64, prob)
    got = p64.forward(yt).cpu().numpy()
    want = osolve.forward_coefficients(prob, y)
    assert _rel(got * sg, want) <= 1e-12
    assert _relmax(got * sg, want) <= 1e-12
    w = synth.normal_batch(2, prob.M, synth.CFG_TEST, 611)
    gw = p64.inverse(torch.from_numpy(w * sg).cuda()).cpu().numpy()
    want_w = osolve.inverse_expansion(prob, w)
    assert _rel(gw, want_w) <= 1e-12
    assert _relmax(gw, want_w) <= 1e-12
    want_u = osolve.solve(prob, y)
    u = p64.solve(yt).cpu().numpy()
    assert _rel(u, want_u) <= 1e-12
    assert _relmax(u, want_u) <= 1e-12
    pmx = Plan(case["n"], case["K"], None, case["a"], case["c"], "mixed", max_nrhs=2)
    um = pmx.solve(yt).cpu().numpy()
    assert _rel(um, want_u) <= 1e-10
    assert _relmax(um, want_u) <= 1e-10
    p64.close()
    pmx.close()
