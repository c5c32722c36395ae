"""Per-axis element orders n_i (Section 4 states the N-D problem with 1D
spaces S_{K_i}^{(n_i)} of their own orders): solves on both algorithms and in
both precisions, the operator, the mass operator, the transforms and
non-zero Dirichlet data, against the oracle's Problem with the same orders."""

import numpy as np
import pytest

from oracle import harness
from oracle import solve as osolve
from paper_1701_03967_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    dict(n=(3, 7), K=(32, 16), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0),
    dict(n=(2, 5, 9), K=(8, 8, 4), X=(1.0, 0.7, 1.2), a=(0.8, 1.3, 2.0), c=0.2),
    dict(n=(7, 3), K=(64, 128), X=(1.0, 1.0), a=(1.0, 1.0), c=0.0),      # register-radix passes on both axes
    dict(n=(1, 9), K=(48, 12), X=(2.0, 1.0), a=(1.5, 0.5), c=0.4),       # shared-memory Stockham passes
]


def _ids(c):
    return "n" + "_".join(map(str, c["n"])) + "_K" + "x".join(map(str, c["K"]))


def _rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def _relmax(x, y):
    return float(np.max(np.abs(x - y)) / np.max(np.abs(y)))


def _prob(case):
    return osolve.Problem(case["n"], case["K"], case["X"], case["a"], case["c"])


def _plan(case, precision, max_nrhs=2):
    from paper_1701_03967_gb300 import Plan
    return Plan(case["n"], case["K"], case["X"], case["a"], case["c"], precision, max_nrhs=max_nrhs)


@pytest.mark.parametrize("case", CASES, ids=_ids)
@pytest.mark.parametrize("algo", ["a", "b"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_solve_with_per_axis_orders(case, algo, precision, tol):
    prob = osolve.Problem(case["n"], case["K"], case["X"], case["a"], case["c"])
    b = synth.normal_batch(2, prob.M, synth.CFG_TEST, 500)
    want = osolve.solve(prob, b)
    plan = _plan(case, precision)
    assert plan.M == prob.M
    plan.set_algorithm(algo)
    got = plan.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    plan.close()
    assert _rel(got, want) <= tol
    assert _relmax(got, want) <= tol


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_operators_and_transforms_with_per_axis_orders(case):
    prob = osolve.Problem(case["n"], case["K"], case["X"], case["a"], case["c"])
    u = synth.normal_batch(2, prob.M, synth.CFG_TEST, 501)
    plan = _plan(case, "fp64")
    ut = torch.from_numpy(u).cuda()
    assert _rel(plan.apply(ut).cpu().numpy(), osolve.apply(prob, u)) <= 1e-13
    assert _rel(plan.apply_mass(ut).cpu().numpy(), osolve.mass_apply(prob, u)) <= 1e-13
    # inverse F_n(direct F_n(u)) = u, and inverse(forward(C u)) = u
    assert _rel(plan.inverse(plan.forward_fn(ut)).cpu().numpy(), u) <= 1e-12
    assert _rel(plan.inverse(plan.forward(plan.apply_mass(ut))).cpu().numpy(), u) <= 1e-12
    plan.close()


@pytest.mark.parametrize("case", CASES[:2], ids=_ids)
def test_dirichlet_polynomial_with_per_axis_orders(case):
    """u = prod_i P_i(x_i) with deg P_i = n_i lies in the FEM space: the
    corrected solve returns it at every node."""
    prob = osolve.Problem(case["n"], case["K"], case["X"], case["a"], case["c"])
    N = prob.N
    rng = np.random.default_rng(23)
    P = [np.polynomial.Polynomial(rng.uniform(-1, 1, prob.ns[i] + 1)) for i in range(N)]

    def u(*x):
        out = np.ones_like(x[0])
        for i in range(N):
            out = out * P[i](x[i])
        return out

    def f(*x):
        out = prob.c * u(*x)
        for i in range(N):
            t = P[i].deriv(2)(x[i])
            for j in range(N):
                if j != i:
                    t = t * P[j](x[j])
            out = out - prob.a[i] * t
        return out

    b = np.ascontiguousarray(harness.load_vector(prob, f))
    grids = [np.arange(prob.M[i] + 2) * prob.h[i] / prob.ns[i] for i in range(N)]
    g = np.ascontiguousarray(u(*np.meshgrid(*grids, indexing="ij")))
    want = harness.nodal_values(prob, u)
    plan = _plan(case, "fp64", 1)
    got = plan.solve_dirichlet(torch.from_numpy(b).cuda(), torch.from_numpy(g).cuda()).cpu().numpy()
    plan.close()
    assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want))


def test_batch_of_per_axis_order_plans_runs_in_stream_mode():
    """A batch holding plans with per-axis orders solves every problem by its
    own plan on the batch's streams (the graph launch, one element order per
    launch, is refused), to the mixed bar against the oracle."""
    from paper_1701_03967_gb300 import Batch, FemFftError
    cases = [CASES[0], CASES[1], dict(n=4, K=(16, 8), X=(1.0, 1.0), a=(1.0, 2.0), c=0.5)]
    plans = [_plan(c, "mixed", 2) for c in cases]
    batch = Batch(plans, [2, 1, 2], tune=False)
    assert batch.n_steps == 0
    with pytest.raises(FemFftError):
        batch.set_mode("graph")
    rhs = [synth.normal_batch(r, _prob(c).M, synth.CFG_TEST, 700 + i) for i, (c, r) in enumerate(zip(cases, [2, 1, 2]))]
    u = batch.solve(batch.pack(rhs))
    torch.cuda.synchronize()
    for c, bp, up in zip(cases, rhs, batch.views(u)):
        want = osolve.solve(_prob(c), bp)
        assert _rel(up.cpu().numpy(), want) <= 1e-10, c
    for pl in plans:
        pl.close()
