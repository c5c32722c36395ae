"""Non-zero Dirichlet data (Section 4 with u = g on the boundary): the
correction b -= L_full G of fem_fft_dirichlet_rhs against the oracle's
``dirichlet_rhs`` on random boundary data (float64 products: relative 1e-12),
and polynomial solutions of degree <= n, which the FEM reproduces exactly, through
the GPU solve of the corrected right-hand side (FP64: 1e-11 of the maximum,
mixed: 1e-10 relative L2)."""

import numpy as np
import pytest

from oracle import harness
from oracle import solve as osolve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [dict(n=4, K=(6,), X=(2.0,), a=(2.0,), c=1.5),
         dict(n=2, K=(6, 16), X=(1.0, 1.5), a=(1.3, 0.7), c=0.4),
         dict(n=9, K=(4, 6), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0),
         dict(n=3, K=(4, 6, 2), X=(1.0, 0.8, 1.2), a=(0.9, 1.1, 2.0), c=0.0)]
IDS = [f"n{c['n']}_{len(c['K'])}d" for c in CASES]


def _plan(case, precision="fp64", max_nrhs=1):
    from paper_1701_03967_gb300 import Plan
    return Plan(case["n"], case["K"], case["X"], case["a"], case["c"], precision, max_nrhs=max_nrhs)


def _prob(case):
    return osolve.Problem(case["n"], case["K"], case["X"], case["a"], case["c"])


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("nrhs", [1, 3])
def test_dirichlet_correction_matches_oracle(case, nrhs):
    prob = _prob(case)
    rng = np.random.default_rng(3)
    ext = tuple(m + 2 for m in prob.M)
    g = rng.standard_normal((nrhs,) + ext)
    b = rng.standard_normal((nrhs,) + prob.M)
    want = b - osolve.dirichlet_rhs(prob, g)
    pl = _plan(case, max_nrhs=nrhs)
    gt = torch.from_numpy(g).cuda()
    if nrhs == 1:
        got = pl.dirichlet_rhs(gt[0].contiguous(), torch.from_numpy(b[0]).cuda())[None]
    else:
        got = pl.dirichlet_rhs(gt, torch.from_numpy(b).cuda())
    got = got.cpu().numpy()
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    # interior entries of g are ignored
    g2 = g.copy()
    g2[(slice(None),) + (slice(1, -1),) * prob.N] = 7.0
    got2 = pl.dirichlet_rhs(torch.from_numpy(g2).cuda() if nrhs > 1 else torch.from_numpy(g2[0]).cuda(),
                            torch.from_numpy(b if nrhs > 1 else b[0]).cuda()).cpu().numpy()
    assert np.array_equal(got2.reshape(got.shape), got)
    pl.close()


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_polynomial_solutions_are_reproduced(case, precision):
    n, N = case["n"], len(case["K"])
    prob = _prob(case)
    rng = np.random.default_rng(5)
    P = [np.polynomial.Polynomial(rng.uniform(-1, 1, n + 1)) for _ in range(N)]

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
    grid = [np.arange(prob.M[i] + 2) * prob.h[i] / n for i in range(N)]
    g = np.ascontiguousarray(u(*np.meshgrid(*grid, indexing="ij")))
    want = harness.nodal_values(prob, u)
    pl = _plan(case, precision)
    got = pl.solve_dirichlet(torch.from_numpy(b).cuda(), torch.from_numpy(g).cuda()).cpu().numpy()
    if precision == "fp64":
        assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want))
    else:
        assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
    pl.close()


def test_dirichlet_rejects_bad_shapes_and_accepts_no_rhs():
    from paper_1701_03967_gb300 import _lib
    pl = _plan(CASES[1])
    b = torch.zeros(pl.M, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        pl.dirichlet_rhs(torch.zeros(pl.M, dtype=torch.float64, device="cuda"), b)
    assert _lib.lib().fem_fft_dirichlet_rhs(pl._h, 0, 0, 0, None) == 0
    pl.close()
