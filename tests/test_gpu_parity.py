"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (relative L2 over all DOF and right-hand sides): 1e-12 for the
FP64 path and 1e-10 for the mixed path after refinement (the solver's
accuracy targets); transforms and the operator apply are checked at 1e-12 /
1e-13."""

import numpy as np
import pytest

from oracle import fem1d, harness, solve as osolve
from paper_1701_03967_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _plan(case, precision="fp64", max_nrhs=1):
    from paper_1701_03967_gb300 import Plan
    return Plan(case["n"], case["K"], case.get("X"), case.get("a"), case.get("c", 0.0), precision,
                max_nrhs=max_nrhs)


def _prob(case):
    return osolve.Problem(case["n"], case["K"], case.get("X"), case.get("a"), case.get("c", 0.0))


def _rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def _relmax(x, y):
    """Relative max-norm error: a localised error (one bad pencil or boundary
    element) that a relative L2 norm over many unknowns would hide."""
    return float(np.max(np.abs(x - y)) / np.max(np.abs(y)))


CASES = [
    dict(n=3, K=(8,), X=(1.3,), a=(0.7,), c=0.2),
    dict(n=9, K=(16,), c=1.0),
    dict(n=1, K=(2,)),
    dict(n=2, K=(6,), X=(2.0,), a=(1.5,), c=-1.0),
    dict(n=5, K=(48,)),
    dict(n=2, K=(16, 16)),
    dict(n=9, K=(16, 32), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0),
    dict(n=4, K=(12, 8), X=(0.7, 1.1), a=(2.0, 0.5), c=0.3),
    dict(n=7, K=(6, 4)),
    dict(n=1, K=(64, 2), c=3.0),
    dict(n=8, K=(32, 16), a=(3.0, 1.0)),
    dict(n=6, K=(24, 18)),
    dict(n=3, K=(4, 8, 6), X=(1.0, 1.5, 0.5), a=(1.0, 0.6, 2.0), c=0.1),
    dict(n=9, K=(4, 4, 4)),
    dict(n=2, K=(16, 8, 12), c=2.0),
    dict(n=5, K=(8, 8, 8)),
    dict(n=4, K=(2, 2, 2)),
]


def _ids(c):
    return f"n{c['n']}_K{'x'.join(map(str, c['K']))}"


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_solve_fp64_matches_oracle(case):
    prob = _prob(case)
    b = synth.normal_batch(2, prob.M, synth.CFG_TEST, 101)
    want = osolve.solve(prob, b)
    plan = _plan(case, "fp64", max_nrhs=2)
    got = plan.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(got, want) <= 1e-12
    assert _relmax(got, want) <= 1e-12


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_solve_mixed_matches_oracle(case):
    prob = _prob(case)
    b = synth.normal_batch(2, prob.M, synth.CFG_TEST, 102)
    want = osolve.solve(prob, b)
    plan = _plan(case, "mixed", max_nrhs=2)
    plan.set_refinement(0.0, 2)
    got = plan.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(got, want) <= 1e-10
    assert _relmax(got, want) <= 1e-10


@pytest.mark.parametrize("case", CASES[::2], ids=_ids)
def test_apply_matches_oracle(case):
    prob = _prob(case)
    u = synth.normal_batch(2, prob.M, synth.CFG_TEST, 103)
    want = osolve.apply(prob, u)
    plan = _plan(case, "fp64", max_nrhs=2)
    got = plan.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    assert _rel(got, want) <= 1e-13
    assert _relmax(got, want) <= 1e-13


def _bubble_signs(plan, prob):
    """Per-axis sign vectors aligning the library's bubble eigenvectors e^(l)
    (sign is free) with the oracle's."""
    signs = []
    for i in range(prob.N):
        lam, cn, p = plan.axis_tables(i)
        _, S, _ = prob.basis1d(i)
        sg = np.ones(prob.M[i])
        n = prob.n
        for l in range(n - 1):
            sg[l] = np.sign(p[0, l] @ S[0:n - 1, l])
        signs.append(sg)
    return signs


@pytest.mark.parametrize("case", CASES[::3], ids=_ids)
def test_forward_and_inverse_transforms_match_oracle(case):
    prob = _prob(case)
    y = synth.normal_field(prob.M, synth.CFG_TEST, 104)
    plan = _plan(case, "fp64")
    got = plan.forward(torch.from_numpy(y).cuda()).cpu().numpy()
    want = osolve.forward_coefficients(prob, y)
    sg = _bubble_signs(plan, prob)
    S = np.ones(prob.M)
    for i, s in enumerate(sg):
        shape = [1] * prob.N
        shape[i] = prob.M[i]
        S = S * s.reshape(shape)
    assert _rel(got * S, want) <= 1e-12
    assert _relmax(got * S, want) <= 1e-12
    w = synth.normal_field(prob.M, synth.CFG_TEST, 105)
    got_w = plan.inverse(torch.from_numpy(w * S).cuda()).cpu().numpy()
    assert _rel(got_w, osolve.inverse_expansion(prob, w)) <= 1e-12
    assert _relmax(got_w, osolve.inverse_expansion(prob, w)) <= 1e-12


@pytest.mark.parametrize("case", CASES[::3] + [dict(n=1, K=(12,), c=0.5), dict(n=8, K=(6, 4), c=0.0)],
                         ids=lambda c: f"n{c['n']}_K{'x'.join(map(str, c['K']))}")
def test_direct_fn_transform_matches_oracle(case):
    """Direct F_n-transform (Theorem 2, item 3), the mass product folded into
    the forward maps: equals the FC_n coefficients of calC w (the oracle's
    dense eigenbasis products of its mass operator), and the inverse F_n
    transform of it returns w."""
    prob = _prob(case)
    w = synth.normal_batch(2, prob.M, synth.CFG_TEST, 106)
    plan = _plan(case, "fp64")
    wt = torch.from_numpy(w).cuda()
    got = plan.forward_fn(wt).cpu().numpy()
    want = osolve.forward_coefficients(prob, osolve.mass_apply(prob, w))
    sg = _bubble_signs(plan, prob)
    S = np.ones(prob.M)
    for i, s_ in enumerate(sg):
        shape = [1] * prob.N
        shape[i] = prob.M[i]
        S = S * s_.reshape(shape)
    assert _rel(got * S, want) <= 1e-12
    assert _relmax(got * S, want) <= 1e-12
    back = plan.inverse(torch.from_numpy(got).cuda()).cpu().numpy()
    assert _rel(back, w) <= 1e-12
    assert _relmax(back, w) <= 1e-12
    # in place
    plan.forward_fn(wt, out=wt)
    assert _rel(wt.cpu().numpy(), got) <= 1e-15


def test_manufactured_solution_error_matches_paper_table():
    """2D, n=5, K=16: max-norm error 5.4e-8 (Section 5 table, algorithm (a))."""
    u, f = harness.manufactured(harness.PAPER_2D, 2, (1, 1), 1.0)
    case = dict(n=5, K=(16, 16), c=1.0)
    prob = _prob(case)
    b = np.ascontiguousarray(harness.load_vector(prob, f))
    plan = _plan(case, "fp64")
    uh = plan.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    err = harness.max_error(prob, uh, u)
    assert abs(err / 5.4e-8 - 1) < 0.06


def test_edge_cases():
    from paper_1701_03967_gb300 import FemFftError, Plan
    case = dict(n=3, K=(8, 4))
    prob = _prob(case)
    plan = _plan(case, "fp64", max_nrhs=2)
    # nrhs larger than the workspace: processed in groups
    b = synth.normal_batch(5, prob.M, synth.CFG_TEST, 106)
    got = plan.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(got, osolve.solve(prob, b)) <= 1e-12
    assert _relmax(got, osolve.solve(prob, b)) <= 1e-12
    # in-place FP64 solve
    bt = torch.from_numpy(b[:2].copy()).cuda()
    plan.solve(bt, out=bt)
    assert _rel(bt.cpu().numpy(), osolve.solve(prob, b[:2])) <= 1e-12
    assert _relmax(bt.cpu().numpy(), osolve.solve(prob, b[:2])) <= 1e-12
    # zero right-hand sides
    z = torch.zeros((0,) + prob.M, dtype=torch.float64, device="cuda")
    plan.solve(z)
    # zero input gives zero output
    assert float(plan.solve(torch.zeros(prob.M, dtype=torch.float64, device="cuda")).abs().max()) == 0.0
    # invalid arguments
    for bad in [dict(n=3, K=(7, 4)), dict(n=0, K=(8,)), dict(n=10, K=(8,)), dict(n=3, K=(8,), c=-100.0),
                dict(n=3, K=(8,), a=(-1.0,)), dict(n=2, K=(4, 4, 4, 4))]:
        with pytest.raises(FemFftError):
            Plan(bad["n"], bad["K"], None, bad.get("a"), bad.get("c", 0.0))
    mixed = _plan(case, "mixed")
    with pytest.raises(FemFftError):
        mixed.solve(bt[0], out=bt[0])
    with pytest.raises(TypeError):
        plan.solve(torch.zeros(prob.M, dtype=torch.float32, device="cuda"))


@pytest.mark.parametrize("case", [dict(n=2, K=(4, 6), a=(1.2, 0.7), c=0.5), dict(n=3, K=(4, 2, 4), c=0.3)],
                         ids=_ids)
def test_grad_coeffs_match_oracle(case):
    prob = _prob(case)
    f = synth.normal_batch(2, prob.M, synth.CFG_TEST, 107)
    ut = synth.normal_batch(2, prob.M, synth.CFG_TEST, 108)
    u = osolve.solve(prob, f)
    gf, ga, gc = osolve.grad(prob, f, 2 * (u - ut))
    plan = _plan(case, "fp64", max_nrhs=2)
    ud = plan.solve(torch.from_numpy(f).cuda())
    lam = plan.solve(2 * (ud - torch.from_numpy(ut).cuda()))
    ga_g, gc_g = plan.grad_coeffs(ud, lam)
    np.testing.assert_allclose(ga_g, ga, rtol=1e-10)
    np.testing.assert_allclose(gc_g, gc, rtol=1e-10)
    assert _rel(lam.cpu().numpy(), gf) <= 1e-12
    assert _relmax(lam.cpu().numpy(), gf) <= 1e-12


@pytest.mark.parametrize("case", [dict(n=9, K=(16, 32), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0),
                                  dict(n=4, K=(8, 12, 8), a=(1.0, 2.0, 0.5), c=0.3),
                                  dict(n=7, K=(48,), c=0.0)], ids=["2d_n9", "3d_n4", "1d_n7"])
def test_mixed_residual_precisions(case):
    """The refinement residual in float64 and in double-float arithmetic: both
    reach the mixed-path target, and the two refined solutions agree to the
    double-float floor."""
    prob = _prob(case)
    b = synth.normal_batch(2, prob.M, synth.CFG_TEST, 7)
    want = osolve.solve(prob, b)
    out = {}
    for mode in ("f64", "df64"):
        plan = _plan(case, "mixed", max_nrhs=2)
        plan.set_residual_precision(mode)
        out[mode] = plan.solve(torch.from_numpy(b).cuda()).cpu().numpy()
        assert _rel(out[mode], want) <= 1e-10, (mode, _rel(out[mode], want))
        assert _relmax(out[mode], want) <= 1e-10
    assert _rel(out["df64"], out["f64"]) <= 1e-11
    assert _relmax(out["df64"], out["f64"]) <= 1e-11


@pytest.mark.parametrize("case", [dict(n=3, K=(8, 12), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0),
                                  dict(n=2, K=(8, 6, 8), a=(1.0, 2.0, 0.5), c=0.3)], ids=["2d", "3d"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_mass_apply_and_heat_steps(case, precision, tol):
    """The mass operator and five implicit Euler steps of C u' + L u = b
    against the oracle's heat step."""
    from paper_1701_03967_gb300 import HeatStepper
    prob = _prob(case)
    u0 = synth.normal_batch(2, prob.M, synth.CFG_TEST, 21)
    b = synth.normal_batch(2, prob.M, synth.CFG_TEST, 22)
    tau = 0.02
    st = HeatStepper(case["n"], case["K"], case.get("X"), case.get("a"), case.get("c", 0.0), tau, precision,
                     max_nrhs=2)
    ut, bt = torch.from_numpy(u0).cuda(), torch.from_numpy(b).cuda()
    assert _rel(st.plan.apply_mass(ut).cpu().numpy(), osolve.mass_apply(prob, u0)) <= 1e-13
    assert _relmax(st.plan.apply_mass(ut).cpu().numpy(), osolve.mass_apply(prob, u0)) <= 1e-13
    want = u0
    for _ in range(5):
        ut = st.step(ut, bt)
        want = osolve.heat_step(prob, want, b, tau)
    assert _rel(ut.cpu().numpy(), want) <= tol
    assert _relmax(ut.cpu().numpy(), want) <= tol
    st.close()


@pytest.mark.parametrize("case", [dict(n=9, K=(16, 32), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0),
                                  dict(n=4, K=(8, 12, 8), a=(1.0, 2.0, 0.5), c=0.3)], ids=["2d_n9", "3d_n4"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_tuned_plan_matches_oracle(case, precision, tol):
    """fem_fft_plan_tune changes only launch shapes: the tuned plan still
    matches the oracle."""
    prob = _prob(case)
    b = synth.normal_batch(2, prob.M, synth.CFG_TEST, 31)
    plan = _plan(case, precision, max_nrhs=2)
    plan.tune()
    got = plan.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(got, osolve.solve(prob, b)) <= tol
    assert _relmax(got, osolve.solve(prob, b)) <= tol


ALGO_B_CASES = [dict(n=9, K=(16, 32), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0),
                dict(n=4, K=(8, 12, 8), a=(1.0, 2.0, 0.5), c=0.3),
                dict(n=1, K=(8, 8)),
                dict(n=2, K=(6, 24), X=(2.0, 1.0), a=(1.5, 0.7), c=-1.0),
                dict(n=7, K=(12, 4, 6), c=2.0)]


@pytest.mark.parametrize("case", ALGO_B_CASES, ids=[f"n{c['n']}_{len(c['K'])}d" for c in ALGO_B_CASES])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_algorithm_b_matches_oracle(case, precision, tol):
    """Algorithm (b) (transforms along x_2..x_N, band solves along x_1)
    against the oracle's solution (algorithm (a), Theorem-1 basis at 40
    digits) at the path's bar, and against the oracle's literal algorithm (b)
    at 1e-11: that route's float64 banded Cholesky is itself only accurate to
    a few 1e-12 at n = 9 (Section 5 reports algorithm (b) stable to about
    1e-11); the GPU's vertex solve avoids the cancellation and is not."""
    prob = _prob(case)
    b = synth.normal_batch(2, prob.M, synth.CFG_TEST, 41)
    plan = _plan(case, precision, max_nrhs=2)
    plan.set_algorithm("b")
    got = plan.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(got, osolve.solve(prob, b)) <= tol
    assert _relmax(got, osolve.solve(prob, b)) <= tol
    assert _rel(got, osolve.solve_b(prob, b)) <= max(tol, 1e-11)
    assert _relmax(got, osolve.solve_b(prob, b)) <= max(tol, 1e-11)
    # new coefficients rebuild the band tables
    a2 = tuple(1.3 * x for x in (case.get("a") or (1.0,) * len(case["K"])))
    plan.set_coefficients(a2, 0.5)
    prob2 = osolve.Problem(case["n"], case["K"], case.get("X"), a2, 0.5)
    got2 = plan.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    assert _rel(got2, osolve.solve(prob2, b)) <= tol
    assert _relmax(got2, osolve.solve(prob2, b)) <= tol


def test_algorithm_b_needs_two_axes():
    from paper_1701_03967_gb300 import FemFftError
    with pytest.raises(FemFftError):
        _plan(dict(n=2, K=(8,)), "fp64").set_algorithm("b")

def test_long_pencil_transforms_and_the_shared_memory_limit():
    """The largest float64 pencil of n = 5 that one CTA holds (K = 2048): the
    direct transform expands calC^-1 y (Theorem 2), so inverse(forward(calC
    y)) = y to float64 rounding, for a batch of pencils with a ragged count.
    One size further (K = 3072) the pencil takes the global four-step path
    with the same result, contiguous (1D) or strided (axis 0 of a 2D
    field)."""
    g = torch.Generator(device="cuda").manual_seed(5)
    for K in (2048, 3072):
        pl = _plan(dict(n=5, K=(K,)), "fp64", max_nrhs=37)
        y = torch.randn(37, pl.M[0], dtype=torch.float64, device="cuda", generator=g)
        w = pl.inverse(pl.forward(pl.apply_mass(y)))
        assert float(torch.linalg.vector_norm(w - y) / torch.linalg.vector_norm(y)) <= 1e-12, K
        pl.close()
    big = _plan(dict(n=5, K=(3072, 2)), "fp64", max_nrhs=3)
    y = torch.randn((3,) + tuple(big.M), dtype=torch.float64, device="cuda", generator=g)
    w = big.inverse(big.forward(big.apply_mass(y)))
    assert float(torch.linalg.vector_norm(w - y) / torch.linalg.vector_norm(y)) <= 1e-12
    big.close()


def test_float64_divide_matches_cuda_division():
    """The float64 passes divide by the spectral denominators with a float
    reciprocal seed and two Newton steps (Section 4, algorithm (a)); against
    CUDA's float64 division over divisors spanning the float range (both
    signs) and numerators over 40 decades: within 4 ulp of the quotient."""
    from paper_1701_03967_gb300 import _lib
    rng = np.random.default_rng(11)
    n = 1 << 20
    x = rng.standard_normal(n) * 10.0 ** rng.uniform(-20, 20, n)
    d = np.where(rng.random(n) < 0.5, -1.0, 1.0) * 10.0 ** rng.uniform(-35, 35, n)
    xt, dt = torch.from_numpy(x).cuda(), torch.from_numpy(d).cuda()
    q, ref = torch.empty_like(xt), torch.empty_like(xt)
    _lib.check(_lib.lib().fem_fft_divide_check(xt.data_ptr(), dt.data_ptr(), q.data_ptr(), ref.data_ptr(), n, None),
               "fem_fft_divide_check")
    q, ref = q.cpu().numpy(), ref.cpu().numpy()
    assert np.array_equal(ref, x / d)     # CUDA's division: the correctly rounded quotient
    assert np.max(np.abs(q - ref) / np.abs(ref)) <= 4 * 2.0 ** -53
