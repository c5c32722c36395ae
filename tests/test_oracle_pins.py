"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test compares the oracle with something other than itself: closed forms
printed in the paper or textbook finite-element matrices, structural facts of
Section 3 (Theorem 1), a brute-force dense solve, the error tables of
Section 5, FEM convergence theory and finite differences.  The last group
plants plausible mistakes in a copy of the oracle and checks that a pin fails.
"""

import json
import math
import os
from fractions import Fraction

import numpy as np
import scipy.linalg
import pytest

from oracle import fem1d, harness, solve
from paper_1701_03967_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Section 2

def test_reference_matrices_textbook_linear_and_quadratic():
    # n=1: linear Lagrange element of length 2
    A, C = fem1d.reference_matrices_exact(1)
    assert A == [[Fraction(1, 2), Fraction(-1, 2)], [Fraction(-1, 2), Fraction(1, 2)]]
    assert C == [[Fraction(2, 3), Fraction(1, 3)], [Fraction(1, 3), Fraction(2, 3)]]
    # n=2: quadratic element of length L=2: stiffness 1/(3L)[[7,-8,1],...],
    # mass L/30 [[4,2,-1],[2,16,2],[-1,2,4]]
    A, C = fem1d.reference_matrices_exact(2)
    assert A == [[Fraction(v, 6) for v in r] for r in ([7, -8, 1], [-8, 16, -8], [1, -8, 7])]
    assert C == [[Fraction(v, 15) for v in r] for r in ([4, 2, -1], [2, 16, 2], [-1, 2, 4])]


@pytest.mark.parametrize("n", range(1, 10))
def test_reference_matrix_invariants(n):
    A, C = fem1d.reference_matrices_exact(n)
    # A (1..1)^T = 0 (Section 2, proof of Lemma 1); sum of C = |[-1,1]| = 2
    assert all(sum(row) == 0 for row in A)
    assert sum(sum(row) for row in C) == 2
    # bisymmetric (Section 2)
    for k in range(n + 1):
        for l in range(n + 1):
            assert A[k][l] == A[l][k] == A[n - k][n - l]
            assert C[k][l] == C[l][k] == C[n - k][n - l]


def test_interior_spectra_closed_forms():
    spec = json.load(open(os.path.join(GOLDEN, "interior_spectra.json")))["S~"]
    for n_str, vals in spec.items():
        want = sorted(eval(v, {"sqrt": math.sqrt}) for v in vals)
        got, _ = fem1d.interior_element_eig(int(n_str))
        np.testing.assert_allclose(got, want, rtol=1e-13)


@pytest.mark.parametrize("n", range(2, 10))
def test_element_eigvecs_even_or_odd_and_assumption_A(n):
    lam0, E = fem1d.interior_element_eig(n)
    for l in range(n - 1):
        e = E[:, l]
        # Section 2, Lemma 1 / Section 3: each e^(l) is even or odd, even for odd
        # l (1-based) when the eigenvalues are ascending
        sign = 1.0 if l % 2 == 0 else -1.0
        np.testing.assert_allclose(fem1d.flip(e), sign * e, atol=1e-12 * np.abs(e).max())
    # the single zero eigenvalue of A e = lambda C e (Section 2, Lemma 1, item 2)
    A, C = fem1d.reference_matrices(n)
    import scipy.linalg
    Sn = scipy.linalg.eigh(A, C, eigvals_only=True)
    assert abs(Sn[0]) < 1e-13 * Sn[-1]


@pytest.mark.parametrize("n", range(2, 10))
def test_assumption_A_exact(n):
    """Assumption (A) of Section 3 (spectra simple, S_n and S~_n disjoint),
    decided exactly over the rationals: the characteristic polynomials
    det(A - lambda C) and det(A~ - lambda C~) are squarefree and coprime.
    (In floating point this cannot be decided for n = 9: the two spectra come
    within 5e-13 of each other near pi^2/4.)"""
    import sympy
    Aex, Cex = fem1d.reference_matrices_exact(n)
    lam = sympy.Symbol("lam")

    def charpoly(idx):
        pts = list(range(len(idx) + 1))
        vals = []
        for x in pts:
            Mx = sympy.Matrix([[sympy.Rational(Aex[i][j].numerator, Aex[i][j].denominator)
                                - x * sympy.Rational(Cex[i][j].numerator, Cex[i][j].denominator)
                                for j in idx] for i in idx])
            vals.append(Mx.det())
        return sympy.Poly(sympy.interpolate(list(zip(pts, vals)), lam), lam)

    pS = charpoly(list(range(n + 1)))
    pT = charpoly(list(range(1, n)))
    assert sympy.degree(sympy.gcd(pS, pT), lam) == 0
    assert sympy.degree(sympy.gcd(pS, pS.diff(lam)), lam) == 0
    if n > 2:
        assert sympy.degree(sympy.gcd(pT, pT.diff(lam)), lam) == 0


# ----------------------------------------------------------------- Section 3

@pytest.mark.parametrize("n,K", [(1, 7), (2, 6), (3, 5), (4, 6), (5, 4), (9, 4)])
def test_spectrum_is_S_tilde_union_dispersion_roots(n, K):
    """Theorem 1, item 1, checked against LAPACK's dense generalized eigh."""
    lam_dense, V = fem1d.eig(n, K)
    lam_thm, S, cn = fem1d.theorem1_basis(n, K)
    np.testing.assert_allclose(np.sort(lam_thm), lam_dense, rtol=1e-10)
    # V^T calC V = I from the library routine (C-orthonormality)
    _, calC = fem1d.assemble(n, K)
    np.testing.assert_allclose(V.T @ calC @ V, np.eye(len(lam_dense)), atol=1e-10)


def test_n1_closed_form_eigenvalues():
    """n=1: the global matrices are (1/2)tridiag(-1,2,-1) and (1/3)tridiag(1,4,1),
    so lambda_k = 3(1 - theta_k) / (2 (2 + theta_k))."""
    K = 12
    lam, S, cn = fem1d.theorem1_basis(1, K)
    th = np.cos(np.pi * np.arange(1, K) / K)
    np.testing.assert_allclose(lam, 3 * (1 - th) / (2 * (2 + th)), rtol=1e-14)
    np.testing.assert_allclose(np.sort(fem1d.eig(1, K)[0]), np.sort(lam), rtol=1e-12)


@pytest.mark.parametrize("n,K", [(2, 8), (3, 6), (5, 8), (9, 6)])
def test_theorem1_eigenpairs_orthogonality_and_norms(n, K):
    lam, S, cn = fem1d.theorem1_basis(n, K)
    calA, calC = fem1d.assemble(n, K)
    # A s = lambda C s for every column (Theorem 1, items 2, 3)
    R = calA @ S - (calC @ S) * lam[None, :]
    assert np.max(np.abs(R)) / np.max(np.abs(calA @ S)) < 1e-12
    # C-orthogonality (Theorem 1, item 4)
    G = S.T @ calC @ S
    off = G - np.diag(np.diag(G))
    assert np.max(np.abs(off)) < 1e-11 * np.max(np.abs(np.diag(G)))
    # ||s_0^(l)||_C^2 = K (Theorem 2, item 2); nodes of s_k: (s_k, s_k) = K/2
    np.testing.assert_allclose(cn[: n - 1], K, rtol=1e-12)
    nodes = np.arange(n - 1, fem1d.dof_count(n, K), n)
    np.testing.assert_allclose(np.sum(S[nodes, n - 1:] ** 2, axis=0), K / 2, rtol=1e-12)


@pytest.mark.parametrize("n,K", [(3, 6), (4, 5), (6, 4)])
def test_norm_formula_of_theorem2(n, K):
    """||s_k||_C^2 = K{c0 + (C~p + 2c).p + theta_k [cn + (C~p + 2c).flip(p)]}
    (Theorem 2, item 2) against the dense s^T calC s."""
    lam, S, cn = fem1d.theorem1_basis(n, K)
    bA, bC = fem1d.element_blocks(n)
    for k in range(1, K):
        th = math.cos(math.pi * k / K)
        for l in range(n):
            col = n - 1 + (k - 1) * n + l
            # recover p from the interiors of element 1: p*0 + flip(p)*sin(pi k/K)
            p = fem1d.flip(S[0:n - 1, col]) / np.sin(np.pi * k / K)
            q = bC["bt"] @ p + 2 * bC["b"]
            want = K * (bC["b0"] + q @ p + th * (bC["bn"] + q @ fem1d.flip(p)))
            assert abs(want - cn[col]) < 1e-10 * abs(cn[col])


# ----------------------------------------------------------------- Section 4

CASES = [
    dict(n=3, K=(9,), X=(1.7,), a=(0.8,), c=0.4),
    dict(n=2, K=(4, 6), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0),
    dict(n=4, K=(3, 4), X=(0.5, 1.5), a=(3.0, 0.7), c=-2.0),
    dict(n=1, K=(5, 7), X=(1.0, 1.0), a=(1.0, 1.0), c=0.0),
    dict(n=2, K=(3, 3, 4), X=(1.0, 1.2, 0.9), a=(1.0, 2.0, 0.5), c=0.3),
    dict(n=3, K=(2, 3, 2), X=(1.0, 1.0, 1.0), a=(1.0, 1.0, 1.0), c=0.0),
    # per-axis orders n_i (Section 4)
    dict(n=(3, 7), K=(4, 3), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0),
    dict(n=(2, 5, 9), K=(3, 2, 2), X=(1.0, 0.7, 1.2), a=(0.8, 1.3, 2.0), c=0.2),
    dict(n=(1, 4), K=(6, 3), X=(1.5, 1.0), a=(1.0, 1.0), c=-1.0),
]


@pytest.mark.parametrize("case", CASES)
def test_solve_matches_brute_force_dense_solve(case):
    p = solve.Problem(case["n"], case["K"], case["X"], case["a"], case["c"])
    b = synth.normal_batch(2, p.M, synth.CFG_TEST, 7)
    L = solve.assemble_dense(p)
    want = np.linalg.solve(L, b.reshape(2, -1).T).T.reshape(b.shape)
    got = solve.solve(p, b)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12
    # apply = L u
    np.testing.assert_allclose(solve.apply(p, want).reshape(2, -1),
                               (L @ want.reshape(2, -1).T).T, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("case", CASES[:5])
def test_heat_step_matches_dense_implicit_euler(case):
    """One implicit Euler step of C u' + L u = b (C the N-D mass operator):
    (C + tau L) u_new = C u + tau b, against dense Kronecker products of the
    assembled 1D matrices and a dense solve."""
    p = solve.Problem(case["n"], case["K"], case["X"], case["a"], case["c"])
    u = synth.normal_batch(2, p.M, synth.CFG_TEST, 11)
    b = synth.normal_batch(2, p.M, synth.CFG_TEST, 12)
    tau = 0.013
    C = np.ones((1, 1))
    for i in range(p.N):
        C = np.kron(C, fem1d.assemble(p.ns[i], p.K[i])[1])
    L = solve.assemble_dense(p)
    rhs = (C @ u.reshape(2, -1).T + tau * b.reshape(2, -1).T)
    want = np.linalg.solve(C + tau * L, rhs).T.reshape(u.shape)
    got = solve.heat_step(p, u, b, tau)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12
    np.testing.assert_allclose(solve.mass_apply(p, u).reshape(2, -1), (C @ u.reshape(2, -1).T).T,
                               rtol=1e-12, atol=1e-13)


def test_heat_step_decays_eigenmodes_exactly():
    """A product of 1D generalized eigenvectors (calA v = lambda calC v, from
    LAPACK) decays in one step with b = 0 by exactly
    1 / (1 + tau (sum_i a_i 4 h_i^-2 lambda_i + c))."""
    p = solve.Problem(3, (5, 4), (1.0, 2.0), (1.3, 0.6), 0.7)
    tau = 0.05
    vecs, lams = [], []
    for i, pick in enumerate((2, 7)):
        calA, calC = fem1d.assemble(p.ns[i], p.K[i])
        w, V = scipy.linalg.eigh(calA, calC)
        vecs.append(V[:, pick])
        lams.append(w[pick])
    u = np.multiply.outer(vecs[0], vecs[1])
    got = solve.heat_step(p, u, np.zeros_like(u), tau)
    factor = 1.0 / (1.0 + tau * (sum(p.a[i] * p.s[i] * lams[i] for i in range(2)) + p.c))
    np.testing.assert_allclose(got, factor * u, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("case", [c for c in CASES if len(c["K"]) > 1])
def test_algorithm_b_matches_brute_force_dense_solve(case):
    """Algorithm (b) (transforms in x_2..x_N, banded Cholesky in x_1) solves
    the same assembled system as the dense solve."""
    p = solve.Problem(case["n"], case["K"], case["X"], case["a"], case["c"])
    b = synth.normal_batch(2, p.M, synth.CFG_TEST, 13)
    L = solve.assemble_dense(p)
    want = np.linalg.solve(L, b.reshape(2, -1).T).T.reshape(b.shape)
    got = solve.solve_b(p, b)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12


def test_paper_error_tables():
    """Section 5 error tables (algorithm (a)) for K <= 32 (2D) and K <= 8 (3D):
    entries above the round-off floor agree to the two printed digits; below
    it the oracle stays at the FP64 round-off level."""
    T = json.load(open(os.path.join(GOLDEN, "paper_error_tables.json")))
    checks = [("2d", 2, harness.PAPER_2D, ks) for ks in ("2", "4", "8", "16", "32")]
    checks += [("3d", 3, harness.PAPER_3D, ks) for ks in ("2", "4", "8")]
    for key, N, expr, ks in checks:
        u, f = harness.manufactured(expr, N, (1,) * N, 1.0)
        for n in range(1, 10):
            p = solve.Problem(n, (int(ks),) * N, None, None, 1.0)
            err = harness.max_error(p, solve.solve(p, harness.load_vector(p, f)), u)
            paper = T[key][ks][n - 1]
            if paper >= 5e-14:
                assert abs(err / paper - 1) < 0.06, (key, ks, n, err, paper)
            else:
                assert err < 5e-14, (key, ks, n, err, paper)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_l2_convergence_order(n):
    """FEM theory: L2 error O(h^{n+1}) for the manufactured u = sin(pi x)sin(2 pi y)."""
    u, f = harness.manufactured("sin(pi*x1)*sin(2*pi*x2)", 2, (1, 1), 0.0)
    errs = []
    for K in (8, 16):
        p = solve.Problem(n, (K, K), None, None, 0.0)
        errs.append(harness.l2_error(p, solve.solve(p, harness.load_vector(p, f)), u))
    rate = errs[0] / errs[1]
    assert 0.8 * 2 ** (n + 1) < rate < 1.25 * 2 ** (n + 1), (n, errs, rate)


def test_gradients_against_central_differences():
    p0 = dict(n=2, K=(4, 3), X=(1.0, 1.3), a=(1.2, 0.7), c=0.5)
    prob = solve.Problem(**p0)
    f = synth.normal_field(prob.M, synth.CFG_TEST, 11)
    ut = synth.normal_field(prob.M, synth.CFG_TEST, 12)

    def loss(a, c, ff):
        q = solve.Problem(p0["n"], p0["K"], p0["X"], a, c)
        return float(np.sum((solve.solve(q, ff) - ut) ** 2))

    u = solve.solve(prob, f)
    gf, ga, gc = solve.grad(prob, f, 2 * (u - ut))
    h = 1e-6
    for i in range(2):
        ap, am = list(p0["a"]), list(p0["a"])
        ap[i] += h
        am[i] -= h
        fd = (loss(ap, p0["c"], f) - loss(am, p0["c"], f)) / (2 * h)
        assert abs(fd - ga[i]) < 1e-6 * max(1.0, abs(fd))
    fd = (loss(p0["a"], p0["c"] + h, f) - loss(p0["a"], p0["c"] - h, f)) / (2 * h)
    assert abs(fd - gc) < 1e-6 * max(1.0, abs(fd))
    for idx in [(0, 0), (3, 2), (5, 4)]:
        e = np.zeros(prob.M)
        e[idx] = h
        fd = (loss(p0["a"], p0["c"], f + e) - loss(p0["a"], p0["c"], f - e)) / (2 * h)
        assert abs(fd - gf[idx]) < 1e-6 * max(1.0, abs(fd))


# ------------------------------------------------- planted mistakes (CPU only)

def _brute_force_error(monkeypatch_fn):
    case = CASES[1]
    p = solve.Problem(case["n"], case["K"], case["X"], case["a"], case["c"])
    b = synth.normal_field(p.M, synth.CFG_TEST, 3)
    want = np.linalg.solve(solve.assemble_dense(p), b.ravel()).reshape(p.M)
    return np.linalg.norm(solve.solve(p, b) - want) / np.linalg.norm(want)


def test_planted_mistakes_are_caught(monkeypatch):
    assert _brute_force_error(None) < 1e-12
    # 1. the zeroth-order term dropped from the denominators
    orig_den = solve.Problem.denominators
    monkeypatch.setattr(solve.Problem, "denominators",
                        lambda self: orig_den(self) - self.c)
    assert _brute_force_error(None) > 1e-6
    monkeypatch.setattr(solve.Problem, "denominators", orig_den)
    # 2. the forward expansion transposed
    orig_fwd = solve.forward_coefficients

    def fwd_T(prob, y):
        x, single = solve._as_batch(prob, y)
        for i in range(prob.N):
            _, S, cn = prob.basis1d(i)
            x = solve._axis_apply(x, S / cn[None, :], i + 1)
        return x[0] if single else x
    monkeypatch.setattr(solve, "forward_coefficients", fwd_T)
    assert _brute_force_error(None) > 1e-6
    monkeypatch.setattr(solve, "forward_coefficients", orig_fwd)
    # 3. the sign of theta flipped in the dispersion relation -> wrong spectrum
    lam_dense, _ = fem1d.eig(3, 5)
    orig_roots = fem1d.dispersion_roots
    monkeypatch.setattr(fem1d, "dispersion_roots",
                        lambda n, theta, dps=40: orig_roots(n, -theta, dps))
    solve._BASIS.clear()
    lam_bad, S_bad, _ = fem1d.theorem1_basis(3, 5)
    # flipping theta maps the roots of k to those of K-k: the set of
    # eigenvalues is unchanged, but the vectors no longer match them
    np.testing.assert_allclose(np.sort(lam_bad), lam_dense, rtol=1e-10)
    calA, calC = fem1d.assemble(3, 5)
    R = calA @ S_bad - (calC @ S_bad) * lam_bad[None, :]
    assert np.max(np.abs(R)) > 1e-3
    monkeypatch.setattr(fem1d, "dispersion_roots", orig_roots)
    solve._BASIS.clear()


def test_full_assembly_structure():
    """The operators with the boundary nodes kept: their interior block is the
    Dirichlet operator, the stiffness annihilates constants (the constant
    function lies in the full space and has zero derivative) and the mass
    entries sum to the measure of (0, K) in reference units, 2K."""
    for n, K in [(1, 3), (2, 4), (5, 3)]:
        fA, fC = fem1d.assemble_full(n, K)
        A, C = fem1d.assemble(n, K)
        assert np.allclose(fA[1:-1, 1:-1], A, atol=1e-14) and np.allclose(fC[1:-1, 1:-1], C, atol=1e-14)
        assert np.max(np.abs(fA.sum(axis=1))) < 1e-12
        assert abs(fC.sum() - 2.0 * K) < 1e-12


DIRICHLET_CASES = [dict(n=2, K=(3, 4), X=(1.0, 1.5), a=(1.3, 0.7), c=0.4),
                   dict(n=3, K=(2, 3, 2), X=(1.0, 0.8, 1.2), a=(0.9, 1.1, 2.0), c=0.0),
                   dict(n=4, K=(5,), X=(2.0,), a=(2.0,), c=1.5),
                   dict(n=(2, 5), K=(3, 2), X=(1.0, 1.5), a=(1.3, 0.7), c=0.4),
                   dict(n=(4, 1, 3), K=(2, 4, 2), X=(1.0, 0.8, 1.2), a=(0.9, 1.1, 2.0), c=0.3)]


@pytest.mark.parametrize("case", DIRICHLET_CASES,
                         ids=[f"n{'_'.join(map(str, np.atleast_1d(c['n'])))}_{len(c['K'])}d" for c in DIRICHLET_CASES])
def test_dirichlet_data_reproduce_polynomials(case):
    """Section 4 with non-zero boundary values: when the exact solution is a
    polynomial of degree <= n_i in variable i it lies in the FEM space, so
    the Galerkin solution equals it; the load vector of its right-hand side
    -sum a_i u_ii + c u is exact with (n+1)-point Gauss (Section 5).  So the
    solve with the boundary correction must return u at every interior node,
    whatever the coefficients; a dropped term, a wrong sign or a wrong
    coupling in the correction breaks the equality."""
    N = len(case["K"])
    prob = solve.Problem(case["n"], case["K"], case["X"], case["a"], case["c"])
    ns = prob.ns
    rng = np.random.default_rng(11)
    P = [np.polynomial.Polynomial(rng.uniform(-1, 1, ns[i] + 1)) for i in range(N)]
    Qp = [np.polynomial.Polynomial(rng.uniform(-1, 1, ns[i] + 1)) for i in range(N)]

    def u(*x):
        prod = np.ones_like(x[0])
        for i in range(N):
            prod = prod * P[i](x[i])
        return prod + sum(Qp[i](x[i]) for i in range(N))

    def f(*x):
        out = prob.c * u(*x)
        for i in range(N):
            t = P[i].deriv(2)(x[i])
            for j in range(N):
                if j != i:
                    t = t * P[j](x[j])
            out = out - prob.a[i] * (t + Qp[i].deriv(2)(x[i]))
        return out

    b = harness.load_vector(prob, f)
    ext_grid = [np.arange(prob.M[i] + 2) * prob.h[i] / ns[i] for i in range(N)]
    g = u(*np.meshgrid(*ext_grid, indexing="ij"))
    got = solve.solve_dirichlet(prob, b, g)
    want = harness.nodal_values(prob, u)
    assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want))
    # without the correction the boundary values are lost
    assert np.max(np.abs(solve.solve(prob, b) - want)) > 1e-3 * np.max(np.abs(want))


def test_basis_node_values_exact_at_long_pencils():
    """Theorem 1, item 3: the node values of s_k^(l) are sin(pi k j / K).
    At the long pencils of Section 5 (pi k j / K up to ~10^4) the oracle's
    basis must keep them to float64 rounding (exact argument reduction),
    checked against 40-digit values; and its interior values against the
    formula p sin(pi k (j-1)/K) + p^ sin(pi k j / K) at 40 digits."""
    import mpmath as mp
    mp.mp.dps = 40
    n, K = 2, 4096
    lam, S, cn = fem1d.theorem1_basis(n, K)
    rng = np.random.default_rng(3)
    # columns of S: bubble modes first, then k = 1..K-1 with n modes each
    for col in rng.choice(np.arange(n - 1, S.shape[1]), 12, replace=False):
        k = (col + 1) // n
        for j in rng.choice(np.arange(1, K), 12, replace=False):
            node = n * j - 1                     # fine index of node j
            want = float(mp.sin(mp.pi * k * j / K))
            assert abs(S[node, col] - want) <= 2e-15, (col, j)   # pi m / K reduced below 2 pi
        # interior of element j: p sin(pi k (j-1)/K) + p^ sin(pi k j/K), p = S[interior of element 1]
        p = S[0:n - 1, col] / max(1e-300, float(mp.sin(mp.pi * k / K)))   # element 1: p^ sin(pi k / K)
        for j in rng.choice(np.arange(1, K + 1), 6, replace=False):
            want = [float(p[n - 2 - i] * mp.sin(mp.pi * k * (j - 1) / K) + p[i] * mp.sin(mp.pi * k * j / K))
                    for i in range(n - 1)]
            got = S[n * (j - 1): n * (j - 1) + n - 1, col]
            assert np.max(np.abs(got - np.array(want)[::-1])) <= 1e-12 * max(1.0, np.max(np.abs(want)))
