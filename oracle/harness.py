"""Load vectors, manufactured solutions and error norms (test infrastructure).

* Section 5, item 2: the right-hand side f^h is computed with multiple Gauss
  quadrature formulas with n+1 nodes in each x_i.  With the scaled operator of
  Section 4 (stiffness 4 h^-2 calA, mass calC, both h-free), f^h is the
  Galerkin load vector multiplied by prod_i (2 / h_i); on each element this is
  sum_q w_q f(x_q) prod_i e_{l_i}(xi_{q,i}) with reference-element weights.
* Section 5, item 2: errors are measured in the mesh uniform norm, read here
  as the maximum over all FEM nodes (element vertices and element-interior
  nodes, i.e. every point of the fine grid).
"""

import numpy as np
import scipy.sparse
import sympy

from . import fem1d


def _lagrange_eval(n, xi):
    """Values e_q(xi_g) of the Lagrange basis on [-1, 1], shape (len(xi), n+1)."""
    nodes = -1.0 + 2.0 * np.arange(n + 1) / n
    B = np.ones((len(xi), n + 1))
    for q in range(n + 1):
        for m in range(n + 1):
            if m != q:
                B[:, q] *= (xi - nodes[m]) / (nodes[q] - nodes[m])
    return B


def _scatter_matrix(n, K, G, rowvals):
    """Sparse map from per-element per-quadrature-point data (K*G) to global
    DOF (M); rowvals[g, q] is the weight of point g for local node q."""
    M = fem1d.dof_count(n, K)
    rows, cols, vals = [], [], []
    for e in range(K):
        for q in range(n + 1):
            gq = fem1d.local_to_global(n, K, e, q)
            if gq is None:
                continue
            for g in range(G):
                rows.append(gq)
                cols.append(e * G + g)
                vals.append(rowvals[g, q])
    return scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(M, K * G))


def _apply_axes(x, mats):
    for ax, mat in enumerate(mats):
        x = np.moveaxis(x, ax, -1)
        x = (mat @ x.reshape(-1, x.shape[-1]).T).T.reshape(x.shape[:-1] + (mat.shape[0],))
        x = np.moveaxis(x, -1, ax)
    return x


def quad_points(n, K, X, G):
    xi, w = np.polynomial.legendre.leggauss(G)
    h = X / K
    pts = (np.arange(K)[:, None] * h + (xi[None, :] + 1.0) * h / 2.0).reshape(-1)
    return xi, w, pts


def load_vector(prob, f):
    """f^h for a callable f(x_1, ..., x_N) (vectorised over numpy arrays),
    (n_i+1)-point Gauss per axis per element (Section 5)."""
    mats, grids = [], []
    for i in range(prob.N):
        n = prob.ns[i]
        G = n + 1
        xi, w, pts = quad_points(n, prob.K[i], prob.X[i], G)
        B = _lagrange_eval(n, xi)
        mats.append(_scatter_matrix(n, prob.K[i], G, w[:, None] * B))
        grids.append(pts)
    mesh = np.meshgrid(*grids, indexing="ij")
    F = f(*mesh)
    return _apply_axes(F, mats)


def fine_grid(prob, i):
    """Coordinates of the M_i fine-grid nodes along axis i (x = m h / n)."""
    return np.arange(1, prob.M[i] + 1) * prob.h[i] / prob.ns[i]


def nodal_values(prob, u):
    mesh = np.meshgrid(*[fine_grid(prob, i) for i in range(prob.N)], indexing="ij")
    return u(*mesh)


def max_error(prob, uh, u):
    """Mesh uniform-norm error: max over all FEM nodes (Section 5)."""
    return float(np.max(np.abs(uh - nodal_values(prob, u))))


def l2_error(prob, uh, u):
    """L2(Omega) error of the FEM function with nodal values uh, by
    (n_i+2)-point Gauss per axis per element."""
    mats, grids, wts = [], [], []
    for i in range(prob.N):
        n = prob.ns[i]
        G = n + 2
        xi, w, pts = quad_points(n, prob.K[i], prob.X[i], G)
        B = _lagrange_eval(n, xi)
        mats.append(_scatter_matrix(n, prob.K[i], G, B).T.tocsr())
        grids.append(pts)
        wts.append(np.tile(w * prob.h[i] / 2.0, prob.K[i]))
    uq = _apply_axes(uh, mats)
    mesh = np.meshgrid(*grids, indexing="ij")
    W = wts[0]
    for wi in wts[1:]:
        W = np.multiply.outer(W, wi)
    return float(np.sqrt(np.sum(W * (uq - u(*mesh)) ** 2)))


# --------------------------------------------------------------------------
# Manufactured solutions
# --------------------------------------------------------------------------

def manufactured(expr_str, N, a, c):
    """(u, f) callables for u given as a sympy expression in x1..xN and
    f = -sum_i a_i u_{x_i x_i} + c u."""
    xs = sympy.symbols(" ".join(f"x{i + 1}" for i in range(N)))
    if N == 1:
        xs = (xs,)
    u = sympy.sympify(expr_str, locals={f"x{i + 1}": xs[i] for i in range(N)})
    f = -sum(sympy.Float(a[i]) * sympy.diff(u, xs[i], 2) for i in range(N)) + sympy.Float(c) * u
    return (sympy.lambdify(xs, u, "numpy"), sympy.lambdify(xs, sympy.simplify(f), "numpy"))


# Section 5 test solutions (alpha = 1, X_i = 1)
PAPER_2D = "sin(2*pi*x1)*sin(3*pi*x2)*cosh(sqrt(2)*x1 - x2)"
PAPER_3D = "sin(2*pi*x1)*sin(3*pi*x2)*sin(4*pi*x3)*cosh(sqrt(2)*x1 - x2 + x3/sqrt(3))"
