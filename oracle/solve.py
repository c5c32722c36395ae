"""N-D solve, apply and gradients of the oracle (test infrastructure only).

Problem (Section 4, the N-dimensional boundary value problem and its FEM form,
generalised to per-axis coefficients a_i and a zeroth-order coefficient c):

    L = sum_i a_i (4 / h_i^2) calA_i (x) prod_{j != i} calC_j  +  c prod_j calC_j,
    h_i = X_i / K_i,   L u = b,

with b the "FEM average" right-hand side f^h and all fields stored as C-order
arrays [M_1, ..., M_N] (axis N fastest), M_i = n K_i - 1, in the fine-grid
ordering of ``fem1d``.

Solve (Section 4, algorithm (a)): the coefficients of b in the expansion in
products of calC_i s_i (the direct FC_n-expansion of Section 3 on every axis,
y_kl = (y, s_k^(l)) / ||s_k^(l)||_C^2), divided by
sum_i a_i 4 h_i^-2 lambda_i + c, then the expansion in products of s_i (the
inverse F_n-expansion).  The oracle forms the 1D eigenbasis of Theorem 1
densely (``fem1d.theorem1_basis``) and applies it by plain matrix products
along each axis -- no FFT and no fast transform formulas.
"""

import numpy as np

from . import fem1d


class Problem:
    """Static description of one problem: N axes with K_i elements of order
    n_i (Section 4 allows a different order per axis; ``n`` is one int for
    all axes or one per axis), lengths X_i, coefficients a_i and c.
    ``self.n`` is the common order (None when the orders differ),
    ``self.ns`` the per-axis orders."""

    def __init__(self, n, K, X=None, a=None, c=0.0):
        self.K = tuple(int(k) for k in K)
        self.N = len(self.K)
        if np.ndim(n) == 0:
            self.ns = (int(n),) * self.N
        else:
            self.ns = tuple(int(x) for x in n)
            if len(self.ns) != self.N:
                raise ValueError("one order per axis")
        self.n = self.ns[0] if len(set(self.ns)) == 1 else None
        self.X = tuple(float(x) for x in (X if X is not None else [1.0] * self.N))
        self.a = tuple(float(x) for x in (a if a is not None else [1.0] * self.N))
        self.c = float(c)
        self.M = tuple(fem1d.dof_count(n_i, k) for n_i, k in zip(self.ns, self.K))
        self.h = tuple(x / k for x, k in zip(self.X, self.K))
        self.s = tuple(4.0 / (h * h) for h in self.h)       # 4 h_i^-2
        self._ops = {}
        self._basis = {}

    @property
    def dof(self):
        return int(np.prod(self.M))

    def basis1d(self, i):
        """(lam, S, cnorm2) of ``fem1d.theorem1_basis`` for axis i (cached per
        (n_i, K_i))."""
        key = (self.ns[i], self.K[i])
        if key not in self._basis:
            self._basis[key] = _basis_cache(self.ns[i], self.K[i])
        return self._basis[key]

    def ops1d(self, i):
        key = (self.ns[i], self.K[i])
        if key not in self._ops:
            self._ops[key] = fem1d.assemble(self.ns[i], self.K[i])
        return self._ops[key]

    def denominators(self):
        """D = sum_i a_i 4 h_i^-2 lambda_i (x) 1 + c over the N-D spectral grid
        (Section 4, algorithm (a), the solution expansion)."""
        D = np.full(self.M, self.c, dtype=np.float64)
        for i in range(self.N):
            lam, _, _ = self.basis1d(i)
            shape = [1] * self.N
            shape[i] = self.M[i]
            D = D + (self.a[i] * self.s[i] * lam).reshape(shape)
        return D


def _axis_apply(x, mat, axis):
    """y = x with matrix ``mat`` applied along ``axis`` (batched leading dim
    allowed): y[..., m, ...] = sum_j mat[m, j] x[..., j, ...]."""
    x = np.moveaxis(x, axis, -1)
    y = x @ mat.T
    return np.moveaxis(y, -1, axis)


def _as_batch(prob, x):
    x = np.asarray(x, dtype=np.float64)
    if x.shape == prob.M:
        return x[None], True
    assert x.shape[1:] == prob.M, (x.shape, prob.M)
    return x, False


_BASIS = {}


def _basis_cache(n, K):
    if (n, K) not in _BASIS:
        _BASIS[(n, K)] = fem1d.theorem1_basis(n, K)
    return _BASIS[(n, K)]


def forward_coefficients(prob, y):
    """Direct FC_n-expansion on every axis (Section 3, Theorem 2, item 2, the
    standard formula y_kl = (y, s_k^(l)) / ||s_k^(l)||_C^2; Section 4, the
    multiple expansion of f^h), by dense products with the Theorem-1 basis."""
    x, single = _as_batch(prob, y)
    for i in range(prob.N):
        _, S, cn = prob.basis1d(i)
        x = _axis_apply(x, S.T / cn[:, None], i + 1)
    return x[0] if single else x


def inverse_expansion(prob, w):
    """Inverse F_n-expansion on every axis: u = sum w_k s_k (Section 3, the
    expansion in eigenvectors), by dense products."""
    x, single = _as_batch(prob, w)
    for i in range(prob.N):
        _, S, _ = prob.basis1d(i)
        x = _axis_apply(x, S, i + 1)
    return x[0] if single else x


def solve(prob, b):
    """u = L^{-1} b by the dense eigenbasis route (Section 4, algorithm (a)).
    ``b`` has shape M or (nrhs,) + M."""
    bhat = forward_coefficients(prob, b)
    return inverse_expansion(prob, bhat / prob.denominators())


def apply(prob, u):
    """b = L u (Section 4, the operator form of the FEM system), by axis-wise
    products with the assembled 1D matrices."""
    x, single = _as_batch(prob, u)
    out = np.zeros_like(x)
    for i in range(prob.N + 1):
        t = x
        for j in range(prob.N):
            calA, calC = prob.ops1d(j)
            t = _axis_apply(t, calA if j == i else calC, j + 1)
        coef = prob.c if i == prob.N else prob.a[i] * prob.s[i]
        out += coef * t
    return out[0] if single else out


def assemble_dense(prob):
    """Full dense L (Kronecker products); for brute-force pins on tiny grids."""
    mats = [prob.ops1d(i) for i in range(prob.N)]
    L = None
    for i in range(prob.N + 1):
        T = np.ones((1, 1))
        for j in range(prob.N):
            T = np.kron(T, mats[j][0] if j == i else mats[j][1])
        coef = prob.c if i == prob.N else prob.a[i] * prob.s[i]
        L = coef * T if L is None else L + coef * T
    return L


def term_apply(prob, u, i):
    """T_i u with T_i = dL/da_i = 4 h_i^-2 calA_i (x) prod_{j!=i} calC_j for
    i < N, and T_N = dL/dc = prod_j calC_j."""
    x, single = _as_batch(prob, u)
    t = x
    for j in range(prob.N):
        calA, calC = prob.ops1d(j)
        t = _axis_apply(t, calA if j == i else calC, j + 1)
    coef = 1.0 if i == prob.N else prob.s[i]
    t = coef * t
    return t[0] if single else t


def solve_b(prob, b):
    """u = L^{-1} b by algorithm (b) of Section 4: the direct FC_n-expansion
    in x_2..x_N only, then for every spectral index (k_2 l_2, ..., k_N l_N)
    the 1D problem in x_1
        [a_1 4 h_1^-2 calA_1 + (sum_{i>=2} a_i 4 h_i^-2 lambda_i + c) calC_1] v = f~
    solved by banded Cholesky (its matrix is symmetric positive definite with
    half-bandwidth n), then the inverse F_n-expansion in x_2..x_N."""
    import scipy.linalg
    x, single = _as_batch(prob, b)
    for i in range(1, prob.N):
        _, S, cn = prob.basis1d(i)
        x = _axis_apply(x, S.T / cn[:, None], i + 1)
    # denominators of the later axes (the x_1 term is the banded solve)
    D = np.full(prob.M[1:], prob.c, dtype=np.float64)
    for i in range(1, prob.N):
        lam, _, _ = prob.basis1d(i)
        shape = [1] * (prob.N - 1)
        shape[i - 1] = prob.M[i]
        D = D + (prob.a[i] * prob.s[i] * lam).reshape(shape)
    calA, calC = prob.ops1d(0)
    n = prob.ns[0]
    alpha = prob.a[0] * prob.s[0]
    M0 = prob.M[0]
    y = np.moveaxis(x, 1, -1).reshape(-1, M0)          # (rhs x later spectral, M0)
    beta = np.broadcast_to(D, x.shape[:1] + D.shape).reshape(-1)
    out = np.empty_like(y)
    for r in range(y.shape[0]):
        Mat = alpha * calA + beta[r] * calC
        ab = np.zeros((n + 1, M0))                    # upper banded storage
        for d in range(n + 1):
            ab[n - d, d:] = np.diagonal(Mat, d)
        out[r] = scipy.linalg.solveh_banded(ab, y[r])
    v = np.moveaxis(out.reshape(x.shape[:1] + x.shape[2:] + (M0,)), -1, 1)
    for i in range(1, prob.N):
        _, S, _ = prob.basis1d(i)
        v = _axis_apply(v, S, i + 1)
    return v[0] if single else v


def dirichlet_rhs(prob, g):
    """d = (L_full G) restricted to the interior nodes, where G is the FEM
    function with the boundary values of ``g`` at the boundary nodes and 0
    inside, and L_full the operator of Section 4 on the space that keeps the
    boundary nodes (``fem1d.assemble_full`` on every axis).  ``g`` has shape
    (M_1+2, ..., M_N+2) or (nrhs,) + that (the fine grid extended by the
    boundary node at each end); only its boundary entries are used.  The
    solution with u = g on the boundary is u = L^{-1}(f^h - d) inside
    (the Dirichlet condition of Section 4 with non-zero data: u - G lies in
    the space with zero boundary values)."""
    x = np.array(g, dtype=np.float64)
    ext = tuple(m + 2 for m in prob.M)
    single = x.shape == ext
    if single:
        x = x[None]
    if x.shape[1:] != ext:
        raise ValueError(f"g has shape {x.shape}, expected {ext} or (nrhs,)+{ext}")
    inner = (slice(None),) + (slice(1, -1),) * prob.N
    x[inner] = 0.0
    full = [fem1d.assemble_full(n_i, k) for n_i, k in zip(prob.ns, prob.K)]
    out = np.zeros_like(x)
    for i in range(prob.N + 1):
        t = x
        for j in range(prob.N):
            fA, fC = full[j]
            t = _axis_apply(t, fA if j == i else fC, j + 1)
        coef = prob.c if i == prob.N else prob.a[i] * prob.s[i]
        out += coef * t
    d = out[inner]
    return d[0] if single else d


def solve_dirichlet(prob, b, g):
    """Interior values of the solution with the boundary values of ``g``:
    L^{-1} (b - dirichlet_rhs(prob, g))."""
    return solve(prob, np.asarray(b, dtype=np.float64) - dirichlet_rhs(prob, g))


def mass_apply(prob, u):
    """(prod_j calC_j) u: the mass operator of the N-D space (Section 2, the
    global 1D mass matrices, in tensor products as in Section 4), by
    axis-wise products with the assembled 1D matrices."""
    return term_apply(prob, u, prob.N)


def heat_step(prob, u, b, tau):
    """One implicit Euler step of the time-dependent problem C u' + L u = b,
    C = prod_j calC_j: (C + tau L) u_new = C u + tau b.  C + tau L has the form
    of L with a_i -> tau a_i and c -> 1 + tau c, so the step is a solve of that
    scaled problem (algorithm (a) with denominators 1 + tau (sum_i a_i 4 h_i^-2
    lambda_i + c))."""
    scaled = Problem(prob.ns, prob.K, prob.X, [tau * a for a in prob.a], 1.0 + tau * prob.c)
    return solve(scaled, mass_apply(prob, u) + tau * np.asarray(b, dtype=np.float64))


def grad(prob, f, gu):
    """Gradients of a scalar loss through u = L^{-1} f, given gu = dloss/du.

    L is symmetric, so dloss/df = L^{-1} gu =: lam, and since
    dL/da_i = T_i, dloss/da_i = -lam^T T_i u, dloss/dc = -lam^T T_N u
    (differentiating L u = f).  Sums run over all right-hand sides.
    Returns (grad_f, grad_a (N,), grad_c)."""
    u = solve(prob, f)
    lam = solve(prob, gu)
    ga = np.array([-np.sum(lam * term_apply(prob, u, i)) for i in range(prob.N)])
    gc = -np.sum(lam * term_apply(prob, u, prob.N))
    return lam, ga, gc
