"""1D pieces of the oracle (test infrastructure only; see ``oracle/__init__``).

Paper passages followed:
* Section 2, definition of the local matrices: A_kl = int e_k' e_l',
  C_kl = int e_k e_l on the reference element [-1, 1], Lagrange basis with
  e_l(-1 + 2k/n) = delta_kl.  Built here in exact rational arithmetic.
* Section 2, the space S_K^(n) (node values v_j, j=1..K-1, and element-interior
  vectors v_{j-1/2} in R^{n-1}) and the explicit global system (node rows and
  interior rows).  The oracle orders the nK-1 unknowns along the fine grid
  x = m h / n, m = 1..nK-1, i.e. element e (0-based) owns fine indices
  n*e .. n*e+n-2 (interior l = 1..n-1) and n*e+n-1 (its right node).
* Section 2, the scaled operator form A v = lambda C v, where the true
  eigenvalues are 4 h^-2 lambda.
* Section 2, the element eigenproblems A e = lambda C e and
  A~ e = lambda C~ e (spectra S_n and S~_n).
* Section 3, the dispersion relation (the equation for lambda with parameter
  theta_k = cos(pi k / K)) and Theorem 1 (eigenvalues and eigenvectors s_0^(l),
  s_k^(l)).  ``theorem1_basis`` builds the eigenbasis the oracle solves with,
  literally from Theorem 1, with the eigenvalues and the vectors p_k^(l) in
  high precision (mpmath), as the paper did (quadruple precision).  The dense
  LAPACK route ``eig`` is kept only as a pin: its small eigenvalues carry
  absolute rather than relative errors (about eps * ||calA||), which limits a
  solve built on it to ~1e-10 relative accuracy at K = 64, n = 9.
"""

from fractions import Fraction

import numpy as np
import scipy.linalg


# --------------------------------------------------------------------------
# Reference element (Section 2)
# --------------------------------------------------------------------------

def _poly_mul(p, q):
    out = [Fraction(0)] * (len(p) + len(q) - 1)
    for i, a in enumerate(p):
        for j, b in enumerate(q):
            out[i + j] += a * b
    return out


def _poly_der(p):
    return [i * p[i] for i in range(1, len(p))] or [Fraction(0)]


def _poly_int(p, lo, hi):
    """Exact integral of sum_i p[i] x^i over [lo, hi]."""
    s = Fraction(0)
    for i, a in enumerate(p):
        s += a * (Fraction(hi) ** (i + 1) - Fraction(lo) ** (i + 1)) / (i + 1)
    return s


def lagrange_basis(n):
    """Coefficients (ascending powers of x) of the Lagrange basis e_0..e_n on
    [-1, 1] with nodes x_k = -1 + 2k/n (Section 2)."""
    nodes = [Fraction(-1) + Fraction(2 * k, n) for k in range(n + 1)]
    basis = []
    for l in range(n + 1):
        p = [Fraction(1)]
        for m in range(n + 1):
            if m == l:
                continue
            den = nodes[l] - nodes[m]
            p = _poly_mul(p, [-nodes[m] / den, Fraction(1) / den])
        basis.append(p)
    return basis


def reference_matrices_exact(n):
    """Exact local stiffness A and mass C ((n+1)x(n+1) lists of Fractions),
    A_kl = int_{-1}^{1} e_k' e_l' dx, C_kl = int_{-1}^{1} e_k e_l dx (Section 2)."""
    e = lagrange_basis(n)
    de = [_poly_der(p) for p in e]
    A = [[_poly_int(_poly_mul(de[k], de[l]), -1, 1) for l in range(n + 1)]
         for k in range(n + 1)]
    C = [[_poly_int(_poly_mul(e[k], e[l]), -1, 1) for l in range(n + 1)]
         for k in range(n + 1)]
    return A, C


def reference_matrices(n):
    """float64 versions of A and C (each entry is the correctly rounded value
    of the exact rational)."""
    A, C = reference_matrices_exact(n)
    return (np.array([[float(x) for x in row] for row in A]),
            np.array([[float(x) for x in row] for row in C]))


# --------------------------------------------------------------------------
# Global 1D operators (Section 2, explicit system)
# --------------------------------------------------------------------------

def dof_count(n, K):
    """dim S_K^(n) = nK - 1 (Section 2)."""
    return n * K - 1


def local_to_global(n, K, e, q):
    """Fine-grid index of local node q (0..n) of element e (0-based), or None
    for the two Dirichlet boundary nodes."""
    g = n * e + q - 1
    if g < 0 or g >= n * K - 1:
        return None
    return g


def assemble(n, K):
    """Dense h-free global operators (calA, calC) of Section 2, M x M with
    M = nK-1, assembled by summing the element blocks of A and C."""
    A, C = reference_matrices(n)
    M = dof_count(n, K)
    calA = np.zeros((M, M))
    calC = np.zeros((M, M))
    for e in range(K):
        idx = [local_to_global(n, K, e, q) for q in range(n + 1)]
        for q in range(n + 1):
            gq = idx[q]
            if gq is None:
                continue
            for r in range(n + 1):
                gr = idx[r]
                if gr is None:
                    continue
                calA[gq, gr] += A[q, r]
                calC[gq, gr] += C[q, r]
    return calA, calC


def assemble_full(n, K):
    """Dense h-free operators of the space with the two boundary nodes kept,
    (nK+1) x (nK+1): the same element blocks summed over the K elements, with
    fine index m = n e + q (0..nK) for local node q of element e (0-based).
    Rows/columns 1..nK-1 are ``assemble``'s; rows 0 and nK and the columns of
    the boundary nodes carry the coupling that Dirichlet data enter through
    (Section 4: u = g on the boundary, f^h modified by the boundary values)."""
    A, C = reference_matrices(n)
    M = n * K + 1
    fA = np.zeros((M, M))
    fC = np.zeros((M, M))
    for e in range(K):
        for q in range(n + 1):
            for r in range(n + 1):
                fA[n * e + q, n * e + r] += A[q, r]
                fC[n * e + q, n * e + r] += C[q, r]
    return fA, fC


def assemble_sparse(n, K):
    """The same (calA, calC) as ``assemble``, as scipy CSR matrices."""
    import scipy.sparse
    A, C = reference_matrices(n)
    M = dof_count(n, K)
    rows, cols, va, vc = [], [], [], []
    for e in range(K):
        idx = [local_to_global(n, K, e, q) for q in range(n + 1)]
        for q in range(n + 1):
            for r in range(n + 1):
                if idx[q] is None or idx[r] is None:
                    continue
                rows.append(idx[q])
                cols.append(idx[r])
                va.append(A[q, r])
                vc.append(C[q, r])
    shape = (M, M)
    return (scipy.sparse.csr_matrix((va, (rows, cols)), shape=shape),
            scipy.sparse.csr_matrix((vc, (rows, cols)), shape=shape))


def eig(n, K):
    """Dense generalized eigendecomposition calA V = calC V diag(lam) with
    V^T calC V = I (scipy/LAPACK).  Returns (lam, V); the true (h-scaled)
    eigenvalues are 4 h^-2 lam (Section 2)."""
    calA, calC = assemble(n, K)
    lam, V = scipy.linalg.eigh(calA, calC)
    return lam, V


# --------------------------------------------------------------------------
# Element eigenproblems, dispersion relation and Theorem 1 (Sections 2, 3)
# --------------------------------------------------------------------------

def flip(p):
    """The flip P of Section 2: (P p)_l = p_{n-l}."""
    return np.asarray(p)[::-1]


def element_blocks(n):
    """Blocks of the 3x3 block form of A and C (Section 2, eq. for A, C, G):
    a0, a (R^{n-1}), a_n, A~ ((n-1)x(n-1)) and likewise for C."""
    A, C = reference_matrices(n)
    def blocks(B):
        return dict(b0=B[0, 0], b=B[1:n, 0].copy(), bn=B[0, n],
                    bt=B[1:n, 1:n].copy())
    return blocks(A), blocks(C)


def interior_element_eig(n):
    """Eigenpairs of A~ e = lambda C~ e (Section 2), C~-normalised
    (C~ e . e = 1).  Returns (lam0 ascending, E with columns e^(l))."""
    bA, bC = element_blocks(n)
    lam0, E = scipy.linalg.eigh(bA["bt"], bC["bt"])
    return lam0, E


def _fraction_det(M):
    """Exact determinant of a square matrix of Fractions (Gaussian elimination)."""
    M = [row[:] for row in M]
    N = len(M)
    d = Fraction(1)
    for c in range(N):
        p = next((r for r in range(c, N) if M[r][c] != 0), None)
        if p is None:
            return Fraction(0)
        if p != c:
            M[c], M[p] = M[p], M[c]
            d = -d
        d *= M[c][c]
        for r in range(c + 1, N):
            f = M[r][c] / M[c][c]
            for cc in range(c, N):
                M[r][cc] -= f * M[c][cc]
    return d


def _fraction_interp(xs, ys):
    """Exact monomial coefficients (ascending) of the polynomial through the
    points (xs, ys) (Gauss-Jordan on the Vandermonde system, Fractions)."""
    N = len(xs)
    M = [[x ** p for p in range(N)] + [y] for x, y in zip(xs, ys)]
    for c in range(N):
        p = next(r for r in range(c, N) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(N):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                for cc in range(c, N + 1):
                    M[r][cc] -= f * M[c][cc]
    return [M[i][N] / M[i][i] for i in range(N)]


def dispersion_polynomials(n):
    """Exact rational coefficients (ascending in lambda) of P0 and P1 with
    P0(lambda) + theta P1(lambda) = det(G~(lambda)) (g0_hat + theta gn_hat)(lambda).

    Section 3 writes the dispersion relation as gamma_hat(lambda) = theta with
    gamma_hat = -g0_hat / gn_hat, g0_hat = g0 - g.G~^{-1} g and
    gn_hat = gn - gcheck.G~^{-1} g (G = A - lambda C in the 3x3 block form of
    Section 2).  Multiplying by det G~ turns the two Schur complements into
    determinants of bordered matrices: det [[g0, g^T], [g, G~]] and
    det [[gn, gcheck^T], [g, G~]], i.e. the leading n x n block of G(lambda)
    and the same block with its first row replaced by the first n entries of
    the last row of G(lambda).  Both are polynomials of degree <= n; they are
    obtained exactly by evaluation at n+1 integers and interpolation."""
    Aex, Cex = reference_matrices_exact(n)
    xs = [Fraction(j) for j in range(n + 1)]
    p0, p1 = [], []
    for x in xs:
        G = [[Aex[i][j] - x * Cex[i][j] for j in range(n + 1)] for i in range(n + 1)]
        B0 = [row[0:n] for row in G[0:n]]
        B1 = [G[n][0:n]] + [row[0:n] for row in G[1:n]]
        p0.append(_fraction_det(B0))
        p1.append(_fraction_det(B1))
    return _fraction_interp(xs, p0), _fraction_interp(xs, p1)


def dispersion_roots(n, theta, dps=40):
    """All n roots lambda of the dispersion relation of Section 3 for one
    theta (float or mpmath number), as mpmath numbers at ``dps`` digits.
    Roots of P0 + theta P1 (``dispersion_polynomials``) by mpmath.polyroots."""
    import mpmath
    with mpmath.workdps(dps):
        P0, P1 = _disp_cache(n)
        th = mpmath.mpf(theta)
        c = [mpmath.mpf(P0[p].numerator) / P0[p].denominator
             + th * mpmath.mpf(P1[p].numerator) / P1[p].denominator
             for p in range(len(P0) - 1, -1, -1)]
        # float64 companion-matrix roots as starting values, then mpmath's
        # simultaneous iteration to full working precision
        init = np.roots([float(x) for x in c])
        r = mpmath.polyroots(c, maxsteps=60, extraprec=2 * dps,
                             roots_init=[mpmath.mpc(complex(z)) for z in init])
        return sorted((mpmath.re(x) for x in r), key=float)


_DISP = {}


def _disp_cache(n):
    if n not in _DISP:
        _DISP[n] = dispersion_polynomials(n)
    return _DISP[n]


def _element_eig_mp(n, dps):
    """High-precision eigenpairs of A~ e = lambda C~ e (Section 2), C~-normalised."""
    import mpmath
    Aex, Cex = reference_matrices_exact(n)
    def mp(x):
        return mpmath.mpf(x.numerator) / x.denominator
    m = n - 1
    At = mpmath.matrix([[mp(Aex[i][j]) for j in range(1, n)] for i in range(1, n)])
    Ct = mpmath.matrix([[mp(Cex[i][j]) for j in range(1, n)] for i in range(1, n)])
    L = mpmath.cholesky(Ct)
    Li = L ** -1
    ev, Q = mpmath.eigsy(Li * At * Li.T)
    E = Li.T * Q
    order = sorted(range(m), key=lambda i: float(ev[i]))
    lam0 = [ev[i] for i in order]
    Ecols = [[E[r, i] for r in range(m)] for i in order]
    return lam0, Ecols


def theorem1_basis(n, K, dps=40):
    """The C-orthogonal eigenbasis of Section 3, Theorem 1, built literally.

    Spectral order: first the n-1 bubble modes s_0^(l) (eigenvalue
    lambda0^(l) in S~_n), then for k = 1..K-1 the n modes s_k^(l) whose
    eigenvalues lambda_k^(l) are the roots of the dispersion relation with
    theta_k = cos(pi k / K) (item 1).  s_0^(l): zero node values, interiors
    (-P)^{j-1} e^(l) (item 2).  s_k^(l): node values sin(pi k j / K),
    interiors p sin(pi k (j-1)/K) + flip(p) sin(pi k j / K) (item 3), with
    p = p_k^(l) from Section 2, Lemma 2:
    p = sum_l' (a^(l') - lambda c^(l')) / (lambda - lambda0^(l')) e^(l').

    Eigenvalues and p are computed at ``dps`` digits (the paper used quadruple
    precision) and rounded to float64.  Returns (lam (M,), S (M x M), with
    columns s in the fine-grid ordering, Cnorm2 (M,) = s^T calC s computed
    densely)."""
    import mpmath
    M = dof_count(n, K)
    lam = np.zeros(M)
    S = np.zeros((M, M))
    col = 0
    with mpmath.workdps(dps):
        if n > 1:
            lam0, Ecols = _element_eig_mp(n, dps)
            Aex, Cex = reference_matrices_exact(n)
            def mp(x):
                return mpmath.mpf(x.numerator) / x.denominator
            avec = [mp(Aex[i][0]) for i in range(1, n)]
            cvec = [mp(Cex[i][0]) for i in range(1, n)]
            al = [sum(avec[i] * e[i] for i in range(n - 1)) for e in Ecols]
            cl = [sum(cvec[i] * e[i] for i in range(n - 1)) for e in Ecols]
            for l in range(n - 1):
                lam[col] = float(lam0[l])
                S[:, col] = theorem1_bubble(n, K, [float(x) for x in Ecols[l]])
                col += 1
        for k in range(1, K):
            theta = mpmath.cos(mpmath.pi * k / K)
            for root in dispersion_roots(n, theta, dps):
                lam[col] = float(root)
                if n > 1:
                    p = [mpmath.mpf(0)] * (n - 1)
                    for l in range(n - 1):
                        coef = (al[l] - root * cl[l]) / (root - lam0[l])
                        for i in range(n - 1):
                            p[i] += coef * Ecols[l][i]
                    p = np.array([float(x) for x in p])
                else:
                    p = np.zeros(0)
                S[:, col] = _theorem1_vector(n, K, k, p)
                col += 1
    assert col == M
    calC = assemble_sparse(n, K)[1]
    cnorm2 = np.einsum("ij,ij->j", S, np.asarray(calC @ S))
    return lam, S, cnorm2


def _sinpi_ratio(m, K):
    """sin(pi m / K) for integer arrays m: the argument is reduced exactly in
    integers (m mod 2K) before the float64 sine, so its error does not grow
    with m (pi m / K reaches ~10^4 for the long pencils of Section 5)."""
    r = np.mod(np.asarray(m, dtype=np.int64), 2 * K)
    return np.sin(np.pi * r / K)


def _theorem1_vector(n, K, k, p):
    """s_k in the fine-grid ordering for a given p (Section 3, Theorem 1,
    item 3): node j (1..K-1) -> sin(pi k j / K); interior of element j
    (1..K) -> p sin(pi k (j-1)/K) + flip(p) sin(pi k j / K)."""
    M = dof_count(n, K)
    s = np.zeros(M)
    j = np.arange(1, K + 1)
    sl = _sinpi_ratio(k * (j - 1), K)             # sin(pi k (j-1) / K) at the element's left node
    sr = _sinpi_ratio(k * j, K)                   # sin(pi k j / K) at the element's right node
    blocks = np.zeros((K, n))
    if n > 1:
        blocks[:, :n - 1] = np.outer(sl, p) + np.outer(sr, flip(p))
    blocks[:, n - 1] = sr
    s[:] = blocks.reshape(-1)[:M]                 # drops the right boundary node
    return s


def theorem1_bubble(n, K, e_vec):
    """Eigenvector s_0^(l) of Section 3, Theorem 1, item 2: zero node values
    and interiors (-P)^{j-1} e^(l)."""
    M = dof_count(n, K)
    s = np.zeros(M)
    v = np.array(e_vec, dtype=float)
    for j in range(1, K + 1):
        s[n * (j - 1): n * (j - 1) + n - 1] = v
        v = -flip(v)
    return s
