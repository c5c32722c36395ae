"""CPU tests of the C-ABI library: it loads, exports every declared symbol,
and its host-side plan precompute (double-double eigenpairs, Section 3,
Theorem 1) agrees with the oracle.  No device call is made."""

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import fem1d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_1701_03967_gb300 import _lib as L
    if not os.path.exists(L.LIB_PATH):
        from paper_1701_03967_gb300 import build
        build.build()
    return L.lib()


def test_library_exports_every_declared_symbol():
    L = _lib()
    header = open(os.path.join(ROOT, "include", "femfft.h")).read()
    names = set(re.findall(r"^\s*(?:int|const char\*)\s+(fem_fft_\w+)\s*\(", header, re.M))
    assert len(names) >= 14
    for name in sorted(names):
        assert hasattr(L, name), name


def _precompute(n, K, X=1.0):
    L = _lib()
    M = max(n * K - 1, 1)
    lam, cn = np.zeros(M), np.zeros(M)
    p = np.zeros(max(K, 1) * max(n, 1) * max(n - 1, 1))
    dp = ctypes.POINTER(ctypes.c_double)
    rc = L.fem_fft_axis_precompute(n, K, X, lam.ctypes.data_as(dp), cn.ctypes.data_as(dp), p.ctypes.data_as(dp))
    return rc, lam, cn, p.reshape(max(K, 1), max(n, 1), max(n - 1, 1))


@pytest.mark.parametrize("n,K", [(1, 8), (2, 6), (3, 16), (4, 12), (5, 8), (6, 4), (7, 8), (8, 6), (9, 16), (9, 2)])
def test_host_eigenpairs_match_oracle(n, K):
    rc, lam, cn, p = _precompute(n, K)
    assert rc == 0
    lo, S, co = fem1d.theorem1_basis(n, K)
    np.testing.assert_allclose(lam, lo, rtol=1e-14)
    np.testing.assert_allclose(cn, co, rtol=1e-13)
    # p_k^(l): interiors of element 1 of s_k^(l) are flip(p) sin(pi k / K)
    for k in range(1, K):
        for l in range(n):
            col = n - 1 + (k - 1) * n + l
            if n > 1:
                want = fem1d.flip(S[0:n - 1, col]) / np.sin(np.pi * k / K)
                np.testing.assert_allclose(p[k, l], want, rtol=1e-11, atol=1e-12 * np.abs(want).max())
    # bubble eigenvectors e^(l) up to sign
    for l in range(n - 1):
        e_or = S[0:n - 1, l]
        e = p[0, l]
        sgn = np.sign(e @ e_or)
        np.testing.assert_allclose(sgn * e, e_or, atol=1e-13)


def test_host_rejects_bad_sizes():
    for n, K in [(0, 8), (10, 8), (3, 5), (3, 1), (3, 10), (3, 7)]:
        rc, *_ = _precompute(n, K)
        assert rc == -1, (n, K)


def test_noalloc_rejects_oversized_and_invalid_problems_without_a_device_call():
    """fem_fft_apply_noalloc validates before any device call: 3D extents
    whose unknown count would overflow a signed 64-bit product, problems
    beyond its static scratch, and coefficients fem_fft_plan_create rejects
    all return FEM_FFT_ERR_ARG (-1), here with nrhs = 0 and NULL buffers."""
    L = _lib()
    f = L.fem_fft_apply_noalloc

    def call(N, n, K, X=None, a=None, c=0.0, nrhs=0):
        Kc = (ctypes.c_int64 * N)(*K)
        Xc = (ctypes.c_double * N)(*(X or [1.0] * N))
        ac = (ctypes.c_double * N)(*(a or [1.0] * N))
        return f(N, n, Kc, Xc, ac, c, None, None, nrhs, None)

    # (3 * 708588 - 1)^3 wraps a signed 64-bit product
    assert call(3, 3, (708588, 708588, 708588)) == -1
    assert call(3, 9, (1 << 20, 1 << 20, 1 << 20)) == -1
    assert call(2, 9, (1024, 1024)) == -1                  # 3 x 680 MB of temporaries
    assert call(1, 9, (3 << 20,)) == -1                    # K beyond 2^20
    assert call(2, 2, (16, 16), a=[1.0, 0.0]) == -1        # a_i must be positive
    assert call(2, 2, (16, 16), c=-2.0 * np.pi ** 2) == -1  # L not positive definite
    assert call(2, 2, (16, 15)) == -1                      # K must be 2^p 3^q, p >= 1
    assert call(2, 2, (16, 16)) == 0                       # valid, nrhs = 0: a no-op


def test_entry_points_reject_bad_arguments_without_a_device_call():
    """Argument checks that return before any CUDA call: null handles, negative
    counts, unknown modes (so they run without a GPU)."""
    import ctypes
    from paper_1701_03967_gb300 import _lib
    L = _lib.lib()
    buf = (ctypes.c_double * 4)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert L.fem_fft_divide_check(p, p, p, p, -1, None) == -1
    assert L.fem_fft_divide_check(None, p, p, p, 4, None) == -1
    assert L.fem_fft_divide_check(None, None, None, None, 0, None) == 0
    assert L.fem_fft_batch_set_mode(None, 1, 4) == -1
    assert L.fem_fft_solve_host(None, p, p, 1, None) == -1
    assert L.fem_fft_host_wait(None, None) == -1
    assert L.fem_fft_batch_solve(None, p, p, None) == -1
