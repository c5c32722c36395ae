"""GB300-native fast Fourier solver for the tensor-product nth-order FEM
(Zlotnik & Zlotnik, arXiv:1701.03967).

Python binding of the C ABI in ``include/femfft.h`` (``libfemfft.so``, built
in-tree by ``build.build()``).  The binding only marshals arguments: torch is
used for device memory and streams; every step of the solve runs in the CUDA
library.

    plan = Plan(n=9, K=(1024, 1024), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0,
                precision="mixed")
    u = plan.solve(b)            # b: cuda float64 tensor [nrhs, M1, M2] or [M1, M2]
"""

import ctypes

from . import _lib
from ._lib import FEM_FFT_FP64, FEM_FFT_MIXED, FemFftError  # noqa: F401

__all__ = ["Plan", "FemFftError", "solve", "lib_path", "fem_solve"]

lib_path = _lib.LIB_PATH


def _torch():
    import torch
    return torch


class Plan:
    """A solver plan for one problem shape (owns device tables and workspace).

    n: element order (1..9); K: elements per axis (N = len(K) in 1..3, each K_i
    even and of the form 2^p 3^q); X: axis lengths; a: per-axis coefficients;
    c: zeroth-order coefficient; precision: "fp64" or "mixed"; max_nrhs:
    right-hand sides per internal group (workspace size)."""

    def __init__(self, n, K, X=None, a=None, c=0.0, precision="fp64", max_nrhs=1, stream=None):
        torch = _torch()
        L = _lib.lib()
        self.N = len(K)
        self.n = int(n)
        self.K = tuple(int(k) for k in K)
        self.X = tuple(float(x) for x in (X if X is not None else (1.0,) * self.N))
        self.a = tuple(float(x) for x in (a if a is not None else (1.0,) * self.N))
        self.c = float(c)
        self.precision = precision
        prec = {"fp64": FEM_FFT_FP64, "mixed": FEM_FFT_MIXED}[precision]
        self.M = tuple(self.n * k - 1 for k in self.K)
        self.dof = 1
        for m in self.M:
            self.dof *= m
        Karr = (ctypes.c_int64 * self.N)(*self.K)
        Xarr = (ctypes.c_double * self.N)(*self.X)
        Aarr = (ctypes.c_double * self.N)(*self.a)
        h = ctypes.c_void_p()
        _lib.check(L.fem_fft_plan_create(ctypes.byref(h), self.N, self.n, Karr, Xarr, Aarr, self.c, prec,
                                         int(max_nrhs), self._stream(stream)), "fem_fft_plan_create")
        self._h = h
        self._torch_device = torch.device("cuda", torch.cuda.current_device())

    # -- helpers ---------------------------------------------------------
    @staticmethod
    def _stream(stream):
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream()
        return ctypes.c_void_p(stream.cuda_stream)

    def _field(self, x, name):
        torch = _torch()
        if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float64:
            raise TypeError(f"{name} must be a CUDA float64 tensor")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if tuple(x.shape) == self.M:
            return 1
        if x.dim() == self.N + 1 and tuple(x.shape[1:]) == self.M:
            return x.shape[0]
        raise ValueError(f"{name} has shape {tuple(x.shape)}, expected {self.M} or (nrhs,)+{self.M}")

    def _out(self, like, out):
        torch = _torch()
        if out is None:
            return torch.empty_like(like)
        self._field(out, "out")
        if out.shape != like.shape:
            raise ValueError("out shape mismatch")
        return out

    # -- solver ----------------------------------------------------------
    def solve(self, b, out=None, stream=None):
        """u = L^{-1} b (Section 4, algorithm (a))."""
        nrhs = self._field(b, "b")
        u = self._out(b, out)
        _lib.check(_lib.lib().fem_fft_solve(self._h, b.data_ptr(), u.data_ptr(), nrhs, self._stream(stream)),
                   "fem_fft_solve")
        return u

    def apply(self, u, out=None, stream=None):
        """b = L u (float64, matrix-free)."""
        nrhs = self._field(u, "u")
        b = self._out(u, out)
        _lib.check(_lib.lib().fem_fft_apply(self._h, u.data_ptr(), b.data_ptr(), nrhs, self._stream(stream)),
                   "fem_fft_apply")
        return b

    def forward(self, y, out=None, stream=None):
        """Direct FC_n coefficients along every axis (float64)."""
        nrhs = self._field(y, "y")
        c = self._out(y, out)
        _lib.check(_lib.lib().fem_fft_forward(self._h, y.data_ptr(), c.data_ptr(), nrhs, self._stream(stream)),
                   "fem_fft_forward")
        return c

    def inverse(self, coef, out=None, stream=None):
        """Inverse F_n-expansion along every axis (float64)."""
        nrhs = self._field(coef, "coef")
        w = self._out(coef, out)
        _lib.check(_lib.lib().fem_fft_inverse(self._h, coef.data_ptr(), w.data_ptr(), nrhs,
                                              self._stream(stream)), "fem_fft_inverse")
        return w

    def set_coefficients(self, a, c, stream=None):
        """Replace a_i and c (only the denominator tables are recomputed)."""
        a = tuple(float(x) for x in a)
        arr = (ctypes.c_double * self.N)(*a)
        _lib.check(_lib.lib().fem_fft_plan_set_coefficients(self._h, arr, float(c), self._stream(stream)),
                   "fem_fft_plan_set_coefficients")
        self.a, self.c = a, float(c)

    def set_refinement(self, rtol=0.0, max_iter=2):
        _lib.check(_lib.lib().fem_fft_set_refinement(self._h, float(rtol), int(max_iter)),
                   "fem_fft_set_refinement")

    def last_info(self):
        it = ctypes.c_int()
        rel = ctypes.c_double()
        _lib.check(_lib.lib().fem_fft_last_info(self._h, ctypes.byref(it), ctypes.byref(rel)), "fem_fft_last_info")
        return it.value, rel.value

    def grad_coeffs(self, u, lam, stream=None):
        """(-lam^T dL/da_i u for each axis i, -lam^T dL/dc u), float64."""
        nrhs = self._field(u, "u")
        self._field(lam, "lam")
        ga = (ctypes.c_double * self.N)()
        gc = ctypes.c_double()
        _lib.check(_lib.lib().fem_fft_grad_coeffs(self._h, u.data_ptr(), lam.data_ptr(), nrhs, ga,
                                                  ctypes.byref(gc), self._stream(stream)), "fem_fft_grad_coeffs")
        return list(ga), gc.value

    KINDS = ("forward", "fused", "inverse", "apply")

    def profile(self, enable=True):
        """Start (or stop and clear) per-kernel CUDA-event timing."""
        _lib.check(_lib.lib().fem_fft_profile(self._h, 1 if enable else 0), "fem_fft_profile")

    def profile_read(self):
        """{kind: dict(launches, ms, bytes, flops64)} since profiling started
        (synchronises)."""
        out = {}
        for k, name in enumerate(self.KINDS):
            cnt = ctypes.c_int64()
            ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            _lib.check(_lib.lib().fem_fft_profile_read(self._h, k, ctypes.byref(cnt), ctypes.byref(ms),
                                                       ctypes.byref(by), ctypes.byref(fl)), "fem_fft_profile_read")
            out[name] = dict(launches=cnt.value, ms=ms.value, bytes=by.value, flops64=fl.value)
        return out

    def axis_tables(self, axis):
        """(lam, cnorm, p) host tables of one axis (numpy arrays)."""
        import numpy as np
        M, K, n = self.M[axis], self.K[axis], self.n
        lam = np.zeros(M)
        cn = np.zeros(M)
        p = np.zeros(K * n * max(n - 1, 1))
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.check(_lib.lib().fem_fft_axis_tables(self._h, axis, lam.ctypes.data_as(dp), cn.ctypes.data_as(dp),
                                                  p.ctypes.data_as(dp)), "fem_fft_axis_tables")
        return lam, cn, p.reshape(K, n, max(n - 1, 1))

    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().fem_fft_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(b, n, K, X=None, a=None, c=0.0, precision="fp64"):
    """One-shot convenience: build a plan, solve, free the plan."""
    nrhs = b.shape[0] if b.dim() == len(K) + 1 else 1
    p = Plan(n, K, X, a, c, precision, max_nrhs=nrhs)
    try:
        return p.solve(b)
    finally:
        p.close()


def fem_solve(plan, f, a=None, c=None):
    """Differentiable u = L(a, c)^{-1} f (see ``autograd.FemSolve``)."""
    from .autograd import fem_solve as _fs
    return _fs(plan, f, a, c)
