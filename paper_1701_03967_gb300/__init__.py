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
from ._lib import FEM_FFT_BATCH_GRAPH, FEM_FFT_BATCH_STREAMS, FEM_FFT_FP64, FEM_FFT_MIXED, FemFftError  # noqa: F401

__all__ = ["Plan", "Batch", "HeatStepper", "HostSolveStream", "FemFftError", "solve", "lib_path", "fem_solve"]

lib_path = _lib.LIB_PATH


def _torch():
    import torch
    return torch


class Plan:
    """A solver plan for one problem shape (owns device tables and workspace).

    n: element order (1..9), one for all axes or one per axis (Section 4);
    K: elements per axis (N = len(K) in 1..3, each K_i
    even and of the form 2^p 3^q); X: axis lengths; a: per-axis coefficients;
    c: zeroth-order coefficient; precision: "fp64" or "mixed"; max_nrhs:
    right-hand sides per internal group (workspace size)."""

    def __init__(self, n, K, X=None, a=None, c=0.0, precision="fp64", max_nrhs=1, stream=None):
        torch = _torch()
        L = _lib.lib()
        self.N = len(K)
        if isinstance(n, (tuple, list)):
            self.ns = tuple(int(x) for x in n)
            if len(self.ns) != self.N:
                raise ValueError("one element order per axis")
        else:
            self.ns = (int(n),) * self.N
        self.n = self.ns[0] if len(set(self.ns)) == 1 else None   # the common order, if any
        self.K = tuple(int(k) for k in K)
        self.X = tuple(float(x) for x in (X if X is not None else (1.0,) * self.N))
        self.a = tuple(float(x) for x in (a if a is not None else (1.0,) * self.N))
        self.c = float(c)
        self.precision = precision
        prec = {"fp64": FEM_FFT_FP64, "mixed": FEM_FFT_MIXED}[precision]
        self.M = tuple(n_i * k - 1 for n_i, k in zip(self.ns, self.K))
        self.dof = 1
        for m in self.M:
            self.dof *= m
        Karr = (ctypes.c_int64 * self.N)(*self.K)
        Xarr = (ctypes.c_double * self.N)(*self.X)
        Aarr = (ctypes.c_double * self.N)(*self.a)
        h = ctypes.c_void_p()
        Narr = (ctypes.c_int * self.N)(*self.ns)
        _lib.check(L.fem_fft_plan_create_orders(ctypes.byref(h), self.N, Narr, Karr, Xarr, Aarr, self.c, prec,
                                                int(max_nrhs), self._stream(stream)), "fem_fft_plan_create_orders")
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
        """u = L^{-1} b (Section 4: algorithm (a), or (b) after set_algorithm("b"))."""
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

    def apply_mass(self, u, out=None, stream=None):
        """b = (C_1 (x) ... (x) C_N) u (float64, matrix-free mass operator)."""
        nrhs = self._field(u, "u")
        b = self._out(u, out)
        _lib.check(_lib.lib().fem_fft_apply_mass(self._h, u.data_ptr(), b.data_ptr(), nrhs, self._stream(stream)),
                   "fem_fft_apply_mass")
        return b

    def dirichlet_rhs(self, g, b, stream=None):
        """b -= L_full G in place (fem_fft_dirichlet_rhs): g holds the boundary
        values on the grid extended by the boundary node at each end of every
        axis, shape (M_1+2, ..., M_N+2) or (nrhs,) + that; b is a field of
        the plan's shape with as many right-hand sides."""
        torch = _torch()
        nrhs = self._field(b, "b")
        ext = tuple(m + 2 for m in self.M)
        want = ext if (nrhs == 1 and tuple(b.shape) == self.M) else (nrhs,) + ext
        if not isinstance(g, torch.Tensor) or not g.is_cuda or g.dtype != torch.float64 or not g.is_contiguous():
            raise TypeError("g must be a contiguous CUDA float64 tensor")
        if tuple(g.shape) != want:
            raise ValueError(f"g has shape {tuple(g.shape)}, expected {want}")
        _lib.check(_lib.lib().fem_fft_dirichlet_rhs(self._h, g.data_ptr(), b.data_ptr(), nrhs, self._stream(stream)),
                   "fem_fft_dirichlet_rhs")
        return b

    def solve_dirichlet(self, f, g, out=None, stream=None):
        """Interior values of the solution with u = g on the boundary:
        L^{-1} (f - L_full G) (Section 4 with non-zero Dirichlet data).  A
        mixed plan may need ``set_refinement(0.0, 3)`` here: the corrected
        right-hand side carries the boundary layer of the data (2D n=9
        K=1024: two steps 1.7e-10, three 3.1e-13)."""
        rhs = f.clone()
        self.dirichlet_rhs(g, rhs, stream=stream)
        return self.solve(rhs, out=out, stream=stream)

    def forward(self, y, out=None, stream=None):
        """Direct FC_n coefficients along every axis (float64)."""
        nrhs = self._field(y, "y")
        c = self._out(y, out)
        _lib.check(_lib.lib().fem_fft_forward(self._h, y.data_ptr(), c.data_ptr(), nrhs, self._stream(stream)),
                   "fem_fft_forward")
        return c

    def solve_host(self, b_host, u_host, stream=None):
        """u_host = L^-1 b_host for float64 CPU tensors (pinned for overlap),
        through fem_fft_solve_host: the copies are pipelined with the solves
        of neighbouring calls inside the library.  Asynchronous: call
        ``host_wait`` (then synchronise the stream) before reading u_host."""
        torch = _torch()
        for x, nm in ((b_host, "b_host"), (u_host, "u_host")):
            if not isinstance(x, torch.Tensor) or x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
                raise TypeError(f"{nm} must be a contiguous float64 CPU tensor")
        if tuple(b_host.shape) == self.M:
            nrhs = 1
        elif b_host.dim() == self.N + 1 and tuple(b_host.shape[1:]) == self.M:
            nrhs = b_host.shape[0]
        else:
            raise ValueError("b_host has the wrong shape")
        if u_host.shape != b_host.shape:
            raise ValueError("u_host shape mismatch")
        _lib.check(_lib.lib().fem_fft_solve_host(self._h, b_host.data_ptr(), u_host.data_ptr(), nrhs,
                                                 self._stream(stream)), "fem_fft_solve_host")
        return u_host

    def host_wait(self, stream=None):
        """Make the stream wait for every download of ``solve_host``."""
        _lib.check(_lib.lib().fem_fft_host_wait(self._h, self._stream(stream)), "fem_fft_host_wait")

    def forward_fn(self, w, out=None, stream=None):
        """Direct F_n coefficients along every axis (float64; the mass product
        folded into the forward maps, Theorem 2 item 3)."""
        nrhs = self._field(w, "w")
        c = self._out(w, out)
        _lib.check(_lib.lib().fem_fft_forward_fn(self._h, w.data_ptr(), c.data_ptr(), nrhs, self._stream(stream)),
                   "fem_fft_forward_fn")
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

    def set_algorithm(self, algo="a", stream=None):
        """Solver of ``solve`` (N >= 2): "a" (transforms along every axis,
        default) or "b" (transforms along x_2..x_N, band solves along x_1)."""
        code = {"a": 0, "b": 1}[algo]
        _lib.check(_lib.lib().fem_fft_set_algorithm(self._h, code, self._stream(stream)), "fem_fft_set_algorithm")

    def tune(self, stream=None):
        """Time the plan's pencil passes over tile shapes and FFT schedules and
        keep the fastest (fem_fft_plan_tune)."""
        _lib.check(_lib.lib().fem_fft_plan_tune(self._h, self._stream(stream)), "fem_fft_plan_tune")

    def set_residual_precision(self, mode="df64"):
        """Arithmetic of the refinement residual of a mixed plan: "df64"
        (double-float on the float pipes, default) or "f64"."""
        code = {"f64": 0, "df64": 1}[mode]
        _lib.check(_lib.lib().fem_fft_set_residual_precision(self._h, code), "fem_fft_set_residual_precision")

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

    KINDS = ("forward", "fused", "inverse", "apply", "apply_df")

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
        M, K, n = self.M[axis], self.K[axis], self.ns[axis]
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


class Batch:
    """Many mixed-precision problems solved together: by one graph launch of
    the recorded work list, or in stream mode (set_mode) by every problem's
    own plan on a few streams -- the only mode for plans with per-axis orders.

    plans: distinct ``Plan`` objects created with precision="mixed" (kept
    alive by the batch); nrhs: right-hand sides per problem (each <= the plan's
    max_nrhs); steps: float64 refinement steps; tune: time tile shapes and
    radix schedules for the passes the batch uses (missing from tune_cache);
    tune_cache: JSON file of tuning results (read and updated).

    Fields are packed: problem p occupies ``offsets[p] : offsets[p] +
    nrhs[p] * plans[p].dof`` of one float64 CUDA tensor of ``total_len``
    elements; ``pack`` / ``views`` convert."""

    MODES = ("forward", "inverse", "fused")

    def __init__(self, plans, nrhs=None, steps=2, tune=True, tune_cache=None, stream=None):
        L = _lib.lib()
        self.plans = list(plans)
        self.nprob = len(self.plans)
        self.nrhs = [1] * self.nprob if nrhs is None else [int(r) for r in nrhs]
        if len(self.nrhs) != self.nprob:
            raise ValueError("nrhs must have one entry per plan")
        handles = (ctypes.c_void_p * self.nprob)(*[p._h for p in self.plans])
        nr = (ctypes.c_int64 * self.nprob)(*self.nrhs)
        h = ctypes.c_void_p()
        cache = tune_cache.encode() if tune_cache else None
        _lib.check(L.fem_fft_batch_create(ctypes.byref(h), handles, self.nprob, nr, int(steps), cache,
                                          1 if tune else 0, Plan._stream(stream)), "fem_fft_batch_create")
        self._h = h
        offs = (ctypes.c_int64 * self.nprob)()
        total, nsteps, nitems = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _lib.check(L.fem_fft_batch_layout(self._h, offs, ctypes.byref(total), ctypes.byref(nsteps),
                                          ctypes.byref(nitems)), "fem_fft_batch_layout")
        self.offsets = list(offs)
        self.total_len = total.value
        self.n_steps = nsteps.value
        self.n_items = nitems.value

    def set_mode(self, mode, nstreams=8):
        """"graph": the recorded work list in one graph launch (default);
        "streams": every problem solved by its own plan on one of nstreams
        streams (fem_fft_batch_set_mode)."""
        m = {"graph": FEM_FFT_BATCH_GRAPH, "streams": FEM_FFT_BATCH_STREAMS}[mode]
        _lib.check(_lib.lib().fem_fft_batch_set_mode(self._h, m, int(nstreams)), "fem_fft_batch_set_mode")

    def solve(self, b, out=None, stream=None, check=False):
        """u = L_p^{-1} b_p for every problem (packed float64 CUDA tensors)."""
        torch = _torch()
        for x, name in ((b, "b"),) + (((out, "out"),) if out is not None else ()):
            if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float64 or \
                    not x.is_contiguous() or x.numel() != self.total_len:
                raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of {self.total_len} elements")
        u = torch.empty_like(b) if out is None else out
        _lib.check(_lib.lib().fem_fft_batch_solve(self._h, b.data_ptr(), u.data_ptr(), Plan._stream(stream)),
                   "fem_fft_batch_solve")
        if check:
            self.check(stream)
        return u

    def status(self, stream=None):
        """(status code, step index of a timed-out wait or -1); synchronises."""
        st, where = ctypes.c_int(), ctypes.c_int64()
        _lib.lib().fem_fft_batch_status(self._h, Plan._stream(stream), ctypes.byref(st), ctypes.byref(where))
        return st.value, where.value

    def check(self, stream=None):
        code, where = self.status(stream)
        if code != 0:
            raise FemFftError(code, f"batched solve (step {where})")

    def views(self, flat):
        """Per-problem views (nrhs_p, M_1..M_N) of a packed tensor."""
        out = []
        for p, pl in enumerate(self.plans):
            n = self.nrhs[p] * pl.dof
            out.append(flat[self.offsets[p]:self.offsets[p] + n].view((self.nrhs[p],) + tuple(pl.M)))
        return out

    def pack(self, fields):
        """Packed CUDA float64 tensor from per-problem arrays (nrhs_p, M...)."""
        torch = _torch()
        flat = torch.empty(self.total_len, dtype=torch.float64, device="cuda")
        for v, f in zip(self.views(flat), fields):
            v.copy_(torch.as_tensor(f).reshape(v.shape))
        return flat

    def tuning(self):
        """The tuned entries used by the batch: dicts with n, K, strided, mode,
        W (pencils per tile), V (FFT values per thread), split, us_per_pencil."""
        L = _lib.lib()
        cnt = L.fem_fft_batch_tuning(self._h, 0, None, None)
        ent = (ctypes.c_int * (7 * max(cnt, 1)))()
        us = (ctypes.c_double * max(cnt, 1))()
        L.fem_fft_batch_tuning(self._h, cnt, ent, us)
        out = []
        for i in range(cnt):
            r = ent[7 * i:7 * i + 7]
            out.append(dict(n=r[0], K=r[1], strided=r[2], mode=self.MODES[r[3]] if r[3] < 3 else r[3], W=r[4],
                            V=r[5], split=r[6], us_per_pencil=us[i]))
        return out

    def set_wait_limit(self, seconds):
        _lib.check(_lib.lib().fem_fft_batch_set_wait_limit(self._h, float(seconds)), "fem_fft_batch_set_wait_limit")

    def hold_step(self, step):
        """Test hook: make step `step` wait for an item count never reached
        (-1 restores the schedule)."""
        _lib.check(_lib.lib().fem_fft_batch_hold_step(self._h, int(step)), "fem_fft_batch_hold_step")

    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().fem_fft_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HeatStepper:
    """Implicit Euler steps of C u' + L u = b (C the N-D mass operator, L the
    operator of ``Plan``): (C + tau L) u_new = C u + tau b.  C + tau L has the
    form of L with a_i -> tau a_i and c -> 1 + tau c, so a step is the mass
    apply of u plus one solve of that scaled operator (denominators
    1 + tau (sum_i a_i 4 h_i^-2 lambda_i + c))."""

    def __init__(self, n, K, X=None, a=None, c=0.0, tau=1e-3, precision="fp64", max_nrhs=1, stream=None):
        N = len(K)
        a = tuple(float(x) for x in (a if a is not None else (1.0,) * N))
        self.tau = float(tau)
        self.plan = Plan(n, K, X, tuple(self.tau * x for x in a), 1.0 + self.tau * float(c), precision,
                         max_nrhs=max_nrhs, stream=stream)

    def step(self, u, b, out=None, stream=None):
        """u_new = (C + tau L)^-1 (C u + tau b), all in the library
        (fem_fft_heat_step)."""
        nrhs = self.plan._field(u, "u")
        self.plan._field(b, "b")
        u_new = self.plan._out(u, out)
        _lib.check(_lib.lib().fem_fft_heat_step(self.plan._h, self.tau, u.data_ptr(), b.data_ptr(), u_new.data_ptr(),
                                                nrhs, self.plan._stream(stream)), "fem_fft_heat_step")
        return u_new

    def close(self):
        self.plan.close()


class HostSolveStream:
    """Solves of right-hand sides held in (pinned) host memory through the
    library's pipelined host-buffer path (fem_fft_solve_host): the upload of a
    right-hand side and the download of a solution run on the plan's copy
    streams under the neighbouring solves, over two device slots the plan
    owns.  ``submit(b_host, u_host)`` queues one solve and returns at once;
    ``wait()`` makes the stream wait for every queued download and
    ``synchronize()`` waits on the host.  Host tensors must stay alive and
    unmodified until their transfer has completed (float64 CPU tensors of the
    plan's field shape, or (nrhs,) + that shape)."""

    def __init__(self, plan, nrhs=1):
        self.plan = plan
        self.shape = tuple(plan.M) if nrhs == 1 else (int(nrhs),) + tuple(plan.M)

    def submit(self, b_host, u_host, stream=None):
        if tuple(b_host.shape) != self.shape or tuple(u_host.shape) != self.shape:
            raise ValueError("host tensors must have the stream's field shape")
        self.plan.solve_host(b_host, u_host, stream=stream)

    def wait(self, stream=None):
        self.plan.host_wait(stream=stream)

    def synchronize(self, stream=None):
        torch = _torch()
        st = stream if stream is not None else torch.cuda.current_stream()
        self.plan.host_wait(stream=st)
        st.synchronize()


def batch_order(nsteps, work=None):
    """Level order of a work list (host only): list of (problem, step)."""
    L = _lib.lib()
    n = len(nsteps)
    tot = sum(nsteps)
    ns = (ctypes.c_int * max(n, 1))(*nsteps)
    w = (ctypes.c_double * max(n, 1))(*work) if work is not None else None
    op = (ctypes.c_int * max(tot, 1))()
    os_ = (ctypes.c_int * max(tot, 1))()
    k = L.fem_fft_batch_order(n, ns, w, op, os_)
    if k < 0:
        raise FemFftError(k, "fem_fft_batch_order")
    return [(op[i], os_[i]) for i in range(k)]


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
