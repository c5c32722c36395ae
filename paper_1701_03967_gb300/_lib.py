"""ctypes loader for libfemfft.so (the C ABI declared in include/femfft.h).

Argument marshalling only: every computation runs in the CUDA library.  There
is no fallback: a missing library raises immediately.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfemfft.so")

FEM_FFT_FP64 = 0
FEM_FFT_MIXED = 1
FEM_FFT_BATCH_GRAPH = 0
FEM_FFT_BATCH_STREAMS = 1

_lib = None


class FemFftError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        L = _lib
        msg = L.fem_fft_strerror(code).decode() if L else str(code)
        detail = L.fem_fft_last_error().decode() if L else ""
        super().__init__(f"{what}: {msg} ({code}){': ' + detail if detail else ''}")


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    P64 = ctypes.POINTER(ctypes.c_int64)
    PD = ctypes.POINTER(ctypes.c_double)
    PI = ctypes.POINTER(ctypes.c_int)
    sig = {
        "fem_fft_plan_create": ([ctypes.POINTER(vp), i32, i32, P64, PD, PD, f64, i32, i64, vp], i32),
        "fem_fft_plan_create_orders": ([vp, i32, PI, P64, PD, PD, f64, i32, i64, vp], i32),
        "fem_fft_plan_orders": ([vp, PI], i32),
        "fem_fft_plan_destroy": ([vp], i32),
        "fem_fft_plan_set_coefficients": ([vp, PD, f64, vp], i32),
        "fem_fft_solve": ([vp, vp, vp, i64, vp], i32),
        "fem_fft_apply": ([vp, vp, vp, i64, vp], i32),
        "fem_fft_apply_mass": ([vp, vp, vp, i64, vp], i32),
        "fem_fft_dirichlet_rhs": ([vp, vp, vp, i64, vp], i32),
        "fem_fft_set_refinement": ([vp, f64, i32], i32),
        "fem_fft_plan_tune": ([vp, vp], i32),
        "fem_fft_set_algorithm": ([vp, i32, vp], i32),
        "fem_fft_set_residual_precision": ([vp, i32], i32),
        "fem_fft_last_info": ([vp, PI, PD], i32),
        "fem_fft_forward": ([vp, vp, vp, i64, vp], i32),
        "fem_fft_forward_fn": ([vp, vp, vp, i64, vp], i32),
        "fem_fft_solve_host": ([vp, vp, vp, i64, vp], i32),
        "fem_fft_host_wait": ([vp, vp], i32),
        "fem_fft_heat_step": ([vp, f64, vp, vp, vp, i64, vp], i32),
        "fem_fft_inverse": ([vp, vp, vp, i64, vp], i32),
        "fem_fft_grad_coeffs": ([vp, vp, vp, i64, PD, PD, vp], i32),
        "fem_fft_plan_dims": ([vp, PI, PI, P64, PI], i32),
        "fem_fft_axis_tables": ([vp, i32, PD, PD, PD], i32),
        "fem_fft_axis_precompute": ([i32, i64, f64, PD, PD, PD], i32),
        "fem_fft_profile": ([vp, i32], i32),
        "fem_fft_profile_read": ([vp, i32, P64, PD, PD, PD], i32),
        "fem_fft_apply_noalloc": ([i32, i32, P64, PD, PD, f64, vp, vp, i64, vp], i32),
        "fem_fft_batch_create": ([ctypes.POINTER(vp), ctypes.POINTER(vp), i32, P64, i32, ctypes.c_char_p, i32, vp],
                                 i32),
        "fem_fft_batch_destroy": ([vp], i32),
        "fem_fft_batch_layout": ([vp, P64, P64, P64, P64], i32),
        "fem_fft_batch_solve": ([vp, vp, vp, vp], i32),
        "fem_fft_batch_status": ([vp, vp, PI, P64], i32),
        "fem_fft_batch_tuning": ([vp, i32, PI, PD], i32),
        "fem_fft_batch_set_wait_limit": ([vp, f64], i32),
        "fem_fft_batch_hold_step": ([vp, i64], i32),
        "fem_fft_batch_set_mode": ([vp, i32, i32], i32),
        "fem_fft_batch_order": ([i32, PI, PD, PI, PI], i32),
        "fem_fft_apply_tiling": ([i64, i64, i64, PI, ctypes.POINTER(ctypes.c_int64)], i32),
        "fem_fft_apply_block_map": ([i64, i64, i64, i64, P64, P64, P64], i32),
        "fem_fft_divide_check": ([vp, vp, vp, vp, i64, vp], i32),
        "fem_fft_strerror": ([i32], ctypes.c_char_p),
        "fem_fft_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def check(code, what):
    if code != 0:
        raise FemFftError(code, what)
