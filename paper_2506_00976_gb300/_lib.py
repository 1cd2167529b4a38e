"""ctypes loader for ``libqwb.so`` (the C ABI declared in ``include/qwb.h``).

There is no fallback: if the shared library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libqwb.so")

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
P_double = ctypes.POINTER(ctypes.c_double)
P_int32 = ctypes.POINTER(ctypes.c_int32)

QWB_OK = 0
QWB_PREC_F64 = 0
QWB_PREC_MIXED = 1
QWB_FLAG_NO_WEIGHTED, QWB_FLAG_NO_PRIMAL, QWB_FLAG_NO_DUAL, QWB_FLAG_MINCOST = 1, 2, 4, 8
QWB_FLAG_SEPARABLE, QWB_FLAG_SYMMETRIC_DUAL, QWB_FLAG_VERIFY = 16, 32, 64
STATUS_NAMES = {0: "QWB_OK", 1: "QWB_ERR_INVALID_ARG", 2: "QWB_ERR_MASS", 3: "QWB_ERR_CUDA",
                4: "QWB_ERR_NOT_CONVERGED", 5: "QWB_ERR_TIMEOUT", 6: "QWB_ERR_OOM",
                7: "QWB_ERR_UNSUPPORTED", 8: "QWB_ERR_VERIFY"}


class QwbProblem(ctypes.Structure):
    _fields_ = [("N", c_int32), ("kappa", c_int32), ("p", c_double), ("d", c_int32),
                ("reserved", c_int32)]


class QwbResult(ctypes.Structure):
    _fields_ = [("ub_weighted", c_double), ("ub_primal", c_double), ("lb", c_double),
                ("lb_p", c_double), ("ub_weighted_p", c_double), ("w_hat_p", c_double),
                ("delta_mu", c_double), ("delta_nu", c_double), ("ipf_residual", c_double),
                ("lb_mincost", c_double),
                ("t_coarse_cost_ms", c_double), ("t_solve_ms", c_double),
                ("t_primal_ms", c_double), ("t_dual_ms", c_double),
                ("ipf_sweeps_done", c_int32), ("status", c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


# (name, restype, argtypes) of every exported symbol of include/qwb.h
SIGNATURES = [
    ("qwb_ctx_create", c_int32, [ctypes.POINTER(c_void_p), c_int32]),
    ("qwb_ctx_destroy", None, [c_void_p]),
    ("qwb_coarse_cost", c_int32, [c_void_p, ctypes.POINTER(QwbProblem), c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    ("qwb_coarse_cost_separable", c_int32, [c_void_p, ctypes.POINTER(QwbProblem), c_void_p, c_void_p,
                                            c_void_p, c_void_p]),
    ("qwb_coarse_solve", c_int32, [c_int32, c_int32, P_double, P_double, P_double, P_int32,
                                   P_int32, P_double, P_int32, P_double, P_double, P_double]),
    ("qwb_coarse_solve_grid", c_int32, [c_int32, P_double, P_double, P_double, P_int32, P_int32,
                                        P_double, P_int32, P_double, P_double, P_double]),
    ("qwb_primal_upscale_ipf", c_int32, [c_void_p, ctypes.POINTER(QwbProblem), c_void_p, c_void_p,
                                         c_void_p, c_void_p, c_void_p, c_int32, c_int32,
                                         c_void_p, c_void_p, ctypes.POINTER(QwbResult), c_int32,
                                         c_void_p]),
    ("qwb_primal_upscale_ipf_kernel", c_int32, [c_void_p, ctypes.POINTER(QwbProblem), c_void_p,
                                                c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                                c_void_p, c_int32, c_void_p, c_void_p,
                                                ctypes.POINTER(QwbResult), c_int32, c_void_p]),
    ("qwb_dual_upscale_ctransform", c_int32, [c_void_p, ctypes.POINTER(QwbProblem), c_void_p,
                                              c_void_p, c_void_p, c_void_p, c_void_p,
                                              ctypes.POINTER(QwbResult), c_int32, c_void_p]),
    ("qwb_ctransform", c_int32, [c_void_p, c_int32, c_double, c_void_p, c_void_p, c_int32,
                                 c_void_p]),
    ("qwb_ctransform_shape", c_int32, [c_void_p, c_int32, c_int32, c_double, c_void_p, c_void_p,
                                       c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p]),
    ("qwb_ctransform_noalloc", c_int32, [c_int32, c_double, c_void_p, c_void_p, c_void_p]),
    ("qwb_ctransform_separable", c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_void_p]),
    ("qwb_lb_adjoint", c_int32, [c_void_p, c_int32, c_double, c_void_p, c_void_p, c_double,
                                 c_void_p, c_void_p]),
    ("qwb_bounds", c_int32, [c_void_p, c_int32, ctypes.POINTER(QwbProblem),
                             ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_int32, c_int32,
                             ctypes.POINTER(QwbResult), c_int32, c_int32, c_int32, c_void_p]),
    ("qwb_batch_create", c_int32, [c_void_p, c_int32, ctypes.POINTER(QwbProblem), c_int32,
                                   c_int32, c_int32, ctypes.POINTER(c_void_p)]),
    ("qwb_batch_destroy", None, [c_void_p]),
    ("qwb_batch_coarse", c_int32, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                   c_int32, c_void_p]),
    ("qwb_batch_solve", c_int32, [c_void_p, c_int32, c_void_p]),
    ("qwb_batch_fine", c_int32, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                 c_int32, c_void_p]),
    ("qwb_batch_results", c_int32, [c_void_p, ctypes.POINTER(QwbResult), c_void_p]),
    ("qwb_batch_potentials", c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    ("qwb_batch_coarse_plan", c_int32, [c_void_p, c_int32, P_int32, P_int32, P_double, c_int32,
                                        P_int32]),
    ("qwb_batch_coarse_potentials", c_int32, [c_void_p, c_int32, P_double, P_double]),
    ("qwb_batch_fine_scalings", c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    ("qwb_batch_set_ipf_cluster", c_int32, [c_void_p, c_int32]),
    ("qwb_batch_set_upscale_kernel", c_int32, [c_void_p, c_int32, c_void_p]),
    ("qwb_batch_set_upscale_cluster", c_int32, [c_void_p, c_int32, c_int32]),
    ("qwb_batch_kernel_times", c_int32, [c_void_p, P_double, c_int32]),
    ("qwb_batch_tuning", c_int32, [c_void_p, ctypes.c_char_p, c_int32]),
    ("qwb_status_string", ctypes.c_char_p, [c_int32]),
    ("qwb_last_error", ctypes.c_char_p, []),
    ("qwb_kernel_launch_count", c_int64, []),
    ("qwb_probe_fp32_rate", c_int32, [c_int32, c_int32, c_int32, P_double]),
]

_LIB = None


class QwbError(RuntimeError):
    def __init__(self, status, where, message=""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}"
                         + (f" ({message})" if message else ""))


def load():
    """Load libqwb.so and declare its signatures; raise if it is not built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2506_00976_gb300.build` (needs nvcc)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def check(status, where):
    if status != QWB_OK:
        msg = load().qwb_last_error()
        raise QwbError(status, where, msg.decode() if msg else "")
