"""Python binding of the qwb C ABI (``include/qwb.h``), one function per entry point.

Argument marshalling only: every step of the method runs in ``libqwb.so``
(CUDA kernels and the host network simplex).  PyTorch provides device memory
(float64 CUDA tensors) and the current stream.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np
import torch

from . import _lib
from ._lib import QwbProblem, QwbResult, check
from ._lib import (QWB_FLAG_MINCOST, QWB_FLAG_NO_DUAL, QWB_FLAG_NO_PRIMAL,  # noqa: F401
                   QWB_FLAG_NO_WEIGHTED, QWB_FLAG_SEPARABLE, QWB_FLAG_SYMMETRIC_DUAL, QWB_FLAG_VERIFY)

_CTX = {}
_CTX_LOCK = threading.Lock()

PREC = {"f64": _lib.QWB_PREC_F64, "mixed": _lib.QWB_PREC_MIXED}


def _prec(prec):
    if prec not in PREC:
        raise ValueError(f"prec must be one of {sorted(PREC)}")
    return PREC[prec]


def context(device=None):
    """The library context of a CUDA device (created once per process)."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else
                       torch.device(device).index or 0)
    with _CTX_LOCK:
        if dev.index not in _CTX:
            h = ctypes.c_void_p()
            check(_lib.load().qwb_ctx_create(ctypes.byref(h), dev.index), "qwb_ctx_create")
            _CTX[dev.index] = h
        return _CTX[dev.index]


def _stream(t):
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _dev64(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


QWB_IPF_BULK = 32   # Batch.set_ipf_cluster(C | QWB_IPF_BULK): the bulk-copy staged sweeps
QWB_IPF_WIDE = 64   # Batch.set_ipf_cluster(C | QWB_IPF_WIDE): the register form with 512-thread CTAs


def problem(N, kappa, p, d=2):
    """One problem on the grid [N]^d (d = 2 images, d = 3 volumes)."""
    return QwbProblem(int(N), int(kappa), float(p), int(d), 0)


def coarse_cost(mu, nu, N, kappa, p, prec="mixed", d=2):
    """qwb_coarse_cost: (C-bar [M, M], mu~ [M], nu~ [M]) on the device."""
    n = N // kappa
    M = n ** d
    cbar = torch.empty((M, M), dtype=torch.float64, device=mu.device)
    mc = torch.empty(M, dtype=torch.float64, device=mu.device)
    nc = torch.empty(M, dtype=torch.float64, device=mu.device)
    pr = problem(N, kappa, p, d)
    check(_lib.load().qwb_coarse_cost(context(mu.device), ctypes.byref(pr), _dev64(mu, "mu"),
                                      _dev64(nu, "nu"), _ptr(cbar), _ptr(mc), _ptr(nc),
                                      _prec(prec), _stream(mu)), "qwb_coarse_cost")
    return cbar, mc, nc


def coarse_cost_separable(mu, nu, N, kappa):
    """qwb_coarse_cost_separable: C-bar [M, M] for p = 2 (d = 2, kappa 4 or 8)
    by separating the squared distance over the axes (FP32 reductions)."""
    M = (N // kappa) ** 2
    cbar = torch.empty((M, M), dtype=torch.float64, device=mu.device)
    pr = problem(N, kappa, 2.0, 2)
    check(_lib.load().qwb_coarse_cost_separable(context(mu.device), ctypes.byref(pr), _dev64(mu, "mu"),
                                                _dev64(nu, "nu"), _ptr(cbar), _stream(mu)),
          "qwb_coarse_cost_separable")
    return cbar


def coarse_solve(C, a, b):
    """qwb_coarse_solve (host network simplex): dict with CSR plan, f, g, obj (numpy)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if C.ndim != 2 or a.shape != (C.shape[0],) or b.shape != (C.shape[1],):
        raise ValueError("coarse_solve: C must be (n, m) with a of n and b of m entries")
    n, m = C.shape
    rowptr = np.zeros(n + 1, dtype=np.int32)
    col = np.zeros(n + m, dtype=np.int32)
    val = np.zeros(n + m, dtype=np.float64)
    nnz = ctypes.c_int32()
    f = np.zeros(n)
    g = np.zeros(m)
    obj = ctypes.c_double()
    pd = lambda x: x.ctypes.data_as(_lib.P_double)  # noqa: E731
    pi = lambda x: x.ctypes.data_as(_lib.P_int32)   # noqa: E731
    check(_lib.load().qwb_coarse_solve(n, m, pd(C), pd(a), pd(b), pi(rowptr), pi(col), pd(val),
                                       ctypes.byref(nnz), pd(f), pd(g), ctypes.byref(obj)),
          "qwb_coarse_solve")
    k = nnz.value
    return {"rowptr": rowptr, "col": col[:k].copy(), "val": val[:k].copy(), "f": f, "g": g,
            "obj": obj.value}


def coarse_solve_grid(tab, a, b):
    """qwb_coarse_solve_grid (host network simplex, offset-table cost on an
    n x n grid): dict with CSR plan, f, g, obj (numpy)."""
    tab = np.ascontiguousarray(tab, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if tab.ndim != 2 or tab.shape[0] != tab.shape[1]:
        raise ValueError("coarse_solve_grid: tab must be a square (n_side, n_side) table")
    ns = tab.shape[0]
    M = ns * ns
    if a.shape != (M,) or b.shape != (M,):
        raise ValueError(f"coarse_solve_grid: a and b must have n_side^2 = {M} entries")
    rowptr = np.zeros(M + 1, dtype=np.int32)
    col = np.zeros(2 * M, dtype=np.int32)
    val = np.zeros(2 * M, dtype=np.float64)
    nnz = ctypes.c_int32()
    f = np.zeros(M)
    g = np.zeros(M)
    obj = ctypes.c_double()
    pd = lambda x: x.ctypes.data_as(_lib.P_double)  # noqa: E731
    pi = lambda x: x.ctypes.data_as(_lib.P_int32)   # noqa: E731
    check(_lib.load().qwb_coarse_solve_grid(ns, pd(tab), pd(a), pd(b), pi(rowptr), pi(col), pd(val),
                                            ctypes.byref(nnz), pd(f), pd(g), ctypes.byref(obj)),
          "qwb_coarse_solve_grid")
    k = nnz.value
    return {"rowptr": rowptr, "col": col[:k].copy(), "val": val[:k].copy(), "f": f, "g": g,
            "obj": obj.value}


def primal_upscale_ipf(mu, nu, N, kappa, p, rowptr, col, val, sweeps=50, prec="mixed",
                       want_scalings=False, d=2):
    """qwb_primal_upscale_ipf: the primal upscaling upper bound from a coarse CSR plan."""
    dev = mu.device
    rp = torch.as_tensor(np.asarray(rowptr, dtype=np.int32), device=dev)
    cl = torch.as_tensor(np.asarray(col, dtype=np.int32), device=dev)
    vl = torch.as_tensor(np.asarray(val, dtype=np.float64), device=dev)
    a = b = None
    if want_scalings:
        a = torch.empty(N ** d, dtype=torch.float64, device=dev)
        b = torch.empty(N ** d, dtype=torch.float64, device=dev)
    res = QwbResult()
    pr = problem(N, kappa, p, d)
    check(_lib.load().qwb_primal_upscale_ipf(context(dev), ctypes.byref(pr), _dev64(mu, "mu"),
                                             _dev64(nu, "nu"), _ptr(rp), _ptr(cl), _ptr(vl),
                                             int(vl.numel()), int(sweeps), _ptr(a), _ptr(b),
                                             ctypes.byref(res), _prec(prec), _stream(mu)),
          "qwb_primal_upscale_ipf")
    out = res.as_dict()
    if want_scalings:
        out["a"], out["b"] = a, b
    return out


def primal_upscale_ipf_kernel(mu, nu, N, kappa, p, rowptr, col, val, K, sweeps=50, prec="mixed",
                              want_scalings=False):
    """qwb_primal_upscale_ipf_kernel: the primal upscaling upper bound with a
    general positive upscaling kernel K [kappa^2, kappa^2] (d = 2, kappa <= 8)."""
    dev = mu.device
    rp = torch.as_tensor(np.asarray(rowptr, dtype=np.int32), device=dev)
    cl = torch.as_tensor(np.asarray(col, dtype=np.int32), device=dev)
    vl = torch.as_tensor(np.asarray(val, dtype=np.float64), device=dev)
    Kd = torch.as_tensor(np.ascontiguousarray(K, dtype=np.float64), device=dev).contiguous()
    if Kd.shape != (kappa * kappa, kappa * kappa):
        raise ValueError("K must be [kappa^2, kappa^2]")
    a = b = None
    if want_scalings:
        a = torch.empty(N * N, dtype=torch.float64, device=dev)
        b = torch.empty(N * N, dtype=torch.float64, device=dev)
    res = QwbResult()
    pr = problem(N, kappa, p, 2)
    check(_lib.load().qwb_primal_upscale_ipf_kernel(context(dev), ctypes.byref(pr), _dev64(mu, "mu"),
                                                    _dev64(nu, "nu"), _ptr(rp), _ptr(cl), _ptr(vl),
                                                    int(vl.numel()), _ptr(Kd), int(sweeps), _ptr(a),
                                                    _ptr(b), ctypes.byref(res), _prec(prec),
                                                    _stream(mu)),
          "qwb_primal_upscale_ipf_kernel")
    out = res.as_dict()
    if want_scalings:
        out["a"], out["b"] = a, b
    return out


def dual_upscale_ctransform(mu, nu, N, kappa, p, f_coarse, prec="mixed", want_potentials=True, d=2):
    """qwb_dual_upscale_ctransform: the dual upscaling lower bound from a coarse potential."""
    dev = mu.device
    fc = torch.as_tensor(np.asarray(f_coarse, dtype=np.float64), device=dev) \
        if not isinstance(f_coarse, torch.Tensor) else f_coarse
    f = g = None
    if want_potentials:
        f = torch.empty(N ** d, dtype=torch.float64, device=dev)
        g = torch.empty(N ** d, dtype=torch.float64, device=dev)
    res = QwbResult()
    pr = problem(N, kappa, p, d)
    check(_lib.load().qwb_dual_upscale_ctransform(context(dev), ctypes.byref(pr), _dev64(mu, "mu"),
                                                  _dev64(nu, "nu"), _dev64(fc, "f_coarse"),
                                                  _ptr(f), _ptr(g), ctypes.byref(res),
                                                  _prec(prec), _stream(mu)),
          "qwb_dual_upscale_ctransform")
    out = res.as_dict()
    if want_potentials:
        out["f"], out["g"] = f, g
    return out


def ctransform(h, N, p, prec="mixed"):
    """qwb_ctransform: out_j = min_i rho(x_i, x_j)^p - h_i, rounded down."""
    out = torch.empty(N * N, dtype=torch.float64, device=h.device)
    check(_lib.load().qwb_ctransform(context(h.device), int(N), float(p), _dev64(h, "h"),
                                     _ptr(out), _prec(prec), _stream(h)), "qwb_ctransform")
    return out


def ctransform_shape(h, N, p, R, TC, packing=0, in_rows=0, prec="mixed", d=2):
    """qwb_ctransform_shape: the lazy c-transform on [N]^d with an explicit launch shape."""
    out = torch.empty(N ** d, dtype=torch.float64, device=h.device)
    check(_lib.load().qwb_ctransform_shape(context(h.device), int(N), int(d), float(p), _dev64(h, "h"),
                                           _ptr(out), int(R), int(TC), int(packing), int(in_rows),
                                           _prec(prec), _stream(h)), "qwb_ctransform_shape")
    return out


def ctransform_separable(h, N, prec="mixed"):
    """qwb_ctransform_separable: the p = 2 c-transform by separation over the grid axes."""
    out = torch.empty(N * N, dtype=torch.float64, device=h.device)
    check(_lib.load().qwb_ctransform_separable(context(h.device), int(N), _dev64(h, "h"), _ptr(out),
                                               _prec(prec), _stream(h)), "qwb_ctransform_separable")
    return out


def lb_adjoint(f, mu, N, p, lb_p):
    """qwb_lb_adjoint: gradient of the lower bound with respect to mu along the simplex."""
    grad = torch.empty(N * N, dtype=torch.float64, device=f.device)
    check(_lib.load().qwb_lb_adjoint(context(f.device), int(N), float(p), _dev64(f, "f"),
                                     _dev64(mu, "mu"), float(lb_p), _ptr(grad), _stream(f)),
          "qwb_lb_adjoint")
    return grad


def _ptr_array(tensors, name):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = _dev64(t, name).value
    return arr


class Batch:
    """The method for many pairs, split into its steps (qwb_batch_*)."""

    def __init__(self, problems, ipf_sweeps=50, prec="mixed", flags=0, device=None):
        self.problems = [problem(*pr) if not isinstance(pr, QwbProblem) else pr for pr in problems]
        self.n = len(self.problems)
        arr = (QwbProblem * self.n)(*self.problems)
        self._h = ctypes.c_void_p()
        self._dev = torch.device("cuda", torch.cuda.current_device() if device is None else
                                 torch.device(device).index or 0)
        check(_lib.load().qwb_batch_create(context(self._dev), self.n, arr, int(ipf_sweeps),
                                           int(flags), _prec(prec), ctypes.byref(self._h)),
              "qwb_batch_create")

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self._dev).cuda_stream)

    def coarse(self, mus, nus, batched=True):
        check(_lib.load().qwb_batch_coarse(self._h, _ptr_array(mus, "mu"), _ptr_array(nus, "nu"),
                                           int(bool(batched)), self._stream()), "qwb_batch_coarse")

    def solve(self, threads=0):
        check(_lib.load().qwb_batch_solve(self._h, int(threads), self._stream()),
              "qwb_batch_solve")

    def fine(self, mus, nus, batched=True):
        check(_lib.load().qwb_batch_fine(self._h, _ptr_array(mus, "mu"), _ptr_array(nus, "nu"),
                                         int(bool(batched)), self._stream()), "qwb_batch_fine")

    def results(self):
        res = (QwbResult * self.n)()
        check(_lib.load().qwb_batch_results(self._h, res, self._stream()), "qwb_batch_results")
        return [r.as_dict() for r in res]

    KERNELS = ("sumpool", "cbar", "primal", "centre", "upsample", "ctransform_g",
               "ctransform_f", "lbsum", "ipf_cluster", "primal_kernel")

    def kernel_times(self):
        """Device ms of each kernel of the last batched passes (after a sync)."""
        out = (ctypes.c_double * 10)()
        check(_lib.load().qwb_batch_kernel_times(self._h, out, 10), "qwb_batch_kernel_times")
        return dict(zip(self.KERNELS, list(out)))

    def tuning(self):
        """The autotuner's choices and candidate timings for this batch (dict)."""
        import json
        buf = ctypes.create_string_buffer(65536)
        check(_lib.load().qwb_batch_tuning(self._h, buf, len(buf)), "qwb_batch_tuning")
        return json.loads(buf.value.decode())

    def potentials(self, t):
        N, d = self.problems[t].N, self.problems[t].d or 2
        f = torch.empty(N ** d, dtype=torch.float64, device=self._dev)
        g = torch.empty(N ** d, dtype=torch.float64, device=self._dev)
        check(_lib.load().qwb_batch_potentials(self._h, int(t), _ptr(f), _ptr(g), self._stream()),
              "qwb_batch_potentials")
        return f, g

    def coarse_plan(self, t):
        """Pair t's exact coarse plan of the last solve as a dense [M, M] numpy array."""
        n = ctypes.c_int32()
        L = _lib.load()
        check(L.qwb_batch_coarse_plan(self._h, int(t), None, None, None, 0, ctypes.byref(n)),
              "qwb_batch_coarse_plan")
        pr = self.problems[t]
        M = (pr.N // pr.kappa) ** (pr.d or 2)
        rowptr = np.zeros(M + 1, dtype=np.int32)
        col = np.zeros(max(1, n.value), dtype=np.int32)
        val = np.zeros(max(1, n.value), dtype=np.float64)
        check(L.qwb_batch_coarse_plan(self._h, int(t), rowptr.ctypes.data_as(_lib.P_int32),
                                      col.ctypes.data_as(_lib.P_int32), val.ctypes.data_as(_lib.P_double),
                                      int(len(col)), ctypes.byref(n)), "qwb_batch_coarse_plan")
        plan = np.zeros((M, M))
        for k in range(M):
            for e in range(rowptr[k], rowptr[k + 1]):
                plan[k, col[e]] = val[e]
        return plan

    def coarse_potentials(self, t):
        """Pair t's exact coarse dual potentials (f~, g~) of the last solve (numpy, M each)."""
        pr = self.problems[t]
        M = (pr.N // pr.kappa) ** (pr.d or 2)
        f = np.zeros(M)
        g = np.zeros(M)
        check(_lib.load().qwb_batch_coarse_potentials(self._h, int(t), f.ctypes.data_as(_lib.P_double),
                                                      g.ctypes.data_as(_lib.P_double)),
              "qwb_batch_coarse_potentials")
        return f, g

    def set_ipf_cluster(self, C):
        """Run the fine IPF sweeps inside the primal kernel (0) or on clusters of C CTAs."""
        check(_lib.load().qwb_batch_set_ipf_cluster(self._h, int(C)), "qwb_batch_set_ipf_cluster")

    def set_upscale_kernel(self, kappa, K):
        """Upscale the plans of the 2-D pairs with block side kappa by the
        general kernel K [kappa^2, kappa^2] (None: the uniform kernel)."""
        Kd = None
        if K is not None:
            Kd = torch.as_tensor(np.ascontiguousarray(K, dtype=np.float64), device=self._dev).contiguous()
            if Kd.shape != (kappa * kappa, kappa * kappa):
                raise ValueError("K must be [kappa^2, kappa^2]")
        check(_lib.load().qwb_batch_set_upscale_kernel(self._h, int(kappa), _ptr(Kd)),
              "qwb_batch_set_upscale_kernel")

    def set_upscale_cluster(self, C, threads=128):
        """Run the general-kernel primal pass one CTA per pair (C = 0), one CTA
        per pair for the sweeps with the evaluation spread over many CTAs
        (C = -1), or on clusters of C in {1, 2, 4, 8} CTAs of `threads`
        threads per pair."""
        check(_lib.load().qwb_batch_set_upscale_cluster(self._h, int(C), int(threads)),
              "qwb_batch_set_upscale_cluster")

    def fine_scalings(self, t):
        """Pair t's fine IPF scalings a, b (pass type widened to FP64)."""
        N, d = self.problems[t].N, self.problems[t].d or 2
        a = torch.empty(N ** d, dtype=torch.float64, device=self._dev)
        b = torch.empty(N ** d, dtype=torch.float64, device=self._dev)
        check(_lib.load().qwb_batch_fine_scalings(self._h, int(t), _ptr(a), _ptr(b), self._stream()),
              "qwb_batch_fine_scalings")
        return a, b

    def close(self):
        if self._h:
            _lib.load().qwb_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bounds(mus, nus, problems, ipf_sweeps=50, prec="mixed", batched=True, threads=0, flags=0):
    """qwb_bounds: every bound for every pair (list of result dicts)."""
    probs = [problem(*pr) if not isinstance(pr, QwbProblem) else pr for pr in problems]
    n = len(probs)
    res = (QwbResult * n)()
    check(_lib.load().qwb_bounds(context(mus[0].device), n, (QwbProblem * n)(*probs),
                                 _ptr_array(mus, "mu"), _ptr_array(nus, "nu"), int(ipf_sweeps),
                                 int(flags), res, _prec(prec), int(bool(batched)), int(threads),
                                 _stream(mus[0])), "qwb_bounds")
    return [r.as_dict() for r in res]


PROBE_KINDS = ("fma.rn.f32", "sub.rm.f32", "min.f32 (2 inputs)", "min.f32 (3 inputs)", "fma.rn.f32x2",
               "sub.rm.f32x2", "sub.rm.f32x2 + 3-input min (2 candidates)",
               "2 x sub.rm.f32 + 3-input min (2 candidates)",
               "c-transform inner block, fused subtraction-and-min (2 candidates)",
               "c-transform inner block, separate subtraction and min (2 candidates)")


def probe_fp32_rate(kind, ctas_per_sm=8, iters=2048):
    """Measured FP32 instruction rate of the current device (qwb_probe_fp32_rate):
    results per cycle per SM, results per second, the cycle counter's rate (MHz),
    the SM count and the CTA placement."""
    out = np.zeros(6)
    check(_lib.load().qwb_probe_fp32_rate(int(kind), int(ctas_per_sm), int(iters),
                                          out.ctypes.data_as(_lib.P_double)), "qwb_probe_fp32_rate")
    return {"kind": PROBE_KINDS[kind], "per_clk_per_sm": float(out[0]), "per_s": float(out[1]),
            "counter_mhz": float(out[2]), "sms": int(out[3]), "ctas_per_sm": int(out[4]),
            "most_ctas_on_one_sm": int(out[5])}


def kernel_launch_count():
    return int(_lib.load().qwb_kernel_launch_count())


class LowerBound(torch.autograd.Function):
    """Dual upscaling lower bound (Alg. 5) as a differentiable function of mu.

    forward(mu, nu, N, kappa, p, prec) -> LB (0-d float64 tensor).
    backward returns d LB / d mu along the simplex, computed by the adjoint
    kernel from the corrected potential f: (1/p) lb_p^(1/p-1) (f - <f, mu>).
    The coarse potential is held fixed (it is piecewise constant in mu).
    """

    @staticmethod
    def forward(ctx, mu, nu, N, kappa, p, prec="mixed"):
        flags = _lib.QWB_FLAG_NO_WEIGHTED | _lib.QWB_FLAG_NO_PRIMAL
        with Batch([(N, kappa, p)], ipf_sweeps=1, prec=prec, flags=flags, device=mu.device) as b:
            b.coarse([mu], [nu])
            b.solve()
            b.fine([mu], [nu])
            r = b.results()[0]
            f, _ = b.potentials(0)
        ctx.save_for_backward(mu, f)
        ctx.N, ctx.p, ctx.lb_p = N, p, r["lb_p"]
        return torch.tensor(r["lb"], dtype=torch.float64, device=mu.device)

    @staticmethod
    def backward(ctx, grad_out):
        mu, f = ctx.saved_tensors
        g = lb_adjoint(f, mu, ctx.N, ctx.p, ctx.lb_p)
        return grad_out * g, None, None, None, None, None
