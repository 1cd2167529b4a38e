"""The allocation-free c-transform entry point (qwb_ctransform_noalloc).

It serves callers that cannot allocate device memory when they need a
c-transform (a frozen or exhausted memory pool, a plugin whose host owns the
device budget).  Called through the C ABI twice in a row, it must give the same
result as qwb_ctransform; sizes beyond its static scratch are rejected.  This
file is collected last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2506_00976_gb300 import _lib, api

pytestmark = pytest.mark.gpu


def _call(N, p, h, out):
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.qwb_ctransform_noalloc(int(N), float(p), ctypes.c_void_p(h.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), stream)


@pytest.mark.parametrize("N,p", [(64, 2.0), (32, 1.0), (12, 1.5), (256, 2.0)])
def test_noalloc_ctransform_matches_twice(N, p):
    rng = np.random.default_rng(N)
    for call in range(2):              # the static scratch keeps the previous call's contents
        h_np = (rng.standard_normal(N * N) * 2.0 * N).astype(np.float32).astype(np.float64)
        h = torch.tensor(h_np, device="cuda")
        ref = api.ctransform(h, N, p, prec="mixed")
        out = torch.full((N * N,), float("nan"), dtype=torch.float64, device="cuda")
        _lib.check(_call(N, p, h, out), "qwb_ctransform_noalloc")
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (call, float((out - ref).abs().max()))


def test_noalloc_rejects_oversize_grid():
    h = torch.zeros(300 * 300, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(h)
    assert _call(300, 2.0, h, out) == 7          # QWB_ERR_UNSUPPORTED
    assert b"256" in _lib.load().qwb_last_error()
