"""The allocation-free c-transform entry point (qwb_ctransform_noalloc).

It serves callers that cannot allocate device memory when they need a
c-transform (a frozen or exhausted memory pool, a plugin whose host owns the
device budget).  Called through the C ABI twice in a row, it must give the same
result as qwb_ctransform; for p = 2 it must also equal the FP64 oracle's
transform rounded down to FP32, bit for bit; a large grid followed by a small
one must not see the large call's leftovers in the shared static scratch;
sizes beyond that scratch are rejected.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import _lib, api

pytestmark = pytest.mark.gpu


def _call(N, p, h, out):
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.qwb_ctransform_noalloc(int(N), float(p), ctypes.c_void_p(h.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), stream)


def _noalloc(N, p, h):
    out = torch.full((N * N,), float("nan"), dtype=torch.float64, device="cuda")
    _lib.check(_call(N, p, h, out), "qwb_ctransform_noalloc")
    torch.cuda.synchronize()
    return out


def _rd32(x):
    """Largest float32 value <= x (elementwise)."""
    y = np.asarray(x, dtype=np.float64).astype(np.float32)
    bad = y.astype(np.float64) > x
    y[bad] = np.nextafter(y[bad], np.float32(-np.inf))
    return y.astype(np.float64)


def _potential(rng, N):
    return torch.tensor((rng.standard_normal(N * N) * 2.0 * N).astype(np.float32).astype(np.float64),
                        device="cuda")


@pytest.mark.parametrize("N,p", [(64, 2.0), (32, 1.0), (12, 1.5), (256, 2.0), (256, 1.0), (256, 1.5)])
def test_noalloc_ctransform_matches_twice(N, p):
    rng = np.random.default_rng(N)
    for call in range(2):              # the static scratch keeps the previous call's contents
        h = _potential(rng, N)
        ref = api.ctransform(h, N, p, prec="mixed")
        out = _noalloc(N, p, h)
        assert torch.equal(out, ref), (call, float((out - ref).abs().max()))


@pytest.mark.parametrize("N", [16, 33])
def test_noalloc_ctransform_p2_matches_oracle(N):
    """p = 2 costs are exact FP32 integers: the result is the oracle's FP64
    transform rounded down, bit for bit."""
    rng = np.random.default_rng(100 + N)
    for _ in range(2):
        h = _potential(rng, N)
        out = _noalloc(N, 2.0, h).cpu().numpy()
        np.testing.assert_array_equal(out, _rd32(O.c_transform(h.cpu().numpy(), N, 2.0)))


def test_noalloc_large_then_small_grid():
    """A 256 x 256 call at p = 1.5 fills the scratch (cost tables, FP32 copies,
    work items); the 12 x 12 call after it must read none of that."""
    rng = np.random.default_rng(5)
    big = _potential(rng, 256)
    assert torch.equal(_noalloc(256, 1.5, big), api.ctransform(big, 256, 1.5, prec="mixed"))
    h = _potential(rng, 12)
    out = _noalloc(12, 1.5, h)
    assert torch.equal(out, api.ctransform(h, 12, 1.5, prec="mixed"))
    g = out.cpu().numpy()
    hn = h.cpu().numpy()
    exact = O.c_transform(hn, 12, 1.5)
    X = O.grid_points(12)
    C = O.ground_cost(X, X, 1.5)
    scale = np.maximum(np.abs(exact), C.max())
    assert np.all(g <= exact + 1e-12 * scale)                                  # rounded down
    assert np.all(g >= exact - 4 * np.spacing(scale.astype(np.float32)).astype(np.float64))
    assert (hn[:, None] + g[None, :] - C).max() <= 1e-9                         # feasible


def test_noalloc_rejects_oversize_grid():
    h = torch.zeros(300 * 300, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(h)
    assert _call(300, 2.0, h, out) == 7          # QWB_ERR_UNSUPPORTED
    assert b"256" in _lib.load().qwb_last_error()
