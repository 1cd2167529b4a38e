"""Failure paths on the GPU, made on the host (no GPU fault is provoked).

* A bounded device wait that runs out: with QWB_FAULT=ipf_bulk_skip_chunk=c
  the bulk-copy IPF sweeps never issue chunk c (no copy is ever in flight for
  it), so the mbarrier wait for it ends at the QWB_WAIT_TIMEOUT_MS limit of the
  global timer; the kernel returns, qwb_batch_results reports QWB_ERR_TIMEOUT
  for the batch, and the next batch on the same context is correct.
* Non-finite input: a NaN in a measure is refused as QWB_ERR_MASS.
"""
import time

import numpy as np
import pytest
import torch

from paper_2506_00976_gb300 import _lib, api, synth
from paper_2506_00976_gb300._lib import QwbError, QwbResult

pytestmark = pytest.mark.gpu


def T(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _pair(N, seed):
    return synth.make_measure(N, "gauss", seed, 0), synth.make_measure(N, "gauss", seed, 1)


def test_bulk_ipf_wait_times_out_and_context_recovers(monkeypatch):
    N, kappa, p = 128, 4, 2.0
    mu, nu = _pair(N, 61)
    md, nd = [T(mu)], [T(nu)]
    monkeypatch.setenv("QWB_WAIT_TIMEOUT_MS", "5")
    monkeypatch.setenv("QWB_FAULT", "ipf_bulk_skip_chunk=3")
    with api.Batch([(N, kappa, p)], ipf_sweeps=10, prec="mixed", flags=1 | 4) as b:
        b.coarse(md, nd)
        b.solve()
        b.set_ipf_cluster(4 | api.QWB_IPF_BULK)
        t0 = time.perf_counter()
        b.fine(md, nd)
        res = (QwbResult * 1)()
        st = _lib.load().qwb_batch_results(b._h, res, b._stream())
        elapsed = time.perf_counter() - t0
        assert st == 5, _lib.STATUS_NAMES.get(st, st)                 # QWB_ERR_TIMEOUT
        assert res[0].status == 5
        assert b"timed out" in _lib.load().qwb_last_error()
        assert elapsed < 30.0                                           # the wait was bounded
    monkeypatch.setenv("QWB_FAULT", "")
    monkeypatch.setenv("QWB_WAIT_TIMEOUT_MS", "2000")
    out = {}
    for form in (4 | api.QWB_IPF_BULK, 0):
        with api.Batch([(N, kappa, p)], ipf_sweeps=10, prec="mixed", flags=1 | 4) as b:
            b.coarse(md, nd)
            b.solve()
            b.set_ipf_cluster(form)
            b.fine(md, nd)
            r = b.results()[0]
            assert r["status"] == 0
            out[form] = r["ub_primal"]
    assert out[4 | api.QWB_IPF_BULK] == out[0]


def test_nan_measure_is_refused():
    N = 16
    mu, nu = _pair(N, 62)
    bad = mu.copy()
    bad[5] = np.nan
    with pytest.raises(QwbError, match="MASS"):
        api.coarse_cost(T(bad), T(nu), N, 4, 2.0)
    with pytest.raises(QwbError, match="MASS"):
        api.bounds([T(mu)], [T(np.where(np.arange(N * N) == 7, np.inf, nu))], [(N, 4, 2.0)], ipf_sweeps=2)
    r = api.bounds([T(mu)], [T(nu)], [(N, 4, 2.0)], ipf_sweeps=2)[0]   # the context still works
    assert r["status"] == 0 and 0 < r["lb"] <= r["ub_weighted"]
