"""Failure paths on the GPU, made on the host (no GPU fault is provoked).

* A bounded device wait that runs out: with QWB_FAULT=ipf_bulk_skip_chunk=c
  the bulk-copy IPF sweeps never issue chunk c (no copy is ever in flight for
  it), so the mbarrier wait for it ends at the QWB_WAIT_TIMEOUT_MS limit of the
  global timer; the kernel returns, qwb_batch_results reports QWB_ERR_TIMEOUT
  for the batch, and the next batch on the same context is correct.
* Non-finite input: a NaN in a measure is refused as QWB_ERR_MASS.
* The certificate check (QWB_FLAG_VERIFY, or QWB_VERIFY=1): it passes on
  correct potentials, and with QWB_FAULT=verify_shift=1 (the check tightened
  by one cost unit) it reports QWB_ERR_VERIFY.
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


def _verify_cases():
    return [(16, 4, 2.0, "gauss"), (24, 4, 1.0, "field"), (32, 8, 1.5, "cauchy"), (32, 4, 2.0, "blobs3")]


@pytest.mark.parametrize("prec", ["mixed", "f64"])
@pytest.mark.parametrize("batched", [True, False])
def test_verify_mode_passes_and_changes_nothing(prec, batched):
    """QWB_FLAG_VERIFY re-checks f_i + g_j <= c_ij on every pair of fine
    points after each dual pass (both sides with the symmetric dual): every
    pair passes, and the bounds are those of the batch without the check."""
    mus, nus, probs = [], [], []
    for t, (N, kappa, p, cls) in enumerate(_verify_cases()):
        mus.append(T(synth.make_measure(N, cls, 66, 2 * t)))
        nus.append(T(synth.make_measure(N, cls, 66, 2 * t + 1)))
        probs.append((N, kappa, p))
    r0 = api.bounds(mus, nus, probs, ipf_sweeps=5, batched=batched, prec=prec, flags=32)
    r1 = api.bounds(mus, nus, probs, ipf_sweeps=5, batched=batched, prec=prec, flags=32 | api.QWB_FLAG_VERIFY)
    for a, b in zip(r0, r1):
        assert b["status"] == 0
        for key in ("lb", "lb_p", "ub_primal", "ub_weighted"):
            assert a[key] == b[key], key


def test_verify_mode_detects_a_violation(monkeypatch):
    """With QWB_FAULT=verify_shift=1 the check compares f_i + g_j with
    c_ij - 1, which the c-transform's tight pairs (slack below one rounding)
    fail: every pair reports QWB_ERR_VERIFY, through the environment switch
    QWB_VERIFY=1 as well; a batch made afterwards without the fault passes."""
    mus, nus, probs = [], [], []
    for t, (N, kappa, p, cls) in enumerate(_verify_cases()):
        mus.append(T(synth.make_measure(N, cls, 67, 2 * t)))
        nus.append(T(synth.make_measure(N, cls, 67, 2 * t + 1)))
        probs.append((N, kappa, p))
    monkeypatch.setenv("QWB_FAULT", "verify_shift=1")
    monkeypatch.setenv("QWB_VERIFY", "1")
    bad = api.bounds(mus, nus, probs, ipf_sweeps=3)
    assert all(r["status"] == 8 for r in bad), [r["status"] for r in bad]
    monkeypatch.delenv("QWB_FAULT")
    good = api.bounds(mus, nus, probs, ipf_sweeps=3)
    assert all(r["status"] == 0 for r in good)
