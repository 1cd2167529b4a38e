"""Planted mistakes: each plausible error in the oracle must fail one of its pins.

The mistakes are planted in copies of oracle functions on the CPU (monkeypatch);
the checks below are the same kinds of pins the oracle tests use.
"""
import numpy as np
import pytest

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import synth


def _moment_closed_form_ok(mu, nu, N, kappa):
    n = N // kappa
    X = O.grid_points(N)

    def moments(w):
        W = w.reshape(n, kappa, n, kappa)
        m0 = W.sum(axis=(1, 3)).ravel()
        xs = [X[:, a].reshape(n, kappa, n, kappa) for a in (0, 1)]
        e = [(W * xa).sum(axis=(1, 3)).ravel() / m0 for xa in xs]
        s2 = (W * (xs[0] ** 2 + xs[1] ** 2)).sum(axis=(1, 3)).ravel() / m0
        return e, s2
    (a1, a2), sa = moments(mu)
    (b1, b2), sb = moments(nu)
    expect = sa[:, None] + sb[None, :] - 2 * (np.outer(a1, b1) + np.outer(a2, b2))
    return np.allclose(O.coarse_cost_weighted(mu, nu, N, kappa, 2), expect, rtol=1e-10, atol=1e-10)


def test_transposed_cbar_is_caught(monkeypatch):
    N, kappa = 8, 2
    mu, nu = synth.make_measure(N, "gauss", 110, 0), synth.make_measure(N, "gauss", 110, 1)
    assert _moment_closed_form_ok(mu, nu, N, kappa)
    orig = O.weighted_cost_numerators
    monkeypatch.setattr(O, "weighted_cost_numerators", lambda *a: orig(*a).T)
    assert not _moment_closed_form_ok(mu, nu, N, kappa)


def test_wrong_block_centre_offset_is_caught(monkeypatch):
    N, kappa = 16, 4
    Xc = O.block_centres(N, kappa)
    f_c = 1.0 + Xc[:, 0] - 2.0 * Xc[:, 1]
    X = O.grid_points(N)
    ok = lambda: np.allclose(O.upsample_potential(f_c, N, kappa), 1.0 + X[:, 0] - 2.0 * X[:, 1])
    assert ok()
    orig = np.arange

    def shifted_arange(*a, **k):       # t = (x - kappa/2)/kappa instead of (x - (kappa-1)/2)/kappa
        r = orig(*a, **k)
        return r - 0.5 if (len(a) == 1 and a[0] == N and not k) else r
    monkeypatch.setattr(O.np, "arange", shifted_arange)
    assert not ok()


def test_sign_error_in_ctransform_is_caught(monkeypatch):
    N = 10
    h = np.random.default_rng(0).standard_normal(N * N) * 5
    X = O.grid_points(N)
    C = O.ground_cost(X, X, 2)
    good = (C - h[:, None]).min(axis=0)
    assert np.allclose(O.c_transform(h, N, 2), good)
    orig = O.c_transform
    monkeypatch.setattr(O, "c_transform", lambda hh, NN, p, chunk=1024, d=2: orig(-hh, NN, p, chunk, d))
    g = O.c_transform(h, N, 2)
    assert (h[:, None] + g[None, :] - C).max() > 1e-6        # feasibility pin fails


def test_dropped_kernel_normalisation_is_caught(monkeypatch):
    N, kappa = 6, 3
    n = N // kappa
    mu, nu = synth.make_measure(N, "field", 111, 0), synth.make_measure(N, "field", 111, 1)
    plan, _, _, _ = O.exact_ot(O.coarse_cost_centre(N, kappa, 2), O.sumpool(mu, N, kappa),
                               O.sumpool(nu, N, kappa))
    rows, cols = np.divmod(np.arange(N * N), N)
    kidx = (rows // kappa) * n + cols // kappa
    dense = plan[kidx][:, kidx] / kappa ** 4
    v = np.random.default_rng(1).random(N * N)
    assert np.allclose(O.upscaled_plan_apply(plan, v, N, kappa), dense @ v)
    orig = O.upscaled_plan_apply
    monkeypatch.setattr(O, "upscaled_plan_apply",
                        lambda pc, vv, NN, kk, d=2: orig(pc, vv, NN, kk, d) * kk ** 4)
    assert not np.allclose(O.upscaled_plan_apply(plan, v, N, kappa), dense @ v)


def test_tv_weights_without_power_is_caught(monkeypatch):
    """Using rho instead of rho^p as TV weight (one reading of Sec. 3.1) breaks
    Villani's bound W_p <= TV_p^w for p = 2 on some pair."""
    N = 8
    rng = np.random.default_rng(2)
    orig = O.tv_weights
    monkeypatch.setattr(O, "tv_weights", lambda NN, p, d=2: orig(NN, 1.0, d))
    broken = False
    for t in range(20):
        mu = np.zeros(N * N); mh = np.zeros(N * N)
        mu[rng.integers(0, N * N)] = 1.0
        mh[rng.integers(0, N * N)] = 1.0
        if O.wasserstein_exact(mh, mu, N, 2) > O.tv_correction(mh, mu, N, 2) * (1 + 1e-12):
            broken = True
            break
    assert broken
