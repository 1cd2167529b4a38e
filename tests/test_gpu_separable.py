"""GPU tests of the separable p = 2 c-transform (exact reformulation of the
lazy c-transform of Sec. 4 over the two grid axes) and of the separable p = 2
C-bar (the same separation of the sum that defines C-bar in Sec. 3.2)
against the oracle's brute-force definitions, and of batches that use them
(QWB_FLAG_SEPARABLE)."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu
SEPARABLE = 16


def T(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _ulp32(x):
    return np.spacing(np.abs(np.asarray(x, dtype=np.float64)).astype(np.float32)).astype(np.float64)


@pytest.mark.parametrize("N", [1, 2, 7, 8, 12, 16, 33, 64])
def test_integer_potential_bit_exact(N):
    """Integer potentials: every candidate and minimum is an exact FP32
    integer, so the separable result equals the definition exactly."""
    h = np.random.default_rng(50 + N).integers(-4 * N * N, 4 * N * N, N * N).astype(np.float64)
    exact = O.c_transform(h, N, 2.0)
    for prec in ("mixed", "f64"):
        g = api.ctransform_separable(T(h), N, prec=prec).cpu().numpy()
        np.testing.assert_array_equal(g, exact)


@pytest.mark.parametrize("N", [5, 16, 33, 48])
@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_real_potential_certified(N, prec):
    """Real potentials: below the exact transform by at most two roundings of
    the largest candidate, and dual feasible on every pair."""
    rng = np.random.default_rng(60 + N)
    h = rng.standard_normal(N * N) * 3.0 * N
    if prec == "mixed":
        h = h.astype(np.float32).astype(np.float64)
    g = api.ctransform_separable(T(h), N, prec=prec).cpu().numpy()
    exact = O.c_transform(h, N, 2.0)
    X = O.grid_points(N)
    C = O.ground_cost(X, X, 2.0)
    big = C.max() + np.abs(h).max()
    assert np.all(g <= exact + 1e-12 * big)
    tol = 4 * _ulp32(big) if prec == "mixed" else 4 * np.spacing(big)
    assert np.all(g >= exact - tol), np.max(exact - g)
    assert (h[:, None] + g[None, :] - C).max() <= (0.0 if prec == "mixed" else 1e-12 * big)


def test_agrees_with_brute_force_kernel():
    """At 128 x 128 the separable and the N^4 kernels differ by at most two
    FP32 roundings of the largest candidate (both are round-down bounds)."""
    N = 128
    h = (np.random.default_rng(70).standard_normal(N * N) * 300.0).astype(np.float32).astype(np.float64)
    g1 = api.ctransform_separable(T(h), N).cpu().numpy()
    g2 = api.ctransform(T(h), N, 2.0).cpu().numpy()
    big = 2 * (N - 1) ** 2 + np.abs(h).max()
    assert np.max(np.abs(g1 - g2)) <= 4 * _ulp32(big)
    J = np.random.default_rng(71).choice(N * N, 32, replace=False)
    exact = O.c_transform_at(h, N, 2.0, J)
    assert np.all(g1[J] <= exact) and np.all(g1[J] >= exact - 4 * _ulp32(big))


def test_256_sampled():
    N = 256
    h = (np.random.default_rng(72).standard_normal(N * N) * 600.0).astype(np.float32).astype(np.float64)
    g = api.ctransform_separable(T(h), N).cpu().numpy()
    J = np.random.default_rng(73).choice(N * N, 32, replace=False)
    exact = O.c_transform_at(h, N, 2.0, J)
    big = 2 * (N - 1) ** 2 + np.abs(h).max()
    assert np.all(g[J] <= exact) and np.all(g[J] >= exact - 4 * _ulp32(big))


@pytest.mark.parametrize("batched", [True, False])
def test_batch_with_separable_flag(batched):
    """A batch of p = 1 and p = 2 pairs with QWB_FLAG_SEPARABLE: p = 1 pairs
    are unchanged, p = 2 lower bounds stay valid and within FP32 rounding of
    the brute-force ones; the primal upper bounds do not depend on the flag,
    and the weighted-cost bounds (the separable C-bar for kappa 4 and 8)
    agree to FP32 rounding and stay above W."""
    cases = [(16, 4, 2.0, "gauss"), (32, 4, 1.0, "cauchy"), (32, 8, 2.0, "field"), (24, 4, 2.0, "white")]
    mus, nus, probs, raw = [], [], [], []
    for t, (N, kappa, p, cls) in enumerate(cases):
        mu, nu = synth.make_measure(N, cls, 74, 2 * t), synth.make_measure(N, cls, 74, 2 * t + 1)
        raw.append((mu, nu)); mus.append(T(mu)); nus.append(T(nu)); probs.append((N, kappa, p))
    r0 = api.bounds(mus, nus, probs, ipf_sweeps=5, batched=batched)
    r1 = api.bounds(mus, nus, probs, ipf_sweeps=5, batched=batched, flags=SEPARABLE)
    for t, (N, kappa, p, cls) in enumerate(cases):
        assert r1[t]["status"] == 0
        assert r1[t]["ub_primal"] == r0[t]["ub_primal"]
        if p != 2.0:
            assert r1[t]["lb"] == r0[t]["lb"] and r1[t]["ub_weighted"] == r0[t]["ub_weighted"]
        else:
            assert abs(r1[t]["lb_p"] - r0[t]["lb_p"]) <= 1e-4 * max(1.0, abs(r0[t]["lb_p"]))
            assert abs(r1[t]["ub_weighted"] - r0[t]["ub_weighted"]) <= 1e-5 * r0[t]["ub_weighted"]
        if N <= 16:
            W = O.wasserstein_exact(raw[t][0], raw[t][1], N, p)
            assert r1[t]["lb"] <= W <= r1[t]["ub_weighted"] * (1 + 1e-12)


@pytest.mark.parametrize("N,kappa", [(16, 4), (32, 4), (24, 4), (64, 4), (128, 4), (36, 4),
                                     (32, 8), (48, 8), (8, 8), (64, 8)])
def test_coarse_cost_separable(N, kappa):
    """The separable p = 2 C-bar (row and column sums of each block, then the
    two axes' squared offsets) against the oracle's direct FP64 reduction
    over every fine pixel pair: every entry an upper bound, within FP32
    rounding (2e-5 relative) of it and of the direct FP32 kernel; power-of-two
    and other coarse sides (6, 9)."""
    mu, nu = synth.make_measure(N, "gauss", 76, 0), synth.make_measure(N, "field", 76, 1)
    got = api.coarse_cost_separable(T(mu), T(nu), N, kappa).cpu().numpy()
    ref = O.coarse_cost_weighted(mu, nu, N, kappa, 2.0)
    assert np.all(got >= ref * (1 - 1e-13))
    assert np.all(got <= ref * (1 + 2e-5) + 1e-300)
    direct = api.coarse_cost(T(mu), T(nu), N, kappa, 2.0, prec="mixed")[0].cpu().numpy()
    np.testing.assert_allclose(got, direct, rtol=2e-5)
    again = api.coarse_cost_separable(T(mu), T(nu), N, kappa).cpu().numpy()
    assert np.array_equal(got, again)


def test_coarse_cost_separable_zero_mass_and_refusals():
    """A zero-mass block takes the unweighted mean of rho^2 over the block
    pair, as the direct kernels do; p != 2, kappa 2 and volumes are refused."""
    N, kappa = 32, 4
    mu = synth.make_measure(N, "gauss", 77, 0).reshape(N, N).copy()
    mu[kappa:2 * kappa, 2 * kappa:3 * kappa] = 0.0
    mu = (mu / mu.sum()).ravel()
    nu = synth.make_measure(N, "gauss", 77, 1)
    got = api.coarse_cost_separable(T(mu), T(nu), N, kappa).cpu().numpy()
    ref = O.coarse_cost_weighted(mu, nu, N, kappa, 2.0)
    np.testing.assert_allclose(got, ref, rtol=2e-5)
    assert np.all(got >= ref * (1 - 1e-13))
    lib = _lib.load()
    for (n2, k2, p2, d2) in ((32, 4, 1.0, 2), (32, 2, 2.0, 2), (16, 4, 2.0, 3)):
        pr = api.problem(n2, k2, p2, d2)
        cb = torch.empty(1, dtype=torch.float64, device="cuda")
        assert lib.qwb_coarse_cost_separable(api.context(torch.device("cuda")), ctypes.byref(pr),
                                             ctypes.c_void_p(T(mu).data_ptr()), ctypes.c_void_p(T(nu).data_ptr()),
                                             ctypes.c_void_p(cb.data_ptr()), None) == 7
