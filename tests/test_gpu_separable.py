"""GPU tests of the separable p = 2 c-transform (exact reformulation of the
lazy c-transform of Sec. 4 over the two grid axes) against the oracle's
brute-force definition, and of batches that use it (QWB_FLAG_SEPARABLE)."""
import numpy as np
import pytest
import torch

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import api, synth

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
    the brute-force ones; the upper bounds do not depend on the flag."""
    cases = [(16, 4, 2.0, "gauss"), (32, 4, 1.0, "cauchy"), (32, 8, 2.0, "field"), (24, 4, 2.0, "white")]
    mus, nus, probs, raw = [], [], [], []
    for t, (N, kappa, p, cls) in enumerate(cases):
        mu, nu = synth.make_measure(N, cls, 74, 2 * t), synth.make_measure(N, cls, 74, 2 * t + 1)
        raw.append((mu, nu)); mus.append(T(mu)); nus.append(T(nu)); probs.append((N, kappa, p))
    r0 = api.bounds(mus, nus, probs, ipf_sweeps=5, batched=batched)
    r1 = api.bounds(mus, nus, probs, ipf_sweeps=5, batched=batched, flags=SEPARABLE)
    for t, (N, kappa, p, cls) in enumerate(cases):
        assert r1[t]["status"] == 0
        assert r1[t]["ub_weighted"] == r0[t]["ub_weighted"] and r1[t]["ub_primal"] == r0[t]["ub_primal"]
        if p != 2.0:
            assert r1[t]["lb"] == r0[t]["lb"]
        else:
            assert abs(r1[t]["lb_p"] - r0[t]["lb_p"]) <= 1e-4 * max(1.0, abs(r0[t]["lb_p"]))
        if N <= 16:
            W = O.wasserstein_exact(raw[t][0], raw[t][1], N, p)
            assert r1[t]["lb"] <= W
