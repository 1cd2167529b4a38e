"""Pins for the oracle's exact Kantorovich solver (Sec. 2.1), CPU only.

The solver (successive shortest paths, oracle/ssp.c) is checked against
things other than itself: the HiGHS LP solver shipped with scipy, the
one-dimensional quantile closed form, the 2 x 2 closed form, exact results for
translated measures, and the LP optimality certificates.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import synth


def _highs(C, a, b):
    n, m = C.shape
    A = sp.vstack([sp.kron(sp.eye(n), np.ones((1, m))), sp.kron(np.ones((1, n)), sp.eye(m))])
    r = linprog(C.ravel(), A_eq=A, b_eq=np.r_[a, b], bounds=(0, None), method="highs",
                options={"primal_feasibility_tolerance": 1e-10,
                         "dual_feasibility_tolerance": 1e-10})
    assert r.status == 0
    return r.fun


def _certificates(C, a, b, plan, f, g, obj):
    assert plan.min() >= 0.0
    assert np.abs(plan.sum(axis=1) - a).max() <= 1e-13
    assert np.abs(plan.sum(axis=0) - b).max() <= 1e-13
    slack = C - f[:, None] - g[None, :]
    assert slack.min() >= -1e-12 * max(1.0, C.max())
    # complementary slackness: no mass on arcs with positive reduced cost
    assert (plan * np.maximum(slack, 0)).sum() <= 1e-12 * max(1.0, C.max())
    dual = float(f @ a + g @ b)
    assert abs(dual - obj) <= 1e-10 * max(1.0, abs(obj))


@pytest.mark.parametrize("seed", range(6))
def test_random_dense_vs_highs(seed):
    rng = np.random.default_rng(seed)
    n, m = rng.integers(1, 40, size=2)
    C = rng.random((n, m)) * 10.0
    a = rng.random(n); a /= a.sum()
    b = rng.random(m); b /= b.sum()
    if seed % 2:
        a[rng.integers(0, n)] = 0.0
        a /= a.sum()
    plan, f, g, obj = O.exact_ot(C, a, b)
    assert abs(obj - _highs(C, a, b)) <= 1e-9 * max(1.0, abs(obj))
    _certificates(C, a, b, plan, f, g, obj)


@pytest.mark.parametrize("p", [1.0, 1.5, 2.0])
@pytest.mark.parametrize("cls", ["white", "gauss", "field"])
def test_grid_vs_highs(p, cls):
    N = 8
    mu, nu = synth.make_measure(N, cls, 90, 0), synth.make_measure(N, cls, 90, 1)
    X = O.grid_points(N)
    C = O.ground_cost(X, X, p)
    plan, f, g, obj = O.exact_ot(C, mu, nu)
    assert abs(obj - _highs(C, mu, nu)) <= 1e-9 * max(1.0, obj)
    _certificates(C, mu, nu, plan, f, g, obj)


def _w_pp_1d(xs, a, ys, b, p):
    """Textbook closed form in one dimension: integral over t of |F^-1(t) - G^-1(t)|^p."""
    ia = [i for i in range(len(xs)) if a[i] > 0]
    ib = [j for j in range(len(ys)) if b[j] > 0]
    ca, cb = np.cumsum(a[ia]), np.cumsum(b[ib])
    ca[-1] = cb[-1] = 1.0
    total, t, u, v = 0.0, 0.0, 0, 0
    while u < len(ia) and v < len(ib):
        nxt = min(ca[u], cb[v])
        total += (nxt - t) * abs(xs[ia[u]] - ys[ib[v]]) ** p
        t = nxt
        if ca[u] <= nxt:
            u += 1
        if cb[v] <= nxt:
            v += 1
    return total


@pytest.mark.parametrize("p", [1.0, 2.0, 3.0])
@pytest.mark.parametrize("seed", range(3))
def test_one_row_closed_form(p, seed):
    """Measures supported on one grid row: the LP equals the 1-D quantile formula."""
    N = 12
    rng = np.random.default_rng(100 + seed)
    mu = np.zeros((N, N)); nu = np.zeros((N, N))
    mu[3] = rng.random(N) * (rng.random(N) < 0.7)
    nu[3] = rng.random(N) * (rng.random(N) < 0.7)
    mu[3, 0] += 0.1; nu[3, N - 1] += 0.1
    mu, nu = mu.ravel() / mu.sum(), nu.ravel() / nu.sum()
    xs = np.arange(N, dtype=float)
    expect = _w_pp_1d(xs, mu.reshape(N, N)[3], xs, nu.reshape(N, N)[3], p)
    got = O.wasserstein_exact(mu, nu, N, p) ** p
    assert got == pytest.approx(expect, rel=1e-12, abs=1e-14)


def test_two_by_two_closed_form():
    """2 x 2 transport: the plan has one free entry t, the cost is linear in t."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        a0, b0 = rng.random(2)
        C = rng.random((2, 2))
        lo, hi = max(0.0, a0 + b0 - 1.0), min(a0, b0)

        def cost(t):
            return (t * C[0, 0] + (a0 - t) * C[0, 1] + (b0 - t) * C[1, 0]
                    + (1.0 - a0 - b0 + t) * C[1, 1])
        expect = min(cost(lo), cost(hi))
        _, _, _, obj = O.exact_ot(C, np.array([a0, 1 - a0]), np.array([b0, 1 - b0]))
        assert obj == pytest.approx(expect, rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("p", [1.0, 2.0])
def test_translation_exact(p):
    """nu = mu translated by an integer vector t (support kept inside): W_p = |t|."""
    N = 10
    rng = np.random.default_rng(3)
    img = np.zeros((N, N))
    img[1:6, 2:6] = rng.random((5, 4)) + 0.1
    t = (3, 2)
    sh = np.zeros((N, N))
    sh[1 + t[0]:6 + t[0], 2 + t[1]:6 + t[1]] = img[1:6, 2:6]
    mu, nu = img.ravel() / img.sum(), sh.ravel() / sh.sum()
    assert O.wasserstein_exact(mu, nu, N, p) == pytest.approx(np.hypot(*t), rel=1e-12)


def test_dirac_to_dirac():
    N = 9
    mu = np.zeros(N * N); nu = np.zeros(N * N)
    mu[2 * N + 1] = 1.0; nu[7 * N + 5] = 1.0
    for p in (1.0, 2.0, 1.5):
        assert O.wasserstein_exact(mu, nu, N, p) == pytest.approx(np.hypot(5, 4), rel=1e-13)
