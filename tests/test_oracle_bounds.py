"""Pins for the oracle's bounds (Sec. 3.2-3.5, Alg. 3-5), CPU only.

Each pin is something the paper or the mathematics fixes independently of the
oracle: the exact LP value (W), theorem inequalities, the zero gap at
kappa = 1, the one-sweep fixed point of IPF under the uniform kernel, a
separable transform for p = 2, closed-form c-transforms of affine potentials,
Villani's weighted-TV bound and finite differences.
"""
import json
import os

import numpy as np
import pytest

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("p", [1.0, 2.0, 1.5])
@pytest.mark.parametrize("cls", ["white", "gauss", "cauchy", "field", "blobs3"])
def test_bound_ordering_small(p, cls):
    """LB_dual, LB_min <= W <= UB_weighted <= UB_primal (Theorems of Sec. 3.2-3.5)."""
    N, kappa = 12, 3
    mu, nu = synth.make_measure(N, cls, 97, 0), synth.make_measure(N, cls, 97, 1)
    W = O.wasserstein_exact(mu, nu, N, p)
    b = O.bounds(mu, nu, N, kappa, p)
    tol = 1e-10 * max(1.0, W)
    assert b["lb"] <= W + tol
    assert O.lb_mincost(mu, nu, N, kappa, p) <= W + tol
    assert W <= b["ub_weighted"] + tol
    assert b["ub_weighted"] <= b["ub_primal"] + tol


@pytest.mark.parametrize("p", [1.0, 2.0])
@pytest.mark.parametrize("cls", ["gauss", "field"])
def test_kappa_one_zero_gap(p, cls):
    """Coarse grid = fine grid: every quantization bound equals W_p."""
    N = 8
    mu, nu = synth.make_measure(N, cls, 98, 0), synth.make_measure(N, cls, 98, 1)
    W = O.wasserstein_exact(mu, nu, N, p)
    b = O.bounds(mu, nu, N, 1, p)
    for key in ("lb", "ub_weighted"):
        assert b[key] == pytest.approx(W, rel=1e-9, abs=1e-9), key
    w_hat = b["w_hat_p"] ** (1 / p)
    assert w_hat == pytest.approx(W, rel=1e-9, abs=1e-9)
    # the corrections obey the proposition: Delta_mu + Delta_nu < 2^(2-2/p) xi^(1/p) r
    r = np.sqrt(2.0) * (N - 1) / 2.0
    xi = b["ipf_residual"] * (1 + 1e-9) + 1e-300
    assert 0.0 <= b["ub_primal"] - w_hat <= 2 ** (2 - 2 / p) * xi ** (1 / p) * r + 1e-15


@pytest.mark.parametrize("cls", ["white", "gauss", "field"])
def test_ipf_fixed_point_after_one_sweep(cls):
    """Uniform kernel: a_i / mu_i is constant per block and the marginals are
    exact after the first sweep (fixed point alpha_k = kappa^d / mu~_k up to
    the shared scale)."""
    N, kappa = 16, 4
    mu, nu = synth.make_measure(N, cls, 99, 0), synth.make_measure(N, cls, 99, 1)
    mt, nt = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    plan, _, _, _ = O.exact_ot(O.coarse_cost_centre(N, kappa, 2), mt, nt)
    fit = O.ipf(mu, nu, plan, N, kappa, xi=1e-13, max_sweeps=50)
    assert fit["sweeps"] == 1
    assert fit["residual"] < 1e-13
    n = N // kappa
    ratio = (fit["a"] / mu).reshape(n, kappa, n, kappa)
    spread = ratio.max(axis=(1, 3)) - ratio.min(axis=(1, 3))
    assert spread.max() <= 1e-12 * ratio.max()


def test_ipf_matches_dense_upscaled_plan():
    """The block form of pi-hat v equals the dense kappa^-4 pi~_{k(i) l(j)} matrix,
    and diag(a) pi-hat diag(b) has marginals (mu, nu) (Alg. 4 steps 1-2)."""
    N, kappa = 6, 3
    n = N // kappa
    mu, nu = synth.make_measure(N, "gauss", 100, 0), synth.make_measure(N, "gauss", 100, 1)
    mt, nt = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    plan, _, _, _ = O.exact_ot(O.coarse_cost_centre(N, kappa, 2), mt, nt)
    rows, cols = np.divmod(np.arange(N * N), N)
    kidx = (rows // kappa) * n + cols // kappa
    dense = plan[kidx][:, kidx] / kappa ** 4
    assert dense.sum() == pytest.approx(1.0, abs=1e-14)
    v = np.random.default_rng(0).random(N * N)
    np.testing.assert_allclose(O.upscaled_plan_apply(plan, v, N, kappa), dense @ v, rtol=1e-13)
    np.testing.assert_allclose(O.upscaled_plan_apply_T(plan, v, N, kappa), dense.T @ v, rtol=1e-13)
    fit = O.ipf(mu, nu, plan, N, kappa)
    fitted = fit["a"][:, None] * dense * fit["b"][None, :]
    np.testing.assert_allclose(fitted.sum(axis=1), mu, rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(fitted.sum(axis=0), nu, rtol=1e-12, atol=1e-16)
    X = O.grid_points(N)
    cost = float((fitted * O.ground_cost(X, X, 2)).sum())
    assert O.upscaled_cost(fit["a"], fit["b"], plan, N, kappa, 2) == pytest.approx(cost, rel=1e-13)


@pytest.mark.parametrize("p", [1.0, 2.0])
@pytest.mark.parametrize("cls", ["gauss", "cauchy", "field"])
def test_primal_ub_equals_plan_on_cbar(p, cls):
    """Uniform kernel + converged IPF gives the quantization coupling, so
    W-hat^p = <pi~*, C-bar> (appendix lemma on the weighted-cost identity)."""
    N, kappa = 16, 4
    mu, nu = synth.make_measure(N, cls, 101, 0), synth.make_measure(N, cls, 101, 1)
    b = O.bounds(mu, nu, N, kappa, p)
    assert b["w_hat_p"] == pytest.approx(float((b["plan_coarse"] * b["cbar"]).sum()), rel=1e-12)
    assert b["delta_mu"] < 1e-5 and b["delta_nu"] < 1e-5


@pytest.mark.parametrize("p", [1.0, 2.0])
def test_tv_bounds(p):
    """TV_p^w(mu-hat, mu) >= W_p(mu-hat, mu) (Villani's weighted-TV bound) and
    TV <= 2^(1-1/p) r ||mu-hat - mu||_1^(1/p) (the radius step of the proposition)."""
    N = 8
    rng = np.random.default_rng(11)
    X = O.grid_points(N)
    r = np.sqrt(((X - X.mean(axis=0)) ** 2).sum(-1)).max()
    for _ in range(5):
        mu = synth.make_measure(N, "gauss", 102, int(rng.integers(0, 100)))
        mh = np.clip(mu * (1.0 + 0.3 * rng.standard_normal(N * N)), 0, None)
        mh /= mh.sum()
        tv = O.tv_correction(mh, mu, N, p)
        assert O.wasserstein_exact(mh, mu, N, p) <= tv * (1 + 1e-12)
        assert tv <= 2 ** (1 - 1 / p) * r * np.abs(mh - mu).sum() ** (1 / p) * (1 + 1e-12)


def test_upsample_reproduces_affine_and_nodes():
    N, kappa = 16, 4
    Xc = O.block_centres(N, kappa)
    f_c = 3.0 - 2.0 * Xc[:, 0] + 0.5 * Xc[:, 1]
    X = O.grid_points(N)
    np.testing.assert_allclose(O.upsample_potential(f_c, N, kappa),
                               3.0 - 2.0 * X[:, 0] + 0.5 * X[:, 1], rtol=0, atol=1e-12)
    v = np.random.default_rng(1).random(N * N)
    np.testing.assert_array_equal(O.upsample_potential(v, N, 1), v)
    np.testing.assert_array_equal(O.upsample_potential(np.array([2.5]), 4, 4), np.full(16, 2.5))


def _separable_ctransform_p2(h, N):
    """p = 2 only: min over x1 of [(x1-y1)^2 + min over x2 of ((x2-y2)^2 - h(x1,x2))]."""
    H = h.reshape(N, N)
    ax = np.arange(N, dtype=float)
    sq = (ax[:, None] - ax[None, :]) ** 2                     # [x, y]
    inner = (sq[None, :, :] - H[:, :, None]).min(axis=1)      # [x1, y2]
    return (sq[:, :, None] + inner[:, None, :]).min(axis=0).ravel()   # [y1, y2]


@pytest.mark.parametrize("cls", ["white", "gauss", "field"])
def test_ctransform_separable_p2(cls):
    N = 16
    rng = np.random.default_rng(12)
    h = rng.standard_normal(N * N) * 30.0
    np.testing.assert_allclose(O.c_transform(h, N, 2), _separable_ctransform_p2(h, N),
                               rtol=0, atol=1e-9)


def test_ctransform_affine_closed_form():
    """p = 2, h(x) = 2<x,t>: h^c(y) = -2<y,t> - |t|^2 wherever y + t lies in the grid."""
    N = 12
    t = np.array([2.0, -3.0])
    X = O.grid_points(N)
    hc = O.c_transform(2.0 * X @ t, N, 2)
    inside = ((X + t >= 0) & (X + t <= N - 1)).all(axis=1)
    np.testing.assert_allclose(hc[inside], (-2.0 * X @ t - t @ t)[inside], atol=1e-9)


@pytest.mark.parametrize("p", [1.0, 2.0, 1.5])
def test_ctransform_triple_and_feasibility(p):
    N = 10
    h = np.random.default_rng(13).standard_normal(N * N) * 10.0
    g = O.c_transform(h, N, p)
    f = O.c_transform(g, N, p)
    np.testing.assert_allclose(O.c_transform(f, N, p), g, atol=1e-9)
    X = O.grid_points(N)
    C = O.ground_cost(X, X, p)
    assert (f[:, None] + g[None, :] - C).max() <= 1e-9
    assert (f >= h - 1e-9).all()                      # f = h^cc dominates h


@pytest.mark.parametrize("cls", ["gauss", "field"])
def test_lb_shift_invariance(cls):
    N, kappa = 12, 3
    mu, nu = synth.make_measure(N, cls, 103, 0), synth.make_measure(N, cls, 103, 1)
    mt = O.sumpool(mu, N, kappa)
    f_c = np.random.default_rng(2).standard_normal(mt.size) * 5
    a = O.lb_from_potential(mu, nu, N, kappa, 2, f_c)["lb_p"]
    b = O.lb_from_potential(mu, nu, N, kappa, 2, f_c + 123.25)["lb_p"]
    assert a == pytest.approx(b, abs=1e-9)


@pytest.mark.parametrize("p", [1.0, 2.0])
def test_gradient_fixed_potential_fd(p):
    """Central finite differences (h = 1e-6) of LB along e_i - mu with the coarse
    potential held fixed match lb_grad_mu."""
    N, kappa = 12, 3
    mu, nu = synth.make_measure(N, "field", 104, 0), synth.make_measure(N, "field", 104, 1)
    out = O.lb_dual(mu, nu, N, kappa, p)
    f_c = out["f_coarse"]
    grad = O.lb_grad_mu(mu, out["f"], out["lb_p"], p)
    h = 1e-6
    for i in np.random.default_rng(3).choice(N * N, 8, replace=False):
        e = np.zeros(N * N); e[i] = 1.0
        lp = O.lb_from_potential((mu + h * e) / (1 + h), nu, N, kappa, p, f_c)["lb"]
        lm = O.lb_from_potential((mu - h * e) / (1 - h), nu, N, kappa, p, f_c)["lb"]
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(grad[i], rel=1e-5, abs=1e-7)


@pytest.mark.slow
def test_small_blob_pair_against_full_lp():
    """32 x 32 three-blob pair, kappa = 4, p = 2: LB <= W (full 1024 x 1024 LP)
    <= UB_weighted <= UB_primal, matching the stored oracle values."""
    with open(os.path.join(GOLDEN, "blobs3_32_k4_p2.json")) as fh:
        gold = json.load(fh)
    N, kappa, p = 32, 4, 2.0
    mu, nu = synth.make_measure(N, "blobs3", 0, 0), synth.make_measure(N, "blobs3", 0, 1)
    b = O.bounds(mu, nu, N, kappa, p)
    W = gold["w_exact"]
    assert b["lb"] <= W <= b["ub_weighted"] <= b["ub_primal"]
    for key in ("lb", "ub_weighted", "ub_primal"):
        assert b[key] == pytest.approx(gold[key], rel=1e-9), key


def test_ctransform_at_closed_form_and_brute_force():
    """The one-output-at-a-time c-transform: the affine closed form (p = 2) on a
    grid too large for the full transform, and a brute-force double loop."""
    N = 200
    t = np.array([3.0, -5.0])
    X = O.grid_points(N)
    J = np.random.default_rng(14).choice(N * N, 40, replace=False)
    inside = ((X[J] + t >= 0) & (X[J] + t <= N - 1)).all(axis=1)
    got = O.c_transform_at(2.0 * X @ t, N, 2.0, J)
    np.testing.assert_allclose(got[inside], (-2.0 * X[J] @ t - t @ t)[inside], atol=1e-7)
    n = 5
    h = np.random.default_rng(15).standard_normal(n * n) * 4.0
    for p in (1.0, 1.5, 2.0):
        for j in range(n * n):
            xj, yj = divmod(j, n)
            brute = min(((xi - xj) ** 2 + (yi - yj) ** 2) ** (p / 2) - h[xi * n + yi]
                        for xi in range(n) for yi in range(n))
            assert O.c_transform_at(h, n, p, [j])[0] == pytest.approx(brute, abs=1e-12)


def test_dual_from_g_is_the_swapped_problem():
    """Starting from g~ is the f~ route of the swapped problem (the cost is
    symmetric): LB_g(mu, nu; g~) = LB_f(nu, mu; f~ = g~), with f and g
    exchanged; and both routes bound the exact W from below."""
    N, kappa, p = 12, 3, 2.0
    mu, nu = synth.make_measure(N, "gauss", 80, 0), synth.make_measure(N, "gauss", 80, 1)
    mt, nt = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    _, f_c, g_c, _ = O.exact_ot(O.coarse_cost_centre(N, kappa, p), mt, nt)
    a = O.lb_dual_from_g(mu, nu, N, kappa, p, g_c)
    b = O.lb_dual(nu, mu, N, kappa, p, f_c=g_c)
    assert a["lb_p"] == pytest.approx(b["lb_p"], rel=1e-13, abs=1e-12)
    np.testing.assert_allclose(a["f"], b["g"], atol=1e-10)
    np.testing.assert_allclose(a["g"], b["f"], atol=1e-10)
    W = O.wasserstein_exact(mu, nu, N, p)
    sym = O.lb_dual_symmetric(mu, nu, N, kappa, p, f_c=f_c, g_c=g_c)
    assert O.lb_dual(mu, nu, N, kappa, p, f_c=f_c)["lb"] <= sym["lb"] <= W + 1e-12
    assert a["lb"] <= W + 1e-12
