"""Pins of the oracle's primal upscaling with a general normalized positive
kernel K (Sec. 3.4, eq. coupling tensor upscale): the uniform kernel
reproduces the uniform path, a separable kernel yields the uniform kernel's
fitted plan, IPF and the cost match a dense construction of pi-hat written
out entry by entry, and every bound sits above the exact LP value."""
import numpy as np
import pytest

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import synth


def dense_upscaled(plan_c, K, N, kappa):
    """pi-hat_ij = pi~_{k(i) l(j)} K[u(i), v(j)], entry by entry."""
    n = N // kappa
    P = np.zeros((N * N, N * N))
    for i in range(N * N):
        r, c = divmod(i, N)
        k, u = (r // kappa) * n + c // kappa, (r % kappa) * kappa + c % kappa
        for j in range(N * N):
            rr, cc = divmod(j, N)
            l, v = (rr // kappa) * n + cc // kappa, (rr % kappa) * kappa + cc % kappa
            P[i, j] = plan_c[k, l] * K[u, v]
    return P


def random_kernel(kappa, seed):
    K = np.random.default_rng(seed).uniform(0.2, 1.0, (kappa * kappa, kappa * kappa))
    return K / K.sum()


def pair(N, cls, seed):
    return synth.make_measure(N, cls, seed, 0), synth.make_measure(N, cls, seed, 1)


def coarse_plan(mu, nu, N, kappa, p):
    mt, nt = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    return O.exact_ot(O.coarse_cost_centre(N, kappa, p), mt, nt)[0]


@pytest.mark.parametrize("kappa", [2, 4])
def test_uniform_kernel_is_the_uniform_path(kappa):
    N, p = 16, 2.0
    mu, nu = pair(N, "gauss", 60)
    plan = coarse_plan(mu, nu, N, kappa, p)
    K = np.full((kappa ** 2, kappa ** 2), float(kappa) ** -4)
    u = O.ipf(mu, nu, plan, N, kappa, max_sweeps=7)
    k = O.ipf_K(mu, nu, plan, K, N, kappa, max_sweeps=7)
    np.testing.assert_allclose(k["a"], u["a"], rtol=1e-13)
    np.testing.assert_allclose(k["b"], u["b"], rtol=1e-13)
    cu = O.upscaled_cost(u["a"], u["b"], plan, N, kappa, p)
    ck = O.upscaled_cost_K(k["a"], k["b"], plan, K, N, kappa, p)
    assert abs(ck - cu) <= 1e-13 * cu


@pytest.mark.parametrize("kappa", [1, 2, 4])
def test_ipf_and_cost_match_dense_construction(kappa):
    """A non-symmetric random kernel: the blocked K-products, IPF and the
    support cost equal the same steps on the dense N^2 x N^2 matrix."""
    N, p, S = 8, 1.5, 5
    mu, nu = pair(N, "cauchy", 61)
    plan = coarse_plan(mu, nu, N, kappa, p)
    K = random_kernel(kappa, 62)
    P = dense_upscaled(plan, K, N, kappa)
    assert abs(P.sum() - 1.0) <= 1e-13                       # a coupling (normalized K)
    v = np.random.default_rng(63).uniform(0.5, 2.0, N * N)
    np.testing.assert_allclose(O.upscaled_plan_apply_K(plan, K, v, N, kappa), P @ v, rtol=1e-12)
    np.testing.assert_allclose(O.upscaled_plan_apply_KT(plan, K, v, N, kappa), P.T @ v, rtol=1e-12)
    b = np.ones(N * N)
    for _ in range(S):
        with np.errstate(divide="ignore", invalid="ignore"):
            a = np.where(P @ b > 0, mu / (P @ b), 0.0)
            b = np.where(P.T @ a > 0, nu / (P.T @ a), 0.0)
    fit = O.ipf_K(mu, nu, plan, K, N, kappa, xi=0.0, max_sweeps=S)
    np.testing.assert_allclose(fit["a"], a, rtol=1e-12)
    np.testing.assert_allclose(fit["b"], b, rtol=1e-12)
    X = O.grid_points(N)
    dense_cost = (a[:, None] * P * b[None, :] * O.ground_cost(X, X, p)).sum()
    assert abs(O.upscaled_cost_K(a, b, plan, K, N, kappa, p) - dense_cost) <= 1e-12 * dense_cost


def test_separable_kernel_yields_the_uniform_fitted_plan():
    """K = k_u (x) k_v: a_i k_u(u(i)) and b_j k_v(v(j)) absorb the factors, so
    the fitted plan diag(a) pi-hat diag(b) is the uniform kernel's."""
    N, kappa, p = 8, 4, 2.0
    mu, nu = pair(N, "field", 64)
    plan = coarse_plan(mu, nu, N, kappa, p)
    rng = np.random.default_rng(65)
    ku, kv = rng.uniform(0.3, 1.0, kappa ** 2), rng.uniform(0.3, 1.0, kappa ** 2)
    K = np.outer(ku, kv)
    K /= K.sum()
    Ku = np.full_like(K, 1.0 / K.size)
    fits = [O.ipf_K(mu, nu, plan, k, N, kappa, max_sweeps=3) for k in (K, Ku)]
    plans = [f["a"][:, None] * dense_upscaled(plan, k, N, kappa) * f["b"][None, :] for f, k in zip(fits, (K, Ku))]
    np.testing.assert_allclose(plans[0], plans[1], rtol=1e-11, atol=1e-18)


@pytest.mark.parametrize("N,kappa,p", [(8, 2, 2.0), (8, 4, 1.0), (12, 3, 2.0)])
def test_kernel_bound_above_exact(N, kappa, p):
    mu, nu = pair(N, "gauss", 66)
    W = O.wasserstein_exact(mu, nu, N, p)
    for K in (random_kernel(kappa, 67), O.gaussian_kernel(kappa, 0.7)):
        r = O.ub_primal_K(mu, nu, N, kappa, p, K, max_sweeps=3000)
        assert r["ub_primal"] >= W * (1 - 1e-12), (r["ub_primal"], W)
        assert r["w_hat"] >= W * (1 - 1e-12) - r["delta_mu"] - r["delta_nu"]


def test_kappa_one_zero_gap():
    """kappa = 1, K = [1]: the upscaled plan is the exact optimum, W-hat = W,
    and the corrections obey the proposition's bound in the IPF residual."""
    N, p = 8, 2.0
    mu, nu = pair(N, "cauchy", 68)
    r = O.ub_primal_K(mu, nu, N, 1, p, np.ones((1, 1)))
    W = O.wasserstein_exact(mu, nu, N, p)
    assert abs(r["w_hat"] - W) <= 1e-9 * W
    rad = np.sqrt(2.0) * (N - 1) / 2.0
    xi = r["residual"] * (1 + 1e-9) + 1e-300
    assert 0.0 <= r["ub_primal"] - r["w_hat"] <= 2 ** (2 - 2 / p) * xi ** (1 / p) * rad + 1e-15


def test_alignment_kernel_on_a_block_translation():
    """nu is mu moved down by one block (kappa rows), so W_2 = kappa.  The
    uniform kernel spreads each pixel over its target block; a kernel
    concentrated on equal offsets maps pixels onto their translates and gets
    close to W, below the uniform kernel's bound."""
    N, kappa, p = 16, 4, 2.0
    rng = np.random.default_rng(69)
    img = np.zeros((N, N))
    img[: N - kappa] = rng.uniform(0.1, 1.0, (N - kappa, N))
    img /= img.sum()
    mu = img.ravel()
    nu = np.roll(img, kappa, axis=0).ravel()
    W = O.wasserstein_exact(mu, nu, N, p)
    assert abs(W - kappa) <= 1e-9
    uni = O.ub_primal(mu, nu, N, kappa, p)["ub_primal"]
    ali = O.ub_primal_K(mu, nu, N, kappa, p, O.gaussian_kernel(kappa, 0.25), max_sweeps=3000)["ub_primal"]
    assert W <= ali < uni
    assert ali - W < 0.1 * (uni - W)
