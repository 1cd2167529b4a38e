"""Pins of the oracle on 3-D grids (volumes; the paper's method on [N]^3).

Each check compares the oracle with something other than itself: closed forms,
an exact LP, brute force over voxel pairs, or invariants."""
import numpy as np
import pytest

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import synth

D = 3


def _vol(N, cls, w, i):
    return synth.make_volume(N, cls, w, i)


def test_grid_and_pooling_by_hand():
    N, kappa = 4, 2
    X = O.grid_points(N, D)
    assert X.shape == (64, 3)
    assert tuple(X[1 * 16 + 2 * 4 + 3]) == (1.0, 2.0, 3.0)        # row-major flat index
    mu = np.arange(64, dtype=np.float64)
    mt = O.sumpool(mu, N, kappa, D)
    # block (1, 0, 1): x1 in {2,3}, x2 in {0,1}, x3 in {2,3}
    want = sum(mu[a * 16 + b * 4 + c] for a in (2, 3) for b in (0, 1) for c in (2, 3))
    assert mt[1 * 4 + 0 * 2 + 1] == want
    assert mt.sum() == mu.sum()
    Xc = O.block_centres(N, kappa, D)
    assert tuple(Xc[1 * 4 + 0 * 2 + 1]) == (2.5, 0.5, 2.5)


@pytest.mark.parametrize("kappa", [2, 4])
def test_cbar_p2_centroid_variance_closed_form(kappa):
    """For p = 2, C-bar_kl = |c_k - c'_l|^2 + var_k + var'_l with c, var the
    block centroid and variance of each measure (E|X-Y|^2 of independent X, Y)."""
    N = 8
    mu, nu = _vol(N, "density", 90, 0), _vol(N, "field3", 90, 1)
    Cb = O.coarse_cost_weighted(mu, nu, N, kappa, 2.0, D)
    X = O.grid_points(N, D)
    n = N // kappa
    blk = (X // kappa).astype(int) @ np.array([n * n, n, 1])
    M = n ** 3

    def stats(w):
        c = np.zeros((M, 3)); v = np.zeros(M)
        for k in range(M):
            sel = blk == k
            wk = w[sel] / w[sel].sum()
            c[k] = wk @ X[sel]
            v[k] = wk @ ((X[sel] - c[k]) ** 2).sum(axis=1)
        return c, v
    c1, v1 = stats(mu)
    c2, v2 = stats(nu)
    want = ((c1[:, None, :] - c2[None, :, :]) ** 2).sum(-1) + v1[:, None] + v2[None, :]
    np.testing.assert_allclose(Cb, want, rtol=1e-11, atol=1e-10)


@pytest.mark.parametrize("p", [1.0, 1.5, 2.0])
def test_cbar_product_coupling_identity(p):
    """<mu~ (x) nu~, C-bar> = <mu (x) nu, C> (the weighted cost is an average)."""
    N, kappa = 4, 2
    mu, nu = _vol(N, "density", 91, 0), _vol(N, "density", 91, 1)
    Cb = O.coarse_cost_weighted(mu, nu, N, kappa, p, D)
    mt, nt = O.sumpool(mu, N, kappa, D), O.sumpool(nu, N, kappa, D)
    X = O.grid_points(N, D)
    assert mt @ Cb @ nt == pytest.approx(mu @ O.ground_cost(X, X, p) @ nu, rel=1e-12)


def test_cmin_and_centre_cost_closed_forms():
    N, kappa = 8, 2
    n = N // kappa
    K = np.array([(a, b, c) for a in range(n) for b in range(n) for c in range(n)], dtype=float)
    for p in (1.0, 2.0):
        gap = np.maximum(0.0, kappa * np.abs(K[:, None, :] - K[None, :, :]) - (kappa - 1))
        want = (gap ** 2).sum(-1) ** (p / 2)
        np.testing.assert_allclose(O.coarse_cost_min(N, kappa, p, D), want, atol=1e-12)
        cen = ((kappa * (K[:, None, :] - K[None, :, :])) ** 2).sum(-1) ** (p / 2)
        np.testing.assert_allclose(O.coarse_cost_centre(N, kappa, p, D), cen, atol=1e-12)


def test_trilinear_upsampling_reproduces_affine_and_identity():
    N, kappa = 8, 2
    Xc = O.block_centres(N, kappa, D)
    f_c = 0.5 + Xc @ np.array([1.0, -2.0, 0.25])
    X = O.grid_points(N, D)
    np.testing.assert_allclose(O.upsample_potential(f_c, N, kappa, D),
                               0.5 + X @ np.array([1.0, -2.0, 0.25]), atol=1e-12)
    h = np.random.default_rng(92).standard_normal(N ** 3)
    np.testing.assert_allclose(O.upsample_potential(h, N, 1, D), h, atol=0)
    # a non-affine value at one voxel against the explicit eight-corner formula
    F = np.random.default_rng(93).standard_normal((4, 4, 4))
    up = O.upsample_potential(F.ravel(), N, kappa, D).reshape(N, N, N)
    t = (np.array([3, 6, 0]) - 0.5) / 2.0
    k0 = np.clip(np.floor(t).astype(int), 0, 2)
    w = t - k0
    val = 0.0
    for e in np.ndindex(2, 2, 2):
        wt = np.prod([w[a] if e[a] else 1.0 - w[a] for a in range(3)])
        val += wt * F[k0[0] + e[0], k0[1] + e[1], k0[2] + e[2]]
    assert up[3, 6, 0] == pytest.approx(val, abs=1e-12)


def test_ctransform_3d_separable_and_affine():
    N = 5
    h = np.random.default_rng(94).standard_normal(N ** 3) * 4.0
    g = O.c_transform(h, N, 2.0, d=D)
    H = h.reshape(N, N, N)
    ax = np.arange(N, dtype=float)
    sq = (ax[:, None] - ax[None, :]) ** 2
    s1 = (sq[None, None, :, :] - H[:, :, :, None]).min(axis=2)                 # over x3
    s2 = (sq[None, :, :, None] + s1[:, :, None, :]).min(axis=1)                # over x2
    s3 = (sq[:, :, None, None] + s2[:, None, :, :]).min(axis=0)                # over x1
    np.testing.assert_allclose(g, s3.ravel(), atol=1e-10)
    t = np.array([1.0, -1.0, 2.0])
    X = O.grid_points(N, D)
    hc = O.c_transform(2.0 * X @ t, N, 2.0, d=D)
    inside = ((X + t >= 0) & (X + t <= N - 1)).all(axis=1)
    np.testing.assert_allclose(hc[inside], (-2.0 * X @ t - t @ t)[inside], atol=1e-9)
    J = [0, 17, 63, 124]
    np.testing.assert_allclose(O.c_transform_at(h, N, 1.0, J, d=D),
                               O.c_transform(h, N, 1.0, d=D)[J], atol=0)


@pytest.mark.parametrize("p", [1.0, 2.0])
def test_bounds_3d_bracket_exact_w(p):
    """8^3 volumes, kappa 2 (coarse 4^3): LB <= W (exact 512 x 512 LP) <= UB_w,
    W <= UB_p; the primal fixed point gives W-hat^p = <pi~*, C-bar>."""
    N, kappa = 8, 2
    mu, nu = _vol(N, "density", 95, 0), _vol(N, "density", 95, 1)
    r = O.bounds(mu, nu, N, kappa, p, d=D)
    W = O.wasserstein_exact(mu, nu, N, p, d=D)
    assert r["lb"] <= W * (1 + 1e-12) <= r["ub_weighted"] * (1 + 1e-12)
    assert W <= r["ub_primal"] * (1 + 1e-12)
    assert r["w_hat_p"] == pytest.approx(float((r["plan_coarse"] * r["cbar"]).sum()), rel=1e-10)
    assert r["ipf_residual"] < 1e-12
    assert O.lb_mincost(mu, nu, N, kappa, p, d=D) <= W * (1 + 1e-12)


def test_kappa_one_zero_gap_3d():
    N = 4
    mu, nu = _vol(N, "field3", 96, 0), _vol(N, "field3", 96, 1)
    W = O.wasserstein_exact(mu, nu, N, 2.0, d=D)
    r = O.bounds(mu, nu, N, 1, 2.0, d=D)
    assert r["lb"] == pytest.approx(W, rel=1e-9)
    assert r["ub_weighted"] == pytest.approx(W, rel=1e-9)
    # the TV corrections take a p-th root of rounding-level marginal errors
    assert r["ub_primal"] == pytest.approx(W, rel=1e-6)
