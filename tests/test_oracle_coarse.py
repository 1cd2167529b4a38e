"""Pins for the oracle's coarsening and coarse costs (Sec. 2.2, Sec. 3.2-3.4), CPU only."""
import itertools

import numpy as np
import pytest

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import synth


def test_sumpool_hand_example():
    mu = np.arange(16, dtype=float)              # 4 x 4 grid, kappa = 2
    # blocks: rows 0-1/cols 0-1 -> 0+1+4+5; cols 2-3 -> 2+3+6+7; ...
    assert O.sumpool(mu, 4, 2).tolist() == [10.0, 18.0, 42.0, 50.0]
    assert O.block_centres(4, 2).tolist() == [[0.5, 0.5], [0.5, 2.5], [2.5, 0.5], [2.5, 2.5]]


@pytest.mark.parametrize("cls", synth.CLASSES)
def test_sumpool_mass(cls):
    mu = synth.make_measure(32, cls, 91, 0)
    assert O.sumpool(mu, 32, 4).sum() == pytest.approx(1.0, abs=1e-15)


def _block_moments(mu, N, kappa):
    n = N // kappa
    out = []
    for k1, k2 in itertools.product(range(n), range(n)):
        m0 = e1 = e2 = s2 = 0.0
        for r in range(k1 * kappa, (k1 + 1) * kappa):
            for c in range(k2 * kappa, (k2 + 1) * kappa):
                w = mu[r * N + c]
                m0 += w; e1 += w * r; e2 += w * c; s2 += w * (r * r + c * c)
        out.append((e1 / m0, e2 / m0, s2 / m0))
    return out


@pytest.mark.parametrize("cls", ["white", "gauss", "cauchy", "field"])
@pytest.mark.parametrize("N,kappa", [(8, 2), (12, 3), (16, 4)])
def test_cbar_p2_moment_closed_form(cls, N, kappa):
    """p = 2: C-bar_kl = E_k|x|^2 + E_l|y|^2 - 2 <E_k x, E_l y> (block moments)."""
    mu, nu = synth.make_measure(N, cls, 92, 0), synth.make_measure(N, cls, 92, 1)
    Cbar = O.coarse_cost_weighted(mu, nu, N, kappa, 2)
    A, B = _block_moments(mu, N, kappa), _block_moments(nu, N, kappa)
    for k, (x1, x2, xs) in enumerate(A):
        for l, (y1, y2, ys) in enumerate(B):
            expect = xs + ys - 2.0 * (x1 * y1 + x2 * y2)
            assert Cbar[k, l] == pytest.approx(expect, rel=1e-11, abs=1e-11)


@pytest.mark.parametrize("kappa", [2, 4])
def test_cbar_uniform_blocks(kappa):
    """Masses uniform within blocks: C-bar = |x~_k - y~_l|^2 + 2 * 2 * (kappa^2 - 1)/12."""
    N = 4 * kappa
    rng = np.random.default_rng(5)
    n = N // kappa
    blk_mu = rng.random((n, n)) + 0.1
    blk_nu = rng.random((n, n)) + 0.1
    mu = np.kron(blk_mu, np.ones((kappa, kappa))).ravel(); mu /= mu.sum()
    nu = np.kron(blk_nu, np.ones((kappa, kappa))).ravel(); nu /= nu.sum()
    Cbar = O.coarse_cost_weighted(mu, nu, N, kappa, 2)
    Xc = O.block_centres(N, kappa)
    d2 = ((Xc[:, None, :] - Xc[None, :, :]) ** 2).sum(-1)
    np.testing.assert_allclose(Cbar, d2 + 4.0 * (kappa ** 2 - 1) / 12.0, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("p", [1.0, 1.5, 2.0])
def test_cbar_kappa1_is_ground_cost(p):
    N = 6
    mu, nu = synth.make_measure(N, "white", 93, 0), synth.make_measure(N, "white", 93, 1)
    X = O.grid_points(N)
    np.testing.assert_allclose(O.coarse_cost_weighted(mu, nu, N, 1, p), O.ground_cost(X, X, p),
                               rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("p", [1.0, 1.5, 2.0])
@pytest.mark.parametrize("cls", ["gauss", "cauchy"])
def test_cbar_product_coupling_identity(p, cls):
    """<mu~ (x) nu~, C-bar> = <mu (x) nu, C> (the quantization-coupling identity
    of the appendix lemma with pi~ = mu~ (x) nu~)."""
    N, kappa = 12, 3
    mu, nu = synth.make_measure(N, cls, 94, 0), synth.make_measure(N, cls, 94, 1)
    Cbar = O.coarse_cost_weighted(mu, nu, N, kappa, p)
    mt, nt = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    X = O.grid_points(N)
    assert float(mt @ Cbar @ nt) == pytest.approx(float(mu @ O.ground_cost(X, X, p) @ nu),
                                                 rel=1e-12)


def test_cbar_transpose_symmetry():
    N, kappa = 12, 2
    mu, nu = synth.make_measure(N, "field", 95, 0), synth.make_measure(N, "field", 95, 1)
    for p in (1.0, 2.0):
        np.testing.assert_allclose(O.coarse_cost_weighted(mu, nu, N, kappa, p),
                                   O.coarse_cost_weighted(nu, mu, N, kappa, p).T, rtol=1e-13)


def test_cbar_zero_mass_block_uses_plain_mean():
    N, kappa = 8, 2
    mu = synth.make_measure(N, "gauss", 96, 0).reshape(N, N).copy()
    mu[0:2, 0:2] = 0.0
    mu = mu.ravel() / mu.sum()
    nu = synth.make_measure(N, "gauss", 96, 1)
    Cbar = O.coarse_cost_weighted(mu, nu, N, kappa, 2)
    # row 0 (the empty block) is the plain mean of |x - y|^2 over the block pair
    Xc = O.block_centres(N, kappa)
    d2 = ((Xc[0][None, :] - Xc) ** 2).sum(-1)
    np.testing.assert_allclose(Cbar[0], d2 + 4.0 * (kappa ** 2 - 1) / 12.0, rtol=1e-13)
    assert np.isfinite(Cbar).all()


@pytest.mark.parametrize("p", [1.0, 2.0, 1.5])
@pytest.mark.parametrize("N,kappa", [(8, 2), (12, 4)])
def test_ctilde_and_cmin_closed_forms(p, N, kappa):
    n = N // kappa
    K = np.array(list(itertools.product(range(n), range(n))), dtype=float)
    dk = np.abs(K[:, None, :] - K[None, :, :])
    ct = (kappa * np.sqrt((dk ** 2).sum(-1))) ** p
    np.testing.assert_allclose(O.coarse_cost_centre(N, kappa, p), ct, rtol=1e-13, atol=1e-12)
    gap = np.maximum(0.0, kappa * dk - (kappa - 1))
    np.testing.assert_allclose(O.coarse_cost_min(N, kappa, p), ((gap ** 2).sum(-1)) ** (p / 2),
                               rtol=1e-13, atol=1e-12)
