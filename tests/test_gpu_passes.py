"""GPU parity of each pass against the FP64 oracle, through the C ABI.

Pass-level tests feed the CUDA path the oracle's own coarse solutions, so both
sides work on identical inputs.  Tolerances: the FP32 path within 1e-4
relative on the bounds, the FP64 path within 1e-6; the c-transform for p = 2
is bit-exact (round-down of the exact minimum); certification inequalities
are checked exactly.
"""
import numpy as np
import pytest
import torch

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import api, synth

pytestmark = pytest.mark.gpu

TOL = {"mixed": 1e-4, "f64": 1e-6}


def T(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def rd32(x):
    """Largest float32 value <= x (elementwise)."""
    y = np.asarray(x, dtype=np.float64).astype(np.float32)
    bad = y.astype(np.float64) > x
    y[bad] = np.nextafter(y[bad], np.float32(-np.inf))
    return y.astype(np.float64)


def fp32_values(rng, n, scale):
    return (rng.standard_normal(n) * scale).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("N", [1, 7, 8, 12, 16, 32, 64])
def test_ctransform_p2_bit_exact(N):
    h = fp32_values(np.random.default_rng(N), N * N, 3.0 * N)
    g = api.ctransform(T(h), N, 2.0, prec="mixed").cpu().numpy()
    np.testing.assert_array_equal(g, rd32(O.c_transform(h, N, 2.0)))


@pytest.mark.parametrize("N", [6, 16, 33])
@pytest.mark.parametrize("p", [1.0, 1.5, 3.0])
def test_ctransform_general_p(N, p):
    h = fp32_values(np.random.default_rng(7 * N), N * N, 2.0 * N)
    g = api.ctransform(T(h), N, p, prec="mixed").cpu().numpy()
    exact = O.c_transform(h, N, p)
    X = O.grid_points(N)
    C = O.ground_cost(X, X, p)
    scale = np.maximum(np.abs(exact), C.max())
    assert np.all(g <= exact + 1e-12 * scale)                      # rounded down
    assert np.all(g >= exact - 4 * np.spacing(scale.astype(np.float32)).astype(np.float64))
    assert (h[:, None] + g[None, :] - C).max() <= 1e-9              # feasible


@pytest.mark.parametrize("N", [8, 16])
@pytest.mark.parametrize("p", [1.0, 2.0])
def test_ctransform_f64(N, p):
    h = np.random.default_rng(3).standard_normal(N * N) * 10
    g = api.ctransform(T(h), N, p, prec="f64").cpu().numpy()
    exact = O.c_transform(h, N, p)
    X = O.grid_points(N)
    C = O.ground_cost(X, X, p)
    assert np.max(np.abs(g - exact)) <= 1e-12 * (1 + np.abs(exact).max() + C.max())
    assert (h[:, None] + g[None, :] - C).max() <= 1e-12 * (1 + C.max())


@pytest.mark.parametrize("N,kappa,p", [(8, 2, 2.0), (12, 3, 2.0), (16, 4, 1.0), (32, 4, 2.0),
                                        (32, 8, 2.0), (16, 1, 2.0), (24, 4, 1.5), (64, 4, 2.0),
                                        (24, 4, 2.0), (64, 4, 1.0), (4, 4, 2.0), (64, 8, 1.0),
                                        (48, 8, 2.0), (8, 8, 2.0)])
@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_coarse_cost(N, kappa, p, prec):
    mu, nu = synth.make_measure(N, "gauss", 20, 0), synth.make_measure(N, "field", 20, 1)
    cbar, mc, nc = api.coarse_cost(T(mu), T(nu), N, kappa, p, prec=prec)
    ref = O.coarse_cost_weighted(mu, nu, N, kappa, p)
    got = cbar.cpu().numpy()
    np.testing.assert_allclose(mc.cpu().numpy(), O.sumpool(mu, N, kappa), rtol=1e-14, atol=1e-17)
    np.testing.assert_allclose(nc.cpu().numpy(), O.sumpool(nu, N, kappa), rtol=1e-14, atol=1e-17)
    assert np.all(got >= ref * (1 - 1e-13))                         # an upper bound
    rel = 2e-5 if prec == "mixed" else 1e-12
    assert np.all(got <= ref * (1 + rel) + 1e-300)


@pytest.mark.parametrize("N,kappa", [(16, 4), (32, 8), (24, 4)])
def test_coarse_cost_zero_mass_block(N, kappa):
    mu = synth.make_measure(N, "gauss", 21, 0).reshape(N, N).copy()
    mu[kappa:2 * kappa, 2 * kappa:3 * kappa] = 0.0
    mu = (mu / mu.sum()).ravel()
    nu = synth.make_measure(N, "gauss", 21, 1)
    for prec in ("mixed", "f64"):
        got = api.coarse_cost(T(mu), T(nu), N, kappa, 2.0, prec=prec)[0].cpu().numpy()
        ref = O.coarse_cost_weighted(mu, nu, N, kappa, 2.0)
        np.testing.assert_allclose(got, ref, rtol=2e-5 if prec == "mixed" else 1e-12)


def _oracle_plan(mu, nu, N, kappa, p):
    mt, nt = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    plan, f, g, obj = O.exact_ot(O.coarse_cost_centre(N, kappa, p), mt, nt)
    return plan, f


def _csr(plan):
    rows, cols = np.nonzero(plan)
    rowptr = np.zeros(plan.shape[0] + 1, dtype=np.int32)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr).astype(np.int32), cols.astype(np.int32), plan[rows, cols]


@pytest.mark.parametrize("N,kappa,p,cls", [(16, 4, 2.0, "gauss"), (32, 4, 2.0, "field"),
                                            (32, 2, 1.0, "cauchy"), (64, 4, 2.0, "white"),
                                            (24, 3, 1.5, "gauss"), (8, 1, 2.0, "field")])
@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_primal_pass(N, kappa, p, cls, prec):
    mu, nu = synth.make_measure(N, cls, 22, 0), synth.make_measure(N, cls, 22, 1)
    plan, _ = _oracle_plan(mu, nu, N, kappa, p)
    ref = O.ub_primal(mu, nu, N, kappa, p, plan_c=plan)
    rowptr, col, val = _csr(plan)
    r = api.primal_upscale_ipf(T(mu), T(nu), N, kappa, p, rowptr, col, val, sweeps=50,
                               prec=prec, want_scalings=True)
    tol = TOL[prec]
    assert r["w_hat_p"] >= ref["w_hat_p"] * (1 - 1e-12)
    assert r["ub_primal"] >= ref["w_hat"] * (1 - 1e-12)
    assert abs(r["w_hat_p"] - ref["w_hat_p"]) <= tol * ref["w_hat_p"]
    assert abs(r["ub_primal"] - ref["ub_primal"]) <= tol * ref["ub_primal"]
    assert r["ipf_residual"] < 1e-12
    # the fitted plan's scalings are the oracle's fixed point
    np.testing.assert_allclose(r["a"].cpu().numpy() * (r["b"].cpu().numpy().sum()),
                               ref["a"] * ref["b"].sum(), rtol=1e-9, atol=0)


@pytest.mark.parametrize("N,kappa,p,cls", [(16, 4, 2.0, "gauss"), (32, 4, 2.0, "field"),
                                            (32, 2, 1.0, "cauchy"), (64, 4, 2.0, "white"),
                                            (24, 3, 1.5, "blobs3"), (8, 1, 2.0, "field"),
                                            (32, 32, 2.0, "gauss")])
@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_dual_pass(N, kappa, p, cls, prec):
    mu, nu = synth.make_measure(N, cls, 23, 0), synth.make_measure(N, cls, 23, 1)
    _, f_c = _oracle_plan(mu, nu, N, kappa, p)
    ref = O.lb_dual(mu, nu, N, kappa, p, f_c=f_c)
    r = api.dual_upscale_ctransform(T(mu), T(nu), N, kappa, p, f_c, prec=prec)
    tol = TOL[prec]
    fmax = np.abs(ref["f"]).max() + np.abs(ref["g"]).max()
    assert abs(r["lb_p"] - ref["lb_p"]) <= tol * max(abs(ref["lb_p"]), 1e-3) + 64 * 6e-8 * fmax * (prec == "mixed")
    if ref["lb"] > 0:
        assert abs(r["lb"] - ref["lb"]) <= tol * ref["lb"] + 1e-6 * (prec == "mixed")
    f, g = r["f"].cpu().numpy(), r["g"].cpu().numpy()
    atol = 8 * np.spacing(np.float32(fmax)) if prec == "mixed" else 1e-10 * (1 + fmax)
    np.testing.assert_allclose(f, ref["f"], rtol=0, atol=atol)
    np.testing.assert_allclose(g, ref["g"], rtol=0, atol=atol)
    if N <= 32:   # certificate: f_i + g_j <= c_ij on every pair
        X = O.grid_points(N)
        assert (f[:, None] + g[None, :] - O.ground_cost(X, X, p)).max() <= 1e-10


@pytest.mark.parametrize("N,p", [(64, 2.0), (128, 1.0), (32, 2.0)])
def test_coarse_cost_kappa4_variants(N, p, monkeypatch):
    """Every compiled variant of the kappa = 4 FP32 C-bar kernel (forced with
    QWB_CBAR_VARIANT) gives the same rounded-up coarse cost, bit for bit, at
    or above the oracle's and within 2e-5 of it; a zero-mass block takes the
    unweighted mean."""
    kappa = 4
    mu, nu = synth.make_measure(N, "gauss", 26, 0), synth.make_measure(N, "cauchy", 26, 1)
    mu = mu.reshape(N, N).copy(); mu[4:8, 8:12] = 0.0; mu = (mu / mu.sum()).ravel()
    ref = O.coarse_cost_weighted(mu, nu, N, kappa, p)
    got = {}
    for v in (2, 3, 6, 7, 8):
        monkeypatch.setenv("QWB_CBAR_VARIANT", str(v))
        cbar, _, _ = api.coarse_cost(T(mu), T(nu), N, kappa, p, prec="mixed")
        got[v] = cbar.cpu().numpy()
        assert np.all(got[v] >= ref * (1 - 1e-15)), v
        np.testing.assert_allclose(got[v], ref, rtol=2e-5, atol=0)
    for v in (3, 6, 7, 8):
        np.testing.assert_array_equal(got[v], got[2])


def test_invalid_inputs():
    from paper_2506_00976_gb300._lib import QwbError
    N = 8
    mu, nu = synth.make_measure(N, "gauss", 24, 0), synth.make_measure(N, "gauss", 24, 1)
    with pytest.raises(QwbError, match="MASS"):
        api.coarse_cost(T(mu * 1.01), T(nu), N, 2, 2.0)
    bad = mu.copy(); bad[3] = -1e-3; bad[4] += 1e-3
    with pytest.raises(QwbError, match="MASS"):
        api.coarse_cost(T(bad), T(nu), N, 2, 2.0)
    with pytest.raises(QwbError, match="INVALID_ARG"):
        api.coarse_cost(T(mu), T(nu), N, 3, 2.0)
    with pytest.raises(QwbError, match="INVALID_ARG"):
        api.ctransform(T(mu), N, 0.5)


SHAPES = [(R, TC, 0) for R, TC in [(1, 1), (2, 2), (4, 4), (8, 8), (16, 8), (16, 16), (8, 16)]] + \
         [(8, 8, 1), (16, 8, 1), (16, 16, 1)] + \
         [(8, 8, 2), (16, 8, 2), (8, 16, 2), (16, 16, 2)] + \
         [(8, 8, 3), (8, 8, 4), (8, 16, 4), (8, 16, 5), (16, 8, 5), (16, 16, 5), (8, 16, 6)] + \
         [(16, 16, 7), (16, 8, 7), (8, 16, 7), (16, 16, 8)]


@pytest.mark.parametrize("R,TC,packing", SHAPES)
@pytest.mark.parametrize("N,in_rows", [(32, 0), (32, 5), (64, 7), (64, 1)])
def test_ctransform_every_shape_p2(R, TC, packing, N, in_rows):
    """Every compiled launch shape gives the p = 2 transform bit for bit
    (round-down of the exact minimum), including odd line splits whose items
    combine by atomic min and the line-paired kernel's odd tail."""
    h = fp32_values(np.random.default_rng(100 + N + in_rows), N * N, 3.0 * N)
    g = api.ctransform_shape(T(h), N, 2.0, R, TC, packing, in_rows).cpu().numpy()
    np.testing.assert_array_equal(g, rd32(O.c_transform(h, N, 2.0)))


@pytest.mark.parametrize("R,TC,packing", SHAPES + [(16, 16, 9), (32, 16, 10), (16, 8, 11), (32, 8, 12)])
@pytest.mark.parametrize("N,in_rows", [(32, 5), (32, 3), (64, 7)])
def test_ctransform_integer_potentials_split(R, TC, packing, N, in_rows):
    """Integer potentials make many candidates exact zeros, which the
    round-down subtraction returns as -0.0; items that see part of the input
    lines combine their minima by atomic min, and -0.0 must not beat a
    negative partial minimum there (its signed-integer image is the most
    negative integer).  The transform must be the exact one, bit for bit, and
    feasible on every pixel pair."""
    h = np.round(fp32_values(np.random.default_rng(700 + N + in_rows), N * N, 3.0 * N))
    g = api.ctransform_shape(T(h), N, 2.0, R, TC, packing, in_rows).cpu().numpy()
    exact = O.c_transform(h, N, 2.0)
    np.testing.assert_array_equal(g, exact)
    X = O.grid_points(N)
    assert (h[:, None] + g[None, :] - O.ground_cost(X, X, 2.0)).max() <= 0.0


@pytest.mark.parametrize("R,TC,packing", [(16, 16, 9), (16, 8, 9), (8, 16, 9), (16, 16, 10), (32, 16, 10),
                                           (32, 8, 10), (16, 16, 11), (16, 8, 11), (8, 16, 11), (16, 16, 12),
                                           (32, 8, 12)])
@pytest.mark.parametrize("N,in_rows", [(32, 0), (32, 5), (64, 7), (64, 1), (128, 0)])
def test_ctransform_shifted_p2(R, TC, packing, N, in_rows):
    """The shifted line-paired kernels (p = 2): every candidate is
    fl_down(D - fl_up(h - A)) <= c - h, so the result never exceeds the exact
    transform and every pair stays feasible (checked on all pixel pairs for
    N <= 64); it lies below the once-rounded transform by at most the rounding
    of h - A plus that of the result: within 3 FP32 ulps of the magnitudes
    involved, and equal to it when every h - A is exact (integer h)."""
    h = fp32_values(np.random.default_rng(500 + N + in_rows), N * N, 3.0 * N)
    g = api.ctransform_shape(T(h), N, 2.0, R, TC, packing, in_rows).cpu().numpy()
    exact = O.c_transform(h, N, 2.0)
    assert np.all(g <= exact)
    scale = np.abs(h).max() + 2.0 * (N - 1) ** 2
    assert np.all(g >= exact - 3 * float(np.spacing(np.float32(scale))))
    if N <= 64:
        X = O.grid_points(N)
        assert (h[:, None] + g[None, :] - O.ground_cost(X, X, 2.0)).max() <= 0.0
    # integer potentials: h - A is exact, so the result is the once-rounded one
    hi = np.round(h)
    gi = api.ctransform_shape(T(hi), N, 2.0, R, TC, packing, in_rows).cpu().numpy()
    np.testing.assert_array_equal(gi, rd32(O.c_transform(hi, N, 2.0)))


@pytest.mark.parametrize("R,TC,packing", [(8, 8, 0), (16, 8, 1), (16, 8, 2), (8, 16, 2), (16, 16, 2),
                                           (8, 8, 3), (8, 16, 4), (16, 16, 5), (8, 16, 6), (16, 16, 7),
                                           (16, 16, 8)])
@pytest.mark.parametrize("p", [1.0, 1.5])
def test_ctransform_every_shape_general_p(R, TC, packing, p):
    N = 32
    h = fp32_values(np.random.default_rng(200), N * N, 2.0 * N)
    g = api.ctransform_shape(T(h), N, p, R, TC, packing, 3).cpu().numpy()
    ref = api.ctransform_shape(T(h), N, p, 1, 1, 0, 0).cpu().numpy()
    np.testing.assert_array_equal(g, ref)        # same round-down table, same minimum
    exact = O.c_transform(h, N, p)
    X = O.grid_points(N)
    C = O.ground_cost(X, X, p)
    assert np.all(g <= exact + 1e-12 * np.maximum(np.abs(exact), C.max()))
    assert (h[:, None] + g[None, :] - C).max() <= 1e-9


@pytest.mark.parametrize("R,TC,packing", [(8, 8, 0), (16, 8, 2), (8, 16, 2)])
@pytest.mark.parametrize("p", [2.0, 1.0])
def test_ctransform_every_shape_3d(R, TC, packing, p):
    """Line-paired packing across the lines of a volume ([N]^3, lines of N)."""
    N = 16
    h = fp32_values(np.random.default_rng(300), N ** 3, 2.0 * N)
    g = api.ctransform_shape(T(h), N, p, R, TC, packing, 5, d=3).cpu().numpy()
    exact = O.c_transform(h, N, p, d=3)
    if p == 2.0:
        np.testing.assert_array_equal(g, rd32(exact))
    else:
        ref = api.ctransform_shape(T(h), N, p, 1, 1, 0, 0, d=3).cpu().numpy()
        np.testing.assert_array_equal(g, ref)
        assert np.all(g <= exact + 1e-9)


def test_ctransform_shape_rejects():
    from paper_2506_00976_gb300._lib import QwbError
    h = T(np.zeros(64))
    with pytest.raises(QwbError, match="INVALID_ARG"):
        api.ctransform_shape(h, 8, 2.0, 3, 8, 0)            # R does not divide N
    with pytest.raises(QwbError, match="INVALID_ARG"):
        api.ctransform_shape(h, 8, 2.0, 8, 8, 2, prec="f64")  # packing is FP32 only
    with pytest.raises(QwbError, match="UNSUPPORTED"):
        api.ctransform_shape(h, 8, 2.0, 2, 8, 0)             # not compiled
    with pytest.raises(QwbError, match="UNSUPPORTED"):
        api.ctransform_shape(T(np.zeros(512)), 8, 2.0, 8, 8, 4, d=3)   # register-cut shapes are 2-D only
    with pytest.raises(QwbError, match="UNSUPPORTED"):
        api.ctransform_shape(T(np.zeros(256)), 16, 1.0, 16, 16, 9)     # shifted form: p = 2 only


@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_primal_pass_dense_coupling(prec):
    """The primal pass accepts any coupling of the coarse marginals, here the
    product coupling mu~ (x) nu~ with all M^2 entries (far more than the 2M - 1
    of a basic plan): the upscaled bound equals the oracle's for that plan."""
    N, kappa, p = 16, 4, 2.0
    mu, nu = synth.make_measure(N, "gauss", 25, 0), synth.make_measure(N, "field", 25, 1)
    mt, nt = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    plan = np.outer(mt, nt)
    ref = O.ub_primal(mu, nu, N, kappa, p, plan_c=plan)
    rowptr, col, val = _csr(plan)
    assert len(val) == plan.size
    r = api.primal_upscale_ipf(T(mu), T(nu), N, kappa, p, rowptr, col, val, sweeps=10, prec=prec)
    tol = TOL[prec]
    assert r["w_hat_p"] >= ref["w_hat_p"] * (1 - 1e-12)
    assert abs(r["ub_primal"] - ref["ub_primal"]) <= tol * ref["ub_primal"]
