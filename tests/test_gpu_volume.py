"""GPU parity on 3-D grids (volumes, d = 3) through the C ABI, against the
oracle's d-generic passes; pass-level tests feed both sides the oracle's own
coarse solution."""
import numpy as np
import pytest
import torch

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import api, synth

pytestmark = pytest.mark.gpu
D = 3
TOL = {"mixed": 1e-4, "f64": 1e-6}


def T(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _pair(N, cls, w):
    return synth.make_volume(N, cls, w, 0), synth.make_volume(N, cls, w, 1)


@pytest.mark.parametrize("N,kappa,p", [(8, 2, 2.0), (8, 4, 1.0), (12, 3, 2.0), (16, 4, 1.5)])
@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_coarse_cost_3d(N, kappa, p, prec):
    mu, nu = _pair(N, "density", 100)
    cbar, mc, nc = api.coarse_cost(T(mu), T(nu), N, kappa, p, prec=prec, d=D)
    ref = O.coarse_cost_weighted(mu, nu, N, kappa, p, D)
    got = cbar.cpu().numpy()
    np.testing.assert_allclose(mc.cpu().numpy(), O.sumpool(mu, N, kappa, D), rtol=1e-14, atol=0)
    assert np.all(got >= ref * (1 - 1e-15))                       # an upper bound
    rel = 2e-5 if prec == "mixed" else 1e-12
    np.testing.assert_allclose(got, ref, rtol=rel, atol=0)


def _oracle_plan(mu, nu, N, kappa, p):
    mt, nt = O.sumpool(mu, N, kappa, D), O.sumpool(nu, N, kappa, D)
    plan, f, g, _ = O.exact_ot(O.coarse_cost_centre(N, kappa, p, D), mt, nt)
    return plan, f, g


def _csr(plan):
    rows, cols = np.nonzero(plan)
    rowptr = np.zeros(plan.shape[0] + 1, dtype=np.int32)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr).astype(np.int32), cols.astype(np.int32), plan[rows, cols]


@pytest.mark.parametrize("N,kappa,p,cls", [(8, 2, 2.0, "density"), (12, 3, 1.0, "field3"),
                                            (16, 4, 2.0, "field3"), (8, 1, 2.0, "density")])
@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_primal_pass_3d(N, kappa, p, cls, prec):
    mu, nu = _pair(N, cls, 101)
    plan, _, _ = _oracle_plan(mu, nu, N, kappa, p)
    ref = O.ub_primal(mu, nu, N, kappa, p, plan_c=plan, d=D)
    rowptr, col, val = _csr(plan)
    r = api.primal_upscale_ipf(T(mu), T(nu), N, kappa, p, rowptr, col, val, sweeps=20,
                               prec=prec, want_scalings=True, d=D)
    tol = TOL[prec]
    assert r["w_hat_p"] >= ref["w_hat_p"] * (1 - 1e-12)
    assert abs(r["w_hat_p"] - ref["w_hat_p"]) <= tol * ref["w_hat_p"]
    assert abs(r["ub_primal"] - ref["ub_primal"]) <= tol * ref["ub_primal"]
    assert r["ipf_residual"] < 1e-12
    np.testing.assert_allclose(r["a"].cpu().numpy() * (r["b"].cpu().numpy().sum()),
                               ref["a"] * ref["b"].sum(), rtol=1e-9, atol=0)


@pytest.mark.parametrize("N,kappa,p,cls", [(8, 2, 2.0, "density"), (12, 3, 1.0, "field3"),
                                            (16, 4, 2.0, "density"), (8, 8, 2.0, "field3")])
@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_dual_pass_3d(N, kappa, p, cls, prec):
    mu, nu = _pair(N, cls, 102)
    _, f_c, _ = _oracle_plan(mu, nu, N, kappa, p)
    ref = O.lb_dual(mu, nu, N, kappa, p, f_c=f_c, d=D)
    r = api.dual_upscale_ctransform(T(mu), T(nu), N, kappa, p, f_c, prec=prec, d=D)
    fmax = np.abs(ref["f"]).max() + np.abs(ref["g"]).max()
    f, g = r["f"].cpu().numpy(), r["g"].cpu().numpy()
    atol = 8 * np.spacing(np.float32(fmax)) if prec == "mixed" else 1e-10 * (1 + fmax)
    np.testing.assert_allclose(f, ref["f"], rtol=0, atol=atol)
    np.testing.assert_allclose(g, ref["g"], rtol=0, atol=atol)
    tol = TOL[prec]
    assert abs(r["lb_p"] - ref["lb_p"]) <= tol * max(abs(ref["lb_p"]), 1e-3) + \
        (64 * 6e-8 * fmax if prec == "mixed" else 0.0)
    X = O.grid_points(N, D)
    assert (f[:, None] + g[None, :] - O.ground_cost(X, X, p)).max() <= 1e-10


@pytest.mark.parametrize("p", [1.0, 2.0])
@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_bounds_3d_certified(p, prec):
    """8^3 volumes, kappa 2: LB <= W (exact 512 x 512 LP) <= UB_w and W <= UB_p;
    UB_w (an LP value) matches the oracle."""
    N, kappa = 8, 2
    mu, nu = _pair(N, "density", 103)
    W = O.wasserstein_exact(mu, nu, N, p, d=D)
    r = api.bounds([T(mu)], [T(nu)], [(N, kappa, p, D)], ipf_sweeps=5, prec=prec)[0]
    assert r["status"] == 0
    assert r["lb"] <= W <= r["ub_weighted"] and W <= r["ub_primal"]
    ref = O.ub_weighted(mu, nu, N, kappa, p, D)["ub_weighted"]
    assert abs(r["ub_weighted"] - ref) <= TOL[prec] * ref


def test_mixed_dimension_batch_matches_single_pairs():
    """2-D and 3-D pairs in one batch (batched and plain forms, all flags of the
    lower bound) give the single-pair results bit for bit."""
    cases = [(8, 2, 2.0, 3, "density"), (16, 4, 1.0, 2, "gauss"), (12, 3, 1.0, 3, "field3"),
             (32, 4, 2.0, 2, "field"), (16, 4, 2.0, 3, "field3")]
    mus, nus, probs = [], [], []
    for t, (N, kappa, p, d, cls) in enumerate(cases):
        if d == 3:
            mu, nu = synth.make_volume(N, cls, 104, 2 * t), synth.make_volume(N, cls, 104, 2 * t + 1)
        else:
            mu, nu = synth.make_measure(N, cls, 104, 2 * t), synth.make_measure(N, cls, 104, 2 * t + 1)
        mus.append(T(mu)); nus.append(T(nu)); probs.append((N, kappa, p, d))
    for flags in (0, 16 | 32):
        rb = api.bounds(mus, nus, probs, ipf_sweeps=5, prec="mixed", batched=True, flags=flags)
        rp = api.bounds(mus, nus, probs, ipf_sweeps=5, prec="mixed", batched=False, flags=flags)
        for t in range(len(cases)):
            rs = api.bounds([mus[t]], [nus[t]], [probs[t]], ipf_sweeps=5, prec="mixed", flags=flags)[0]
            for k in ("lb", "ub_weighted", "ub_primal"):
                assert rb[t][k] == rs[k] == rp[t][k], (flags, t, k)


@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_separable_3d(prec):
    """The separable p = 2 transform in three stages on volumes: certified
    lower bounds within rounding of the lazy transform's."""
    N, kappa = 16, 4
    mu, nu = _pair(N, "density", 105)
    r0 = api.bounds([T(mu)], [T(nu)], [(N, kappa, 2.0, D)], ipf_sweeps=3, prec=prec)[0]
    r1 = api.bounds([T(mu)], [T(nu)], [(N, kappa, 2.0, D)], ipf_sweeps=3, prec=prec, flags=16)[0]
    assert r1["status"] == 0
    assert abs(r1["lb_p"] - r0["lb_p"]) <= (1e-4 if prec == "mixed" else 1e-10) * abs(r0["lb_p"])
    assert r1["ub_weighted"] == r0["ub_weighted"]


def test_volume_32_sampled():
    """32^3 volumes, kappa 4 (coarse 8^3): bounds ordered; sampled voxels of
    the dual pass against the oracle's one-at-a-time transform."""
    N, kappa, p = 32, 4, 2.0
    mu, nu = _pair(N, "density", 106)
    _, f_c, _ = _oracle_plan(mu, nu, N, kappa, p)
    r = api.dual_upscale_ctransform(T(mu), T(nu), N, kappa, p, f_c, d=D)
    fc = O.centre_potential(f_c, O.sumpool(mu, N, kappa, D))
    f_hat = O.upsample_potential(fc, N, kappa, D)
    J = np.random.default_rng(107).choice(N ** 3, 24, replace=False)
    g_ref = O.c_transform_at(f_hat, N, p, J, d=D)
    g = r["g"].cpu().numpy()
    # f-hat is rounded to FP32 on the device, so g is compared both ways
    scale = np.abs(f_hat).max() + np.abs(g_ref).max() + 3.0 * N * N
    np.testing.assert_allclose(g[J], g_ref, rtol=0, atol=8 * np.spacing(np.float32(scale)))
    b = api.bounds([T(mu)], [T(nu)], [(N, kappa, p, D)], ipf_sweeps=10)[0]
    assert b["status"] == 0 and 0 <= b["lb"] <= min(b["ub_weighted"], b["ub_primal"])


def test_plane_and_volume_of_same_side_do_not_share_state():
    """A 2-D call and a 3-D call with equal N, kappa and p use separate
    per-problem workspaces (the 3-D measures hold N^3 values)."""
    N, kappa = 8, 8
    h = np.random.default_rng(5).standard_normal(N * N).astype(np.float32).astype(np.float64)
    api.ctransform(T(h), N, 2.0)                   # 2-D workspace for (8, 8, 2)
    mu, nu = _pair(N, "field3", 103)
    _, f_c, _ = _oracle_plan(mu, nu, N, kappa, 2.0)
    r = api.dual_upscale_ctransform(T(mu), T(nu), N, kappa, 2.0, f_c, prec="mixed", d=D)
    ref = O.lb_dual(mu, nu, N, kappa, 2.0, f_c=f_c, d=D)
    fmax = np.abs(ref["f"]).max() + np.abs(ref["g"]).max()
    assert abs(r["lb_p"] - ref["lb_p"]) <= 1e-4 * max(abs(ref["lb_p"]), 1e-3) + 64 * 6e-8 * fmax
