"""End-to-end GPU tests of the whole method (qwb_bounds / batches) and the
differentiable lower bound, against the FP64 oracle and exact LP values."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import api, synth

pytestmark = pytest.mark.gpu

TOL = {"mixed": 1e-4, "f64": 1e-6}   # relative, on the bounds
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def T(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_blob_pair_32_certified(prec):
    """32 x 32 three-blob pair, kappa 4, p 2: LB <= W (exact 1024 x 1024 LP)
    <= UB_weighted <= UB_primal; the weighted-cost bound (a unique LP value)
    matches the oracle."""
    with open(os.path.join(GOLDEN, "blobs3_32_k4_p2.json")) as fh:
        gold = json.load(fh)
    N, kappa, p = 32, 4, 2.0
    mu, nu = synth.make_measure(N, "blobs3", 0, 0), synth.make_measure(N, "blobs3", 0, 1)
    r = api.bounds([T(mu)], [T(nu)], [(N, kappa, p)], ipf_sweeps=50, prec=prec)[0]
    W = gold["w_exact"]
    assert r["status"] == 0
    assert r["lb"] <= W <= r["ub_weighted"] <= r["ub_primal"] * (1 + 1e-9)
    tol = 1e-6 if prec == "f64" else 1e-4
    assert abs(r["ub_weighted"] - gold["ub_weighted"]) <= tol * gold["ub_weighted"]
    # LB and UB_primal depend on which optimal coarse solution (the C~ LP is
    # degenerate on a grid) the solver returns; pass-level tests pin them on
    # identical inputs, here they are valid and close to the oracle's
    assert abs(r["lb"] - gold["lb"]) <= 5e-3 * gold["lb"]
    assert abs(r["ub_primal"] - gold["ub_primal"]) <= 5e-3 * gold["ub_primal"]


@pytest.mark.parametrize("p", [1.0, 2.0])
def test_batched_equals_plain(p):
    """The batched (graph-captured, persistent) form gives bit-identical results
    to one pair per launch."""
    N, kappa = 32, 4
    pairs = synth.class_pairs(N, "gauss", 30, count=4)
    mus = [T(a) for a, _ in pairs]
    nus = [T(b) for _, b in pairs]
    probs = [(N, kappa, p)] * len(pairs)
    rb = api.bounds(mus, nus, probs, ipf_sweeps=10, prec="mixed", batched=True)
    rp = api.bounds(mus, nus, probs, ipf_sweeps=10, prec="mixed", batched=False)
    for a, b in zip(rb, rp):
        for k in ("lb", "lb_p", "ub_weighted", "ub_primal", "w_hat_p"):
            assert a[k] == b[k], k


@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_uneven_batch_matches_single_pairs(prec):
    """Pairs of different N, kappa and p in one batch (the C-bar kernels of
    kappa 4, kappa 8 and other block sides in one pass; the c-transform's
    p = 2 and table launches): each result equals the single-pair result, and
    every bound is valid against the exact LP."""
    cases = [(16, 4, 2.0, "gauss"), (32, 8, 1.0, "cauchy"), (24, 4, 2.0, "field"),
             (16, 2, 1.0, "white"), (32, 4, 2.0, "blobs3"), (16, 8, 2.0, "field"),
             (48, 8, 1.5, "gauss")]
    mus, nus, probs, raw = [], [], [], []
    for t, (N, kappa, p, cls) in enumerate(cases):
        mu, nu = synth.make_measure(N, cls, 31, 2 * t), synth.make_measure(N, cls, 31, 2 * t + 1)
        raw.append((mu, nu))
        mus.append(T(mu)); nus.append(T(nu)); probs.append((N, kappa, p))
    rb = api.bounds(mus, nus, probs, ipf_sweeps=5, prec=prec, batched=True)
    for t, (N, kappa, p, cls) in enumerate(cases):
        rs = api.bounds([mus[t]], [nus[t]], [probs[t]], ipf_sweeps=5, prec=prec, batched=False)[0]
        for k in ("lb", "ub_weighted", "ub_primal"):
            assert rb[t][k] == rs[k], (t, k)
        if N <= 16:
            W = O.wasserstein_exact(raw[t][0], raw[t][1], N, p)
            assert rb[t]["lb"] <= W <= min(rb[t]["ub_weighted"], rb[t]["ub_primal"])


@pytest.mark.parametrize("cls", ["gauss", "field", "white"])
def test_small_grid_certified_all_classes(cls):
    N, kappa = 16, 4
    mu, nu = synth.make_measure(N, cls, 32, 0), synth.make_measure(N, cls, 32, 1)
    for p in (1.0, 2.0):
        W = O.wasserstein_exact(mu, nu, N, p)
        for prec in ("mixed", "f64"):
            r = api.bounds([T(mu)], [T(nu)], [(N, kappa, p)], ipf_sweeps=3, prec=prec)[0]
            assert r["lb"] <= W <= r["ub_weighted"] and W <= r["ub_primal"], (p, prec, r, W)


def test_kappa_one_zero_gap():
    N = 8
    mu, nu = synth.make_measure(N, "gauss", 33, 0), synth.make_measure(N, "gauss", 33, 1)
    W = O.wasserstein_exact(mu, nu, N, 2.0)
    r = api.bounds([T(mu)], [T(nu)], [(N, 1, 2.0)], ipf_sweeps=2, prec="f64")[0]
    assert r["lb"] <= W <= r["ub_weighted"]
    assert abs(r["lb"] - W) <= 1e-9 * W
    assert abs(r["ub_weighted"] - W) <= 1e-6 * W
    assert abs(r["ub_primal"] - W) <= 1e-6 * W


@pytest.mark.parametrize("p", [1.0, 2.0])
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_adjoint_kernel_fd(p, prec):
    """The adjoint kernel's gradient vs central finite differences of the
    oracle LB (h = 1e-6, FP64) along e_i - mu, for the same fixed coarse
    potential (the oracle's)."""
    N, kappa = 16, 4
    mu, nu = synth.make_measure(N, "field", 34, 0), synth.make_measure(N, "field", 34, 1)
    mt, nt = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    _, f_c, _, _ = O.exact_ot(O.coarse_cost_centre(N, kappa, p), mt, nt)
    r = api.dual_upscale_ctransform(T(mu), T(nu), N, kappa, p, f_c, prec=prec)
    grad = api.lb_adjoint(r["f"], T(mu), N, p, r["lb_p"]).cpu().numpy()
    ref = O.lb_dual(mu, nu, N, kappa, p, f_c=f_c)
    h = 1e-6
    for i in np.random.default_rng(5).choice(N * N, 20, replace=False):
        e = np.zeros(N * N); e[i] = 1.0
        lp = O.lb_from_potential((mu + h * e) / (1 + h), nu, N, kappa, p, ref["f_coarse"])["lb"]
        lm = O.lb_from_potential((mu - h * e) / (1 - h), nu, N, kappa, p, ref["f_coarse"])["lb"]
        fd = (lp - lm) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-3 if prec == "mixed" else 1e-5, abs=1e-6)


@pytest.mark.parametrize("p", [1.0, 2.0])
@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_adjoint_vs_oracle_64(p, prec):
    """At 64 x 64 the adjoint kernel's gradient, from the GPU dual pass on the
    oracle's coarse potential, against the oracle's gradient formula on the
    oracle's own potentials (lb_grad_mu, pinned to finite differences on the
    CPU), element by element."""
    N, kappa = 64, 4
    mu, nu = synth.make_measure(N, "field", 36, 0), synth.make_measure(N, "cauchy", 36, 1)
    mt, nt = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    _, f_c, _, _ = O.exact_ot(O.coarse_cost_centre(N, kappa, p), mt, nt)
    r = api.dual_upscale_ctransform(T(mu), T(nu), N, kappa, p, f_c, prec=prec)
    grad = api.lb_adjoint(r["f"], T(mu), N, p, r["lb_p"]).cpu().numpy()
    ref = O.lb_dual(mu, nu, N, kappa, p, f_c=f_c)
    want = O.lb_grad_mu(mu, ref["f"], ref["lb_p"], p)
    scale = np.abs(want).max()
    np.testing.assert_allclose(grad, want, rtol=0, atol=(1e-4 if prec == "mixed" else 1e-9) * scale)


def test_lower_bound_autograd():
    """LowerBound.apply: forward equals the batch LB; backward is the adjoint of
    its own potential; finite differences through the whole method (coarse
    re-solve included) agree wherever the coarse basis does not change."""
    N, kappa, p = 16, 4, 2.0
    mu, nu = synth.make_measure(N, "field", 35, 0), synth.make_measure(N, "field", 35, 1)
    mu_t = T(mu).requires_grad_(True)
    lb = api.LowerBound.apply(mu_t, T(nu), N, kappa, p, "f64")
    r = api.bounds([T(mu)], [T(nu)], [(N, kappa, p)], ipf_sweeps=1, prec="f64")[0]
    assert float(lb) == r["lb"]
    lb.backward()
    grad = mu_t.grad.cpu().numpy()
    assert np.isfinite(grad).all() and abs(float(grad @ mu)) <= 1e-9 * np.abs(grad).max()
    h = 1e-6
    agree = 0
    picks = np.random.default_rng(6).choice(N * N, 10, replace=False)
    for i in picks:
        e = np.zeros(N * N); e[i] = 1.0
        lp = float(api.LowerBound.apply(T((mu + h * e) / (1 + h)), T(nu), N, kappa, p, "f64"))
        lm = float(api.LowerBound.apply(T((mu - h * e) / (1 - h)), T(nu), N, kappa, p, "f64"))
        agree += abs((lp - lm) / (2 * h) - grad[i]) <= 1e-4 * (1 + abs(grad[i]))
    assert agree >= 8, agree


@pytest.mark.parametrize("p", [1.0, 2.0])
def test_mincost_lower_bound(p):
    """Min-cost lower bound (Sec. 3.3): the LP value is unique, so the library's
    certified value sits just below the oracle's and below the exact W; it is
    not above the dual-upscaling LB's coarse counterpart by more than rounding
    and is reported as 0 when the flag is off."""
    N, kappa = 16, 4
    for cls in ("gauss", "blobs3"):
        mu, nu = synth.make_measure(N, cls, 36, 0), synth.make_measure(N, cls, 36, 1)
        ref = O.lb_mincost(mu, nu, N, kappa, p)
        W = O.wasserstein_exact(mu, nu, N, p)
        r = api.bounds([T(mu)], [T(nu)], [(N, kappa, p)], ipf_sweeps=2, prec="f64",
                       flags=8)[0]
        assert r["status"] == 0
        assert r["lb_mincost"] <= ref * (1 + 1e-12) and r["lb_mincost"] <= W
        assert abs(r["lb_mincost"] - ref) <= 1e-9 * max(ref, 1e-300), (cls, r["lb_mincost"], ref)
        r0 = api.bounds([T(mu)], [T(nu)], [(N, kappa, p)], ipf_sweeps=2, prec="f64")[0]
        assert r0["lb_mincost"] == 0.0
        assert r0["lb"] == r["lb"]


def test_mincost_lower_bound_larger_grid():
    """32 x 32, kappa 2 (M = 256 coarse pixels per side of the LP): the grid
    network simplex's value matches the oracle's SSP value."""
    N, kappa, p = 32, 2, 2.0
    mu, nu = synth.make_measure(N, "cauchy", 37, 0), synth.make_measure(N, "cauchy", 37, 1)
    ref = O.lb_mincost(mu, nu, N, kappa, p)
    r = api.bounds([T(mu)], [T(nu)], [(N, kappa, p)], ipf_sweeps=2, prec="mixed", flags=8)[0]
    assert abs(r["lb_mincost"] - ref) <= 1e-9 * ref and r["lb_mincost"] <= ref * (1 + 1e-12)


@pytest.mark.parametrize("prec", ["f64", "mixed"])
@pytest.mark.parametrize("batched", [True, False])
def test_symmetric_dual(prec, batched):
    """QWB_FLAG_SYMMETRIC_DUAL (Sec. 3.5 from both coarse potentials): the
    bound is the larger of the two certified ones, so at least the one-sided
    bound of the same coarse solution and at most the exact W; the kept
    potentials are dual feasible on every pixel pair and reproduce lb_p; the
    upper bounds do not change."""
    N, kappa = 16, 4
    pairs = [(synth.make_measure(N, c, 81, 2 * t), synth.make_measure(N, c, 81, 2 * t + 1))
             for t, c in enumerate(["gauss", "cauchy", "field", "white", "blobs3", "gauss"])]
    X = O.grid_points(N)
    sides = 0
    for p in (1.0, 2.0):
        mus = [T(a) for a, _ in pairs]
        nus = [T(b) for _, b in pairs]
        probs = [(N, kappa, p)] * len(pairs)
        with api.Batch(probs, ipf_sweeps=3, prec=prec) as b0, \
                api.Batch(probs, ipf_sweeps=3, prec=prec, flags=32) as b1:
            for b in (b0, b1):
                b.coarse(mus, nus, batched=batched); b.solve(); b.fine(mus, nus, batched=batched)
            r0, r1 = b0.results(), b1.results()
            C = O.ground_cost(X, X, p)
            for t, (mu, nu) in enumerate(pairs):
                assert r1[t]["status"] == 0
                assert r1[t]["lb"] >= r0[t]["lb"] and r1[t]["lb_p"] >= r0[t]["lb_p"]
                assert r1[t]["ub_weighted"] == r0[t]["ub_weighted"]
                W = O.wasserstein_exact(mu, nu, N, p)
                assert r1[t]["lb"] <= W
                f, g = (x.cpu().numpy() for x in b1.potentials(t))
                assert (f[:, None] + g[None, :] - C).max() <= 1e-10
                s = float(f @ mu + g @ nu)
                assert r1[t]["lb_p"] <= s + 1e-12 and s - r1[t]["lb_p"] <= 1e-9 * (1 + abs(s))
                sides += r1[t]["lb_p"] > r0[t]["lb_p"]
    assert sides >= 1, "the side started from g~ never won: its path went unexercised"


@pytest.mark.parametrize("prec", ["f64", "mixed"])
@pytest.mark.parametrize("batched", [True, False])
def test_symmetric_dual_vs_oracle(prec, batched):
    """The dual pass from g~ against the oracle (Sec. 3.5 started from the
    other coarse potential).  Both sides consume the batch's own exact coarse
    potentials (f~, g~): the batch's lb_p equals the oracle's
    lb_dual_symmetric (the larger of lb_dual from f~ and lb_dual_from_g from
    g~), and the kept potentials f, g equal the oracle's on the kept side,
    element by element.  The single-pair entry point run from g~ with the
    measures swapped computes the same g~-side pass (the cost is symmetric):
    its potentials equal lb_dual_from_g's with f and g exchanged."""
    N, kappa = 16, 4
    pairs = [(synth.make_measure(N, c, 81, 2 * t), synth.make_measure(N, c, 81, 2 * t + 1))
             for t, c in enumerate(["gauss", "cauchy", "field", "white", "blobs3", "gauss"])]
    tol = TOL[prec]
    g_side_kept = 0
    for p in (1.0, 2.0):
        mus = [T(a) for a, _ in pairs]
        nus = [T(b) for _, b in pairs]
        with api.Batch([(N, kappa, p)] * len(pairs), ipf_sweeps=3, prec=prec, flags=32) as b:
            b.coarse(mus, nus, batched=batched); b.solve(); b.fine(mus, nus, batched=batched)
            res = b.results()
            for t, (mu, nu) in enumerate(pairs):
                f_c, g_c = b.coarse_potentials(t)
                A = O.lb_dual(mu, nu, N, kappa, p, f_c=f_c)
                B = O.lb_dual_from_g(mu, nu, N, kappa, p, g_c)
                S = O.lb_dual_symmetric(mu, nu, N, kappa, p, f_c=f_c, g_c=g_c)
                fmax = max(np.abs(X["f"]).max() + np.abs(X["g"]).max() for X in (A, B))
                slack = tol * max(abs(S["lb_p"]), 1e-3) + 64 * 6e-8 * fmax * (prec == "mixed")
                assert res[t]["status"] == 0
                assert abs(res[t]["lb_p"] - S["lb_p"]) <= slack, (p, t, res[t]["lb_p"], A["lb_p"], B["lb_p"])
                atol = 8 * np.spacing(np.float32(fmax)) if prec == "mixed" else 1e-10 * (1 + fmax)
                f, g = (x.cpu().numpy() for x in b.potentials(t))
                if abs(A["lb_p"] - B["lb_p"]) > 2 * slack:     # the kept side is unambiguous
                    np.testing.assert_allclose(f, S["f"], rtol=0, atol=atol)
                    np.testing.assert_allclose(g, S["g"], rtol=0, atol=atol)
                    g_side_kept += B["lb_p"] > A["lb_p"]
                else:                                           # either side is a correct choice
                    assert any(np.abs(f - X["f"]).max() <= atol and np.abs(g - X["g"]).max() <= atol
                               for X in (A, B))
                r = api.dual_upscale_ctransform(T(nu), T(mu), N, kappa, p, g_c, prec=prec)
                np.testing.assert_allclose(r["f"].cpu().numpy(), B["g"], rtol=0, atol=atol)
                np.testing.assert_allclose(r["g"].cpu().numpy(), B["f"], rtol=0, atol=atol)
                assert abs(r["lb_p"] - B["lb_p"]) <= slack
    assert g_side_kept >= 1, "no pair kept the g~ side: its potentials were never compared"


@pytest.mark.parametrize("sweeps", [1, 7, 50])
@pytest.mark.parametrize("batched", [True, False])
@pytest.mark.parametrize("cluster", [2, 4, 8, 16])
def test_fine_ipf_scalings_bulk(sweeps, batched, cluster):
    """The bulk-copy staged sweeps (cluster | QWB_IPF_BULK; groups whose pairs
    share N): several chunks per half sweep and a stage ring that wraps across
    half sweeps (256^2 at kappa 8: 16 KB chunks of two block rows; 128^2 at
    kappa 4: chunks of eight block rows).  The scalings reach the uniform
    kernel's fixed point and equal the register-streaming cluster sweeps up to
    FP32 rounding; the certified bound, which the FP64 block-scalar sweeps
    define, is bit-identical; no bounded wait times out (status 0)."""
    cases = [(256, 8, 2.0, "gauss"), (256, 8, 1.0, "field"), (128, 4, 2.0, "white"),
             (128, 4, 2.0, "cauchy")]
    mus, nus, probs = [], [], []
    for i, (N, kappa, p, cls) in enumerate(cases):
        mu, nu = synth.make_measure(N, cls, 50 + i, 0), synth.make_measure(N, cls, 50 + i, 1)
        if i == 3:   # a zero-mass block on each side
            mu = mu.reshape(N, N).copy(); mu[8:12, 4:8] = 0.0; mu = (mu / mu.sum()).ravel()
            nu = nu.reshape(N, N).copy(); nu[0:4, 60:64] = 0.0; nu = (nu / nu.sum()).ravel()
        mus.append(mu); nus.append(nu); probs.append((N, kappa, p))
    md, nd = [T(x) for x in mus], [T(x) for x in nus]
    out = {}
    for form in ("bulk", "registers"):
        with api.Batch(probs, ipf_sweeps=sweeps, prec="mixed", flags=1 | 4) as b:
            b.coarse(md, nd, batched=batched)
            b.solve()
            b.set_ipf_cluster(cluster | (api.QWB_IPF_BULK if form == "bulk" else 0))
            b.fine(md, nd, batched=batched)
            res = b.results()
            assert all(r["status"] == 0 for r in res)
            out[form] = ([r["ub_primal"] for r in res], [[x.cpu().numpy() for x in b.fine_scalings(t)]
                                                          for t in range(len(probs))])
    for t, (N, kappa, p) in enumerate(probs):
        assert out["bulk"][0][t] == out["registers"][0][t], t
        for side, meas in enumerate((mus[t], nus[t])):
            got = out["bulk"][1][t][side]
            coarse = O.sumpool(meas, N, kappa)
            blk = np.repeat(np.repeat(coarse.reshape(N // kappa, N // kappa), kappa, 0), kappa, 1).ravel()
            want = np.where(blk > 0, kappa ** 2 * meas / np.where(blk > 0, blk, 1.0), 0.0)
            np.testing.assert_allclose(got, want, rtol=2e-5, atol=0)
            np.testing.assert_allclose(got, out["registers"][1][t][side], rtol=2e-5, atol=0)


@pytest.mark.parametrize("sweeps", [1, 7, 50])
@pytest.mark.parametrize("batched", [True, False])
@pytest.mark.parametrize("cluster", [0, 2, 8, 16, 3, 3 | 64, 4 | 64])
def test_fine_ipf_scalings(sweeps, batched, cluster):
    """The fine FP32 IPF sweeps (inside the primal kernel, or on clusters of up
    to 2, 8 or 16 CTAs per pair, of 3 CTAs that split the block rows unevenly
    (coarse sides 8, 12, 16: rows 3 + 3 + 2, 4 + 4 + 4, 6 + 6 + 4), and with
    512-thread CTAs (| QWB_IPF_WIDE = 64)): from b = 1 the uniform kernel reaches its fixed point
    a = kappa^2 mu / mu~, b = kappa^2 nu / nu~ after one sweep whatever the
    coarse plan (Sec. 3.4, IPF paragraph), and further sweeps stay there up to
    FP32 rounding.  The oracle's FP64 IPF on its own plan agrees."""
    cases = [(32, 4, 2.0, "gauss"), (64, 8, 2.0, "field"), (32, 2, 1.0, "white"),
             (48, 4, 1.0, "cauchy"), (64, 4, 2.0, "gauss")]
    if cluster == 16:    # coarse sides divisible by 16, so both groups take 16 CTAs
        cases = [(128, 8, 2.0, "gauss"), (64, 4, 1.0, "field"), (64, 2, 2.0, "white"),
                 (128, 4, 2.0, "cauchy"), (64, 4, 2.0, "gauss")]
    mus, nus, probs = [], [], []
    for i, (N, kappa, p, cls) in enumerate(cases):
        mu, nu = synth.make_measure(N, cls, 40 + i, 0), synth.make_measure(N, cls, 40 + i, 1)
        if i == 4:   # a zero-mass block on each side
            mu = mu.reshape(N, N).copy(); mu[8:12, 4:8] = 0.0; mu = (mu / mu.sum()).ravel()
            nu = nu.reshape(N, N).copy(); nu[0:4, 60:64] = 0.0; nu = (nu / nu.sum()).ravel()
        mus.append(mu); nus.append(nu); probs.append((N, kappa, p))
    with api.Batch(probs, ipf_sweeps=sweeps, prec="mixed") as b:
        md, nd = [T(x) for x in mus], [T(x) for x in nus]
        b.coarse(md, nd, batched=batched)
        b.solve()
        b.set_ipf_cluster(cluster)
        b.fine(md, nd, batched=batched)
        assert all(r["status"] == 0 for r in b.results())
        for t, (N, kappa, p) in enumerate(probs):
            a, bb = (x.cpu().numpy() for x in b.fine_scalings(t))
            for got, meas in ((a, mus[t]), (bb, nus[t])):
                coarse = O.sumpool(meas, N, kappa)
                blk = np.repeat(np.repeat(coarse.reshape(N // kappa, N // kappa), kappa, 0), kappa, 1).ravel()
                want = np.where(blk > 0, kappa ** 2 * meas / np.where(blk > 0, blk, 1.0), 0.0)
                np.testing.assert_allclose(got, want, rtol=2e-5, atol=0)
            if t == 0:
                plan, _, _, _ = O.exact_ot(O.coarse_cost_centre(N, kappa, p),
                                           O.sumpool(mus[t], N, kappa), O.sumpool(nus[t], N, kappa))
                ref = O.ipf(mus[t], nus[t], plan, N, kappa, max_sweeps=sweeps)
                np.testing.assert_allclose(a, ref["a"], rtol=2e-5, atol=0)
                np.testing.assert_allclose(bb, ref["b"], rtol=2e-5, atol=0)


@pytest.mark.parametrize("cluster", [2, 4 | 64, 8, 16])
def test_fine_ipf_warp_rows_kappa8(cluster):
    """Cluster sweeps at kappa 8 where whole warps own 32 blocks of one block
    row (coarse sides 32 and 64), which move the fine rows as 64 consecutive
    float4 per warp: the scalings reach the fixed point a = kappa^2 mu / mu~
    (and b likewise) and the certified bound equals the in-kernel sweeps' bit
    for bit (the FP64 block-scalar sweeps define it)."""
    cases = [(256, 8, 2.0, "field"), (512, 8, 2.0, "gauss")]
    mus, nus, probs = [], [], []
    for i, (N, kappa, p, cls) in enumerate(cases):
        mus.append(synth.make_measure(N, cls, 90 + i, 0)); nus.append(synth.make_measure(N, cls, 90 + i, 1))
        probs.append((N, kappa, p))
    md, nd = [T(x) for x in mus], [T(x) for x in nus]
    ub = {}
    for form in (0, cluster):
        with api.Batch(probs, ipf_sweeps=7, prec="mixed", flags=1 | 4) as b:
            b.coarse(md, nd)
            b.solve()
            b.set_ipf_cluster(form)
            b.fine(md, nd)
            res = b.results()
            assert all(r["status"] == 0 for r in res)
            ub[form] = [r["ub_primal"] for r in res]
            if form:
                for t, (N, kappa, p) in enumerate(probs):
                    a, bb = (x.cpu().numpy() for x in b.fine_scalings(t))
                    for got, meas in ((a, mus[t]), (bb, nus[t])):
                        coarse = O.sumpool(meas, N, kappa)
                        blk = np.repeat(np.repeat(coarse.reshape(N // kappa, N // kappa), kappa, 0), kappa, 1).ravel()
                        want = np.where(blk > 0, kappa ** 2 * meas / np.where(blk > 0, blk, 1.0), 0.0)
                        np.testing.assert_allclose(got, want, rtol=2e-5, atol=0)
    assert ub[0] == ub[cluster]
