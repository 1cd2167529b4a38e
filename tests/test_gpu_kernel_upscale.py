"""GPU parity of the primal pass with a general normalized positive upscaling
kernel K (Sec. 3.4, eq. coupling tensor upscale) against the FP64 oracle.

Tolerances.  The plan's cost W-hat^p matches the oracle's to 1e-6 (F64) or
1e-4 (MIXED) relative.  The TV corrections are p-th roots of weighted sums of
|mu-hat - mu|: with FP32 scalings each marginal entry carries a relative
rounding error of at most about (kappa^2 + row degree + 2) u (the FP32 sums
of the half sweep that produced it, and its division), which the oracle's
FP64 state does not have, and the certified evaluation encloses each entry
in an interval of relative half-width (kappa^2 + deg + 3) 2^-52 and the total
mass in one wider by its summation bound (m / 256 + 42) 2^-52; the sums
therefore agree to within
    floor = 2^(p-1) (c u + (4 (kappa^2 + deg + 3) + 2 (m / 256 + 42)) 2^-52)
            sum_i w_i (mu_i + nu_i),  c = 4 (kappa^2 + deg + 2),
and each Delta to within (its oracle value^p + floor)^(1/p) above and the
same with - floor below (u = 2^-24 for MIXED, 2^-53 for F64)."""
import numpy as np
import pytest
import torch

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import api, synth

pytestmark = pytest.mark.gpu
TOL = {"mixed": 1e-4, "f64": 1e-6}
UNIT = {"mixed": 2.0 ** -24, "f64": 2.0 ** -53}


def T(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _plan(mu, nu, N, kappa, p):
    mt, nt = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    plan, _, _, _ = O.exact_ot(O.coarse_cost_centre(N, kappa, p), mt, nt)
    return plan


def _csr(plan):
    rows, cols = np.nonzero(plan)
    rowptr = np.zeros(plan.shape[0] + 1, dtype=np.int32)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr).astype(np.int32), cols.astype(np.int32), plan[rows, cols]


def _random_kernel(kappa, seed):
    rng = np.random.default_rng(seed)
    K = rng.uniform(0.05, 1.0, size=(kappa * kappa, kappa * kappa))
    return K / K.sum()


def _check(r, ref, mu, nu, N, kappa, p, prec, plan):
    deg = int(max((plan > 0).sum(axis=1).max(), (plan > 0).sum(axis=0).max()))
    w = O.tv_weights(N, p)
    # the scalings' rounding (above) and the certified evaluation's own
    # enclosures: a relative (kappa^2 + deg + 3) 2^-52 either side of each
    # marginal entry and, plus the summation bound (m / 256 + 42) 2^-52, of
    # the mass s (which enters through |1/s - 1|)
    m_terms = (N * N + 255) // 256 + 42
    rel = (4 * (kappa * kappa + deg + 2) * UNIT[prec]
           + (4 * (kappa * kappa + deg + 3) + 2 * m_terms) * 2.0 ** -52)
    floor = 2.0 ** (p - 1) * rel * float(np.dot(w, mu + nu))
    tol = TOL[prec]
    assert abs(r["w_hat_p"] - ref["w_hat_p"]) <= tol * ref["w_hat_p"]
    for key in ("delta_mu", "delta_nu"):
        d_o = ref[key] ** p / 2.0 ** (p - 1)          # the weighted sum behind Delta
        hi = (2.0 ** (p - 1) * (d_o * (1 + tol)) + floor) ** (1.0 / p)
        lo = max(2.0 ** (p - 1) * d_o * (1 - tol) - floor, 0.0) ** (1.0 / p)
        assert lo * (1 - 1e-12) <= r[key] <= hi * (1 + 1e-12), (key, r[key], ref[key], lo, hi)
    # the bound adds up from its parts (rounded up)
    assert r["ub_primal"] >= r["w_hat_p"] ** (1.0 / p) + r["delta_mu"] + r["delta_nu"] - 1e-12


@pytest.mark.parametrize("N,kappa,p,cls", [(16, 4, 2.0, "gauss"), (32, 4, 1.0, "field"),
                                            (32, 8, 2.0, "cauchy"), (24, 2, 2.0, "white"),
                                            (40, 8, 1.5, "blobs3"), (36, 6, 2.0, "gauss"),
                                            (27, 3, 2.0, "field"), (20, 5, 1.0, "gauss"),
                                            (21, 7, 2.0, "blobs3"), (8, 1, 2.0, "cauchy")])
@pytest.mark.parametrize("kind", ["gauss1", "random"])
@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_primal_kernel_pass(N, kappa, p, cls, kind, prec):
    """The general-kernel primal pass against the oracle's ub_primal_K on the
    same coarse plan and the same number of sweeps (the oracle runs them all:
    xi = 0), for a Gaussian kernel over the in-block offsets and a random
    positive kernel; tails of ragged blocks per CTA (N / kappa not a multiple
    of anything) are covered by N = 24, 36, 40; odd kappa and kappa = 1 take
    the scalar sweep and evaluation paths, kappa 2, 4, 8 the fused sweep."""
    mu, nu = synth.make_measure(N, cls, 41, 0), synth.make_measure(N, cls, 41, 1)
    plan = _plan(mu, nu, N, kappa, p)
    K = O.gaussian_kernel(kappa, 1.0) if kind == "gauss1" else _random_kernel(kappa, 7)
    sweeps = 40
    ref = O.ub_primal_K(mu, nu, N, kappa, p, K, xi=0.0, max_sweeps=sweeps, plan_c=plan)
    rowptr, col, val = _csr(plan)
    r = api.primal_upscale_ipf_kernel(T(mu), T(nu), N, kappa, p, rowptr, col, val, K, sweeps=sweeps,
                                      prec=prec, want_scalings=True)
    assert r["ipf_sweeps_done"] == sweeps
    _check(r, ref, mu, nu, N, kappa, p, prec, plan)
    # the scalings follow the oracle's trajectory (same start b = 1, same sweeps)
    a, b = r["a"].cpu().numpy(), r["b"].cpu().numpy()
    rt = 1e-9 if prec == "f64" else 2e-3
    s = ref["b"].sum() / b.sum()                      # a, b are defined up to a b -> b t, a -> a / t
    np.testing.assert_allclose(b * s, ref["b"], rtol=rt, atol=0)
    np.testing.assert_allclose(a / s, ref["a"], rtol=rt, atol=0)


@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_primal_kernel_uniform_equals_uniform_pass(prec):
    """K = kappa^-4 on every offset pair gives the uniform pass's bound (the
    uniform pass finishes with exact FP64 block sweeps; the general pass
    reaches the same fixed point after one sweep in exact arithmetic)."""
    N, kappa, p = 32, 4, 2.0
    mu, nu = synth.make_measure(N, "field", 42, 0), synth.make_measure(N, "field", 42, 1)
    plan = _plan(mu, nu, N, kappa, p)
    K = np.full((kappa * kappa, kappa * kappa), float(kappa) ** -4)
    rowptr, col, val = _csr(plan)
    ru = api.primal_upscale_ipf(T(mu), T(nu), N, kappa, p, rowptr, col, val, sweeps=3, prec=prec)
    rk = api.primal_upscale_ipf_kernel(T(mu), T(nu), N, kappa, p, rowptr, col, val, K, sweeps=3, prec=prec)
    ref = O.ub_primal(mu, nu, N, kappa, p, plan_c=plan)
    assert abs(rk["w_hat_p"] - ru["w_hat_p"]) <= TOL[prec] * ru["w_hat_p"]
    _check(rk, {**ref}, mu, nu, N, kappa, p, prec, plan)


@pytest.mark.parametrize("N,kappa,p,cls", [(8, 2, 2.0, "gauss"), (16, 4, 1.0, "cauchy"),
                                            (16, 4, 2.0, "white"), (16, 8, 2.0, "blobs3")])
@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_primal_kernel_certified(N, kappa, p, cls, prec):
    """UB_primal with a Gaussian kernel is an upper bound of the exact W_p
    (full LP), also after few sweeps (the TV corrections cover the unfitted
    marginals) and for a sharply peaked kernel."""
    mu, nu = synth.make_measure(N, cls, 43, 0), synth.make_measure(N, cls, 43, 1)
    W = O.wasserstein_exact(mu, nu, N, p)
    plan = _plan(mu, nu, N, kappa, p)
    rowptr, col, val = _csr(plan)
    for sigma, sweeps in ((1.0, 2), (1.0, 60), (0.3, 30)):
        K = O.gaussian_kernel(kappa, sigma)
        r = api.primal_upscale_ipf_kernel(T(mu), T(nu), N, kappa, p, rowptr, col, val, K, sweeps=sweeps,
                                          prec=prec)
        assert r["ub_primal"] >= W * (1 - 1e-12), (sigma, sweeps, r["ub_primal"], W)


def test_primal_kernel_rejects_bad_kernels():
    """Non-positive or non-finite kernels, kappa > 8 and volumes are refused."""
    N, kappa, p = 16, 4, 2.0
    mu, nu = synth.make_measure(N, "gauss", 44, 0), synth.make_measure(N, "gauss", 44, 1)
    plan = _plan(mu, nu, N, kappa, p)
    rowptr, col, val = _csr(plan)
    K = O.gaussian_kernel(kappa, 1.0)
    for bad in (np.where(np.eye(16) > 0, 0.0, K), np.where(np.eye(16) > 0, np.nan, K), -K):
        with pytest.raises(RuntimeError):
            api.primal_upscale_ipf_kernel(T(mu), T(nu), N, kappa, p, rowptr, col, val, bad, sweeps=2)
    N2, k2 = 32, 16
    mu2, nu2 = synth.make_measure(N2, "gauss", 44, 2), synth.make_measure(N2, "gauss", 44, 3)
    plan2 = _plan(mu2, nu2, N2, k2, p)
    r2 = _csr(plan2)
    with pytest.raises(RuntimeError):
        api.primal_upscale_ipf_kernel(T(mu2), T(nu2), N2, k2, p, *r2, np.full((256, 256), 1.0 / 65536),
                                      sweeps=2)


@pytest.mark.parametrize("prec", ["mixed", "f64"])
def test_batch_kernel_pairs(prec):
    """A batch of uneven pairs where those of block side 4 and 8 use general
    kernels: the batched form equals one pair per launch bit for bit, the
    other pairs are unchanged, every bound is valid against the exact LP, and
    the K pairs match the oracle's bound on the batch's own coarse plan."""
    cases = [(16, 4, 2.0, "gauss"), (32, 8, 1.0, "cauchy"), (16, 2, 2.0, "field"),
             (32, 4, 2.0, "blobs3"), (16, 8, 2.0, "white"), (24, 4, 1.0, "field")]
    mus, nus, probs, raw = [], [], [], []
    for t, (N, kappa, p, cls) in enumerate(cases):
        mu, nu = synth.make_measure(N, cls, 45, 2 * t), synth.make_measure(N, cls, 45, 2 * t + 1)
        raw.append((mu, nu))
        mus.append(T(mu)); nus.append(T(nu)); probs.append((N, kappa, p))
    K4, K8 = O.gaussian_kernel(4, 1.0), _random_kernel(8, 3)
    sweeps = 30

    plans = {}

    def run(batched, with_k):
        with api.Batch(probs, ipf_sweeps=sweeps, prec=prec) as bt:
            if with_k:
                bt.set_upscale_kernel(4, K4)
                bt.set_upscale_kernel(8, K8)
            bt.coarse(mus, nus, batched=batched)
            bt.solve()
            bt.fine(mus, nus, batched=batched)
            if batched and with_k:
                for t in range(len(cases)):
                    plans[t] = bt.coarse_plan(t)
            return bt.results()

    rb, rp, r0 = run(True, True), run(False, True), run(True, False)
    for t, (N, kappa, p, cls) in enumerate(cases):
        for key in ("ub_primal", "w_hat_p", "lb"):
            assert rb[t][key] == rp[t][key], (t, key)
        if kappa not in (4, 8):
            assert rb[t]["ub_primal"] == r0[t]["ub_primal"], t
        assert rb[t]["lb"] == r0[t]["lb"], t
        if N <= 16:
            W = O.wasserstein_exact(raw[t][0], raw[t][1], N, p)
            assert rb[t]["lb"] <= W <= rb[t]["ub_primal"] * (1 + 1e-12), t
        if kappa in (4, 8):
            K = K4 if kappa == 4 else K8
            plan = plans[t]
            ref = O.ub_primal_K(raw[t][0], raw[t][1], N, kappa, p, K, xi=0.0, max_sweeps=sweeps, plan_c=plan)
            _check(rb[t], ref, raw[t][0], raw[t][1], N, kappa, p, prec, plan)


def test_batch_kernel_scalings_layout():
    """With the uniform kernel given as a general K, the fitted a / mu is
    constant on every block (the exact fixed point) in the scalings the batch
    returns: they come back in the pixel layout."""
    N, kappa, p = 32, 4, 2.0
    mu, nu = synth.make_measure(N, "field", 46, 0), synth.make_measure(N, "field", 46, 1)
    K = np.full((16, 16), 1.0 / 256)
    with api.Batch([(N, kappa, p)], ipf_sweeps=4, prec="f64") as bt:
        bt.set_upscale_kernel(kappa, K)
        bt.coarse([T(mu)], [T(nu)])
        bt.solve()
        bt.fine([T(mu)], [T(nu)])
        a, _ = bt.fine_scalings(0)
    ratio = (a.cpu().numpy() / mu).reshape(N // kappa, kappa, N // kappa, kappa)
    spread = ratio.max(axis=(1, 3)) - ratio.min(axis=(1, 3))
    assert np.all(spread <= 1e-9 * ratio.max(axis=(1, 3)))


def _kernel_batch(cases, K, kappa, sweeps, batched, form, seed=47):
    """Run the primal pass of a batch whose pairs all take the kernel K;
    form: None (the autotuner's choice) or (C, threads)."""
    mus, nus, probs = [], [], []
    for t, (N, p, cls) in enumerate(cases):
        mus.append(T(synth.make_measure(N, cls, seed, 2 * t)))
        nus.append(T(synth.make_measure(N, cls, seed, 2 * t + 1)))
        probs.append((N, kappa, p))
    with api.Batch(probs, ipf_sweeps=sweeps, prec="mixed", flags=api.QWB_FLAG_NO_DUAL) as bt:
        bt.set_upscale_kernel(kappa, K)
        if form is not None:
            bt.set_upscale_cluster(*form)
        bt.coarse(mus, nus, batched=batched)
        bt.solve()
        bt.fine(mus, nus, batched=batched)
        res = bt.results()
        scal = [bt.fine_scalings(t) for t in range(len(cases))]
        plans = [bt.coarse_plan(t) for t in range(len(cases))]
        tuning = bt.tuning()
    return res, scal, plans, tuning


@pytest.mark.parametrize("kappa,cases,forms", [
    (4, [(16, 2.0, "gauss"), (32, 2.0, "blobs3"), (24, 1.0, "field"), (40, 2.0, "cauchy")],
     [(-1, 128), (1, 256), (2, 128), (4, 128), (4, 64), (8, 64)]),
    (8, [(32, 2.0, "field"), (16, 1.0, "gauss"), (48, 2.0, "white")],
     [(-1, 128), (1, 128), (2, 64), (4, 128), (8, 64)]),
    (2, [(16, 2.0, "blobs3"), (10, 2.0, "gauss")], [(-1, 128), (2, 256), (4, 64), (8, 128)]),
])
def test_batch_kernel_cluster_form(kappa, cases, forms):
    """The cluster form of the general-kernel primal pass (one pair on a
    cluster of C CTAs that split its block rows), and the form that keeps the
    one-CTA sweeps and spreads the evaluation over many CTAs (C = -1).  Its fine sweeps are those
    of the one-CTA kernel item for item, so the scalings agree bit for bit;
    its certified sums run in another order with tighter enclosures, so its
    bounds are no larger than the one-CTA kernel's and agree with the
    oracle's on the same coarse plan within the usual floors; batched equals
    one pair per launch bit for bit.  Covers CTAs that own no block row (C > n) and
    uneven row splits (n = 6, 10, 5)."""
    K = O.gaussian_kernel(kappa, 1.0) if kappa != 8 else _random_kernel(8, 5)
    sweeps = 20
    r0, s0, plans, _ = _kernel_batch(cases, K, kappa, sweeps, True, (0, 128))
    for form in forms:
        rb, sb, _, _ = _kernel_batch(cases, K, kappa, sweeps, True, form)
        rp, sp, _, _ = _kernel_batch(cases, K, kappa, sweeps, False, form)
        for t, (N, p, cls) in enumerate(cases):
            for side in range(2):
                assert torch.equal(sb[t][side], s0[t][side]), (form, t, side)
                assert torch.equal(sp[t][side], s0[t][side]), (form, t, side)
            for key in ("ub_primal", "w_hat_p", "delta_mu", "delta_nu"):
                assert rb[t][key] == rp[t][key], (form, t, key)
            # the plan cost differs by its summation order only; the TV terms
            # drop the one-CTA kernel's summation bound on the total mass
            # (about 43 2^-52 of the weighted mass B) and add 2^-53 of the
            # weighted sums, so they come out no larger
            assert abs(rb[t]["w_hat_p"] - r0[t]["w_hat_p"]) <= 1e-12 * r0[t]["w_hat_p"], (form, t)
            for key in ("ub_primal", "delta_mu", "delta_nu"):
                assert rb[t][key] <= r0[t][key] * (1 + 1e-12), (form, t, key)
            mu = synth.make_measure(N, cls, 47, 2 * t)
            nu = synth.make_measure(N, cls, 47, 2 * t + 1)
            ref = O.ub_primal_K(mu, nu, N, kappa, p, K, xi=0.0, max_sweeps=sweeps, plan_c=plans[t])
            _check(rb[t], ref, mu, nu, N, kappa, p, "mixed", plans[t])
            if N <= 16:
                W = O.wasserstein_exact(mu, nu, N, p)
                assert W <= rb[t]["ub_primal"] * (1 + 1e-12), (form, t)


def test_batch_kernel_cluster_tuned_and_refused():
    """The autotuner times the one-CTA and the cluster forms and reports
    them; the cluster form is refused for FP64 batches and unknown shapes."""
    cases = [(32, 2.0, "gauss"), (32, 2.0, "field")]
    K = O.gaussian_kernel(4, 1.0)
    _, _, _, tuning = _kernel_batch(cases, K, 4, 5, True, None)
    uk = tuning["upscale_kernel"]
    assert "single" in uk["candidates_ms"] and "single_sweeps_spread_eval" in uk["candidates_ms"]
    assert any(k.startswith("cluster") for k in uk["candidates_ms"])
    N = 16
    mu, nu = T(synth.make_measure(N, "gauss", 48, 0)), T(synth.make_measure(N, "gauss", 48, 1))
    with api.Batch([(N, 4, 2.0)], ipf_sweeps=3, prec="f64") as bt:
        bt.set_upscale_kernel(4, K)
        with pytest.raises(RuntimeError):
            bt.set_upscale_cluster(4, 128)
        with pytest.raises(RuntimeError):
            bt.set_upscale_cluster(3, 128)
        with pytest.raises(RuntimeError):
            bt.set_upscale_cluster(4, 96)
