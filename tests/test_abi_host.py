"""CPU checks of the C ABI: the library builds, loads without a GPU, exports
every function include/qwb.h declares, and its host exact solver (network
simplex) agrees with the oracle's successive-shortest-path solver."""
import os
import re

import numpy as np
import pytest

from oracle import qwb_oracle as O
from paper_2506_00976_gb300 import _lib, build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "qwb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qwb_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name
    bound = {s[0] for s in _lib.SIGNATURES}
    assert set(names) == bound, set(names) ^ bound


def test_status_strings(lib):
    assert lib.qwb_status_string(0) == b"QWB_OK"
    assert lib.qwb_status_string(2) == b"QWB_ERR_MASS"


def _solve(C, a, b):
    from paper_2506_00976_gb300 import api
    return api.coarse_solve(C, a, b)


@pytest.mark.parametrize("seed", range(5))
def test_network_simplex_random_dense(lib, seed):
    rng = np.random.default_rng(seed)
    n, m = rng.integers(1, 60, size=2)
    C = rng.random((n, m)) * 100
    a = rng.random(n); a /= a.sum()
    b = rng.random(m); b /= b.sum()
    r = _solve(C, a, b)
    _, _, _, obj = O.exact_ot(C, a, b)
    assert r["obj"] == pytest.approx(obj, rel=1e-10, abs=1e-12)
    assert len(r["val"]) <= n + m - 1
    plan = np.zeros((n, m))
    for i in range(n):
        for e in range(r["rowptr"][i], r["rowptr"][i + 1]):
            plan[i, r["col"][e]] += r["val"][e]
    assert np.abs(plan.sum(1) - a).max() < 1e-13 and np.abs(plan.sum(0) - b).max() < 1e-13
    assert (C - r["f"][:, None] - r["g"][None, :]).min() >= -1e-12 * C.max()
    assert float(r["f"] @ a + r["g"] @ b) == pytest.approx(obj, rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("seed", range(12))
def test_network_simplex_degenerate_dense(lib, seed):
    """Integer costs from a few values (many ties, degenerate pivots) and
    zero masses on both sides, rectangular shapes: the oracle's optimum,
    exact marginals, a basic plan and feasible potentials.  Exercises the
    tree updates of long pivot sequences (re-rooted subtrees, empty and
    re-filled subtrees, zero-flow arcs)."""
    rng = np.random.default_rng(100 + seed)
    n, m = rng.integers(2, 70, size=2)
    C = rng.integers(0, 4 if seed % 2 else 40, size=(n, m)).astype(np.float64)
    a = rng.random(n) * (rng.random(n) > 0.25)
    b = rng.random(m) * (rng.random(m) > 0.2)
    a[0] += 0.1; b[-1] += 0.1
    a /= a.sum(); b /= b.sum()
    r = _solve(C, a, b)
    obj = O.exact_ot(C, a, b)[3]
    assert r["obj"] == pytest.approx(obj, rel=1e-10, abs=1e-13)
    assert len(r["val"]) <= n + m - 1
    plan = np.zeros((n, m))
    for i in range(n):
        for e in range(r["rowptr"][i], r["rowptr"][i + 1]):
            plan[i, r["col"][e]] += r["val"][e]
    assert np.abs(plan.sum(1) - a).max() < 1e-13 and np.abs(plan.sum(0) - b).max() < 1e-13
    assert (C - r["f"][:, None] - r["g"][None, :]).min() >= -1e-12 * max(C.max(), 1.0)


@pytest.mark.parametrize("p", [1.0, 2.0])
@pytest.mark.parametrize("cls", ["white", "gauss", "field"])
def test_network_simplex_grid_costs(lib, p, cls):
    """Degenerate grid costs (many ties): objective equals the oracle's."""
    N, kappa = 32, 2
    mu, nu = synth.make_measure(N, cls, 40, 0), synth.make_measure(N, cls, 40, 1)
    C = O.coarse_cost_centre(N, kappa, p)
    a, b = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    r = _solve(C, a, b)
    _, _, _, obj = O.exact_ot(C, a, b)
    assert r["obj"] == pytest.approx(obj, rel=1e-10)
    assert len(r["val"]) <= 2 * len(a) - 1
    assert (C - r["f"][:, None] - r["g"][None, :]).min() >= -1e-10


def test_network_simplex_zero_masses(lib):
    rng = np.random.default_rng(9)
    C = rng.random((20, 15))
    a = rng.random(20); a[[0, 5, 7]] = 0; a /= a.sum()
    b = rng.random(15); b[[3]] = 0; b /= b.sum()
    r = _solve(C, a, b)
    assert r["obj"] == pytest.approx(O.exact_ot(C, a, b)[3], rel=1e-10)


def test_network_simplex_rejects_bad_input(lib):
    from paper_2506_00976_gb300._lib import QwbError
    with pytest.raises(QwbError, match="INVALID_ARG"):
        _solve(-np.ones((2, 2)), np.array([0.5, 0.5]), np.array([0.5, 0.5]))
    with pytest.raises(QwbError, match="INVALID_ARG"):
        _solve(np.ones((2, 2)), np.array([np.nan, 1.0]), np.array([0.5, 0.5]))


@pytest.mark.parametrize("ns,kappa,p,cls", [(8, 4, 2.0, "gauss"), (16, 4, 2.0, "white"), (16, 2, 1.0, "field"),
                                           (20, 4, 1.5, "cauchy"), (24, 4, 2.0, "field"), (24, 2, 1.0, "gauss")])
def test_network_simplex_grid_table(lib, ns, kappa, p, cls):
    """qwb_coarse_solve_grid (offset-table cost, coarse to fine for even sides
    >= 16, the separable row-minimum filter for p = 2) against the oracle's
    exact solver on the dense C~ matrix: the same optimal objective, a basic
    plan with the given marginals, and potentials feasible up to rounding
    (g = f^c, f = g^c in FP64) whose dual objective is the optimum."""
    from paper_2506_00976_gb300 import api
    N = ns * kappa
    mu, nu = synth.make_measure(N, cls, 41, 0), synth.make_measure(N, cls, 41, 1)
    if cls == "field":                               # zero-mass cells on both sides
        mu = mu.reshape(N, N).copy(); mu[:kappa, :kappa] = 0.0; mu = (mu / mu.sum()).ravel()
        nu = nu.reshape(N, N).copy(); nu[-kappa:, -2 * kappa:] = 0.0; nu = (nu / nu.sum()).ravel()
    a, b = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    C = O.coarse_cost_centre(N, kappa, p)
    tab = np.array([[C[0, d1 * ns + d2] for d2 in range(ns)] for d1 in range(ns)])
    r = api.coarse_solve_grid(tab, a, b)
    _, _, _, obj = O.exact_ot(C, a, b)
    assert r["obj"] == pytest.approx(obj, rel=1e-10)
    M = ns * ns
    assert len(r["val"]) <= 2 * M - 1
    plan = np.zeros((M, M))
    for i in range(M):
        for e in range(r["rowptr"][i], r["rowptr"][i + 1]):
            plan[i, r["col"][e]] += r["val"][e]
    assert np.abs(plan.sum(1) - a).max() < 1e-13 and np.abs(plan.sum(0) - b).max() < 1e-13
    assert (C - r["f"][:, None] - r["g"][None, :]).min() >= -1e-12 * C.max()
    assert float(r["f"] @ a + r["g"] @ b) == pytest.approx(obj, rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("p", [1.0, 2.0])
def test_network_simplex_grid_empty_parent_cells(lib, p):
    """Coarse to fine with whole 2 x 2 parent cells of zero mass: their
    children have no arc in the half-resolution plan, so the fine starting
    tree built from that plan hangs them from the root alone.  Objective,
    marginals and basis size against the oracle's exact solver."""
    from paper_2506_00976_gb300 import api
    ns, kappa = 16, 2
    N = ns * kappa
    mu = synth.make_measure(N, "gauss", 45, 0).reshape(N, N).copy()
    nu = synth.make_measure(N, "white", 45, 1).reshape(N, N).copy()
    mu[:2 * kappa, :2 * kappa] = 0.0
    mu[6 * kappa:8 * kappa, 4 * kappa:6 * kappa] = 0.0
    nu[-2 * kappa:, -4 * kappa:] = 0.0
    mu = (mu / mu.sum()).ravel(); nu = (nu / nu.sum()).ravel()
    a, b = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    C = O.coarse_cost_centre(N, kappa, p)
    tab = np.array([[C[0, d1 * ns + d2] for d2 in range(ns)] for d1 in range(ns)])
    r = api.coarse_solve_grid(tab, a, b)
    assert r["obj"] == pytest.approx(O.exact_ot(C, a, b)[3], rel=1e-10)
    M = ns * ns
    assert len(r["val"]) <= 2 * M - 1
    plan = np.zeros((M, M))
    for i in range(M):
        for e in range(r["rowptr"][i], r["rowptr"][i + 1]):
            plan[i, r["col"][e]] += r["val"][e]
    assert np.abs(plan.sum(1) - a).max() < 1e-13 and np.abs(plan.sum(0) - b).max() < 1e-13


def test_pivot_cap_reports_not_converged(lib, monkeypatch):
    """Host-side fault injection (QWB_FAULT=ns_pivot_cap=k): a network simplex
    stopped after a few pivots on a problem that needs many reports
    QWB_ERR_NOT_CONVERGED with a message, and the next call without the fault
    solves the same problem to the oracle's optimum."""
    from paper_2506_00976_gb300 import api
    from paper_2506_00976_gb300._lib import QwbError
    rng = np.random.default_rng(11)
    n = 40
    C = rng.random((n, n)) * 100
    a = rng.random(n); a /= a.sum()
    b = rng.random(n); b /= b.sum()
    monkeypatch.setenv("QWB_FAULT", "ns_pivot_cap=3")
    with pytest.raises(QwbError, match="NOT_CONVERGED"):
        api.coarse_solve(C, a, b)
    assert b"pivot cap" in lib.qwb_last_error()
    side = 8
    tab = (np.arange(side)[:, None] ** 2 + np.arange(side)[None, :] ** 2).astype(np.float64)
    ga = rng.random(side * side); ga /= ga.sum()
    gb = rng.random(side * side); gb /= gb.sum()
    with pytest.raises(QwbError, match="NOT_CONVERGED"):
        api.coarse_solve_grid(tab, ga, gb)
    monkeypatch.setenv("QWB_FAULT", "")
    r = api.coarse_solve(C, a, b)
    assert r["obj"] == pytest.approx(O.exact_ot(C, a, b)[3], rel=1e-10)


@pytest.fixture(scope="module")
def warm_driver(tmp_path_factory):
    """The host solver's warm C-bar solve as a small program (g++, no GPU)."""
    import shutil
    import subprocess
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("nsdrv") / "ns_warm_driver")
    src = [os.path.join(ROOT, "tests", "ns_warm_driver.cpp"),
           os.path.join(ROOT, "paper_2506_00976_gb300", "csrc", "netsimplex.cpp")]
    subprocess.run([gxx, "-O2", "-std=c++17", "-o", exe, *src], check=True, capture_output=True)
    return exe


def _run_warm(exe, tmp_path, tab, a, b, C, bound):
    import subprocess
    path = str(tmp_path / "prob.bin")
    with open(path, "wb") as fh:
        np.array([tab.shape[0]], dtype=np.int32).tofile(fh)
        for arr in (tab, a, b, C, np.array([bound])):
            np.ascontiguousarray(arr, dtype=np.float64).tofile(fh)
    out = subprocess.run([exe, path], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), float(out[1]), int(out[2]), float(out[3]), float(out[4])


@pytest.mark.parametrize("N,kappa,p,cls", [(32, 2, 2.0, "gauss"), (40, 4, 1.5, "cauchy"), (32, 2, 1.0, "white")])
def test_warm_cbar_solve_with_cost_bound(warm_driver, tmp_path, N, kappa, p, cls):
    """The C-bar solve of a batch pair (Sec. 3.2): started from the C~
    optimum's basis, the C~ plan's neighbourhoods priced first, with the
    entries checked against a caller's bound inside the full scans (and,
    bound < 0, by a pass of their own): the oracle's optimal objective and a
    basic plan with the given marginals either way."""
    ns = N // kappa
    M = ns * ns
    mu, nu = synth.make_measure(N, cls, 43, 0), synth.make_measure(N, cls, 43, 1)
    a, b = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    Ct = O.coarse_cost_centre(N, kappa, p)
    tab = np.array([[Ct[0, d1 * ns + d2] for d2 in range(ns)] for d1 in range(ns)])
    Cb = O.coarse_cost_weighted(mu, nu, N, kappa, p)
    obj = O.exact_ot(Cb, a, b)[3]
    bound = 2.0 * (2.0 * (N - 1) ** 2) ** (p / 2) + 1.0
    for bd in (bound, -1.0):
        st, val, nnz, re, ce = _run_warm(warm_driver, tmp_path, tab, a, b, Cb, bd)
        assert st == 0
        assert val == pytest.approx(obj, rel=1e-10)
        assert nnz <= 2 * M - 1 and re < 1e-13 and ce < 1e-13


@pytest.mark.parametrize("bad", [np.nan, -1.0, np.inf, "over"])
@pytest.mark.parametrize("where", ["far", "near"])
def test_warm_cbar_solve_rejects_bad_entries(warm_driver, tmp_path, bad, where):
    """A NaN, negative, infinite or above-bound C-bar entry makes the warm
    solve return INVALID_ARG, whether it lies among the arcs priced first
    (checked before the solve) or only in the full scans ("far": the corner
    arc from block 0 to block M - 1)."""
    N, kappa, p = 32, 2, 2.0
    ns = N // kappa
    M = ns * ns
    mu, nu = synth.make_measure(N, "gauss", 44, 0), synth.make_measure(N, "gauss", 44, 1)
    a, b = O.sumpool(mu, N, kappa), O.sumpool(nu, N, kappa)
    Ct = O.coarse_cost_centre(N, kappa, p)
    tab = np.array([[Ct[0, d1 * ns + d2] for d2 in range(ns)] for d1 in range(ns)])
    Cb = O.coarse_cost_weighted(mu, nu, N, kappa, p).copy()
    bound = 2.0 * (2.0 * (N - 1) ** 2) + 1.0
    k, l = (0, M - 1) if where == "far" else (0, 0)
    Cb[k, l] = 3.0 * bound if bad == "over" else bad
    for bd in ((bound, -1.0) if bad != "over" else (bound,)):
        st = _run_warm(warm_driver, tmp_path, tab, a, b, Cb, bd)[0]
        assert st == 1
