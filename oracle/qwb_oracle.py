"""Plain FP64 CPU oracle for the quantization-based W_p bounds.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or call
this module.  It shares no code, header, table or helper with the CUDA library
(``paper_2506_00976_gb300``) and never imports it.

Every function follows the paper (Bobrutsky & Moscovich, "Quantization-based
Bounds on the Wasserstein Metric") step by step in numpy float64, in the
paper's order and notation; the citation in each docstring names the section,
equation or algorithm.  Library primitives (reshape, sum, min, matmul, sqrt)
serve as steps; there is no blocking or fusion beyond what the definitions
state, apart from chunking loops over output indices to bound memory.

Conventions (readings where the paper is silent):
  * the grid is [N]^d with d = 2 (images, the default) or d = 3 (volumes);
    grid points are 0-based coordinates with unit spacing, flattened
    row-major (i = row * N + col in 2-D, ((x1 * N) + x2) * N + x3 in 3-D);
  * rho is the Euclidean distance and C_ij = rho(x_i, y_j)^p (Sec. 5);
  * coarse index k = k1 * n + k2 (3-D: (k1 * n + k2) * n + k3) for the block
    of coordinates k_a*kappa .. k_a*kappa + kappa - 1 on each axis; block
    centres are the AvgPool of coordinates (Sec. 2.2);
  * a coarse block of zero mass gets C-bar equal to the unweighted mean of the
    cost over the block pair, and IPF sets a_i = 0 where (pi-hat b)_i = 0;
  * the coarse potential is shifted so that <f~, mu~> = 0 before upscaling
    (the lower bound does not change under such shifts);
  * the upscaling interpolation R is multilinear (bilinear, trilinear) in
    block-centre coordinates with linear extrapolation outside the hull of
    the centres.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, a library LP solver, brute force or invariants.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_SSP = None


def _ssp_lib():
    global _SSP
    if _SSP is None:
        lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_ssp.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp, dp,
                                   ctypes.POINTER(ctypes.c_int)]
        lib.oracle_ssp.restype = ctypes.c_int
        _SSP = lib
    return _SSP


# --------------------------------------------------------------------------
# Grid model: Sec. 2.1 (Kantorovich problem, W_p = L_C^(1/p)), Sec. 2.2
# (regular grid [N]^d), Sec. 5 (rho = Euclidean).
# --------------------------------------------------------------------------
def grid_points(N: int, d: int = 2) -> np.ndarray:
    """All points of the grid [N]^d as an (N^d, d) float64 array, row-major."""
    axes = np.meshgrid(*([np.arange(N, dtype=np.float64)] * d), indexing="ij")
    return np.stack([a.ravel() for a in axes], axis=1)


def _blocked(N: int, kappa: int, d: int):
    """Shape that splits every axis into (block index, offset in block), and
    the offset axes of that shape."""
    n = N // kappa
    return (n, kappa) * d, tuple(2 * a + 1 for a in range(d))


def ground_cost(X: np.ndarray, Y: np.ndarray, p: float) -> np.ndarray:
    """C_ij = rho(x_i, y_j)^p with rho the Euclidean distance (Sec. 2.1, Sec. 5)."""
    d2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(axis=-1)
    if p == 2:
        return d2
    if p == 1:
        return np.sqrt(d2)
    return d2 ** (p / 2.0)


# --------------------------------------------------------------------------
# Coarsening: Sec. 2.2 (SumPool of the measure, AvgPool of the coordinates).
# --------------------------------------------------------------------------
def sumpool(mu: np.ndarray, N: int, kappa: int, d: int = 2) -> np.ndarray:
    """mu~_k = mu(X_k): the mass of each kappa^d block (Sec. 2.2)."""
    shape, off = _blocked(N, kappa, d)
    return mu.reshape(shape).sum(axis=off).ravel()


def block_centres(N: int, kappa: int, d: int = 2) -> np.ndarray:
    """x~_k = mean(X_k), the AvgPool of the grid coordinates (Sec. 2.2)."""
    shape, off = _blocked(N, kappa, d)
    return grid_points(N, d).reshape(shape + (d,)).mean(axis=off).reshape(-1, d)


def _block_row_pixels(N: int, kappa: int, k1: int, d: int = 2) -> np.ndarray:
    """Flat indices of the slab of points whose first coordinate lies in block k1."""
    rows = np.arange(k1 * kappa, (k1 + 1) * kappa)
    rest = N ** (d - 1)
    return (rows[:, None] * rest + np.arange(rest)[None, :]).ravel()


def _slab_to_blocks(T, N, kappa, d, reduce):
    """Reduce a (slab points, ...) array over the offsets of the slab's blocks:
    the slab of first-axis block k1 has shape (kappa,) + (N,) * (d-1)."""
    n = N // kappa
    lead = (kappa,) + (n, kappa) * (d - 1)
    axes = (0,) + tuple(2 + 2 * a for a in range(d - 1))
    return reduce(T.reshape(lead + T.shape[1:]), axis=axes).reshape((n ** (d - 1),) + T.shape[1:])


# --------------------------------------------------------------------------
# Coarse costs.
# --------------------------------------------------------------------------
def weighted_cost_numerators(mu, nu, N, kappa, p, d=2):
    """num_kl = sum over x in X_k, y in Y_l of rho(x,y)^p mu(x) nu(y).

    The numerator of the marginally weighted coarse cost (Sec. 3.2, the
    equation defining C-bar; Alg. 3), summed over every fine point pair inside
    each block pair.  Processed one slab of source blocks (fixed first block
    coordinate) at a time.
    """
    n = N // kappa
    M = n ** d
    X = grid_points(N, d)
    shape, off = _blocked(N, kappa, d)
    num = np.empty((M, M))
    for k1 in range(n):
        I = _block_row_pixels(N, kappa, k1, d)
        T = ground_cost(X[I], X, p) * nu[None, :]                          # rho^p nu(y)
        T = T.reshape((len(I),) + shape).sum(axis=tuple(a + 1 for a in off))  # sum y in Y_l
        T = T.reshape(len(I), M) * mu[I][:, None]                           # times mu(x)
        rows = n ** (d - 1)
        num[k1 * rows:(k1 + 1) * rows] = _slab_to_blocks(T, N, kappa, d, np.sum)   # sum x in X_k
    return num


def coarse_cost_weighted(mu, nu, N, kappa, p, d=2):
    """C-bar_kl = num_kl / (mu(X_k) nu(Y_l))  (Sec. 3.2, eq. for C-bar; Alg. 3).

    Where mu(X_k) nu(Y_l) = 0 the paper's quotient is undefined; this oracle
    then uses the unweighted mean of rho^p over the block pair (any finite
    value is valid there because the coarse plan puts no mass on that entry).
    """
    num = weighted_cost_numerators(mu, nu, N, kappa, p, d)
    mt, nt = sumpool(mu, N, kappa, d), sumpool(nu, N, kappa, d)
    den = np.outer(mt, nt)
    Cbar = np.empty_like(num)
    pos = den > 0
    Cbar[pos] = num[pos] / den[pos]
    if not pos.all():
        ones = np.ones(N ** d)
        mean = weighted_cost_numerators(ones, ones, N, kappa, p, d) / float(kappa) ** (2 * d)
        Cbar[~pos] = mean[~pos]
    return Cbar


def coarse_cost_centre(N, kappa, p, d=2):
    """C~_kl = rho(x~_k, x~_l)^p between block centres (Alg. 4 and Alg. 5)."""
    Xc = block_centres(N, kappa, d)
    return ground_cost(Xc, Xc, p)


def coarse_cost_min(N, kappa, p, d=2):
    """C^min_kl = min over x in X_k, y in Y_l of rho(x,y)^p (Sec. 3.3)."""
    n = N // kappa
    M = n ** d
    X = grid_points(N, d)
    shape, off = _blocked(N, kappa, d)
    out = np.empty((M, M))
    rows = n ** (d - 1)
    for k1 in range(n):
        I = _block_row_pixels(N, kappa, k1, d)
        T = ground_cost(X[I], X, p)
        T = T.reshape((len(I),) + shape).min(axis=tuple(a + 1 for a in off)).reshape(len(I), M)
        out[k1 * rows:(k1 + 1) * rows] = _slab_to_blocks(T, N, kappa, d, np.min)
    return out


# --------------------------------------------------------------------------
# Exact Kantorovich problem (Sec. 2.1) by successive shortest paths (ssp.c).
# --------------------------------------------------------------------------
def exact_ot(C, a, b):
    """Solve min <pi, C> over pi in Pi(a, b) and its dual exactly (Sec. 2.1).

    Returns (plan, f, g, objective): an optimal coupling (dense) and optimal
    Kantorovich potentials with f_i + g_j <= C_ij (Sec. 2.1, the set R(C)).
    """
    C = np.ascontiguousarray(C, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n, m = C.shape
    plan = np.empty((n, m))
    f = np.empty(n)
    g = np.empty(m)
    obj = ctypes.c_double()
    rounds = ctypes.c_int()
    dp = ctypes.POINTER(ctypes.c_double)
    st = _ssp_lib().oracle_ssp(n, m, C.ctypes.data_as(dp), a.ctypes.data_as(dp),
                               b.ctypes.data_as(dp), plan.ctypes.data_as(dp),
                               f.ctypes.data_as(dp), g.ctypes.data_as(dp),
                               ctypes.byref(obj), ctypes.byref(rounds))
    if st != 0:
        raise RuntimeError(f"oracle_ssp failed with status {st}")
    return plan, f, g, obj.value


def wasserstein_exact(mu, nu, N, p, d=2):
    """W_p(mu, nu) = L_C(mu, nu)^(1/p) on the full grid (Sec. 2.1).  Small N only."""
    X = grid_points(N, d)
    _, _, _, obj = exact_ot(ground_cost(X, X, p), mu, nu)
    return max(obj, 0.0) ** (1.0 / p)


# --------------------------------------------------------------------------
# Weighted-cost upper bound: Sec. 3.2, Theorem (weighted cost UB), Alg. 3.
# --------------------------------------------------------------------------
def ub_weighted(mu, nu, N, kappa, p, d=2):
    mt, nt = sumpool(mu, N, kappa, d), sumpool(nu, N, kappa, d)
    Cbar = coarse_cost_weighted(mu, nu, N, kappa, p, d)
    plan, _, _, L = exact_ot(Cbar, mt, nt)
    return {"ub_weighted": max(L, 0.0) ** (1.0 / p), "L_cbar": L, "plan": plan,
            "cbar": Cbar}


# --------------------------------------------------------------------------
# Min-cost lower bound: Sec. 3.3, Theorem (locally minimal cost LB).
# --------------------------------------------------------------------------
def lb_mincost(mu, nu, N, kappa, p, d=2):
    mt, nt = sumpool(mu, N, kappa, d), sumpool(nu, N, kappa, d)
    _, _, _, L = exact_ot(coarse_cost_min(N, kappa, p, d), mt, nt)
    return max(L, 0.0) ** (1.0 / p)


# --------------------------------------------------------------------------
# Primal upscaling upper bound: Sec. 3.4, Alg. 4.
# --------------------------------------------------------------------------
def upscaled_plan_apply(plan_c, v, N, kappa, d=2):
    """(pi-hat v)_i where pi-hat = reshape^-1(P~* (x) K), K = kappa^(-2d) (Alg. 4).

    With the uniform kernel, pi-hat_ij = kappa^-2d pi~*_{k(i) l(j)}, so
    (pi-hat v)_i = kappa^-2d sum_l pi~*_{k(i) l} sum_{j in Y_l} v_j.
    """
    n = N // kappa
    V = sumpool(v, N, kappa, d)
    r = (plan_c @ V) * float(kappa) ** (-2 * d)
    r = r.reshape((n,) * d)
    for a in range(d):
        r = np.repeat(r, kappa, axis=a)
    return r.ravel()


def upscaled_plan_apply_T(plan_c, u, N, kappa, d=2):
    """(pi-hat^T u)_j, the transpose of ``upscaled_plan_apply`` (Alg. 4)."""
    return upscaled_plan_apply(plan_c.T, u, N, kappa, d)


def _safe_div(num, den):
    out = np.zeros_like(num)
    pos = den > 0
    out[pos] = num[pos] / den[pos]
    return out


def ipf(mu, nu, plan_c, N, kappa, xi=1e-13, max_sweeps=1000, d=2):
    """Iterative proportional fitting of pi-hat to (mu, nu) (Sec. 3.4 step 2, Alg. 4).

    b <- 1; repeat a <- mu / (pi-hat b); b <- nu / (pi-hat^T a);
    mu-hat <- a * (pi-hat b); nu-hat <- b * (pi-hat^T a)
    until ||mu-hat - mu||_1 + ||nu - nu-hat||_1 < xi (or max_sweeps sweeps).
    """
    b = np.ones(N ** d)
    sweeps = 0
    resid = np.inf
    while sweeps < max_sweeps:
        a = _safe_div(mu, upscaled_plan_apply(plan_c, b, N, kappa, d))
        b = _safe_div(nu, upscaled_plan_apply_T(plan_c, a, N, kappa, d))
        sweeps += 1
        mu_hat = a * upscaled_plan_apply(plan_c, b, N, kappa, d)
        nu_hat = b * upscaled_plan_apply_T(plan_c, a, N, kappa, d)
        resid = np.abs(mu_hat - mu).sum() + np.abs(nu - nu_hat).sum()
        if resid < xi:
            break
    return {"a": a, "b": b, "mu_hat": mu_hat, "nu_hat": nu_hat, "sweeps": sweeps,
            "residual": resid}


def upscaled_cost(a, b, plan_c, N, kappa, p, d=2):
    """<pi-hat_xi, C> = sum over supp(pi-hat) of a_i pi-hat_ij b_j rho(x_i,y_j)^p.

    Sec. 4 (the sum over the support of the upscaled coupling); Alg. 4 step 3.
    supp(pi-hat) is the union of the fine block pairs X_k x Y_l with pi~*_kl > 0.
    """
    n = N // kappa
    X = grid_points(N, d)
    shape, off = _blocked(N, kappa, d)
    perm = tuple(2 * a for a in range(d)) + off          # block axes first, then offsets
    blk = np.arange(N ** d).reshape(shape).transpose(perm).reshape(n ** d, -1)
    total = 0.0
    for k, l in zip(*np.nonzero(plan_c)):
        I, J = blk[k], blk[l]
        pij = plan_c[k, l] * float(kappa) ** (-2 * d)
        total += (a[I][:, None] * pij * b[J][None, :] * ground_cost(X[I], X[J], p)).sum()
    return total


def tv_weights(N, p, d=2):
    """w_i = rho(x-bar, x_i)^p with x-bar = mean of the grid (Alg. 2 and Alg. 4)."""
    X = grid_points(N, d)
    xbar = X.mean(axis=0, keepdims=True)
    return ground_cost(xbar, X, p)[0]


def tv_correction(mu_hat, mu, N, p, d=2):
    """Delta = TV_p^w(mu-hat, mu) = 2^(1-1/p) <w, |mu-hat - mu|>^(1/p) (eq. weighted TV)."""
    s = float(np.dot(tv_weights(N, p, d), np.abs(mu_hat - mu)))
    return 2.0 ** (1.0 - 1.0 / p) * s ** (1.0 / p)


def ub_primal(mu, nu, N, kappa, p, xi=1e-13, max_sweeps=1000, plan_c=None, d=2):
    """Upscaling upper bound W-hat_p + Delta_mu-hat + Delta_nu-hat (Sec. 3.4, Alg. 4)."""
    if plan_c is None:
        mt, nt = sumpool(mu, N, kappa, d), sumpool(nu, N, kappa, d)
        plan_c, _, _, _ = exact_ot(coarse_cost_centre(N, kappa, p, d), mt, nt)
    fit = ipf(mu, nu, plan_c, N, kappa, xi, max_sweeps, d)
    w_hat_p = upscaled_cost(fit["a"], fit["b"], plan_c, N, kappa, p, d)
    d_mu = tv_correction(fit["mu_hat"], mu, N, p, d)
    d_nu = tv_correction(nu, fit["nu_hat"], N, p, d)
    w_hat = max(w_hat_p, 0.0) ** (1.0 / p)
    return {"ub_primal": w_hat + d_mu + d_nu, "w_hat": w_hat, "w_hat_p": w_hat_p,
            "delta_mu": d_mu, "delta_nu": d_nu, "plan": plan_c, **fit}


# --------------------------------------------------------------------------
# Primal upscaling with a general normalized positive kernel K (Sec. 3.4, eq.
# coupling tensor upscale; the uniform kernel above is K = kappa^-2d).  d = 2.
# K is a (kappa^2, kappa^2) array: K[u, v] weighs the pair (offset u in the
# source block, offset v in the target block); offsets are row-major in the
# block, u = u1 * kappa + u2.  pi-hat_ij = pi~_{k(i) l(j)} K[u(i), v(j)].
# --------------------------------------------------------------------------
def _to_blocks(v, N, kappa):
    """Flat pixel vector -> (n^2, kappa^2) array [block k, offset u]."""
    n = N // kappa
    return np.asarray(v, dtype=np.float64).reshape(n, kappa, n, kappa).transpose(0, 2, 1, 3).reshape(
        n * n, kappa * kappa)


def _from_blocks(Bk, N, kappa):
    """(n^2, kappa^2) block array -> flat pixel vector (inverse of _to_blocks)."""
    n = N // kappa
    return Bk.reshape(n, n, kappa, kappa).transpose(0, 2, 1, 3).reshape(N * N)


def upscaled_plan_apply_K(plan_c, K, v, N, kappa):
    """(pi-hat v)_i = sum_l pi~_{k(i) l} sum_v K[u(i), v'] v_{(l, v')}."""
    V = _to_blocks(v, N, kappa)
    return _from_blocks(plan_c @ (V @ np.asarray(K).T), N, kappa)


def upscaled_plan_apply_KT(plan_c, K, u, N, kappa):
    """(pi-hat^T u)_j = sum_k pi~_{k l(j)} sum_u K[u', v(j)] u_{(k, u')}."""
    U = _to_blocks(u, N, kappa)
    return _from_blocks(plan_c.T @ (U @ np.asarray(K)), N, kappa)


def ipf_K(mu, nu, plan_c, K, N, kappa, xi=1e-13, max_sweeps=1000):
    """IPF of pi-hat = pi~ (x) K to (mu, nu) (Sec. 3.4 step 2, Alg. 4), b = 1 first."""
    b = np.ones(N * N)
    sweeps, resid = 0, np.inf
    while sweeps < max_sweeps:
        a = _safe_div(mu, upscaled_plan_apply_K(plan_c, K, b, N, kappa))
        b = _safe_div(nu, upscaled_plan_apply_KT(plan_c, K, a, N, kappa))
        sweeps += 1
        mu_hat = a * upscaled_plan_apply_K(plan_c, K, b, N, kappa)
        nu_hat = b * upscaled_plan_apply_KT(plan_c, K, a, N, kappa)
        resid = np.abs(mu_hat - mu).sum() + np.abs(nu - nu_hat).sum()
        if resid < xi:
            break
    return {"a": a, "b": b, "mu_hat": mu_hat, "nu_hat": nu_hat, "sweeps": sweeps,
            "residual": resid}


def upscaled_cost_K(a, b, plan_c, K, N, kappa, p):
    """<pi-hat_xi, C> over supp(pi-hat): sum over (k, l) in supp pi~ of
    pi~_kl sum_{u,v} a_(k,u) K[u,v] b_(l,v) rho(x_(k,u), y_(l,v))^p (Sec. 4)."""
    X = grid_points(N)
    idx = _to_blocks(np.arange(N * N), N, kappa).astype(np.int64)
    Ab, Bb = _to_blocks(a, N, kappa), _to_blocks(b, N, kappa)
    K = np.asarray(K, dtype=np.float64)
    total = 0.0
    for k, l in zip(*np.nonzero(plan_c)):
        c = ground_cost(X[idx[k]], X[idx[l]], p)
        total += plan_c[k, l] * (Ab[k][:, None] * K * Bb[l][None, :] * c).sum()
    return total


def ub_primal_K(mu, nu, N, kappa, p, K, xi=1e-13, max_sweeps=1000, plan_c=None):
    """Upscaling upper bound with kernel K: W-hat_p + Delta_mu-hat + Delta_nu-hat (Sec. 3.4)."""
    if plan_c is None:
        mt, nt = sumpool(mu, N, kappa), sumpool(nu, N, kappa)
        plan_c, _, _, _ = exact_ot(coarse_cost_centre(N, kappa, p), mt, nt)
    fit = ipf_K(mu, nu, plan_c, K, N, kappa, xi, max_sweeps)
    w_hat_p = upscaled_cost_K(fit["a"], fit["b"], plan_c, K, N, kappa, p)
    d_mu = tv_correction(fit["mu_hat"], mu, N, p)
    d_nu = tv_correction(nu, fit["nu_hat"], N, p)
    w_hat = max(w_hat_p, 0.0) ** (1.0 / p)
    return {"ub_primal": w_hat + d_mu + d_nu, "w_hat": w_hat, "w_hat_p": w_hat_p,
            "delta_mu": d_mu, "delta_nu": d_nu, "plan": plan_c, **fit}


def gaussian_kernel(kappa, sigma):
    """A normalized positive kernel favouring equal offsets: K[u, v] proportional
    to exp(-|u - v|^2 / (2 sigma^2)) over the in-block offsets, sum 1."""
    o = np.array([(u // kappa, u % kappa) for u in range(kappa * kappa)], dtype=np.float64)
    d2 = ((o[:, None, :] - o[None, :, :]) ** 2).sum(-1)
    K = np.exp(-d2 / (2.0 * sigma * sigma))
    return K / K.sum()


# --------------------------------------------------------------------------
# Dual upscaling lower bound: Sec. 3.5, eq. (lazy c-transform), Alg. 5.
# --------------------------------------------------------------------------
def upsample_potential(f_c, N, kappa, d=2):
    """f-hat = {R_{f~, X~}(x_i)}: multilinear interpolation of f~ at the block centres.

    Sec. 3.5 allows any interpolation R; this one is bilinear (d = 2) or
    trilinear (d = 3) in block-centre coordinates, extrapolated linearly from
    the edge cells outside the hull of the centres.  Coordinate
    t = (x - (kappa-1)/2) / kappa per axis.
    """
    n = N // kappa
    if d != 2:
        return _upsample_multilinear(f_c, N, kappa, d)
    F = np.asarray(f_c, dtype=np.float64).reshape(n, n)
    if n == 1:
        return np.full(N * N, F[0, 0])
    t = (np.arange(N) - (kappa - 1) / 2.0) / kappa
    k0 = np.clip(np.floor(t).astype(np.int64), 0, n - 2)
    w = t - k0
    r0, r1 = k0[:, None], (k0 + 1)[:, None]
    c0, c1 = k0[None, :], (k0 + 1)[None, :]
    wr, wc = w[:, None], w[None, :]
    top = (1.0 - wc) * F[r0, c0] + wc * F[r0, c1]
    bot = (1.0 - wc) * F[r1, c0] + wc * F[r1, c1]
    return ((1.0 - wr) * top + wr * bot).ravel()


def _upsample_multilinear(f_c, N, kappa, d):
    """The same interpolation for any d: per axis, the value at t is
    (1 - w) F[k0] + w F[k0 + 1] with k0 = clip(floor(t), 0, n-2), w = t - k0,
    applied along the axes one after another (a tensor-product rule)."""
    n = N // kappa
    F = np.asarray(f_c, dtype=np.float64).reshape((n,) * d)
    if n == 1:
        return np.full(N ** d, F.ravel()[0])
    t = (np.arange(N) - (kappa - 1) / 2.0) / kappa
    k0 = np.clip(np.floor(t).astype(np.int64), 0, n - 2)
    w = t - k0
    L = np.zeros((N, n))                   # 1-D interpolation matrix, N x n
    L[np.arange(N), k0] = 1.0 - w
    L[np.arange(N), k0 + 1] += w
    for a in range(d):
        F = np.moveaxis(np.tensordot(L, F, axes=([1], [a])), 0, a)
    return F.ravel()


def c_transform(h, N, p, chunk=1024, d=2):
    """h^c_j = min_i rho(x_i, y_j)^p - h_i over the whole grid (Sec. 3.5; eq. lazy c-transform)."""
    X = grid_points(N, d)
    m = N ** d
    out = np.empty(m)
    for j0 in range(0, m, chunk):
        J = slice(j0, min(m, j0 + chunk))
        out[J] = (ground_cost(X, X[J], p) - h[:, None]).min(axis=0)
    return out


def c_transform_at(h, N, p, J, d=2):
    """h^c_j for the listed outputs j only (the same definition as
    ``c_transform``, one output at a time): for spot checks on grids whose
    full transform the oracle cannot afford."""
    X = grid_points(N, d)
    J = np.asarray(J, dtype=np.int64)
    return np.array([float((ground_cost(X, X[j:j + 1], p)[:, 0] - h).min()) for j in J])


def centre_potential(f_c, mu_c):
    """Shift f~ so that <f~, mu~> = 0; the dual objective is unchanged (masses are 1)."""
    return f_c - float(np.dot(f_c, mu_c))


def lb_from_potential(mu, nu, N, kappa, p, f_c, d=2):
    """Alg. 5 from the coarse potential on: f-hat, g = f-hat^c, f = g^c, LB."""
    f_hat = upsample_potential(f_c, N, kappa, d)
    g = c_transform(f_hat, N, p, d=d)
    f = c_transform(g, N, p, d=d)       # the cost is symmetric, so g^c uses the same map
    s = float(np.dot(f, mu) + np.dot(g, nu))
    return {"lb": max(s, 0.0) ** (1.0 / p), "lb_p": s, "f_hat": f_hat, "f": f, "g": g}


def lb_dual(mu, nu, N, kappa, p, f_c=None, d=2):
    """Upscaling lower bound (<f, mu> + <g, nu>)^(1/p) (Sec. 3.5, eq. upscaling LB, Alg. 5)."""
    mt = sumpool(mu, N, kappa, d)
    if f_c is None:
        nt = sumpool(nu, N, kappa, d)
        _, f_c, _, _ = exact_ot(coarse_cost_centre(N, kappa, p, d), mt, nt)
    f_c = centre_potential(np.asarray(f_c, dtype=np.float64), mt)
    out = lb_from_potential(mu, nu, N, kappa, p, f_c, d)
    out["f_coarse"] = f_c
    return out


def lb_dual_from_g(mu, nu, N, kappa, p, g_c, d=2):
    """The same upscaling lower bound started from the other coarse potential
    (Sec. 3.5 applies to either side): g-hat = R(g~ - <g~, nu~>), f = g-hat^c,
    g = f^c, LB = (<f, mu> + <g, nu>)^(1/p)."""
    nt = sumpool(nu, N, kappa, d)
    g_c = np.asarray(g_c, dtype=np.float64)
    g_c = g_c - float(np.dot(g_c, nt))
    g_hat = upsample_potential(g_c, N, kappa, d)
    f = c_transform(g_hat, N, p, d=d)   # the cost is symmetric: the same map
    g = c_transform(f, N, p, d=d)
    s = float(np.dot(f, mu) + np.dot(g, nu))
    return {"lb": max(s, 0.0) ** (1.0 / p), "lb_p": s, "g_hat": g_hat, "f": f, "g": g}


def lb_dual_symmetric(mu, nu, N, kappa, p, f_c=None, g_c=None, d=2):
    """The larger of the two upscaling lower bounds, from f~ and from g~
    (both coarse potentials of one exact coarse solution, Sec. 3.5)."""
    if f_c is None or g_c is None:
        mt, nt = sumpool(mu, N, kappa, d), sumpool(nu, N, kappa, d)
        _, f_c, g_c, _ = exact_ot(coarse_cost_centre(N, kappa, p, d), mt, nt)
    a = lb_dual(mu, nu, N, kappa, p, f_c=f_c, d=d)
    b = lb_dual_from_g(mu, nu, N, kappa, p, g_c, d)
    return a if a["lb_p"] >= b["lb_p"] else b


def lb_grad_mu(mu, f, lb_p, p):
    """Derivative of the lower bound along the simplex, d LB / d mu_i.

    For fixed potentials the dual objective S = <f, mu> + <g, nu> is linear in
    mu (Sec. 3.5, the proposition that a c-transformed pair is admissible);
    along the mass-preserving direction e_i - mu its derivative is
    f_i - <f, mu>, and LB = S^(1/p) gives (1/p) S^(1/p - 1) (f_i - <f, mu>).
    """
    if lb_p <= 0.0:
        return np.zeros_like(f)
    return (1.0 / p) * lb_p ** (1.0 / p - 1.0) * (f - float(np.dot(f, mu)))


# --------------------------------------------------------------------------
# Whole method for one pair.
# --------------------------------------------------------------------------
def bounds(mu, nu, N, kappa, p, xi=1e-13, max_sweeps=1000, d=2):
    """All quantization bounds of Sec. 3 for one pair of measures on [N]^d."""
    mt, nt = sumpool(mu, N, kappa, d), sumpool(nu, N, kappa, d)
    Ct = coarse_cost_centre(N, kappa, p, d)
    plan_c, f_c, g_c, Lt = exact_ot(Ct, mt, nt)
    ubw = ub_weighted(mu, nu, N, kappa, p, d)
    ubp = ub_primal(mu, nu, N, kappa, p, xi, max_sweeps, plan_c=plan_c, d=d)
    lbd = lb_dual(mu, nu, N, kappa, p, f_c=f_c, d=d)
    return {"ub_weighted": ubw["ub_weighted"], "ub_primal": ubp["ub_primal"],
            "lb": lbd["lb"], "lb_p": lbd["lb_p"], "w_hat_p": ubp["w_hat_p"],
            "delta_mu": ubp["delta_mu"], "delta_nu": ubp["delta_nu"],
            "ipf_sweeps": ubp["sweeps"], "ipf_residual": ubp["residual"],
            "plan_coarse": plan_c, "f_coarse": lbd["f_coarse"], "L_ctilde": Lt,
            "cbar": ubw["cbar"], "f": lbd["f"], "g": lbd["g"], "f_hat": lbd["f_hat"]}
