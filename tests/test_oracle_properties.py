"""Property tests of the oracle on random tiny grids (hypothesis): the
quantization bounds bracket the exact W_p from the full LP in the order the
paper's statements give (Sec. 3.2 theorem: UB_w >= W; Sec. 3.3 theorem:
L_Cmin^(1/p) <= W; Sec. 3.4: UB_primal >= W, and with the uniform kernel
UB_primal >= UB_w since W-hat^p = <pi~*, C-bar> >= L_C-bar; Sec. 3.5
proposition: LB <= W).  The measures are random with some zero-mass pixels;
N, kappa | N and p vary."""
import numpy as np
import pytest

from oracle import qwb_oracle as O

hypothesis = pytest.importorskip("hypothesis")
st = hypothesis.strategies


@st.composite
def problems(draw):
    N = draw(st.sampled_from([2, 4, 6, 8]))
    kappa = draw(st.sampled_from([k for k in (1, 2, 3, 4, 8) if N % k == 0]))
    p = draw(st.sampled_from([1.0, 1.5, 2.0]))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    rng = np.random.default_rng(seed)
    mus = []
    for _ in range(2):
        w = rng.gamma(0.5, size=N * N)
        w[rng.random(N * N) < 0.2] = 0.0          # some empty pixels
        if w.sum() == 0.0:
            w[rng.integers(N * N)] = 1.0
        mus.append(w / w.sum())
    return N, kappa, p, mus[0], mus[1]


@hypothesis.settings(max_examples=200, deadline=None)
@hypothesis.given(problems())
def test_bounds_bracket_the_exact_distance(prob):
    N, kappa, p, mu, nu = prob
    W = O.wasserstein_exact(mu, nu, N, p)
    b = O.bounds(mu, nu, N, kappa, p)
    lmin = O.lb_mincost(mu, nu, N, kappa, p)
    tol = 1e-9 * max(1.0, W)
    assert b["lb"] <= W + tol, (b["lb"], W)
    assert lmin <= W + tol, (lmin, W)
    assert W <= b["ub_weighted"] + tol, (W, b["ub_weighted"])
    assert b["ub_weighted"] <= b["ub_primal"] + tol, (b["ub_weighted"], b["ub_primal"])
    if kappa == 1:                                 # no quantization: every bound is exact
        assert abs(b["ub_weighted"] - W) <= tol and abs(b["lb"] - W) <= 1e-7 * max(1.0, W)
