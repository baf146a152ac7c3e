"""The oracle against the closed-form expectation of the estimator in the
accuracy experiment (Sec. 3.2): the Monte Carlo mean of the oracle's Sigma
over seeded replications lies within four standard errors of
E[Sigma_ab] = sum_{u,v} K_N(t_u - t_v) (Cov(d_u^a, d_v^b) + E d_u^a E d_v^b)
for both bases (Eqs. (2), (3)) at small, middle and Nyquist cutoffs; and the
closed form itself reproduces the paper's statements: no bias of the
integrated volatility at any N (Dirichlet), a co-volatility bias that grows
with N under asynchrony. The variance, for the MSE of the same experiment:
the estimator is a Gaussian bilinear form in the step increments, whose mean
(checked against the pair sum above) and variance are closed forms, and the
oracle's Monte Carlo variance lies within four standard errors of the
latter."""
import numpy as np
import pytest

import oracle
from paper_2003_02842_gb300 import synth

from stat_helpers import expected_sigma, sigma_moments, variance_se

REPS = 3000


@pytest.fixture(scope="module")
def replications():
    ev = synth.mse_bias_replications(17, REPS)
    out = {}
    for basis in ("dirichlet", "fejer"):
        for N in (1, 5, 50):
            v = []
            for r in range(REPS):
                a, b = ev.offsets[2 * r], ev.offsets[2 * r + 2]
                off = ev.offsets[2 * r:2 * r + 3] - a
                v.append(oracle.estimate(off, ev.t[a:b], ev.logp[a:b], N=N, basis=basis)["Sigma"])
            out[(basis, N)] = np.array(v)
    return ev.meta, out


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
@pytest.mark.parametrize("N", [1, 5, 50])
def test_oracle_mean_matches_closed_form(replications, basis, N):
    meta, out = replications
    v = out[(basis, N)]
    E = expected_sigma(meta, N, basis)
    se = v.std(axis=0, ddof=1) / np.sqrt(REPS)
    assert np.all(np.abs(v.mean(axis=0) - E) <= 4.0 * se), (v.mean(axis=0), E, se)


def test_closed_form_volatility_unbiased_covolatility_epps():
    meta = synth.mse_bias_replications(0, 1).meta
    C, m = meta["step_cov"], meta["step_mean"]
    for N in (1, 2, 10, 25, 50):
        E = expected_sigma(meta, N, "dirichlet")
        # the first asset's integrated variance over its 99 steps, up to the
        # drift's contribution m^2 sum_{u,v} K_N(t_u - t_v) <= 99^2 m^2 (|K_N| <= 1)
        assert abs(E[0, 0] - 99 * C[0, 0]) <= 99 ** 2 * m[0] ** 2
    E = [expected_sigma(meta, N, "dirichlet")[0, 1] for N in (1, 10, 25, 50)]
    assert all(a > b for a, b in zip(E, E[1:]))


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
@pytest.mark.parametrize("N", [1, 5, 50])
def test_quadratic_form_mean_agrees_with_pair_sum(basis, N):
    # two routes to E[Sigma]: the sum over return pairs and the trace of the
    # bilinear form in the step increments
    meta = synth.mse_bias_replications(0, 1).meta
    E1 = expected_sigma(meta, N, basis)
    E2, _ = sigma_moments(meta, N, basis)
    assert np.allclose(E1, E2, rtol=1e-10, atol=1e-16)


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
@pytest.mark.parametrize("N", [1, 5, 50])
def test_oracle_variance_matches_closed_form(replications, basis, N):
    meta, out = replications
    v = out[(basis, N)]
    _, Var = sigma_moments(meta, N, basis)
    for a, b in [(0, 0), (1, 1), (0, 1)]:
        x = v[:, a, b]
        assert abs(x.var() - Var[a, b]) <= 4.0 * variance_se(x), (basis, N, a, b, x.var(), Var[a, b])


def test_variance_closed_form_special_case():
    # one step (n = 2), no drift: asset 1 has a single return d at time 0,
    # the kernel there is K_N(0) = sum_k w_k = 1, so Sigma_11 = d^2 with d
    # ~ N(0, C_11): mean C_11 and variance 2 C_11^2 (a centred Gaussian's square)
    meta = {"n": 2, "step_cov": np.array([[0.3, 0.1], [0.1, 0.2]]), "step_mean": np.zeros(2)}
    E, Var = sigma_moments(meta, 1, "dirichlet")
    assert np.isclose(E[0, 0], 0.3) and np.isclose(Var[0, 0], 2 * 0.3 ** 2)


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_grid_pair_conditional_expectation_agrees_with_pair_sum(basis):
    # the histogram-and-FFT closed form of E[Sigma | times] for the
    # arrival-time experiment against the pairwise sum over returns with
    # explicit step sets and mode-by-mode kernels
    from stat_helpers import grid_pair_conditional_sigma, grid_pair_conditional_sigma_bruteforce
    rng = np.random.default_rng(3)
    C = np.array([[2.0, 0.7], [0.7, 1.5]])
    m = np.array([0.3, -0.2])
    for trial in range(4):
        t1 = np.sort(rng.choice(80, size=14, replace=False))
        t2 = np.sort(rng.choice(80, size=11, replace=False))
        cut = [1, 3, 9, 17]
        got = grid_pair_conditional_sigma(t1, t2, cut, basis, C, m)
        for j, N in enumerate(cut):
            want = grid_pair_conditional_sigma_bruteforce(t1, t2, N, basis, C, m)
            assert np.allclose(got[j], want, rtol=1e-12, atol=1e-12), (trial, N, got[j], want)


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_oracle_epps_sigma_matches_conditional_expectation(basis):
    # the arrival-time experiment (Sec. 4.1) at a short horizon: the oracle's
    # Sigma minus its expectation given each replication's arrival times has
    # mean zero within four standard errors
    from stat_helpers import grid_pair_conditional_sigma
    reps, T = 300, 1500
    ev = synth.epps_replications(77, reps, T=T, rate=1 / 5)
    C, m = ev.meta["step_cov"], ev.meta["step_mean"]
    cut = [5, 30, 140]
    res = np.zeros((reps, len(cut), 2, 2))
    for r in range(reps):
        a0, a1 = 2 * r, 2 * r + 2
        o0, o1 = int(ev.offsets[a0]), int(ev.offsets[a1])
        e = synth.Events(ev.offsets[a0:a1 + 1] - o0, ev.t[o0:o1], ev.logp[o0:o1])
        E = grid_pair_conditional_sigma(e.asset(0)[0], e.asset(1)[0], cut, basis, C, m)
        for j, N in enumerate(cut):
            res[r, j] = oracle.estimate(e.offsets, e.t, e.logp, N=N, basis=basis)["Sigma"] - E[j]
    for j, N in enumerate(cut):
        for a, b in [(0, 0), (1, 1), (0, 1)]:
            x = res[:, j, a, b]
            assert abs(x.mean()) <= 4.0 * x.std(ddof=1) / np.sqrt(reps), (basis, N, a, b)
