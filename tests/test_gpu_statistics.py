"""Statistical validation of the GPU library against the paper's time-scale
experiment (Sec. 4.1, the arrival-time Epps effect): Monte Carlo replications
of a bivariate GBM (correlation 0.35) observed at Poisson arrivals of rate
1/5 on a 1-s grid over T = 28,800 s, correlations from the batched sweep at
the cutoffs Eq. (19) gives for sampling intervals of 1 to 100 s.

What is checked:
- given each replication's arrival times, the estimator's expectation has a
  closed form (Eqs. (2)/(3) with the grid increments' moments; see
  stat_helpers.grid_pair_conditional_sigma): for every interval, basis and
  entry, Sigma minus that conditional expectation has mean zero within four
  standard errors over the replications (the law of total expectation makes
  this exact, whatever the interval-to-cutoff conversion of Eq. (19));
- R_12 against the ratio of those expectations, corrected to second order
  for the ratio's own bias (the Sigma entries fluctuate by a few per cent
  around their expectations), within four standard errors plus 1e-3 for
  the neglected third-order terms;
- the Dirichlet curve rises with the interval (the Epps effect itself) and
  the Fejer estimator is biased upwards against the Dirichlet one, as the
  paper states. The replication means against the theoretical curve
  Eq. (18) are recorded in the design notes, not asserted: Eq. (19) is an
  approximate conversion (the paper's footnote).

Second, the accuracy experiment (Sec. 3.2): a bivariate GBM of 100 points over
one day, the second asset observed at every second point of the first. With
independent Gaussian increments the estimator's expectation has a closed
form, Eq. (2) / (3) with the increments' moments,
  E[Sigma_ab] = sum_{u,v} K_N(t_u - t_v) (Cov(d_u^a, d_v^b) + E d_u^a E d_v^b),
K_N(x) = sum_{|k|<=N} w_k e^{-ikx} (Dirichlet or Fejer weights), summed here
over the return pairs directly; the replication means of the GPU's Sigma lie
within four standard errors of it at every cutoff, and the co-volatility
shows the asynchrony bias growing with N that the paper reports.

The same replications give the other curve of the accuracy figure, the MSE:
the estimator is a Gaussian bilinear form in the step increments, so its
variance has a closed form (2 tr(BVBV) + 4 mu^T BVB mu); the replication
variance of every entry lies within four standard errors of it, and the
replication MSE against the true integrated covariance within four standard
errors of variance + bias^2.

Third, the sensitivity test (App. B): synchronous bivariate GBMs of 10^4
points over one day with integrated variances in 0.1-0.3 and covariances in
-0.1-0.1; the estimates at the Nyquist cutoff lie on a line of slope 1
through 0 against the truth, for both bases.
"""
import numpy as np
import pytest

import oracle
from paper_2003_02842_gb300 import synth

from gpu_helpers import to_dev
from stat_helpers import expected_sigma, grid_pair_conditional_sigma, sigma_moments, variance_se

pytestmark = pytest.mark.gpu

REPS = 512
T = 28800
RATE = 1.0 / 5.0
RHO = 0.35
INTERVALS = [1, 2, 3, 5, 10, 20, 30, 50, 100]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def sweep():
    import paper_2003_02842_gb300 as mm
    ev = synth.epps_replications(2003, REPS, T=T, rate=RATE, rho=RHO)
    off, t, p = to_dev(ev)
    # ascending cutoffs: the largest interval first
    dts = sorted(INTERVALS, reverse=True)
    cut = [oracle.n_from_dt(T, dt) for dt in dts]
    assert all(a < b for a, b in zip(cut, cut[1:]))
    out = {}
    for basis in ("dirichlet", "fejer"):
        b = mm.mm_batch_create(REPS, 2, cut[-1], ev.n_events, tol=1e-6, kernel="es", basis=basis)
        S, R = mm.mm_batch_epps(b, off, t, p, cut)
        assert mm.mm_batch_sync(b) == 0
        S = S.double().cpu().numpy()  # [reps, cutoffs, 2, 2]
        r12 = R[:, :, 0, 1].double().cpu().numpy()
        mm.mm_batch_destroy(b)
        E = np.zeros_like(S)
        C, m = ev.meta["step_cov"], ev.meta["step_mean"]
        for r in range(REPS):
            E[r] = grid_pair_conditional_sigma(ev.asset(2 * r)[0], ev.asset(2 * r + 1)[0], cut, basis, C, m)
        out[basis] = {dt: r12[:, j] for j, dt in enumerate(dts)}
        out[basis + "_S"] = {dt: S[:, j] for j, dt in enumerate(dts)}
        out[basis + "_E"] = {dt: E[:, j] for j, dt in enumerate(dts)}
    return out


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_sigma_matches_its_expectation_given_the_arrival_times(sweep, basis):
    for dt in INTERVALS:
        S, E = sweep[basis + "_S"][dt], sweep[basis + "_E"][dt]
        for a, b in [(0, 0), (1, 1), (0, 1)]:
            x = S[:, a, b] - E[:, a, b]
            se = x.std(ddof=1) / np.sqrt(REPS)
            assert abs(x.mean()) <= 4.0 * se, (basis, dt, a, b, x.mean(), se, E[:, a, b].mean())


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_correlation_matches_the_ratio_of_expectations(sweep, basis):
    # R = S12 / sqrt(S11 S22) with relative deviations x, y, z of the three
    # entries from their expectations: E[R] / rho_E - 1 = -Cov(x, y)/2
    # - Cov(x, z)/2 + 3 Var(y)/8 + 3 Var(z)/8 + Cov(y, z)/4 to second order
    for dt in INTERVALS:
        S, E, r12 = sweep[basis + "_S"][dt], sweep[basis + "_E"][dt], sweep[basis][dt]
        rho_e = E[:, 0, 1] / np.sqrt(E[:, 0, 0] * E[:, 1, 1])
        x = S[:, 0, 1] / E[:, 0, 1] - 1.0
        y = S[:, 0, 0] / E[:, 0, 0] - 1.0
        z = S[:, 1, 1] / E[:, 1, 1] - 1.0
        assert max(y.std(), z.std()) <= 0.1  # the expansion's regime
        cv = lambda u, v: float(np.mean((u - u.mean()) * (v - v.mean())))
        corr2 = -cv(x, y) / 2 - cv(x, z) / 2 + 3 * cv(y, y) / 8 + 3 * cv(z, z) / 8 + cv(y, z) / 4
        d = r12 - rho_e * (1.0 + corr2)
        se = d.std(ddof=1) / np.sqrt(REPS)
        assert abs(d.mean()) <= 4.0 * se + 1e-3, (basis, dt, r12.mean(), rho_e.mean(), corr2, se)


def test_epps_curve_rises_with_the_interval(sweep):
    m = {dt: sweep["dirichlet"][dt].mean() for dt in INTERVALS}
    se = {dt: sweep["dirichlet"][dt].std(ddof=1) / np.sqrt(REPS) for dt in INTERVALS}
    for a, b in [(1, 5), (5, 20), (20, 100)]:
        assert m[b] - m[a] > 3.0 * np.hypot(se[a], se[b]), (a, b, m[a], m[b])


def test_fejer_biased_upwards(sweep):
    diffs = []
    for dt in INTERVALS:
        d = sweep["fejer"][dt] - sweep["dirichlet"][dt]  # paired: the same replications
        se = d.std(ddof=1) / np.sqrt(len(d))
        assert d.mean() > -3.0 * se, (dt, d.mean(), se)
        diffs.append(d.mean())
    assert np.mean(diffs) > 0.0


MB_REPS = 8192
MB_N = 100
MB_CUTS = [1, 2, 3, 5, 10, 20, 30, 40, 49, 50]


@pytest.fixture(scope="module")
def accuracy_sweep():
    import paper_2003_02842_gb300 as mm
    ev = synth.mse_bias_replications(2003, MB_REPS, n=MB_N)
    off, t, p = to_dev(ev)
    out = {}
    for basis in ("dirichlet", "fejer"):
        b = mm.mm_batch_create(MB_REPS, 2, MB_CUTS[-1], ev.n_events, tol=1e-6, kernel="es", basis=basis)
        S, _ = mm.mm_batch_epps(b, off, t, p, MB_CUTS)
        assert mm.mm_batch_sync(b) == 0
        out[basis] = S.double().cpu().numpy()  # [reps, cutoffs, 2, 2]
        mm.mm_batch_destroy(b)
    return ev.meta, out


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_monte_carlo_mean_matches_the_estimators_expectation(accuracy_sweep, basis):
    meta, out = accuracy_sweep
    S = out[basis]
    for j, N in enumerate(MB_CUTS):
        E = expected_sigma(meta, N, basis)
        for a, b in [(0, 0), (1, 1), (0, 1)]:
            x = S[:, j, a, b]
            se = x.std(ddof=1) / np.sqrt(len(x))
            assert abs(x.mean() - E[a, b]) <= 4.0 * se, (basis, N, a, b, x.mean(), E[a, b], se)


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_monte_carlo_variance_and_mse_match_closed_form(accuracy_sweep, basis):
    meta, out = accuracy_sweep
    S = out[basis]
    C = meta["step_cov"]
    # the integrated (co)variance over the steps each pair of returns covers
    truth = np.array([[(MB_N - 1) * C[0, 0], (MB_N - 2) * C[0, 1]], [(MB_N - 2) * C[1, 0], (MB_N - 2) * C[1, 1]]])
    for j, N in enumerate(MB_CUTS):
        E, Var = sigma_moments(meta, N, basis)
        for a, b in [(0, 0), (1, 1), (0, 1)]:
            x = S[:, j, a, b]
            assert abs(x.var() - Var[a, b]) <= 4.0 * variance_se(x), (basis, N, a, b, x.var(), Var[a, b])
            e2 = (x - truth[a, b]) ** 2
            mse = Var[a, b] + (E[a, b] - truth[a, b]) ** 2
            se = e2.std(ddof=1) / np.sqrt(len(e2))
            assert abs(e2.mean() - mse) <= 4.0 * se, (basis, N, a, b, e2.mean(), mse, se)


def test_covolatility_bias_grows_with_the_cutoff(accuracy_sweep):
    meta, out = accuracy_sweep
    x = out["dirichlet"][:, :, 0, 1]
    lo, hi = MB_CUTS.index(5), MB_CUTS.index(50)
    se = np.hypot(x[:, lo].std(ddof=1), x[:, hi].std(ddof=1)) / np.sqrt(MB_REPS)
    truth = (MB_N - 2) * meta["step_cov"][0, 1]  # the steps both assets' returns cover
    assert x[:, hi].mean() < x[:, lo].mean() - 4.0 * se
    assert x[:, hi].mean() < 0.75 * truth  # the Epps drop at the finest time-scale


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_sensitivity_estimates_track_the_true_covariance(basis):
    # App. B: synchronous GBMs, true integrated variances 0.1..0.3 and
    # covariance -0.1..0.1, estimated at the synchronous Nyquist cutoff
    # (Algorithm 2: floor((n - 1) / 2)); both bases are unbiased here (their
    # weights sum to one over independent returns), so estimate against truth
    # is a line of slope 1 through 0. Noise: about 0.003 per estimate, a slope
    # standard error near 0.01 over 96 problems.
    import paper_2003_02842_gb300 as mm
    covs = synth.sensitivity_covariances(2003, 24)
    reps, n = 4, 10000
    ev = synth.sensitivity_replications(2003, covs, reps=reps, n=n)
    off, t, p = to_dev(ev)
    N = (n - 1) // 2
    b = mm.mm_batch_create(len(covs) * reps, 2, N, ev.n_events, tol=1e-6, kernel="es", basis=basis)
    S, _ = mm.mm_batch_epps(b, off, t, p, [N])
    assert mm.mm_batch_sync(b) == 0
    S = S[:, 0].double().cpu().numpy()
    mm.mm_batch_destroy(b)
    truth = ev.meta["truth"]
    for a, c in [(0, 0), (1, 1), (0, 1)]:
        slope, icpt = np.polyfit(truth[:, a, c], S[:, a, c], 1)
        assert abs(slope - 1.0) <= 0.05 and abs(icpt) <= 0.01, (basis, a, c, slope, icpt)
