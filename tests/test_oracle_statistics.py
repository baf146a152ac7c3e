"""The oracle against the closed-form expectation of the estimator in the
accuracy experiment (Sec. 3.2): the Monte Carlo mean of the oracle's Sigma
over seeded replications lies within four standard errors of
E[Sigma_ab] = sum_{u,v} K_N(t_u - t_v) (Cov(d_u^a, d_v^b) + E d_u^a E d_v^b)
for both bases (Eqs. (2), (3)) at small, middle and Nyquist cutoffs; and the
closed form itself reproduces the paper's statements: no bias of the
integrated volatility at any N (Dirichlet), a co-volatility bias that grows
with N under asynchrony."""
import numpy as np
import pytest

import oracle
from paper_2003_02842_gb300 import synth

from stat_helpers import expected_sigma

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
