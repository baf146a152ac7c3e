"""The seeded generators on the CPU: the same seed gives the same data, the
workload shapes are the stated ones, and the draws have the distributions the
workload recipes state (checked statistically against their definitions, not
against the generators' own formulas)."""
import numpy as np

from paper_2003_02842_gb300 import synth


def test_same_seed_same_events():
    a, b = synth.c2_async(3), synth.c2_async(3)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.t, b.t) and np.array_equal(a.logp, b.logp)
    c = synth.c2_async(4)
    assert not np.array_equal(a.t[:50], c.t[:50])


def test_event_lists_sorted_and_distinct():
    ev = synth.c2_async(0)
    for i in range(ev.D):
        t, _ = ev.asset(i)
        assert np.all(np.diff(t) > 0)


def test_gbm_grid_increments_have_the_daily_covariance():
    # Algorithm 1: log-price increments over a step of dt days have covariance
    # cov * dt and mean (mu - sigma^2 / 2) dt
    cov = synth.bivariate_cov(0.1, 0.2, 0.35)
    n, dt = 200001, 1.0 / 1000.0
    lp = synth.gbm_grid(n, 0.01, cov, synth.rng_for(99, 0), dt_days=dt)
    inc = np.diff(lp, axis=0)
    emp = np.cov(inc.T) / dt
    assert np.allclose(emp, cov, rtol=0.02, atol=2e-3)


def test_gram_coefficients_shape_and_scale():
    D, N = 6, 5000
    F = synth.gram_coefficients(0, D, N)
    assert F.shape == (D, N + 1) and F.dtype == np.complex64
    assert np.array_equal(F, synth.gram_coefficients(0, D, N))
    # E|F(k)|^2 = (daily variance x the window in days) / (2 pi)^2
    expect = 0.1 * 28800 / 86400 / (2 * np.pi) ** 2
    emp = np.mean(np.abs(F.astype(np.complex128)) ** 2)
    assert abs(emp / expect - 1.0) < 0.03
    # real and imaginary parts independent and centred
    assert abs(np.mean(F.real * F.imag)) < 0.05 * expect


def test_sensitivity_covariances_in_range_and_definite():
    covs = synth.sensitivity_covariances(1, 200)
    for c in covs:
        assert 0.1 <= c[0, 0] <= 0.3 and 0.1 <= c[1, 1] <= 0.3 and -0.1 <= c[0, 1] <= 0.1
        assert c[0, 1] == c[1, 0] and np.linalg.eigvalsh(c).min() > 0
    ev = synth.sensitivity_replications(1, covs[:2], reps=2, n=500)
    assert ev.D == 8 and ev.meta["truth"].shape == (4, 2, 2)
    assert np.allclose(ev.meta["truth"][0], covs[0] * 499 / 500)


def test_request_stream_default_and_standing_windows():
    a = synth.c5_requests(2, n=200, D=50, T=3000, w_range=(300, 3000), k_range=(3, 20))
    # the default stream draws a fresh window per request
    assert len({(r["t0"], r["t1"]) for r in a}) == len(a)
    for r in a:
        assert 0.0 <= r["t0"] < r["t1"] <= 3000.0 and 300.0 <= r["t1"] - r["t0"] <= 3000.0
        assert 3 <= len(r["assets"]) <= 20 and len(set(r["assets"].tolist())) == len(r["assets"])
        assert r["dt"] in (0.0, 60.0, 600.0)
    b = synth.c5_requests(2, n=200, D=50, T=3000, w_range=(300, 3000), k_range=(3, 20), windows=5)
    assert len({(r["t0"], r["t1"]) for r in b}) == 5
