"""GPU parity of the float32 spreading where one grid tile holds a whole busy
asset: at a low cutoff the oversampled grid has only a few hundred cells
(M_r ~ 4N), so a full day of one-second observations (28,800 events) or a
continuous-time asset of 50,000 or more events lands in a single tile. The
tile's integer accumulation must keep Eq. (15) within the float32 bound
there as well as for sparse tiles.

Cutoffs are the serving workload's: Eq. (19) for sampling intervals of
600 s and 60 s over an 8-hour day (N = 23 and 239), the Nyquist cutoff,
and a few others from N = 1 up.

Tolerances: coefficients, Eq. (15) per asset <= 1e-5 at tolerance 1e-6
(float32 path), the bound of the other parity tests; Sigma relative to the
assets' realised variances <= 1e-5 (float32 coefficients and the 3xTF32
contraction, whose relative product error is about 2^-21); R <= 1e-4.
"""
import numpy as np
import pytest

import oracle
from paper_2003_02842_gb300 import synth

from gpu_helpers import rel_l2_rows, run, to_dev

pytestmark = pytest.mark.gpu

COEF = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def full_day():
    # two assets observed every second of an 8-hour day
    return synth.c1_sync(7, n=28800)


@pytest.mark.parametrize("N", [1, 5, 23, 239, 2000])
@pytest.mark.parametrize("kernel", ["es", "kb", "gauss"])
def test_full_day_on_the_one_second_grid(full_day, N, kernel):
    ev = full_day
    out = run(dict(tol=1e-6, kernel=kernel, basis="dirichlet", prec="bf16x3"), ev, N)
    assert out["status"] == 0 and out["info"]["spread_poly"] == 1
    ref = oracle.coeffs_F(ev.offsets, ev.t, ev.logp, N)
    err = rel_l2_rows(out["F"], ref)
    assert np.all(err <= COEF), err


@pytest.mark.parametrize("n,N", [(50000, 1), (50000, 100), (50000, 1000), (200000, 10), (200000, 1000)])
def test_dense_continuous_time_assets(n, N):
    ev = synth.random_events(8 + n // 50000, D=2, n_range=(n, n), T=28800.0)
    out = run(dict(tol=1e-6, kernel="es", basis="dirichlet", prec="bf16x3"), ev, N)
    assert out["status"] == 0
    ref = oracle.coeffs_F(ev.offsets, ev.t, ev.logp, N)
    err = rel_l2_rows(out["F"], ref)
    assert np.all(err <= COEF), err


@pytest.fixture(scope="module")
def busy_day():
    # six assets, each observing about 95 % of the day's seconds
    return synth.c5_day(9, D=6, T=28800, lam_lo=3.0, lam_hi=3.0)


@pytest.mark.parametrize("mode", ["nyquist", "dt60", "dt600"])
def test_full_day_window_at_each_serving_cutoff(busy_day, mode):
    # the serving form's window rescaling over the whole day, at each of its
    # three cutoff rules, through the coefficient call the serving slots use
    import paper_2003_02842_gb300 as mm
    ev = busy_day
    win = (0.0, 28800.0)
    if mode == "nyquist":
        N = min(14399, oracle.nyquist(ev.offsets, ev.t, *win))
    else:
        N = int(oracle.n_from_dt(28800.0, {"dt60": 60.0, "dt600": 600.0}[mode]))
    plan = mm.mm_plan_create(D=ev.D, N_max=N, max_events=ev.n_events, tol=1e-6, kernel="es", basis="fejer",
                             prec="bf16x3")
    off, t, p = to_dev(ev)
    F, Nu = mm.mm_coeffs(plan, off, t, p, N, window=win)
    assert mm.mm_plan_sync(plan) == 0 and Nu == N
    ref = oracle.coeffs_F(ev.offsets, ev.t, ev.logp, N, window=win)
    err = rel_l2_rows(F.cpu().numpy(), ref)
    assert np.all(err <= COEF), (N, err)
    mm.mm_destroy(plan)


@pytest.mark.parametrize("dt", [0.0, 60.0, 600.0])
def test_full_day_server_request(busy_day, dt):
    # one request over the whole day for every asset: Sigma against the
    # oracle relative to the realised variances, R directly
    import time
    import paper_2003_02842_gb300 as mm
    ev = busy_day
    srv = mm.mm_server_create(D=ev.D, N_max=14399, max_events=ev.n_events, max_slots=2, tol=1e-6, kernel="es",
                              basis="fejer", prec="3xtf32")
    mm.mm_server_load(srv, ev.offsets, ev.t, ev.logp)
    assets = np.arange(ev.D, dtype=np.int32)
    tk = mm.mm_server_submit(srv, 0.0, 28800.0, assets, dt=dt, sigma=True)
    got, t_end = [], time.time() + 120.0
    while not got and time.time() < t_end:
        got = mm.mm_server_poll(srv, wait=0.05)
    assert len(got) == 1 and got[0]["ticket"] == tk
    c = got[0]
    assert c["status"] == 0, c
    o = oracle.estimate(ev.offsets, ev.t, ev.logp, N=c["N"], basis="fejer", window=(0.0, 28800.0))
    V = np.array([np.sum(np.diff(ev.asset(i)[1]) ** 2) for i in range(ev.D)])
    err = np.abs(c["Sigma"].astype(np.float64) - o["Sigma"]) / np.sqrt(np.outer(V, V))
    assert np.max(err) <= 1e-5, (c["N"], np.max(err))
    assert np.max(np.abs(c["R"].astype(np.float64) - o["R"])) <= 1e-4
    mm.mm_server_destroy(srv)


def test_batched_sweep_with_full_day_assets():
    # replications whose assets observe every second, swept up to N = 239:
    # the whole asset falls in one spreading tile
    import paper_2003_02842_gb300 as mm
    reps, D = 3, 2
    ev = synth.c4_batch(6, reps=reps, D=D, T=28800, median_n=40000, sdlog=0.0)
    assert np.all(np.diff(ev.offsets) == 28800)
    cutoffs = [1, 5, 23, 239]
    b = mm.mm_batch_create(reps=reps, D=D, N_max=max(cutoffs), max_events=ev.n_events, tol=1e-6, kernel="es",
                           basis="dirichlet")
    off, t, p = to_dev(ev)
    S, R = mm.mm_batch_epps(b, off, t, p, cutoffs)
    assert mm.mm_batch_sync(b) == 0
    F = mm.mm_batch_coeffs(b).cpu().numpy()
    S = S.cpu().numpy().astype(np.float64)
    for r in range(reps):
        a0, a1 = r * D, (r + 1) * D
        o0, o1 = int(ev.offsets[a0]), int(ev.offsets[a1])
        e = synth.Events(ev.offsets[a0:a1 + 1] - o0, ev.t[o0:o1].copy(), ev.logp[o0:o1].copy())
        ref = oracle.coeffs_F(e.offsets, e.t, e.logp, max(cutoffs))
        err = rel_l2_rows(F[a0:a1], ref)
        assert np.all(err <= COEF), (r, err)
        V = np.array([np.sum(np.diff(e.asset(i)[1]) ** 2) for i in range(D)])
        for j, N in enumerate(cutoffs):
            o = oracle.estimate(e.offsets, e.t, e.logp, N=N, basis="dirichlet")
            assert np.max(np.abs(S[r, j] - o["Sigma"]) / np.sqrt(np.outer(V, V))) <= 1e-5, (r, N)
    mm.mm_batch_destroy(b)
