"""GPU parity of the serving form against the FP64 CPU oracle: each request
(asset subset, window, cutoff) matches the oracle run on that subset's
window events with the window rescaling of Algorithm 4 over [t0, t1]; a
request gives the same result alone and in a mix of concurrent requests;
the scheduler runs several requests at once and reports failures per
request; resident coefficient rows serve later requests over the same
window and cutoff (hits and misses counted exactly, eviction, no caching of
device-found Nyquist cutoffs, concurrent requests). Tolerances: R, max |dR| <= 1e-4; Sigma, max |dSigma_ij| /
sqrt(V_i V_j) <= 1e-4 with V the realised variances of the window."""
import numpy as np
import pytest

import oracle
from paper_2003_02842_gb300 import synth

from gpu_helpers import sigma_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def day():
    return synth.c5_day(3, D=24, T=3000, lam_lo=0.05, lam_hi=0.6)


def _server(day, **kw):
    import paper_2003_02842_gb300 as mm
    args = dict(D=day.D, N_max=1500, max_events=day.n_events, max_slots=4, tol=1e-6, kernel="es", basis="fejer")
    args.update(kw)
    srv = mm.mm_server_create(**args)
    mm.mm_server_load(srv, day.offsets, day.t, day.logp)
    return srv


def _wait(srv, n, timeout=60.0):
    import paper_2003_02842_gb300 as mm
    import time
    got, t_end = [], time.time() + timeout
    while len(got) < n and time.time() < t_end:
        got += mm.mm_server_poll(srv, wait=0.05)
    assert len(got) == n
    return {c["ticket"]: c for c in got}


def _check(day, req, c):
    assert c["status"] == 0, c
    w = synth.window_events(day, req["assets"], req["t0"], req["t1"])
    o = oracle.estimate(w.offsets, w.t, w.logp, N=c["N"], basis="fejer", window=(req["t0"], req["t1"]))
    # Sigma against the realised variances of the window (the scale the
    # NUFFT's whole-vector error bound of Eq. (15) controls; at a small cutoff
    # Sigma_ii(N) itself can be far smaller), R directly
    V = np.array([np.sum(np.diff(w.asset(i)[1]) ** 2) for i in range(w.D)])
    err = np.abs(c["Sigma"].astype(np.float64) - o["Sigma"]) / np.sqrt(np.outer(V, V))
    assert np.max(err) <= 1e-4
    assert np.max(np.abs(c["R"].astype(np.float64) - o["R"])) <= 1e-4


def test_requests_match_oracle_on_their_window(day):
    import paper_2003_02842_gb300 as mm
    srv = _server(day)
    reqs = synth.c5_requests(4, n=12, D=day.D, T=3000, w_range=(300, 3000), k_range=(2, day.D))
    reqs[0]["dt"], reqs[1]["dt"] = 0.0, 60.0  # the Nyquist and Eq. (19) modes both appear
    tk = [mm.mm_server_submit(srv, r["t0"], r["t1"], r["assets"], dt=r["dt"], sigma=True) for r in reqs]
    done = _wait(srv, len(reqs))
    for t, r in zip(tk, reqs):
        c = done[t]
        if r["dt"] > 0:
            T = r["t1"] - r["t0"]
            assert c["N"] == max(1, min(1500, int(np.floor(0.5 * (T / r["dt"] - 1.0)))))
        else:
            w = synth.window_events(day, r["assets"], r["t0"], r["t1"])
            assert c["N"] == min(1500, oracle.nyquist(w.offsets, w.t, r["t0"], r["t1"]))
        _check(day, r, c)
    mm.mm_server_destroy(srv)


def test_same_result_alone_and_in_a_mix(day):
    import paper_2003_02842_gb300 as mm
    srv = _server(day)
    x = {"t0": 400.0, "t1": 2600.0, "assets": np.array([3, 5, 7, 11, 13, 17, 19, 23], np.int32), "dt": 30.0}
    t_alone = mm.mm_server_submit(srv, x["t0"], x["t1"], x["assets"], dt=x["dt"], sigma=True)
    alone = _wait(srv, 1)[t_alone]
    _check(day, x, alone)
    mix = synth.c5_requests(5, n=40, D=day.D, T=3000, w_range=(300, 3000), k_range=(2, day.D))
    tks = [mm.mm_server_submit(srv, r["t0"], r["t1"], r["assets"], dt=r["dt"], sigma=True) for r in mix[:20]]
    t_mix = mm.mm_server_submit(srv, x["t0"], x["t1"], x["assets"], dt=x["dt"], sigma=True)
    tks += [mm.mm_server_submit(srv, r["t0"], r["t1"], r["assets"], dt=r["dt"], sigma=True) for r in mix[20:]]
    done = _wait(srv, 41)
    inmix = done[t_mix]
    assert inmix["N"] == alone["N"]
    # float32 spreading sums in a different order, otherwise the same work
    assert np.max(np.abs(inmix["R"] - alone["R"])) <= 1e-6
    assert sigma_err(inmix["Sigma"], alone["Sigma"].astype(np.float64)) <= 1e-6
    st = mm.mm_server_get_stats(srv)
    assert st["peak_inflight"] >= 2 and st["completed"] == 42
    # every request: the window gather (two kernels) and the slot plan's
    # coefficient and contraction kernels (at least four)
    assert st["launches"] >= 6 * 42
    # the mix itself is right too
    for t, r in zip(tks[:5], mix[:5]):
        _check(day, r, done[t])
    mm.mm_server_destroy(srv)


def test_budget_sets_slots_and_bad_requests_fail_alone(day):
    import paper_2003_02842_gb300 as mm
    srv = _server(day, max_slots=8)
    slot = mm.mm_server_get_stats(srv)["slot_bytes"]
    mm.mm_server_destroy(srv)
    srv = _server(day, max_slots=8, hbm_budget=int(2.5 * slot))
    assert mm.mm_server_get_stats(srv)["slots"] == 2
    good = {"t0": 100.0, "t1": 2900.0, "assets": np.arange(6, dtype=np.int32), "dt": 0.0}
    t_bad = mm.mm_server_submit(srv, 100.0, 2900.0, np.array([0, 99], np.int32), N=10)  # asset 99 does not exist
    t_good = mm.mm_server_submit(srv, good["t0"], good["t1"], good["assets"], sigma=True)
    done = _wait(srv, 2)
    assert done[t_bad]["status"] == 1  # MM_ERR_INVALID_ARG
    _check(day, good, done[t_good])
    with pytest.raises(mm.MMError):
        mm.mm_server_submit(srv, 5.0, 1.0, good["assets"])  # empty window
    mm.mm_server_destroy(srv)


def test_resident_coefficients_serve_repeated_windows(day):
    import paper_2003_02842_gb300 as mm
    srv = _server(day, cache_rows=16)

    def run(req, N):
        t = mm.mm_server_submit(srv, req["t0"], req["t1"], req["assets"], N=N, sigma=True)
        return _wait(srv, 1)[t]

    def counts():
        st = mm.mm_server_get_stats(srv)
        return st["cache_hits"], st["cache_misses"]

    a = {"t0": 200.0, "t1": 2800.0, "assets": np.array([1, 2, 3, 4, 5, 6], np.int32)}
    b = {"t0": 200.0, "t1": 2800.0, "assets": np.array([4, 5, 6, 7, 8, 9], np.int32)}
    da = run(a, 120)
    assert counts() == (0, 6)
    db = run(b, 120)  # assets 4, 5, 6 over the same window at the same cutoff are resident
    assert counts() == (3, 9)
    _check(day, a, da)
    _check(day, b, db)
    da2 = run(a, 120)  # every row resident
    assert counts() == (9, 9)
    assert np.max(np.abs(da2["R"] - da["R"])) <= 1e-6
    dc = run(a, 60)  # another cutoff: other rows
    assert counts() == (9, 15)
    _check(day, a, dc)
    # more (asset, window) rows than the cache holds: older rows are evicted
    for k in range(4):
        w = {"t0": 100.0 + 50.0 * k, "t1": 2900.0, "assets": np.arange(6, dtype=np.int32)}
        _check(day, w, run(w, 90))
    assert counts() == (9, 39)
    # the window's Nyquist cutoff is found on the device: not cached
    dn = run(a, 0)
    assert counts() == (9, 39)
    _check(day, a, dn)
    mm.mm_server_destroy(srv)


def test_resident_coefficients_under_concurrent_requests(day):
    # overlapping windows and subsets in flight together: rows written by one
    # request become visible only once it has finished, so every result
    # matches the oracle
    import paper_2003_02842_gb300 as mm
    srv = _server(day, cache_rows=48, max_slots=4)
    base = synth.c5_requests(11, n=12, D=day.D, T=3000, w_range=(600, 2400), k_range=(3, 10))
    reqs = []
    for r in base:
        reqs.append({"t0": 300.0, "t1": 2700.0, "assets": r["assets"]})  # one shared window
    tks = [mm.mm_server_submit(srv, r["t0"], r["t1"], r["assets"], N=75, sigma=True) for r in reqs * 2]
    done = _wait(srv, len(tks))
    st = mm.mm_server_get_stats(srv)
    assert st["cache_hits"] > 0 and st["cache_hits"] + st["cache_misses"] == sum(len(r["assets"]) for r in reqs * 2)
    for t, r in zip(tks, reqs * 2):
        _check(day, r, done[t])
    mm.mm_server_destroy(srv)
