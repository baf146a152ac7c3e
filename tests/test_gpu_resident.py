"""GPU parity of the resident form of stages (a2)-(c) (spread_algo "fused" on
the mixed path): one launch after the prep kernel spreads each asset's
records straight into its grid row held in shared memory (Eq. (12)),
transforms it (Eq. (13)) and writes the deconvolved coefficients (Eq. (14)).
One CTA holds a row that fits; a cluster of two CTAs holds the halves of a
larger one (decimation in time by 2). The row is accumulated in sub-ranges:
these tests cover one to many sub-ranges, the periodic wrap of Eq. (11)
across the first and last sub-range, sparse and dense rows, assets with 0,
1 and 2 events, and the batched form.

Tolerances, as for the separate kernels: coefficients, Eq. (15) per asset
<= 1e-5 at tolerance 1e-6 (float32 path); R, max |dR| <= 1e-4.
"""
import numpy as np
import pytest

import oracle
from paper_2003_02842_gb300 import synth

from gpu_helpers import rel_l2_rows, run, to_dev

pytestmark = pytest.mark.gpu

COEF = 1e-5
RTOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _resident(ev, N, kernel="es", basis="dirichlet", fft_algo="default", prec="bf16x3", status=0):
    out = run(dict(tol=1e-6, kernel=kernel, basis=basis, prec=prec, spread_algo="fused", fft_algo=fft_algo), ev, N)
    assert out["status"] == status
    assert out["info"]["res_sub"] > 0 and out["info"]["spread_algo"] == 3, out["info"]
    return out


@pytest.mark.parametrize("N", [1, 7, 100, 333, 1000, 5000, 10000])
@pytest.mark.parametrize("kernel", ["gauss", "kb", "es"])
def test_one_cta_per_row(N, kernel):
    # events on a continuum over a day: the first and last events sit at the
    # window's ends, so their stencils wrap around the row
    ev = synth.random_events(21, D=4, n_range=(200, 3000), T=28800.0)
    out = _resident(ev, N, kernel)
    info = out["info"]
    assert info["fft_split"] == 1
    nsub = -(-info["Mr"] // info["res_sub"])
    if N >= 5000:
        assert nsub >= 2  # several sub-ranges per row
    ref = oracle.coeffs_F(ev.offsets, ev.t, ev.logp, N)
    err = rel_l2_rows(out["F"], ref)
    assert np.all(err <= COEF), err


@pytest.mark.parametrize("N", [100, 5000, 14399])
@pytest.mark.parametrize("kernel", ["gauss", "kb", "es"])
def test_cluster_pair_rows(N, kernel):
    # the one-second grid of a day: at the Nyquist cutoff a row (n = 28,800
    # complex points) fits only as two halves; smaller ones on request
    ev = synth.random_events(12, D=3, n_range=(200, 1500), T=28800.0, grid=28800)
    out = _resident(ev, N, kernel, fft_algo="asset_pair")
    assert out["info"]["fft_split"] == 3
    ref = oracle.coeffs_F(ev.offsets, ev.t, ev.logp, N)
    err = rel_l2_rows(out["F"], ref)
    assert np.all(err <= COEF), err


def test_default_form_picks_the_pair_for_the_largest_rows():
    ev = synth.random_events(13, D=2, n_range=(500, 900), T=28800.0, grid=28800)
    out = _resident(ev, 14399)
    assert out["info"]["fft_split"] == 3
    ref = oracle.coeffs_F(ev.offsets, ev.t, ev.logp, 14399)
    assert np.all(rel_l2_rows(out["F"], ref) <= COEF)


def test_ragged_assets_and_covariance():
    # assets with 0, 1, 2 and many events; Sigma and R through the same call
    ev = synth.random_events(3, D=6, n_range=(3, 300), T=5000.0)
    ts = [ev.asset(i)[0] for i in range(ev.D)]
    ps = [ev.asset(i)[1] for i in range(ev.D)]
    for i, k in ((1, 0), (2, 1), (3, 2)):
        ts[i], ps[i] = ts[i][:k], ps[i][:k]
    ev = synth.from_lists(ts, ps)
    N = 97
    out = _resident(ev, N, status=9)  # MM_ERR_ZERO_VARIANCE: non-fatal, R has NaN rows
    ref = oracle.estimate(ev.offsets, ev.t, ev.logp, N=N, basis="dirichlet")
    assert np.all(rel_l2_rows(out["F"], ref["F"]) <= COEF)
    ok = np.diag(ref["Sigma"]) > 0
    sub = np.ix_(ok, ok)
    assert np.max(np.abs(out["R"][sub].astype(np.float64) - ref["R"][sub])) <= RTOL
    assert np.all(np.isnan(out["R"][~ok, :]))


@pytest.mark.parametrize("n,N", [(28800, 5), (28800, 239), (50000, 1), (50000, 1000), (200000, 10)])
def test_dense_rows(n, N):
    # many events per cell: the dense mapping (runs of records in one cell
    # summed in registers) inside the resident kernel
    ev = synth.random_events(8 + n // 50000, D=2, n_range=(n, n), T=28800.0)
    out = _resident(ev, N)
    ref = oracle.coeffs_F(ev.offsets, ev.t, ev.logp, N)
    err = rel_l2_rows(out["F"], ref)
    assert np.all(err <= COEF), err


def test_agrees_with_the_separate_kernels():
    # the same records and the same per-tap polynomials; only the tiles'
    # boundaries (hence their integer scales) differ: agreement to rounding
    ev = synth.c2_async(5)
    N = ev.meta["N"]
    a = run(dict(tol=1e-6, kernel="es", basis="dirichlet", prec="bf16x3", spread_algo="fused"), ev, N)
    b = run(dict(tol=1e-6, kernel="es", basis="dirichlet", prec="bf16x3", spread_algo="scatter"), ev, N)
    assert a["info"]["res_sub"] > 0 and b["info"]["res_sub"] == 0
    d = rel_l2_rows(a["F"], b["F"].astype(np.complex128))
    assert np.all(d <= 2e-6), d


@pytest.mark.parametrize("bad,code", [("unsorted", 2), ("nan", 10)])
def test_bad_event_data_reports_status(bad, code):
    import paper_2003_02842_gb300 as mm
    ev = synth.random_events(51, D=3, n_range=(30, 60), T=100.0)
    t = ev.t.copy()
    lp = ev.logp.copy()
    a = int(ev.offsets[1]) + 5
    if bad == "unsorted":
        t[a], t[a + 1] = t[a + 1], t[a]
    else:
        lp[a] = np.nan
    ev2 = synth.Events(ev.offsets.copy(), t, lp)
    plan = mm.mm_plan_create(D=3, N_max=20, max_events=ev.n_events, tol=1e-6, spread_algo="fused")
    off, tt, p = to_dev(ev2)
    mm.mm_estimate(plan, off, tt, p, 20)
    assert mm.mm_plan_sync(plan) == code
    assert mm.mm_plan_get_info(plan)["res_sub"] > 0
    mm.mm_destroy(plan)


def _split(ev, reps, D):
    out = []
    for r in range(reps):
        a, b = r * D, (r + 1) * D
        off = ev.offsets[a:b + 1]
        e0, e1 = int(off[0]), int(off[-1])
        out.append(synth.Events(off - e0, ev.t[e0:e1].copy(), ev.logp[e0:e1].copy()))
    return out


@pytest.mark.parametrize("T,median_n", [(2000, 300), (28800, 1500)])
def test_batched_form(T, median_n):
    # replications rescaled one by one (Algorithm 4) by the prep kernel, then
    # the resident rows; at T = 28,800 s the rows are cluster pairs
    import paper_2003_02842_gb300 as mm
    reps, D = 4, 3
    ev = synth.c4_batch(17, reps=reps, D=D, T=T, median_n=median_n)
    Nmax = int(ev.meta["nyquist"].min())
    cut = [1, 10, Nmax // 3, Nmax]
    b = mm.mm_batch_create(reps=reps, D=D, N_max=Nmax, max_events=ev.n_events, tol=1e-6, spread_algo="fused")
    off, t, p = to_dev(ev)
    S, R = mm.mm_batch_epps(b, off, t, p, cut)
    assert mm.mm_batch_sync(b) == 0
    prof = mm.mm_batch_get_info(b)
    assert prof["graph_kernels"] >= 3
    F = mm.mm_batch_coeffs(b).cpu().numpy()
    R = R.cpu().numpy().astype(np.float64)
    for r, e in enumerate(_split(ev, reps, D)):
        ref = oracle.coeffs_F(e.offsets, e.t, e.logp, Nmax)
        assert np.all(rel_l2_rows(F[r * D:(r + 1) * D], ref) <= COEF), r
        for j, N in enumerate(cut):
            # Sigma from the oracle's own coefficients at k = -N..N (Algorithm 3 step C)
            c = np.concatenate([np.conj(ref[:, 1:N + 1][:, ::-1]), ref[:, :N + 1]], axis=1) * (2 * np.pi)
            S_ref, _ = oracle.cov_from_coeffs(c, N, "dirichlet")
            R_ref = oracle.corr(S_ref)
            assert np.max(np.abs(R[r, j] - R_ref)) <= RTOL, (r, N)
    mm.mm_batch_destroy(b)
