"""GPU parity of the batched form (replications x cutoff sweep) against the
FP64 CPU oracle applied to each replication on its own: per-replication
rescaling (Algorithm 4), coefficients at the largest cutoff (Eq. (4)), and
Sigma / R at every cutoff of the sweep (Eqs. (2), (3); Algorithm 3), plus
the CUDA-graph replay of repeated sweeps.

Tolerances: coefficients, Eq. (15) per asset <= 1e-5 (NUFFT at 1e-6, float32);
R, max |dR| <= 1e-4 at every cutoff. Sigma errors are measured against the
assets' realised variances (Sigma_ii at the largest cutoff, Dirichlet):
the NUFFT bounds the error of the whole coefficient vector (Eq. (15)), so at
a tiny cutoff, where Sigma_ii(N) rests on a few low modes (N = 1: the total
return alone), an error relative to Sigma_ii(N) itself is not bounded by
the method; relative to the realised variance it stays near the float32
level (bound used: 1e-5).
"""
import numpy as np
import pytest

import oracle
from paper_2003_02842_gb300 import synth

from gpu_helpers import rel_l2_rows, to_dev

pytestmark = pytest.mark.gpu

TOL = dict(coef=1e-5, sig_rv=1e-5, R=1e-4)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _split(ev, reps, D):
    """Replication r of a batch as its own Events (offsets rebased)."""
    out = []
    for r in range(reps):
        a, b = r * D, (r + 1) * D
        off = ev.offsets[a:b + 1]
        e0, e1 = int(off[0]), int(off[-1])
        out.append(synth.Events(off - e0, ev.t[e0:e1].copy(), ev.logp[e0:e1].copy()))
    return out


def _check_batch(ev, reps, D, cutoffs, basis, kernel="es"):
    import paper_2003_02842_gb300 as mm
    b = mm.mm_batch_create(reps=reps, D=D, N_max=max(cutoffs), max_events=ev.n_events, tol=1e-6, kernel=kernel,
                           basis=basis)
    off, t, p = to_dev(ev)
    S, R = mm.mm_batch_epps(b, off, t, p, cutoffs)
    st = mm.mm_batch_sync(b)
    F = mm.mm_batch_coeffs(b).cpu().numpy()
    S, R = S.cpu().numpy().astype(np.float64), R.cpu().numpy().astype(np.float64)
    Nmax = max(cutoffs)
    for r, e in enumerate(_split(ev, reps, D)):
        ref = oracle.coeffs_F(e.offsets, e.t, e.logp, Nmax)
        assert np.all(rel_l2_rows(F[r * D:(r + 1) * D], ref) <= TOL["coef"]), r
        V = np.diag(oracle.estimate(e.offsets, e.t, e.logp, N=Nmax, basis="dirichlet")["Sigma"])
        scale = np.sqrt(np.outer(V, V))
        for j, N in enumerate(cutoffs):
            o = oracle.estimate(e.offsets, e.t, e.logp, N=N, basis=basis)
            assert np.max(np.abs(S[r, j] - o["Sigma"]) / scale) <= TOL["sig_rv"], (r, N)
            ok = np.diag(o["Sigma"]) > 0
            sub = np.ix_(ok, ok)
            assert np.max(np.abs(R[r, j][sub] - o["R"][sub])) <= TOL["R"], (r, N)
            assert np.all(np.diag(R[r, j])[ok] == 1.0)
    return b, st, (off, t, p), S, R


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_batch_sweep_matches_oracle_per_replication(basis):
    reps, D = 6, 4
    ev = synth.c4_batch(5, reps=reps, D=D, T=2000, median_n=300)
    cutoffs = [1, 2, 3, 5, 8, 13, 40, 97, 250, 600]
    b, st, _, _, _ = _check_batch(ev, reps, D, cutoffs, basis)
    assert st == 0


def test_batch_each_replication_rescaled_on_its_own():
    # replications with different time origins and spans: Algorithm 4 per
    # replication, so each one matches the oracle run on it alone
    reps, D = 4, 3
    parts = []
    for r in range(reps):
        e = synth.random_events(70 + r, D=D, n_range=(40, 300), T=500.0 * (r + 1))
        e = synth.Events(e.offsets, e.t * (1.0 + 0.5 * r) + 1.0e6 * r, e.logp)
        parts.append(e)
    ev = synth.concat_events(parts)
    _check_batch(ev, reps, D, [1, 4, 9, 33, 120], "fejer", kernel="kb")


def test_batch_graph_replay_and_new_cutoffs():
    import torch
    import paper_2003_02842_gb300 as mm
    reps, D = 5, 3
    ev = synth.c4_batch(9, reps=reps, D=D, T=1500, median_n=200)
    cut = [1, 3, 10, 30, 100, 300]
    b, _, (off, t, p), S0, R0 = _check_batch(ev, reps, D, cut, "dirichlet")
    info = mm.mm_batch_get_info(b)
    assert info["graph_captures"] == 1 and info["graph_launches"] == 0 and info["graph_kernels"] >= 4
    # the graph is bound to its inputs and outputs: the same buffers replay it
    S1 = torch.empty((reps, len(cut), D, D), dtype=torch.float32, device="cuda")
    R1 = torch.empty_like(S1)
    mm.mm_batch_epps(b, off, t, p, cut, sigma=S1, R=R1)  # new outputs: captured again
    for _ in range(3):
        mm.mm_batch_epps(b, off, t, p, cut, sigma=S1, R=R1)
    assert mm.mm_batch_sync(b) == 0
    info = mm.mm_batch_get_info(b)
    assert info["graph_launches"] == 3 and info["graph_captures"] == 2
    # the replayed graph computes the same sweep (shared-memory atomics make
    # the float32 spreading order vary, so to rounding)
    assert np.allclose(R1.cpu().numpy(), R0, atol=1e-6)
    assert np.allclose(S1.cpu().numpy(), S0, rtol=1e-5, atol=0)
    # other cutoffs: a new capture
    S2, R2 = mm.mm_batch_epps(b, off, t, p, [2, 7, 150])
    assert mm.mm_batch_sync(b) == 0
    assert mm.mm_batch_get_info(b)["graph_captures"] == 3
    e0 = _split(ev, reps, D)[0]
    o = oracle.estimate(e0.offsets, e0.t, e0.logp, N=150, basis="dirichlet")
    assert np.max(np.abs(R2.cpu().numpy()[0, 2].astype(np.float64) - o["R"])) <= TOL["R"]


def test_batch_autotune_keeps_results():
    import paper_2003_02842_gb300 as mm
    reps, D = 8, 10
    ev = synth.c4_batch(11, reps=reps, D=D, T=3000, median_n=400)
    cut = synth.sweep_cutoffs(int(ev.meta["nyquist"].min()), 16)
    b = mm.mm_batch_create(reps=reps, D=D, N_max=max(cut), max_events=ev.n_events, tol=1e-6)
    off, t, p = to_dev(ev)
    info = mm.mm_batch_autotune(b, off, t, p, max(cut), reps=2)
    assert info["tuned_ms"] > 0
    S, R = mm.mm_batch_epps(b, off, t, p, cut)
    assert mm.mm_batch_sync(b) == 0
    R = R.cpu().numpy().astype(np.float64)
    for r, e in enumerate(_split(ev, reps, D)[:3]):
        for j in (0, len(cut) // 2, len(cut) - 1):
            o = oracle.estimate(e.offsets, e.t, e.logp, N=cut[j], basis="dirichlet")
            assert np.max(np.abs(R[r, j] - o["R"])) <= TOL["R"]


def test_batch_rejects_bad_requests():
    import paper_2003_02842_gb300 as mm
    with pytest.raises(mm.MMError):
        mm.mm_batch_create(reps=2, D=13, N_max=10, max_events=100)  # D above the sweep kernel's limit
    ev = synth.c4_batch(1, reps=2, D=3, T=500, median_n=100)
    b = mm.mm_batch_create(reps=2, D=3, N_max=50, max_events=ev.n_events, basis="fejer")
    off, t, p = to_dev(ev)
    for bad in ([0, 5], [5, 5], [3, 2], [10, 51]):
        with pytest.raises(mm.MMError):
            mm.mm_batch_epps(b, off, t, p, bad)


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_sweep_contraction_relative_to_sigma_itself(basis):
    # the sweep against Eqs. (2) / (3) evaluated in float64 on the sweep's own
    # coefficients, each entry relative to sqrt(Sigma_ii Sigma_jj) at its own
    # cutoff (no NUFFT error enters). One replication has a tiny total return
    # in its first asset, so that at N = 1 its diagonal (a single k = 0 term)
    # is small against the k = 1 term: a sweep that forms the Fejer weights as
    # a difference of two prefix sums loses it.
    import paper_2003_02842_gb300 as mm
    reps, D = 3, 2
    evs = _split(synth.concat_events([synth.random_events(40 + r, D=D, n_range=(80, 200), T=3000.0)
                                      for r in range(reps)]), reps, D)
    e = evs[1]
    a0, a1 = int(e.offsets[0]), int(e.offsets[1])
    lp = e.logp.copy()
    lp[a1 - 1] = lp[a0] + 1e-7  # total return of asset 0 in replication 1
    evs[1] = synth.Events(e.offsets, e.t, lp)
    ev = synth.concat_events(evs)
    cutoffs = [1, 2, 3, 8, 40]
    b = mm.mm_batch_create(reps=reps, D=D, N_max=max(cutoffs), max_events=ev.n_events, tol=1e-6, kernel="es",
                           basis=basis)
    off, t, p = to_dev(ev)
    S, _ = mm.mm_batch_epps(b, off, t, p, cutoffs)
    assert mm.mm_batch_sync(b) == 0
    F = mm.mm_batch_coeffs(b).cpu().numpy().astype(np.complex128)  # [reps * D, N_max + 1]
    S = S.cpu().numpy().astype(np.float64)
    mm.mm_batch_destroy(b)
    for r in range(reps):
        c = F[r * D:(r + 1) * D] * 2 * np.pi  # c-convention
        for j, N in enumerate(cutoffs):
            k = np.arange(N + 1)
            w = np.full(N + 1, 1.0 / (2 * N + 1)) if basis == "dirichlet" else (1.0 - k / N) / (N + 1)
            w = w * np.where(k == 0, 1.0, 2.0)  # the -k half folded in
            ref = np.real((c[:, None, :N + 1] * np.conj(c[None, :, :N + 1]) * w).sum(axis=2))
            scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
            assert np.all(np.diag(ref) > 0)
            assert np.max(np.abs(S[r, j] - ref) / scale) <= 2e-5, (r, N, S[r, j], ref)


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_fp64_batch_matches_oracle_per_replication(basis):
    # the batched form in float64 throughout (the mixed form's comparator):
    # coefficients, Sigma and R of every replication and cutoff against the
    # oracle at the FP64 path's tolerances (Eq. (15) <= 1e-10 at tol 1e-12;
    # Sigma relative to the realised variances and R <= 1e-9)
    import paper_2003_02842_gb300 as mm
    reps, D = 5, 3
    ev = synth.c4_batch(9, reps=reps, D=D, T=2000, median_n=300)
    cutoffs = [1, 2, 7, 40, 333, 800]
    b = mm.mm_batch_create(reps=reps, D=D, N_max=max(cutoffs), max_events=ev.n_events, tol=1e-12, kernel="es",
                           basis=basis, prec="fp64")
    off, t, p = to_dev(ev)
    for _ in range(2):  # the eager first call, then the graph replay
        S, R = mm.mm_batch_epps(b, off, t, p, cutoffs)
    assert mm.mm_batch_sync(b) == 0
    assert S.dtype == torch_float64()
    F = mm.mm_batch_coeffs(b).cpu().numpy()
    S, R = S.cpu().numpy(), R.cpu().numpy()
    for r, e in enumerate(_split(ev, reps, D)):
        ref = oracle.coeffs_F(e.offsets, e.t, e.logp, max(cutoffs))
        assert np.all(rel_l2_rows(F[r * D:(r + 1) * D], ref) <= 1e-10), r
        V = np.array([np.sum(np.diff(e.asset(i)[1]) ** 2) for i in range(D)])
        for j, N in enumerate(cutoffs):
            o = oracle.estimate(e.offsets, e.t, e.logp, N=N, basis=basis)
            assert np.max(np.abs(S[r, j] - o["Sigma"]) / np.sqrt(np.outer(V, V))) <= 1e-9, (r, N)
            assert np.max(np.abs(R[r, j] - o["R"])) <= 1e-9, (r, N)
            assert np.all(np.diag(R[r, j]) == 1.0)
    mm.mm_batch_destroy(b)


def test_mixed_batch_agrees_with_fp64_batch():
    # the like-for-like comparison of the two forms on one batch
    import paper_2003_02842_gb300 as mm
    reps, D = 64, 10
    ev = synth.c4_batch(10, reps=reps, D=D, T=4000, median_n=600)
    cutoffs = synth.sweep_cutoffs(int(ev.meta["nyquist"].min()), 16)
    off, t, p = to_dev(ev)
    out = {}
    for prec, tol in (("fp64", 1e-12), ("bf16x3", 1e-6)):
        b = mm.mm_batch_create(reps=reps, D=D, N_max=max(cutoffs), max_events=ev.n_events, tol=tol, kernel="es",
                               basis="dirichlet", prec=prec)
        _, R = mm.mm_batch_epps(b, off, t, p, cutoffs, sigma=False)
        assert mm.mm_batch_sync(b) == 0
        out[prec] = R.double().cpu().numpy()
        mm.mm_batch_destroy(b)
    assert np.max(np.abs(out["bf16x3"] - out["fp64"])) <= 1e-4


def torch_float64():
    import torch
    return torch.float64
