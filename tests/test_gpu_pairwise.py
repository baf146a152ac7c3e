"""GPU parity of the pairwise-cutoff covariance and its nearest positive
semi-definite repair (Sec. 3.1) against the oracle.

Tolerances: Sigma, max |dSigma_ij| / sqrt(Sigma_ii Sigma_jj) <= 1e-4 (mixed)
and 1e-9 (FP64), R <= 1e-4 / 1e-9, as for the common cutoff. The repair maps
a symmetric matrix to its nearest positive semi-definite one, a map that
moves no two inputs further apart in the Frobenius norm than they were: the
repaired matrices may differ by at most twice the input matrices' difference
plus the eigensolver's own rounding, 1e-12 of the norm for the float64
Jacobi iteration (FP64 plans) and 1e-5 for the float32 one (mixed
precisions, whose Sigma is itself correct to about 1e-5 of its scale).
"""
import numpy as np
import pytest

import oracle
from paper_2003_02842_gb300 import synth

from gpu_helpers import sigma_err, to_dev

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(tol=1e-12, sig=1e-9, R=1e-9, eig=1e-12), "bf16x3": dict(tol=1e-6, sig=1e-4, R=1e-4, eig=1e-5)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _case(seed, D=24):
    # per-asset cutoffs from 2 to 119 (fewer distinct values for many assets:
    # the oracle evaluates Algorithm 3 once per distinct pairwise cutoff)
    ev = synth.random_events(80 + seed, D=D, n_range=(30, 300), T=3000.0)
    Ns = np.random.default_rng(seed).integers(2, 120 if D <= 24 else 30, size=D)
    return ev, [int(x) for x in Ns]


def _run(ev, Ns, prec, basis, repair):
    import torch
    import paper_2003_02842_gb300 as mm
    tl = TOL[prec]
    Nc = max(Ns)
    plan = mm.mm_plan_create(D=ev.D, N_max=Nc, max_events=ev.n_events, tol=tl["tol"], kernel="es", basis=basis,
                             prec=prec)
    off, t, p = to_dev(ev)
    F, _ = mm.mm_coeffs(plan, off, t, p, Nc)
    S, R, clipped = mm.mm_corr_pairwise(plan, F, Nc, Ns, psd_repair=repair)
    torch.cuda.synchronize()
    st = mm.mm_plan_sync(plan)
    out = dict(S=S.cpu().numpy().astype(np.float64), R=R.cpu().numpy().astype(np.float64),
               clipped=int(clipped.item()), status=st)
    mm.mm_destroy(plan)
    return out


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_pairwise_cutoffs_match_oracle(prec, basis):
    ev, Ns = _case(0)
    out = _run(ev, Ns, prec, basis, repair=False)
    S_ref, R_ref = oracle.cov_pairwise_cutoffs(ev.offsets, ev.t, ev.logp, Ns, basis=basis)
    assert out["status"] == 0 and out["clipped"] == 0
    assert sigma_err(out["S"], S_ref) <= TOL[prec]["sig"]
    assert np.max(np.abs(out["R"] - R_ref)) <= TOL[prec]["R"]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
@pytest.mark.parametrize("seed,D", [(1, 24), (3, 24), (5, 200), (7, 500)])
def test_psd_repair_matches_oracle(prec, basis, seed, D):
    # D = 24: the one-CTA Jacobi iteration in shared memory; D = 200 and 500
    # (the serving workload's largest request): the iteration over every SM.
    # The iteration stops once the off-diagonal norm is below 2 D eps of the
    # matrix norm (eps of its working type), and every element meets about 2D
    # rotations per sweep, so the decomposition's backward error is of order
    # D eps of the norm: the repaired matrix is held to 8 D eps of the norm
    # (about 1e-4 in float32 at D = 200-500, the mixed path's own Sigma
    # tolerance) beyond twice the input's own distance from the oracle's.
    ev, Ns = _case(seed, D=D)
    raw = _run(ev, Ns, prec, basis, repair=False)
    out = _run(ev, Ns, prec, basis, repair=True)
    S_ref, _ = oracle.cov_pairwise_cutoffs(ev.offsets, ev.t, ev.logp, Ns, basis=basis)
    P_ref, neg = oracle.nearest_psd(S_ref)
    assert neg >= 1  # the pairwise estimate is not positive semi-definite here
    assert out["status"] == 0
    # eigenvalues within the iteration's accuracy of zero may fall either way
    lam = np.linalg.eigvalsh(0.5 * (S_ref + S_ref.T))
    eps_w = 1.1e-16 if prec == "fp64" else 6e-8
    tiny = np.sum(np.abs(lam) <= 4 * D * eps_w * np.abs(lam).max())
    assert abs(out["clipped"] - neg) <= tiny
    d_in = np.linalg.norm(raw["S"] - S_ref)
    tol_eig = max(TOL[prec]["eig"], 8 * D * eps_w)
    assert np.linalg.norm(out["S"] - P_ref) <= 2.0 * d_in + tol_eig * np.linalg.norm(S_ref)
    assert np.linalg.eigvalsh(out["S"]).min() >= -max(1e-5, tol_eig) * np.abs(lam).max()
    assert np.max(np.abs(out["R"] - oracle.corr(P_ref))) <= 10 * max(TOL[prec]["R"], tol_eig)


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_equal_cutoffs_reduce_to_common_estimate_and_need_no_repair(basis):
    import torch
    import paper_2003_02842_gb300 as mm
    ev, _ = _case(2, D=10)
    N = 60
    plan = mm.mm_plan_create(D=ev.D, N_max=N, max_events=ev.n_events, tol=1e-6, kernel="es", basis=basis)
    off, t, p = to_dev(ev)
    F, _ = mm.mm_coeffs(plan, off, t, p, N)
    S0, R0 = mm.mm_corr(plan, F, N)
    S1, R1, c1 = mm.mm_corr_pairwise(plan, F, N, [N] * ev.D, psd_repair=True)
    torch.cuda.synchronize()
    assert mm.mm_plan_sync(plan) == 0
    assert int(c1.item()) == 0  # a Gram matrix: nothing to clip
    assert sigma_err(S1.cpu().numpy(), S0.cpu().numpy().astype(np.float64)) <= 2e-5
    assert np.max(np.abs(R1.cpu().numpy() - R0.cpu().numpy())) <= 2e-5
    mm.mm_destroy(plan)


def test_pairwise_rejects_bad_arguments():
    import torch
    import paper_2003_02842_gb300 as mm
    ev, Ns = _case(4, D=6)
    Nc = max(Ns)
    plan = mm.mm_plan_create(D=ev.D, N_max=Nc, max_events=ev.n_events, tol=1e-6, kernel="es", basis="fejer")
    off, t, p = to_dev(ev)
    F, _ = mm.mm_coeffs(plan, off, t, p, Nc)
    for bad in ([0] + Ns[1:], [Nc + 1] + Ns[1:], Ns[:-1]):
        with pytest.raises((mm.MMError, ValueError)):
            mm.mm_corr_pairwise(plan, F, Nc, bad)
    mm.mm_destroy(plan)
    D = 4001  # beyond the repair's limit (its rotation arrays fill 48 KB)
    plan = mm.mm_plan_create(D=D, N_max=8, max_events=0, tol=1e-6, kernel="es")
    F = torch.zeros((D, 9), dtype=torch.complex64, device="cuda")
    F[:, 1] = 1.0
    with pytest.raises(mm.MMError):
        mm.mm_corr_pairwise(plan, F, 8, [8] * D, psd_repair=True)
    S, R, c = mm.mm_corr_pairwise(plan, F, 8, [8] * D)
    torch.cuda.synchronize()
    mm.mm_destroy(plan)
