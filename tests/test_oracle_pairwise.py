"""Pins of the oracle's pairwise-cutoff covariance and nearest positive
semi-definite repair (Sec. 3.1).

- Each entry of the pairwise estimate equals the independent closed-kernel
  route (Eq. (2) / (3) summed over event pairs with the Dirichlet or Fejer
  kernel in closed form) at that pair's cutoff, with the common window.
- The repair: a textbook 2 x 2 case, positive semi-definiteness of the
  result, no change to a positive semi-definite input, the distance
  sqrt(sum of the squared negative eigenvalues) the eigenvalue method
  attains, and no random positive semi-definite matrix closer to the input.
"""
import numpy as np
import pytest

import oracle
from paper_2003_02842_gb300 import synth


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_pairwise_entries_match_closed_kernels(basis):
    ev = synth.random_events(71, D=5, n_range=(20, 60), T=500.0)
    Ns = [3, 17, 9, 17, 30]
    S, R = oracle.cov_pairwise_cutoffs(ev.offsets, ev.t, ev.logp, Ns, basis=basis)
    t0, t1 = oracle.bounds(ev.offsets, ev.t)
    roff, rt, rd = oracle.returns(ev.offsets, ev.t, ev.logp)
    for i in range(5):
        for j in range(5):
            N = min(Ns[i], Ns[j])
            ref = oracle.cov_pairwise(roff, rt, rd, t0, t1 - t0, N, basis)[i, j]
            assert abs(S[i, j] - ref) <= 1e-10 * max(1.0, abs(ref)), (i, j, S[i, j], ref)
    assert np.allclose(S, S.T)
    assert np.allclose(np.diag(R), 1.0)


def test_equal_cutoffs_reduce_to_the_common_estimate():
    ev = synth.random_events(72, D=4, n_range=(20, 60), T=500.0)
    S, _ = oracle.cov_pairwise_cutoffs(ev.offsets, ev.t, ev.logp, [12] * 4, basis="fejer")
    ref = oracle.estimate(ev.offsets, ev.t, ev.logp, N=12, basis="fejer")["Sigma"]
    assert np.allclose(S, ref, rtol=0, atol=0)


def test_nearest_psd_textbook_case():
    S = np.array([[1.0, 2.0], [2.0, 1.0]])  # eigenvalues 3 and -1
    P, neg = oracle.nearest_psd(S)
    assert neg == 1
    assert np.allclose(P, [[1.5, 1.5], [1.5, 1.5]], atol=1e-14)


def test_nearest_psd_properties():
    rng = np.random.default_rng(5)
    for D in (3, 8, 20):
        X = rng.standard_normal((D, D))
        S = 0.5 * (X + X.T)
        lam = np.linalg.eigvalsh(S)
        P, neg = oracle.nearest_psd(S)
        assert neg == int(np.sum(lam < 0))
        assert np.linalg.eigvalsh(P).min() >= -1e-12 * np.abs(lam).max()
        # the eigenvalue method's distance: the clipped eigenvalues' norm
        d = np.linalg.norm(S - P)
        assert abs(d - np.sqrt(np.sum(lam[lam < 0] ** 2))) <= 1e-12 * np.abs(lam).max() * D
        for _ in range(50):
            Y = rng.standard_normal((D, D))
            B = P + 0.1 * (Y @ Y.T) / D  # another positive semi-definite matrix
            assert np.linalg.norm(S - B) >= d - 1e-12
        # already positive semi-definite: its `neg` zero eigenvalues may round
        # to tiny negatives, and clipping those changes nothing visible
        Q, n2 = oracle.nearest_psd(P)
        assert n2 <= neg and np.allclose(Q, P, rtol=0, atol=1e-12 * np.abs(lam).max())
    G = rng.standard_normal((6, 6))
    S = G @ G.T
    P, neg = oracle.nearest_psd(S)
    assert neg == 0 and np.array_equal(P, 0.5 * (S + S.T))
