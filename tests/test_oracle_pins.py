"""Pins of the FP64 CPU oracle to facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a value
worked out by hand from Eq. (4), a closed form, a brute-force evaluation of
Eqs. (2)/(3) as printed, a printed constant, or a library routine. Together
they are chosen so that a dropped term, a flipped sign, an off-by-one index or
a wrong weight in the oracle fails at least one of them.
"""
import cmath
import math
import os

import numpy as np
import pytest

from paper_2003_02842_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# Eq. (4): coefficient definition, sign and index conventions
# --------------------------------------------------------------------------
def test_worked_example_sign_and_left_endpoint(orc):
    # Raw times 0, 1, 4 -> t~ = 0, pi/2, 2 pi (Algorithm 4). Returns sit at the
    # left end points: d0 at t~ = 0 and d1 at t~ = pi/2 (Sec. 2.1). Eq. (4)
    # (times 2 pi) gives c_k = d0 + d1 e^{-i k pi/2}.
    p = np.array([4.60, 4.63, 4.58])
    d0, d1 = p[1] - p[0], p[2] - p[1]
    ev = synth.from_lists([[0.0, 1.0, 4.0]], [p])
    out = orc.estimate(ev.offsets, ev.t, ev.logp, N=3)
    c = out["c_full"][0]  # k = -3..3
    want = {0: d0 + d1, 1: d0 - 1j * d1, 2: d0 - d1, 3: d0 + 1j * d1,
            -1: d0 + 1j * d1, -2: d0 - d1, -3: d0 - 1j * d1}
    for k, v in want.items():
        assert abs(c[k + 3] - v) < 1e-15, k
    assert np.allclose(out["F"][0], [want[k] / (2 * np.pi) for k in range(4)], atol=1e-16)


def test_c0_telescopes(orc):
    # F(dp)(0) = sum of returns / 2 pi (Sec. 2.2.2) = (p_last - p_first) / 2 pi.
    ev = synth.random_events(1, D=5, n_range=(2, 40))
    F = orc.coeffs_F(ev.offsets, ev.t, ev.logp, N=4)
    for i in range(ev.D):
        _, p = ev.asset(i)
        assert abs(F[i, 0].imag) < 1e-17
        assert abs(F[i, 0].real * 2 * np.pi - (p[-1] - p[0])) < 1e-14


def test_hermitian_symmetry(orc):
    # c(-k) = conj(c(k)) for real returns (Sec. 2.2.2); both sides are
    # evaluated by independent direct sums.
    ev = synth.random_events(2, D=3, n_range=(5, 30))
    out = orc.estimate(ev.offsets, ev.t, ev.logp, N=12)
    c = out["c_full"]
    assert np.max(np.abs(c[:, ::-1] - np.conj(c))) < 1e-14


def test_shift_theorem(orc):
    # Moving every time of an asset by Delta inside a fixed window multiplies
    # c_k by exp(-i k 2 pi Delta / span): catches any error in the k index.
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(0, 500, 40))
    d = rng.normal(0, 0.01, 40)
    t0, span, delta = 0.0, 1000.0, 137.25
    a = orc.coeffs(t, d, t0, span, -9, 9)
    b = orc.coeffs(t + delta, d, t0, span, -9, 9)
    k = np.arange(-9, 10)
    assert np.max(np.abs(b - a * np.exp(-1j * k * 2 * np.pi * delta / span))) < 1e-14


def test_phase_exact_at_large_k(orc):
    # At k t~ ~ 1e6 the oracle still evaluates the phase of the exact rescaled
    # time: an event at raw time span/8 has c_k = d e^{-i k pi/4} exactly.
    span = 28800.0
    t = np.array([span / 8.0])
    d = np.array([0.5])
    ks = np.array([8 * 10**5 + 1, 8 * 10**5 + 2, 12345679])
    c = orc.coeffs_at(t, d, 0.0, span, ks)
    want = 0.5 * np.exp(-1j * np.pi / 4 * (ks % 8))
    assert np.max(np.abs(c - want)) < 1e-15
    # A time whose rescaled value is not a binary fraction (t / span =
    # 1/28800): for k = 28800 m + r the exact phase is 2 pi r / 28800, which
    # needs the low-order part of k * t / span at m ~ 1e3.
    t = np.array([1.0])
    r = np.array([1, 7, 12345, 28799])
    ks = 28800 * 1000 + r
    c = orc.coeffs_at(t, d, 0.0, span, ks)
    want = 0.5 * np.exp(-2j * np.pi * r / 28800.0)
    assert np.max(np.abs(c - want)) < 1e-15


# --------------------------------------------------------------------------
# Eqs. (2)/(3), Algorithm 3 step C
# --------------------------------------------------------------------------
def _brute(ev, N, basis, orc):
    """Eqs. (2)/(3) literally: triple sum over s, h, l of the paper's summand."""
    t0, t1 = orc.bounds(ev.offsets, ev.t)
    D = ev.D
    S = np.zeros((D, D))
    for i in range(D):
        ti, pi_ = ev.asset(i)
        for j in range(D):
            tj, pj = ev.asset(j)
            acc = 0j
            for s in range(-N, N + 1):
                if basis == "dirichlet":
                    w = 1.0 / (2 * N + 1)
                else:
                    w = (1.0 - abs(s) / N) / (N + 1)
                for h in range(len(ti) - 1):
                    for l in range(len(tj) - 1):
                        th = 2 * math.pi * (ti[h] - t0) / (t1 - t0)
                        tl = 2 * math.pi * (tj[l] - t0) / (t1 - t0)
                        acc += w * cmath.exp(1j * s * (tl - th)) * (pi_[h + 1] - pi_[h]) * (pj[l + 1] - pj[l])
            S[i, j] = acc.real
            assert abs(acc.imag) < 1e-12
    return S


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
@pytest.mark.parametrize("N", [1, 2, 4])
def test_bruteforce_triple_sum(orc, basis, N):
    ev = synth.random_events(10 + N, D=3, n_range=(2, 6), T=50.0)
    S = orc.estimate(ev.offsets, ev.t, ev.logp, N=N, basis=basis)["Sigma"]
    B = _brute(ev, N, basis, orc)
    assert np.max(np.abs(S - B)) < 1e-13 * max(1.0, np.max(np.abs(B)))


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
@pytest.mark.parametrize("N", [1, 7, 60])
def test_coefficient_route_equals_closed_kernel_route(orc, basis, N):
    # Step C of Algorithm 3 (products of coefficients) against Eqs. (2)/(3)
    # with the s-sum in closed form (Dirichlet / Fejer kernels).
    ev = synth.random_events(20 + N, D=4, n_range=(2, 40), T=3000.0)
    out = orc.estimate(ev.offsets, ev.t, ev.logp, N=N, basis=basis)
    S = out["Sigma"]
    P = orc.cov_pairwise(out["roff"], out["rt"], out["rd"], out["t0"], out["t1"] - out["t0"], N, basis)
    sc = np.sqrt(np.outer(np.diag(P), np.diag(P)))
    assert np.max(np.abs(S - P) / sc) < 1e-12
    assert out["imag_worst"] < 1e-13


def test_dirichlet_on_exact_grid_is_realized_covariance(orc):
    # Returns on t~ = 2 pi m / M (M = 2N+1): the Dirichlet kernel vanishes at
    # every non-zero grid offset, so Sigma_ij is the sum of products of
    # returns that share a left end point (Sec. 2.3 sampling argument).
    N = 20
    M = 2 * N + 1
    rng = np.random.default_rng(7)
    ts, ps = [], []
    for i in range(3):
        keep = np.sort(rng.choice(np.arange(1, M), size=25, replace=False))
        t = np.concatenate([[0.0], keep.astype(float), [float(M)]])
        ts.append(t)
        ps.append(4.6 + np.cumsum(rng.normal(0, 0.01, len(t))))
    ev = synth.from_lists(ts, ps)
    S = orc.estimate(ev.offsets, ev.t, ev.logp, N=N, basis="dirichlet")["Sigma"]
    for i in range(3):
        for j in range(3):
            ri = {ts[i][h]: ps[i][h + 1] - ps[i][h] for h in range(len(ts[i]) - 1)}
            rj = {ts[j][h]: ps[j][h + 1] - ps[j][h] for h in range(len(ts[j]) - 1)}
            rc = sum(ri[x] * rj[x] for x in ri if x in rj)
            assert abs(S[i, j] - rc) < 1e-14


def test_dirichlet_N0_is_product_of_total_returns(orc):
    ev = synth.random_events(30, D=4, n_range=(2, 20))
    S = orc.estimate(ev.offsets, ev.t, ev.logp, N=0, basis="dirichlet")["Sigma"]
    tot = np.array([ev.asset(i)[1][-1] - ev.asset(i)[1][0] for i in range(ev.D)])
    assert np.max(np.abs(S - np.outer(tot, tot))) < 1e-15


@pytest.mark.parametrize("N", [1, 5, 100])
def test_single_return_weights(orc, N):
    # One return d: Dirichlet gives d^2 (weights sum to 1); Fejer with the
    # paper's weights (1-|s|/N)/(N+1) gives d^2 N/(N+1).
    ev = synth.from_lists([[0.0, 10.0]], [[4.6, 4.65]])
    d = 0.05
    Sd = orc.estimate(ev.offsets, ev.t, ev.logp, N=N, basis="dirichlet")["Sigma"][0, 0]
    Sf = orc.estimate(ev.offsets, ev.t, ev.logp, N=N, basis="fejer")["Sigma"][0, 0]
    assert abs(Sd - d * d) < 1e-16
    assert abs(Sf - d * d * N / (N + 1)) < 1e-16


@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_sigma_symmetric_psd_and_correlation(orc, basis):
    ev = synth.random_events(40, D=6, n_range=(5, 60), T=2000.0)
    out = orc.estimate(ev.offsets, ev.t, ev.logp, N=25, basis=basis)
    S, R = out["Sigma"], out["R"]
    assert np.max(np.abs(S - S.T)) < 1e-15 * np.max(np.abs(S))
    assert np.min(np.linalg.eigvalsh(S)) > -1e-13 * np.max(np.abs(S))
    assert np.max(np.abs(np.diag(R) - 1.0)) < 4e-16
    assert np.max(np.abs(R)) <= 1.0 + 1e-13


def test_correlation_invariant_to_units_and_scale(orc):
    ev = synth.random_events(41, D=4, n_range=(5, 30), T=100.0)
    R1 = orc.estimate(ev.offsets, ev.t, ev.logp, N=9, basis="fejer")["R"]
    t2 = 3.5 * ev.t + 1234.0            # other time unit and origin
    p2 = 2.0 * ev.logp                  # returns scaled by 2
    R2 = orc.estimate(ev.offsets, t2, p2, N=9, basis="fejer")["R"]
    assert np.max(np.abs(R1 - R2)) < 1e-13


def test_zero_variance_asset_gives_nan(orc):
    ev = synth.from_lists([[0.0, 1.0, 2.0], [0.0, 2.0]], [[1.0, 1.0, 1.0], [1.0, 1.1]])
    R = orc.estimate(ev.offsets, ev.t, ev.logp, N=1)["R"]
    assert np.isnan(R[0, 1]) and np.isnan(R[0, 0]) and R[1, 1] == pytest.approx(1.0)


# --------------------------------------------------------------------------
# Algorithms 2 and 4, Eq. (19)
# --------------------------------------------------------------------------
def test_rescale_endpoints_and_bounds(orc):
    ev = synth.from_lists([[3.0, 5.0, 9.0], [1.0, 4.0], [2.0, 11.0]], [[0, 0, 0], [0, 0], [0, 0]])
    t0, t1 = orc.bounds(ev.offsets, ev.t)
    assert (t0, t1) == (1.0, 11.0)
    tt = orc.rescale(ev.t, t0, t1)
    assert tt[3] == 0.0 and abs(tt[6] - 2 * np.pi) < 1e-15
    assert abs(tt[0] - 2 * np.pi * 0.2) < 1e-15


def test_returns_count_and_left_endpoint(orc):
    ev = synth.from_lists([[0.0, 1.0, 3.0], [0.5], []], [[1.0, 2.0, 4.0], [7.0], []])
    roff, rt, rd = orc.returns(ev.offsets, ev.t, ev.logp)
    assert list(roff) == [0, 2, 2, 2]
    assert list(rt) == [0.0, 1.0] and list(rd) == [1.0, 2.0]


def test_nyquist_hand_example(orc):
    # Times 0, 1, 3, 4: smallest gap 1 -> rescaled gap 2 pi / 4, N_1 =
    # floor((2 pi / (2 pi / 4)) / 2) = 2; times 0, 2, 4: N_2 = floor(2 / 2) = 1;
    # N = min_i N_i (Algorithm 2).
    one = synth.from_lists([[0.0, 1.0, 3.0, 4.0]], [[0] * 4])
    assert orc.nyquist(one.offsets, one.t, 0.0, 4.0) == 2
    ev = synth.from_lists([[0.0, 1.0, 3.0, 4.0], [0.0, 2.0, 4.0]], [[0] * 4, [0] * 3])
    assert orc.nyquist(ev.offsets, ev.t, 0.0, 4.0) == 1
    ev2 = synth.from_lists([[0.0, 2.0, 4.0], [0.0, 3.0], [1.0]], [[0] * 3, [0] * 2, [0]])
    assert orc.nyquist(ev2.offsets, ev2.t, 0.0, 4.0) == 0
    # synchronous 1-s grid of n points: N = floor((n-1)/2) (Sec. 3.1: N = n/2)
    c1 = synth.c1_sync(0)
    assert orc.nyquist(c1.offsets, c1.t, 0.0, 999.0) == 499


def test_eq19_cutoffs(orc):
    for T, dt, N in _golden("eq19_cutoffs.txt"):
        assert orc.n_from_dt(float(T), float(dt)) == int(N)


# --------------------------------------------------------------------------
# Sec. 2.2.5 constants and the CPU NUFFT
# --------------------------------------------------------------------------
def test_msp_printed_values(orc):
    for kern, eps, m in _golden("msp_printed.txt"):
        assert orc.msp(kern, float(eps)) == int(m)
    # Sec. 3.2 also quotes omega ~ 24 (Gaussian) vs 13 (KB) for 12 digits
    # from the literature; the paper's own rule is at least as wide.
    assert 2 * orc.msp("gauss", 1e-12) >= 24


def test_grid_sizes_printed(orc):
    rng = np.random.default_rng(5)
    tt = np.sort(rng.uniform(0, 2 * np.pi, 20))
    d = rng.normal(size=20)
    for N, Mr in _golden("grid_sizes.txt"):
        _, used = orc.nufft("gauss", 1e-6, tt, d, int(N))
        assert used == int(Mr)


def test_bessel_i0_textbook(orc):
    for x, v in _golden("bessel_i0.txt"):
        assert orc.bessel_i0(float(x)) == pytest.approx(float(v), rel=2e-15)
    sp = pytest.importorskip("scipy.special")
    for x in np.linspace(0, 40, 81):
        assert orc.bessel_i0(x) == pytest.approx(float(sp.i0(x)), rel=5e-15)


def test_gauss_legendre_nodes(orc):
    # exact for polynomials of degree <= 2n-1, and integrates the Gaussian
    # whose transform is known in closed form (the pair behind step D.1 of
    # Algorithm 8: int e^{-x^2/4 tau} e^{-ikx} dx = sqrt(4 pi tau) e^{-k^2 tau}).
    x, w = orc.gauss_legendre(24)
    for p in range(0, 47):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.dot(w, x ** p) - exact) < 1e-14
    x, w = orc.gauss_legendre(400)
    tau, L = 0.01, 3.0
    for k in [0.0, 3.0, 10.0, 25.0]:
        v = L * np.dot(w, np.exp(-(L * x) ** 2 / (4 * tau)) * np.cos(k * L * x))
        assert v == pytest.approx(np.sqrt(4 * np.pi * tau) * np.exp(-k * k * tau), rel=1e-12)


@pytest.mark.parametrize("msp_,Mr", [(3, 22), (6, 2000), (9, 40000)])
def test_es_transform_against_adaptive_quadrature(orc, msp_, Mr):
    # Eq. (10) by an adaptive Gauss-Kronrod routine (QUADPACK, the same family
    # as the paper's QuadGK) on the original variable, against the oracle's
    # Gauss-Legendre rule in theta.
    integ = pytest.importorskip("scipy.integrate")
    beta, alpha = 2.3 * 2 * msp_, np.pi * 2 * msp_ / Mr
    for k in [0, 1, Mr // 8, Mr // 4]:
        f = lambda y: np.exp(beta * (np.sqrt(max(0.0, 1 - y * y)) - 1)) * np.cos(alpha * k * y)
        ref = 2 * alpha * integ.quad(f, 0, 1, epsabs=1e-300, epsrel=1e-13, limit=400)[0]
        assert orc.es_phihat(msp_, Mr, k) == pytest.approx(ref, rel=1e-12)
        assert orc.es_phihat(msp_, Mr, k, 400) == pytest.approx(orc.es_phihat(msp_, Mr, k, 200), rel=1e-14)


@pytest.mark.parametrize("kernel", ["gauss", "kb", "es"])
@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-6, 1e-9, 1e-12])
def test_cpu_nufft_meets_requested_tolerance(orc, kernel, eps):
    # The paper tunes M_sp so that every kernel strictly meets the requested
    # relative l2 error of Eq. (15) (Sec. 2.2.5 footnote).
    rng = np.random.default_rng(int(-np.log10(eps)) * 3 + len(kernel))
    n, N = 400, 150
    tt = np.sort(rng.uniform(0, 2 * np.pi, n))
    d = rng.normal(0, 0.01, n)
    c, _ = orc.nufft(kernel, eps, tt, d, N)
    ref = orc.coeffs(tt, d, 0.0, 2 * np.pi, -N, N)
    err = orc.rel_l2(c, ref)
    assert err <= max(eps, 2e-14), err


@pytest.mark.parametrize("kernel", ["gauss", "kb", "es"])
def test_cpu_nufft_smooth_grid_reading(orc, kernel):
    # Reading of the grid size: any even M_r >= 2M (sigma >= 2) with sigma,
    # tau, b, alpha recomputed from M_r and M_sp from the sigma = 2 rule keeps
    # the tolerance; e.g. N = 720 -> 2M = 2882 = 2 * 11 * 131 replaced by 2916.
    rng = np.random.default_rng(11)
    n, N, eps = 600, 720, 1e-6
    tt = np.sort(rng.uniform(0, 2 * np.pi, n))
    d = rng.normal(0, 0.01, n)
    ref = orc.coeffs(tt, d, 0.0, 2 * np.pi, -N, N)
    for Mr in [2882, 2916, 3000, 3456]:
        c, used = orc.nufft(kernel, eps, tt, d, N, Mr)
        assert used == Mr
        assert orc.rel_l2(c, ref) <= eps


def test_cpu_nufft_recovers_estimates(orc):
    # Sec. 3.2: with eps < 1e-4 the NUFFT coefficients reproduce the direct
    # estimates. Sigma from NUFFT coefficients vs from direct sums.
    ev = synth.c2_async(0)
    out = orc.estimate(ev.offsets, ev.t, ev.logp, N=200, basis="fejer")
    roff, rt = out["roff"], out["rt"]
    tt = orc.rescale(rt, out["t0"], out["t1"])
    c = np.stack([orc.nufft("gauss", 1e-6, tt[roff[i]:roff[i + 1]], out["rd"][roff[i]:roff[i + 1]], 200)[0]
                  for i in range(2)])
    S, _ = orc.cov_from_coeffs(c, 200, "fejer")
    assert np.max(np.abs(orc.corr(S) - out["R"])) < 1e-6


# --------------------------------------------------------------------------
# Statistical pin: consistency for a synchronous correlated GBM
# --------------------------------------------------------------------------
def test_convergence_to_integrated_covariance(orc):
    # Synchronous bivariate GBM over one day with n = 2000 points (dt = 1/n
    # day, as in the sensitivity test of Appendix B). E[Sigma_hat] equals the
    # integrated covariance (n-1) dt Sigma under Dirichlet, and N/(N+1) of it
    # under the paper's Fejer weights; the spread shrinks as N grows.
    n, reps = 2000, 120
    cov = synth.bivariate_cov()
    target = cov * (n - 1) / n
    est = {(b, N): [] for b in ("dirichlet", "fejer") for N in (20, 200)}
    for r in range(reps):
        rng = synth.rng_for(77, r)
        lp = synth.gbm_grid(n, 0.01, cov, rng, dt_days=1.0 / n)
        t = np.arange(n, dtype=float)
        ev = synth.from_lists([t, t], [lp[:, 0], lp[:, 1]])
        roff, rt, rd = orc.returns(ev.offsets, ev.t, ev.logp)
        t0, t1 = 0.0, float(n - 1)
        c = np.stack([orc.coeffs(rt[roff[i]:roff[i + 1]], rd[roff[i]:roff[i + 1]], t0, t1 - t0, -200, 200)
                      for i in range(2)])
        for (b, N) in est:
            S, _ = orc.cov_from_coeffs(c[:, 200 - N:200 + N + 1], N, b)
            est[(b, N)].append(S)
    for (b, N), v in est.items():
        v = np.array(v)
        mean, se = v.mean(0), v.std(0, ddof=1) / np.sqrt(reps)
        scale = N / (N + 1) if b == "fejer" else 1.0
        assert np.all(np.abs(mean - scale * target) < 4 * se + 1e-4), (b, N, mean, scale * target)
    for b in ("dirichlet", "fejer"):
        mse = {N: np.mean((np.array(est[(b, N)])[:, 0, 1] - target[0, 1]) ** 2) for N in (20, 200)}
        assert mse[200] < mse[20]
