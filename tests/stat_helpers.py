"""Closed-form expectations used by the statistical tests (the oracle's on
the CPU, the GPU library's on the device)."""
import numpy as np


def expected_sigma(meta, N, basis):
    """E[Sigma] of Eq. (2) (Dirichlet) or Eq. (3) (Fejer) for the accuracy
    experiment: returns of asset 1 over each step, of asset 2 over each pair
    of steps, each carried by its left end point, times rescaled to
    [0, 2 pi] by the data's first and last time."""
    n = meta["n"]
    C, m = meta["step_cov"], meta["step_mean"]
    t1 = np.arange(n - 1, dtype=np.float64)        # asset 1: return u covers step u
    t2 = np.arange(0, n - 2, 2, dtype=np.float64)  # asset 2: return v covers steps 2v/2, 2v/2 + 1
    steps = [[{int(u)} for u in t1], [{int(v), int(v) + 1} for v in t2]]
    times = [t1 * 2 * np.pi / (n - 1), t2 * 2 * np.pi / (n - 1)]
    k = np.arange(-N, N + 1)
    w = np.full(2 * N + 1, 1.0 / (2 * N + 1)) if basis == "dirichlet" else (1.0 - np.abs(k) / N) / (N + 1)
    out = np.zeros((2, 2))
    for a in range(2):
        for b in range(2):
            x = times[a][:, None] - times[b][None, :]
            K = (w[None, None, :] * np.cos(k[None, None, :] * x[:, :, None])).sum(axis=2)
            E = np.array([[len(su & sv) * C[a, b] + len(su) * m[a] * len(sv) * m[b] for sv in steps[b]]
                          for su in steps[a]])
            out[a, b] = (K * E).sum()
    return out


def sigma_moments(meta, N, basis):
    """Mean and variance of Sigma_ab in the accuracy experiment, from the
    estimator as a bilinear form in the Gaussian step increments.

    With S the 2(n-1) step increments (asset 1's, then asset 2's), each step
    N(m, C) and the steps independent, asset a's returns are P_a S (asset 1:
    one step each, asset 2: two steps each) and Sigma_ab = S^T G S with
    G = P_a^T K_ab P_b, K_ab[u, v] = K_N(t_u - t_v). For the symmetric part
    B = (G + G^T) / 2 and S ~ N(mu, V):
      E[Sigma_ab]   = tr(B V) + mu^T B mu,
      Var[Sigma_ab] = 2 tr(B V B V) + 4 mu^T B V B mu
    (the moments of a Gaussian quadratic form). Returns (E, Var), each 2 x 2."""
    n = meta["n"]
    C, m = meta["step_cov"], meta["step_mean"]
    ns = n - 1
    t1 = np.arange(n - 1, dtype=np.float64)
    t2 = np.arange(0, n - 2, 2, dtype=np.float64)
    P = [np.zeros((len(t1), 2 * ns)), np.zeros((len(t2), 2 * ns))]
    for u in range(len(t1)):
        P[0][u, u] = 1.0
    for v in range(len(t2)):
        P[1][v, ns + 2 * v] = 1.0
        P[1][v, ns + 2 * v + 1] = 1.0
    V = np.kron(C, np.eye(ns))
    mu = np.concatenate([np.full(ns, m[0]), np.full(ns, m[1])])
    times = [t1 * 2 * np.pi / (n - 1), t2 * 2 * np.pi / (n - 1)]
    k = np.arange(-N, N + 1)
    w = np.full(2 * N + 1, 1.0 / (2 * N + 1)) if basis == "dirichlet" else (1.0 - np.abs(k) / N) / (N + 1)
    E, Var = np.zeros((2, 2)), np.zeros((2, 2))
    for a in range(2):
        for b in range(2):
            x = times[a][:, None] - times[b][None, :]
            K = (w[None, None, :] * np.cos(k[None, None, :] * x[:, :, None])).sum(axis=2)
            G = P[a].T @ K @ P[b]
            B = 0.5 * (G + G.T)
            BV = B @ V
            E[a, b] = np.trace(BV) + mu @ B @ mu
            Var[a, b] = 2.0 * np.trace(BV @ BV) + 4.0 * mu @ BV @ B @ mu
    return E, Var


def variance_se(x):
    """Standard error of the sample variance of x (from its fourth central
    moment)."""
    x = np.asarray(x, dtype=np.float64)
    d = x - x.mean()
    s2 = (d ** 2).mean()
    m4 = (d ** 4).mean()
    return np.sqrt(max(m4 - s2 ** 2, 0.0) / len(x))


def basis_kernel(N, basis, x):
    """K_N(x) = sum_{|k|<=N} w_k e^{ikx} in closed form: the Dirichlet
    kernel sin((N + 1/2) x) / ((2N + 1) sin(x/2)) (Eq. (2)'s weights) or the
    Fejer kernel sin^2(N x/2) / (N (N + 1) sin^2(x/2)) (Eq. (3)'s weights,
    (1 - |k|/N) / (N + 1)); limits 1 and N / (N + 1) at x = 0."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sin(0.5 * x)
    zero = np.abs(s) < 1e-300
    s = np.where(zero, 1.0, s)
    if basis == "dirichlet":
        v = np.sin((N + 0.5) * x) / ((2 * N + 1) * s)
        return np.where(zero, 1.0, v)
    v = (np.sin(0.5 * N * x) / s) ** 2 / (N * (N + 1.0))
    return np.where(zero, N / (N + 1.0), v)


def grid_pair_conditional_sigma(t1, t2, cutoffs, basis, C, m):
    """E[Sigma | observation times] for two assets of a GBM on a 1-s grid
    (per-step covariance C, per-step mean m), observed at the distinct sorted
    integer times t1 and t2, each return carried by its left end point, times
    rescaled by Algorithm 4 over both assets. From Eqs. (2)/(3),
      E[Sigma_ab] = sum_{u,v} K_N(t~_u - t~_v) E[d_u^a d_v^b],
      E[d_u^a d_v^b] = C_ab |S_u^a n S_v^b| + m_a m_b |S_u^a| |S_v^b|,
    S_u the grid steps return u spans. The covariance part is a sum over the
    steps both assets cover of K_N at the difference of the two returns'
    left end points (a histogram of those differences); the drift part is
    sum_k w_k A_k conj(B_k) with A_k = sum_u |S_u| e^{-ik t~_u}, one FFT of
    the grid. Returns an array [len(cutoffs), 2, 2]."""
    t0 = min(int(t1[0]), int(t2[0]))
    span = max(int(t1[-1]), int(t2[-1])) - t0
    js = [np.asarray(t1, np.int64) - t0, np.asarray(t2, np.int64) - t0]
    # left end point of the return covering step s (s spans j_u -> j_u + 1)
    def left(a, s):
        return js[a][np.searchsorted(js[a], s, side="left") - 1]
    hist = {}
    for a in range(2):
        for b in range(a, 2):
            lo = max(js[a][0], js[b][0]) + 1
            hi = min(js[a][-1], js[b][-1])
            s = np.arange(lo, hi + 1)
            d = left(a, s) - left(b, s) if len(s) else np.zeros(0, np.int64)
            hist[a, b] = np.unique(d, return_counts=True)
    A = []
    for a in range(2):
        g = np.zeros(span)
        np.add.at(g, js[a][:-1], np.diff(js[a]).astype(np.float64))
        A.append(np.fft.fft(g))
    out = np.zeros((len(cutoffs), 2, 2))
    for j, N in enumerate(cutoffs):
        k = np.arange(N + 1)
        w = np.full(N + 1, 1.0 / (2 * N + 1)) if basis == "dirichlet" else (1.0 - k / N) / (N + 1)
        for a in range(2):
            for b in range(a, 2):
                d, cnt = hist[a, b]
                cov = C[a, b] * float(np.sum(cnt * basis_kernel(N, basis, 2 * np.pi * d / span)))
                p = A[a][:N + 1] * np.conj(A[b][:N + 1])
                drift = m[a] * m[b] * (w[0] * p[0].real + 2.0 * np.sum(w[1:] * p[1:].real))
                out[j, a, b] = out[j, b, a] = cov + drift
    return out


def grid_pair_conditional_sigma_bruteforce(t1, t2, N, basis, C, m):
    """The same expectation by the pairwise sum over returns, with the step
    sets intersected explicitly and K_N summed mode by mode (small inputs)."""
    t0 = min(t1[0], t2[0])
    span = max(t1[-1], t2[-1]) - t0
    ts = [np.asarray(t1, np.int64), np.asarray(t2, np.int64)]
    k = np.arange(-N, N + 1)
    w = np.full(2 * N + 1, 1.0 / (2 * N + 1)) if basis == "dirichlet" else (1.0 - np.abs(k) / N) / (N + 1)
    out = np.zeros((2, 2))
    for a in range(2):
        for b in range(2):
            tot = 0.0
            for u in range(len(ts[a]) - 1):
                Su = set(range(int(ts[a][u]) + 1, int(ts[a][u + 1]) + 1))
                for v in range(len(ts[b]) - 1):
                    Sv = set(range(int(ts[b][v]) + 1, int(ts[b][v + 1]) + 1))
                    x = 2 * np.pi * (ts[a][u] - ts[b][v]) / span
                    K = float(np.sum(w * np.cos(k * x)))
                    tot += K * (C[a, b] * len(Su & Sv) + m[a] * m[b] * len(Su) * len(Sv))
            out[a, b] = tot
    return out
