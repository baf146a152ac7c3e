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
