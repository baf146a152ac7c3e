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
