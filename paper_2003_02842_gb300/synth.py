"""Seeded synthetic event data shaped like the paper's workloads.

This module only draws inputs: correlated geometric Brownian motions
(Algorithm 1, Sec. 3 Eq. (16)) observed synchronously or at Poisson arrival
times (Sec. 3, "arrival time representation"). It holds none of the
estimator's arithmetic, and both the GPU library's tests and the CPU oracle
consume exactly the arrays it returns.

Every workload is returned in CSR form: ``offsets`` (int64, D+1),
``t`` (float64 event times in seconds, strictly increasing per asset) and
``logp`` (float64 log-prices at those times).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SECONDS_PER_DAY = 86400.0
BASE_SEED = 20032842


@dataclass
class Events:
    offsets: np.ndarray
    t: np.ndarray
    logp: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def D(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_events(self) -> int:
        return int(self.offsets[-1])

    def counts(self) -> np.ndarray:
        return np.diff(self.offsets)

    def asset(self, i):
        a, b = self.offsets[i], self.offsets[i + 1]
        return self.t[a:b], self.logp[a:b]


def rng_for(*stream) -> np.random.Generator:
    """Philox counter-based generator keyed by (base seed, stream ids)."""
    key = [BASE_SEED] + [int(s) for s in stream]
    return np.random.Generator(np.random.Philox(np.random.SeedSequence(key)))


def from_lists(ts, ps) -> Events:
    offs = np.zeros(len(ts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(x) for x in ts])
    t = np.concatenate([np.asarray(x, np.float64) for x in ts]) if ts else np.zeros(0)
    p = np.concatenate([np.asarray(x, np.float64) for x in ps]) if ps else np.zeros(0)
    return Events(offs, t, p)


def gbm_grid(n, mu, cov_daily, rng, s0=100.0, dt_days=1.0 / SECONDS_PER_DAY):
    """Algorithm 1: log S_{k+1} = log S_k + (mu - sigma^2/2) dt + sqrt(dt) A Z,
    A the Cholesky factor of the daily covariance; n synchronous points
    (times 0, 1, ..., n-1 seconds). Returns an (n, D) array of log-prices."""
    cov = np.asarray(cov_daily, np.float64)
    D = cov.shape[0]
    mu = np.broadcast_to(np.asarray(mu, np.float64), (D,))
    A = np.linalg.cholesky(cov)
    Z = rng.standard_normal((n - 1, D))
    inc = (mu - 0.5 * np.diag(cov)) * dt_days + np.sqrt(dt_days) * Z @ A.T
    logp = np.empty((n, D))
    logp[0] = np.log(s0)
    logp[1:] = np.log(s0) + np.cumsum(inc, axis=0)
    return logp


def bivariate_cov(var1=0.1, var2=0.2, rho=0.35):
    c = rho * np.sqrt(var1 * var2)
    return np.array([[var1, c], [c, var2]])


def poisson_grid_sample(n_grid, rate, rng):
    """Arrival-time asynchrony on a 1-s grid: exponential inter-arrival times
    with the given rate, each arrival moved up to the next grid second (never
    into the past), repeated seconds merged. Returns sorted grid indices."""
    mean_n = rate * n_grid
    m = int(mean_n + 10 * np.sqrt(mean_n + 1) + 20)
    arr = np.cumsum(rng.exponential(1.0 / rate, size=m))
    while arr[-1] < n_grid - 1:
        arr = np.concatenate([arr, arr[-1] + np.cumsum(rng.exponential(1.0 / rate, size=m))])
    idx = np.ceil(arr[arr <= n_grid - 1]).astype(np.int64)
    return np.unique(idx)


def c1_sync(seed=0, n=1000):
    """D=2 synchronous correlated GBM (mu = 0.01, sigma^2 = 0.1, 0.2,
    rho = 0.35, dt = 1 s), n equally spaced times 0..n-1 s."""
    rng = rng_for(1, seed)
    lp = gbm_grid(n, 0.01, bivariate_cov(), rng)
    t = np.arange(n, dtype=np.float64)
    ev = from_lists([t, t], [lp[:, 0], lp[:, 1]])
    ev.meta = {"workload": "c1_sync_gbm_D2_n1000", "N": n // 2}
    return ev


def c2_async(seed=0, T=28800, rates=(1 / 15, 1 / 20)):
    """D=2 GBM on the 1-s grid over T seconds, each asset observed at Poisson
    arrival times with the given rates; N = floor(min n / 2)."""
    rng = rng_for(2, seed)
    lp = gbm_grid(T, 0.01, bivariate_cov(), rng)
    ts, ps = [], []
    for j, r in enumerate(rates):
        idx = poisson_grid_sample(T, r, rng)
        ts.append(idx.astype(np.float64))
        ps.append(lp[idx, j])
    ev = from_lists(ts, ps)
    ev.meta = {"workload": "c2_async_gbm_D2", "N": int(min(len(x) for x in ts) // 2)}
    return ev


def epps_replications(seed, reps, T=28800, rate=1 / 5, rho=0.35, var=(0.1, 0.2)):
    """The arrival-time Epps experiment (Sec. 4.1): per replication a
    bivariate GBM (mu = 0.01, variances `var`, correlation rho) on a 1-s grid
    of T seconds, each asset observed at its own Poisson arrivals of the same
    rate on that grid (exponential inter-arrival times moved up to the next
    second, repeats merged). Returns the replications stacked as one Events
    (reps problems of 2 assets each)."""
    ts, ps = [], []
    cov = bivariate_cov(var[0], var[1], rho)
    for r in range(reps):
        rng = rng_for(6, seed, r)
        lp = gbm_grid(T, 0.01, cov, rng)
        for j in range(2):
            idx = poisson_grid_sample(T, rate, rng)
            ts.append(idx.astype(np.float64))
            ps.append(lp[idx, j])
    ev = from_lists(ts, ps)
    dt = 1.0 / SECONDS_PER_DAY
    ev.meta = {"workload": f"epps_R{reps}_T{T}", "reps": reps, "T": T, "rate": rate, "rho": rho,
               "step_cov": cov * dt, "step_mean": (0.01 - 0.5 * np.diag(cov)) * dt}
    return ev


def mse_bias_replications(seed, reps, n=100, rho=0.35, var=(0.1, 0.2), mu=0.01):
    """The accuracy experiment (Sec. 3.2): per replication a bivariate GBM of n
    synchronous points spanning one day (times 0..n-1, step 1/n day), the
    first asset observed at every point, the second at every second point
    (regular non-synchronous trading). Returns the replications stacked as
    one Events (reps problems of 2 assets each); meta holds the per-step
    covariance and mean of the log-price increments."""
    cov = bivariate_cov(var[0], var[1], rho)
    dt = 1.0 / n
    ts, ps = [], []
    t1 = np.arange(n, dtype=np.float64)
    t2 = np.arange(0, n, 2, dtype=np.float64)
    for r in range(reps):
        rng = rng_for(7, seed, r)
        lp = gbm_grid(n, mu, cov, rng, dt_days=dt)
        ts += [t1, t2]
        ps += [lp[:, 0], lp[::2, 1]]
    ev = from_lists(ts, ps)
    ev.meta = {"workload": f"mse_bias_R{reps}_n{n}", "reps": reps, "n": n, "step_cov": cov * dt,
               "step_mean": (mu - 0.5 * np.diag(cov)) * dt}
    return ev


def sensitivity_covariances(seed, count, var=(0.1, 0.3), cov=(-0.1, 0.1), max_corr=0.9):
    """Daily 2x2 covariance matrices for the sensitivity test (App. B): both
    variances uniform on `var`, the covariance uniform on `cov` and clipped to
    a correlation of at most max_corr (a definite matrix)."""
    rng = rng_for(9, seed)
    out = []
    for _ in range(count):
        v1, v2 = rng.uniform(*var, size=2)
        lim = max_corr * np.sqrt(v1 * v2)
        c = float(np.clip(rng.uniform(*cov), -lim, lim))
        out.append(np.array([[v1, c], [c, v2]]))
    return out


def sensitivity_replications(seed, covs, reps=1, n=10000, mu=0.01):
    """The sensitivity test (App. B): synchronous bivariate GBMs of n points
    over one day (step 1/n day), `reps` replications of each daily 2x2
    covariance in covs; all stacked as one Events (2 assets per problem).
    meta["truth"] holds each problem's integrated covariance over the path,
    (n - 1)/n times the daily one."""
    ts, ps, truth = [], [], []
    t = np.arange(n, dtype=np.float64)
    for i, cov in enumerate(covs):
        cov = np.asarray(cov, np.float64)
        for r in range(reps):
            rng = rng_for(8, seed, i, r)
            lp = gbm_grid(n, mu, cov, rng, dt_days=1.0 / n)
            ts += [t, t]
            ps += [lp[:, 0], lp[:, 1]]
            truth.append(cov * (n - 1) / n)
    ev = from_lists(ts, ps)
    ev.meta = {"workload": f"sensitivity_n{n}", "truth": np.array(truth), "n": n}
    return ev


def _continuous_poisson(T, rate, rng):
    n = rng.poisson(rate * T)
    return np.sort(rng.uniform(0.0, T, size=n))


def block_factor_gbm(times_per_asset, sig2, mu, block_of, rho_in, rho_out, rng, s0=100.0):
    """Correlated GBM observed at arbitrary (continuous) per-asset times, exact
    in law: log p_i(t) = log s0 + (mu - sig2_i/2) t + sigma_i W_i(t) with
    W_i = sqrt(rho_out) G + sqrt(rho_in - rho_out) B_block(i) + sqrt(1 - rho_in) E_i
    (G, B_b, E_i independent Brownian motions; t in days). Pairwise correlation
    rho_in inside a block and rho_out across blocks."""
    D = len(times_per_asset)
    nb = int(max(block_of)) + 1
    allt = np.unique(np.concatenate([x for x in times_per_asset if len(x)] + [np.zeros(1)]))
    days = allt / SECONDS_PER_DAY
    dtd = np.diff(days, prepend=0.0)
    sq = np.sqrt(dtd)[:, None]
    G = np.cumsum(rng.standard_normal((len(allt), 1)) * sq, axis=0)[:, 0]
    B = np.cumsum(rng.standard_normal((len(allt), nb)) * sq, axis=0)
    ts, ps = [], []
    for i in range(D):
        ti = np.asarray(times_per_asset[i], np.float64)
        pos = np.searchsorted(allt, ti)
        di = ti / SECONDS_PER_DAY
        ddi = np.diff(di, prepend=0.0)
        E = np.cumsum(rng.standard_normal(len(ti)) * np.sqrt(ddi))
        W = (np.sqrt(rho_out) * G[pos] + np.sqrt(max(rho_in - rho_out, 0.0)) * B[pos, block_of[i]]
             + np.sqrt(1.0 - rho_in) * E)
        s = np.sqrt(sig2[i])
        ps.append(np.log(s0) + (mu - 0.5 * sig2[i]) * di + s * W)
        ts.append(ti)
    return ts, ps


def c3_block(seed=0, D=100, T=28800.0, N=10000, n_blocks=10, rho_in=0.5, rho_out=0.1,
             sig2_range=(0.05, 0.3), rate_range=(1 / 60, 1 / 2)):
    """D correlated GBM assets with block correlation (n_blocks blocks, intra
    rho_in, inter rho_out), sigma^2 ~ U(sig2_range), each observed at
    continuous-time Poisson arrivals with rate ~ U(rate_range) per second over
    T seconds."""
    rng = rng_for(3, seed)
    sig2 = rng.uniform(*sig2_range, size=D)
    rates = rng.uniform(*rate_range, size=D)
    block_of = np.arange(D) * n_blocks // D
    times = [_continuous_poisson(T, r, rng) for r in rates]
    ts, ps = block_factor_gbm(times, sig2, 0.01, block_of, rho_in, rho_out, rng)
    ev = from_lists(ts, ps)
    ev.meta = {"workload": f"c3_block_gbm_D{D}_N{N}", "N": N, "T": T,
               "rates": rates, "sig2": sig2}
    return ev


def batch_replications(seed, reps, D=10, T=28800.0, rho=0.35, sig2_range=(0.1, 0.2),
                       median_n=2000, sdlog=1.0, clip=(100, 50000)):
    """Monte Carlo replications of D equicorrelated GBM assets; per-asset event
    counts lognormal (median median_n, log-sd sdlog) clipped to `clip`, event
    times uniform order statistics on [0, T] (a Poisson process given its
    count). Returns one Events per replication."""
    out = []
    for r in range(reps):
        rng = rng_for(4, seed, r)
        sig2 = rng.uniform(*sig2_range, size=D)
        n = np.clip(np.round(np.exp(np.log(median_n) + sdlog * rng.standard_normal(D))),
                    clip[0], clip[1]).astype(np.int64)
        times = [np.sort(rng.uniform(0.0, T, size=k)) for k in n]
        ts, ps = block_factor_gbm(times, sig2, 0.01, np.zeros(D, np.int64), rho, rho, rng)
        ev = from_lists(ts, ps)
        ev.meta = {"rep": r}
        out.append(ev)
    return out


def c4_batch(seed=0, reps=4096, D=10, T=28800, rho=0.35, sig2_range=(0.1, 0.2), median_n=2000, sdlog=1.0,
             clip=(100, 50000), mu=0.01, s0=100.0):
    """Batched Monte Carlo workload: `reps` replications of D equicorrelated
    GBM assets (pairwise rho, sigma^2 ~ U(sig2_range)) observed on the 1-s
    grid over T seconds. Per-asset event counts are lognormal (median
    median_n, log-sd sdlog) clipped to `clip` and then to the T grid
    seconds; an asset observes each second independently with probability
    count / T (so its count is Binomial around the drawn value). Log-prices
    are exact in law at the observed seconds (one common Brownian factor
    plus one per asset). Returns one CSR Events over reps * D assets in
    replication-major order, plus meta with the per-replication Nyquist
    cutoff floor(span / 2) (unit gaps)."""
    rng = rng_for(4, seed)
    ts, ps = [], []
    nyq = np.empty(reps, dtype=np.int64)
    a_c, a_i = np.sqrt(rho), np.sqrt(1.0 - rho)
    for r in range(reps):
        sig2 = rng.uniform(*sig2_range, size=D)
        n = np.clip(np.round(np.exp(np.log(median_n) + sdlog * rng.standard_normal(D))), clip[0], clip[1])
        n = np.minimum(n, T)
        keep = rng.random((D, T)) < (n / T)[:, None]
        keep[:, 0] |= ~keep.any(axis=1)  # every asset keeps at least one second
        union = keep.any(axis=0)
        sec = np.flatnonzero(union)
        dtd = np.diff(sec, prepend=0).astype(np.float64) / SECONDS_PER_DAY
        G = np.cumsum(rng.standard_normal(len(sec)) * np.sqrt(dtd))
        gpos = np.full(T, -1, dtype=np.int64)
        gpos[sec] = np.arange(len(sec))
        lo, hi = T, 0
        for i in range(D):
            si = np.flatnonzero(keep[i])
            di = si.astype(np.float64) / SECONDS_PER_DAY
            E = np.cumsum(rng.standard_normal(len(si)) * np.sqrt(np.diff(di, prepend=0.0)))
            W = a_c * G[gpos[si]] + a_i * E
            ps.append(np.log(s0) + (mu - 0.5 * sig2[i]) * di + np.sqrt(sig2[i]) * W)
            ts.append(si.astype(np.float64))
            lo, hi = min(lo, int(si[0])), max(hi, int(si[-1]))
        nyq[r] = (hi - lo) // 2
    ev = from_lists(ts, ps)
    ev.meta = {"workload": f"c4_batch_gbm_R{reps}_D{D}", "reps": reps, "D": D, "nyquist": nyq}
    return ev


def gram_coefficients(seed, D, N, day_var=0.1, T=28800):
    """Synthetic Fourier coefficients for the contraction alone: D x (N + 1)
    complex64, each mode complex Gaussian with the variance that one asset's
    returns over T seconds of a GBM with daily variance day_var give every
    mode, (day_var T / 86400) / (2 pi)^2 (returns summed against unit-modulus
    phases), independent across assets and modes."""
    rng = rng_for(10, seed, D, N)
    sd = np.sqrt(day_var * T / SECONDS_PER_DAY / 2.0) / (2.0 * np.pi)  # per real and imaginary part
    F = (rng.standard_normal((D, N + 1)) + 1j * rng.standard_normal((D, N + 1))) * sd
    return F.astype(np.complex64)


def c5_day(seed=0, D=500, T=28800, n_factors=3, load_sd=0.3, idio_var=0.1, mu=0.01, s0=100.0,
           lam_lo=0.01, lam_hi=1.0, shape=0.45):
    """Serving workload: one trading day of D assets on the 1-s grid. Arrival
    intensity is U-shaped, lambda(t) = lam_lo + (lam_hi - lam_lo) |2t/T - 1|^shape
    per second (busy open and close, quiet midday); an asset observes second
    t with probability 1 - exp(-lambda(t)). Log-prices follow a factor GBM,
    exact in law at the observed seconds: n_factors common Brownian factors
    with loadings ~ N(0, load_sd^2) plus an idiosyncratic one of variance
    idio_var (per day)."""
    rng = rng_for(5, seed)
    tsec = np.arange(T)
    lam = lam_lo + (lam_hi - lam_lo) * np.abs(2.0 * tsec / T - 1.0) ** shape
    pobs = 1.0 - np.exp(-lam)
    dt = 1.0 / SECONDS_PER_DAY
    Fac = np.cumsum(rng.standard_normal((T, n_factors)) * np.sqrt(dt), axis=0)  # factors on every second
    L = rng.normal(0.0, load_sd, size=(D, n_factors))
    ts, ps = [], []
    for i in range(D):
        sec = np.flatnonzero(rng.random(T) < pobs)
        if len(sec) == 0:
            sec = np.array([0])
        di = sec.astype(np.float64) * dt
        E = np.cumsum(rng.standard_normal(len(sec)) * np.sqrt(np.diff(di, prepend=0.0)))
        var_i = float(L[i] @ L[i]) + idio_var
        W = Fac[sec] @ L[i] + np.sqrt(idio_var) * E
        ps.append(np.log(s0) + (mu - 0.5 * var_i) * di + W)
        ts.append(sec.astype(np.float64))
    ev = from_lists(ts, ps)
    ev.meta = {"workload": f"c5_day_D{D}", "T": T}
    return ev


def c5_requests(seed=0, n=10000, D=500, T=28800, w_range=(300, 28800), k_range=(10, 500),
                dt_modes=(0.0, 60.0, 600.0), windows=0):
    """Request stream of the serving workload: window length ~ U(w_range)
    seconds at a uniform start, asset subset of size ~ U{k_range} drawn
    without replacement, cutoff mode uniform over dt_modes (0: the window's
    Nyquist cutoff, else Eq. (19) at that sampling interval). windows > 0:
    that many such windows are drawn first and every request takes one of
    them uniformly (clients polling a few standing windows)."""
    rng = rng_for(6, seed)
    pool = []
    for _ in range(windows):
        W = float(rng.uniform(*w_range))
        t0 = float(rng.uniform(0.0, T - W))
        pool.append((t0, t0 + W))
    out = []
    for _ in range(n):
        if pool:
            t0, t1 = pool[int(rng.integers(len(pool)))]
            W = t1 - t0
        else:
            W = float(rng.uniform(*w_range))
            t0 = float(rng.uniform(0.0, T - W))
        k = int(rng.integers(k_range[0], min(k_range[1], D) + 1))
        assets = np.sort(rng.choice(D, size=k, replace=False)).astype(np.int32)
        dtm = float(dt_modes[int(rng.integers(len(dt_modes)))])
        out.append({"t0": t0, "t1": t0 + W, "assets": assets, "dt": dtm})
    return out


def window_events(ev, assets, t0, t1):
    """The events of the given assets inside [t0, t1], as their own Events."""
    ts, ps = [], []
    for a in assets:
        t, p = ev.asset(int(a))
        m = (t >= t0) & (t <= t1)
        ts.append(t[m])
        ps.append(p[m])
    return from_lists(ts, ps)


def sweep_cutoffs(N_max, count=64):
    """`count` strictly increasing cutoffs, log-spaced from 1 to N_max."""
    x = np.exp(np.linspace(0.0, np.log(max(N_max, 1)), count))
    out = []
    for v in x:
        c = max(int(round(v)), out[-1] + 1 if out else 1)
        out.append(c)
    out = [min(c, N_max) for c in out]
    return sorted(set(out))


def random_events(seed, D, n_range=(2, 50), T=1000.0, grid=None, scale=1e-2):
    """Small random test inputs: per-asset event counts uniform in n_range,
    times uniform on [0, T] (or distinct grid points if grid is an integer),
    log-prices a random walk with step sd `scale`."""
    rng = rng_for(9, seed)
    ts, ps = [], []
    for _ in range(D):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        if grid:
            t = np.sort(rng.choice(grid, size=min(n, grid), replace=False)).astype(np.float64)
        else:
            t = np.sort(rng.uniform(0.0, T, size=n))
        p = 4.6 + np.cumsum(scale * rng.standard_normal(len(t)))
        ts.append(t)
        ps.append(p)
    return from_lists(ts, ps)


def concat_events(evs):
    """Stack several Events into one CSR set (replications side by side)."""
    ts, ps = [], []
    for ev in evs:
        for i in range(ev.D):
            a, b = ev.asset(i)
            ts.append(a)
            ps.append(b)
    return from_lists(ts, ps)
