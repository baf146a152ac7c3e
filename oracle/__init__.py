"""FP64 CPU oracle for the Malliavin-Mancino NUFFT covariance estimator.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline and ``--impl reference`` legs may import this
package. The GPU library never calls it and shares no code with it.

The arithmetic lives in ``mm_oracle.c`` (plain C, FP64, OpenMP over modes);
this module only marshals numpy arrays through ctypes and strings the steps of
Algorithm 3 (rescale, returns, Nyquist cutoff, coefficients, contraction,
correlation) together in the paper's order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

GAUSS, KB, ES = 0, 1, 2
DIRICHLET, FEJER = 0, 1
KERNELS = {"gauss": GAUSS, "kb": KB, "es": ES}
BASES = {"dirichlet": DIRICHLET, "fejer": FEJER}


def build(force: bool = False) -> str:
    """Compile mm_oracle.c into liboracle.so (no contraction of a*b+c, so the
    compensated sums and TwoSum steps stay exact on Arm as on x86)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    compile_c(_SRC, tmp)
    os.replace(tmp, _LIB)
    return _LIB


def compile_c(src: str, out: str) -> None:
    """The oracle's compiler line, also used by the tests that build copies of
    the oracle with planted mistakes."""
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_d = ctypes.c_double
_i = ctypes.c_int
_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def _declare(L):
    L.orc_bounds.argtypes = [_i, _p, _p, _p, _p]
    L.orc_rescale.argtypes = [_i64, _p, _d, _d, _p]
    L.orc_returns.argtypes = [_i, _p, _p, _p, _p, _p, _p]
    L.orc_nyquist.argtypes = [_i, _p, _p, _d, _d]
    L.orc_nyquist.restype = _i64
    L.orc_coeffs.argtypes = [_i64, _p, _p, _d, _d, _i64, _i64, _p]
    L.orc_coeffs_at.argtypes = [_i64, _p, _p, _d, _d, _i64, _p, _p]
    L.orc_weight.argtypes = [_i, _i64, _i64]
    L.orc_weight.restype = _d
    L.orc_cov_from_coeffs.argtypes = [_i, _i64, _i, _p, _p]
    L.orc_cov_from_coeffs.restype = _d
    L.orc_cov_pairwise.argtypes = [_i, _p, _p, _p, _d, _d, _i64, _i, _p]
    L.orc_corr.argtypes = [_i, _p, _p]
    L.orc_msp.argtypes = [_i, _d]
    L.orc_msp.restype = _i
    L.orc_bessel_i0.argtypes = [_d]
    L.orc_bessel_i0.restype = _d
    L.orc_gauss_legendre.argtypes = [_i, _p, _p]
    L.orc_es_phihat.argtypes = [_i, _i64, _d, _i]
    L.orc_es_phihat.restype = _d
    L.orc_nufft.argtypes = [_i, _d, _i64, _p, _p, _i64, _i64, _p]
    L.orc_nufft.restype = _i64
    L.orc_rel_l2.argtypes = [_i64, _p, _p]
    L.orc_rel_l2.restype = _d
    L.orc_n_from_dt.argtypes = [_d, _d]
    L.orc_n_from_dt.restype = _i64
    L.orc_num_threads.argtypes = []
    L.orc_num_threads.restype = _i


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64a(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _kernel(k):
    return KERNELS[k] if isinstance(k, str) else int(k)


def _basis(b):
    return BASES[b] if isinstance(b, str) else int(b)


# --------------------------------------------------------------------------
# Thin wrappers, one per C function
# --------------------------------------------------------------------------
def bounds(offsets, t):
    """Algorithm 4: (t_min, t_max) over every asset's times."""
    off, tt = _i64a(offsets), _f64(t)
    lo, hi = np.zeros(1), np.zeros(1)
    lib().orc_bounds(len(off) - 1, _ptr(off), _ptr(tt), _ptr(lo), _ptr(hi))
    return float(lo[0]), float(hi[0])


def rescale(t, t0, t1):
    """Algorithm 4: t~ = 2 pi (t - t0) / (t1 - t0)."""
    tt = _f64(t)
    out = np.empty_like(tt)
    lib().orc_rescale(len(tt), _ptr(tt), t0, t1, _ptr(out))
    return out


def returns(offsets, t, logp):
    """Algorithm 3 step F.3: per-asset returns at left end points, as CSR."""
    off, tt, lp = _i64a(offsets), _f64(t), _f64(logp)
    D = len(off) - 1
    n = int(off[-1] - off[0])
    roff = np.zeros(D + 1, dtype=np.int64)
    rt = np.zeros(max(n, 1))
    rd = np.zeros(max(n, 1))
    lib().orc_returns(D, _ptr(off), _ptr(tt), _ptr(lp), _ptr(roff), _ptr(rt), _ptr(rd))
    m = int(roff[-1])
    return roff, rt[:m].copy(), rd[:m].copy()


def nyquist(offsets, t, t0, t1):
    """Algorithm 2: N = min_i floor(span / (2 min-gap_i)); -1 if undefined."""
    off, tt = _i64a(offsets), _f64(t)
    return int(lib().orc_nyquist(len(off) - 1, _ptr(off), _ptr(tt), t0, t1))


def coeffs(rt, rd, t0, span, kmin, kmax):
    """Eq. (4) times 2 pi: c_k = sum_h delta_h exp(-i k t~_h), k = kmin..kmax."""
    a, b = _f64(rt), _f64(rd)
    out = np.zeros(2 * (kmax - kmin + 1))
    lib().orc_coeffs(len(a), _ptr(a), _ptr(b), t0, span, kmin, kmax, _ptr(out))
    return out[0::2] + 1j * out[1::2]


def coeffs_at(rt, rd, t0, span, ks):
    """Eq. (4) times 2 pi at an explicit list of modes."""
    a, b, k = _f64(rt), _f64(rd), _i64a(ks)
    out = np.zeros(2 * len(k))
    lib().orc_coeffs_at(len(a), _ptr(a), _ptr(b), t0, span, len(k), _ptr(k), _ptr(out))
    return out[0::2] + 1j * out[1::2]


def weight(basis, N, k):
    return float(lib().orc_weight(_basis(basis), N, k))


def cov_from_coeffs(c, N, basis):
    """Algorithm 3 step C from c[D, 2N+1] (k = -N..N). Returns (Sigma, worst |Im|)."""
    c = np.ascontiguousarray(c, dtype=np.complex128)
    D = c.shape[0]
    S = np.zeros(2 * D * D)
    worst = lib().orc_cov_from_coeffs(D, N, _basis(basis), _ptr(c.view(np.float64)), _ptr(S))
    return S[: D * D].reshape(D, D), float(worst)


def cov_pairwise(roff, rt, rd, t0, span, N, basis):
    """Eqs. (2)/(3) with the sum over s in closed form: O(n_i n_j) per pair."""
    ro, a, b = _i64a(roff), _f64(rt), _f64(rd)
    D = len(ro) - 1
    S = np.zeros(D * D)
    lib().orc_cov_pairwise(D, _ptr(ro), _ptr(a), _ptr(b), t0, span, N, _basis(basis), _ptr(S))
    return S.reshape(D, D)


def corr(S):
    """Algorithm 3 last step: R_ij = S_ij / (sqrt(S_ii) sqrt(S_jj))."""
    S = _f64(S)
    D = S.shape[0]
    R = np.zeros(D * D)
    lib().orc_corr(D, _ptr(S), _ptr(R))
    return R.reshape(D, D)


def msp(kernel, eps):
    """M_sp(eps) rule of Sec. 2.2.5 (sigma = 2)."""
    return int(lib().orc_msp(_kernel(kernel), eps))


def bessel_i0(x):
    return float(lib().orc_bessel_i0(x))


def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    lib().orc_gauss_legendre(n, _ptr(x), _ptr(w))
    return x, w


def es_phihat(msp_, Mr, k, nq=200):
    """Eq. (10) scaled to the grid: alpha * int phi_ES(y) e^{i alpha k y} dy."""
    return float(lib().orc_es_phihat(msp_, Mr, float(k), nq))


def nufft(kernel, eps, tt, d, N, Mr=0):
    """Paper-faithful CPU type-1 NUFFT (Algorithms 8/9/10): c_k, k = -N..N."""
    a, b = _f64(tt), _f64(d)
    out = np.zeros(2 * (2 * N + 1))
    Mr_used = lib().orc_nufft(_kernel(kernel), eps, len(a), _ptr(a), _ptr(b), N, Mr, _ptr(out))
    return out[0::2] + 1j * out[1::2], int(Mr_used)


def rel_l2(F, Fref):
    """Eq. (15): ||F - Fref||_2 / ||Fref||_2."""
    F = np.ascontiguousarray(F, dtype=np.complex128)
    Fr = np.ascontiguousarray(Fref, dtype=np.complex128)
    return float(lib().orc_rel_l2(F.size, _ptr(F.view(np.float64)), _ptr(Fr.view(np.float64))))


def n_from_dt(T, dt):
    """Eq. (19): N = floor((T/dt - 1)/2)."""
    return int(lib().orc_n_from_dt(T, dt))


def num_threads():
    return int(lib().orc_num_threads())


# --------------------------------------------------------------------------
# Algorithm 3 end to end
# --------------------------------------------------------------------------
def estimate(offsets, t, logp, N=None, basis="dirichlet", window=None, ks=None):
    """Algorithm 3: rescale (Algorithm 4, data min/max or the given window),
    returns, Nyquist cutoff (Algorithm 2) unless N is given, coefficients by
    the direct sum of Eq. (4), Sigma by step C, R by the last step.

    Returns a dict with F (D x (N+1) complex, k = 0..N, F-convention c/2pi),
    c_full (D x (2N+1), k = -N..N, no 1/2pi), Sigma, R, N, (t0, t1)."""
    off = _i64a(offsets)
    D = len(off) - 1
    t0, t1 = window if window is not None else bounds(off, t)
    if N is None:
        N = nyquist(off, t, t0, t1)
    roff, rt, rd = returns(off, t, logp)
    span = t1 - t0
    c = np.zeros((D, 2 * N + 1), dtype=np.complex128)
    for i in range(D):
        a, b = rt[roff[i]:roff[i + 1]], rd[roff[i]:roff[i + 1]]
        if len(a):
            c[i] = coeffs(a, b, t0, span, -N, N)
    S, worst = cov_from_coeffs(c, N, basis)
    R = corr(S)
    F = c[:, N:] / (2.0 * np.pi)
    return {"F": F, "c_full": c, "Sigma": S, "R": R, "N": N, "t0": t0, "t1": t1,
            "imag_worst": worst, "roff": roff, "rt": rt, "rd": rd}


def cov_pairwise_cutoffs(offsets, t, logp, Ns, basis="dirichlet", window=None):
    """Sec. 3.1, per-asset cutoffs: Sigma_ij by Eq. (2) or (3) at
    N_ij = min(Ns[i], Ns[j]), every asset rescaled with the problem's common
    window (data min/max unless given). Each distinct pairwise cutoff is one
    evaluation of Algorithm 3 at that N; its entries (i, j) with N_ij = N are
    kept. Returns (Sigma, R)."""
    off = _i64a(offsets)
    D = len(off) - 1
    Ns = np.asarray(Ns, dtype=np.int64)
    t0, t1 = window if window is not None else bounds(off, t)
    Nij = np.minimum(Ns[:, None], Ns[None, :])
    S = np.zeros((D, D))
    for N in np.unique(Nij):
        est = estimate(off, t, logp, N=int(N), basis=basis, window=(t0, t1))
        sel = Nij == N
        S[sel] = est["Sigma"][sel]
    return S, corr(S)


def nearest_psd(S):
    """The positive semi-definite matrix nearest to the symmetric S in the
    Frobenius norm (the eigenvalue method the paper cites for repairing a
    pairwise estimate, Sec. 3.1): V max(Lambda, 0) V^T from S = V Lambda V^T
    (numpy's symmetric eigendecomposition). Returns (matrix, number of
    negative eigenvalues); S itself when none is negative."""
    S = 0.5 * (np.asarray(S, dtype=np.float64) + np.asarray(S, dtype=np.float64).T)
    lam, V = np.linalg.eigh(S)
    neg = int(np.sum(lam < 0.0))
    if neg == 0:
        return S, 0
    return (V * np.maximum(lam, 0.0)) @ V.T, neg


def coeffs_F(offsets, t, logp, N, window=None, assets=None, ks=None):
    """F(dp_i)(k) = c_k / (2 pi) (Eq. (4)) for k = 0..N (or the modes ks) of the
    selected assets; rescale bounds from the data unless a window is given."""
    off = _i64a(offsets)
    D = len(off) - 1
    t0, t1 = window if window is not None else bounds(off, t)
    roff, rt, rd = returns(off, t, logp)
    span = t1 - t0
    assets = range(D) if assets is None else assets
    out = []
    for i in assets:
        a, b = rt[roff[i]:roff[i + 1]], rd[roff[i]:roff[i + 1]]
        if ks is None:
            v = coeffs(a, b, t0, span, 0, N) if len(a) else np.zeros(N + 1, complex)
        else:
            v = coeffs_at(a, b, t0, span, ks) if len(a) else np.zeros(len(ks), complex)
        out.append(v / (2.0 * np.pi))
    return np.array(out)
