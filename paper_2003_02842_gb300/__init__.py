"""GB300-native Malliavin-Mancino Fourier covariance estimator via type-1 NUFFTs.

Thin Python binding over the C ABI of ``include/mm.h`` (library
``lib/libmm_gb300.so``). The functions below carry the C names and only
marshal arguments: torch tensors give device (or pinned host) pointers and
the current CUDA stream; every step of the computation runs in the library's
CUDA kernels. There is no CPU fallback.

    plan = mm_plan_create(D=100, N_max=10000, max_events=2_000_000, tol=1e-6,
                          kernel="es", basis="dirichlet", prec="bf16x3")
    F, N = mm_coeffs(plan, offsets, t, logp, N=10000)   # D x (N+1) complex
    Sigma, R = mm_corr(plan, F, N)
    mm_destroy(plan)
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import BASES, KERNELS, PRECISIONS, STAGES, STATUS_NAMES

__all__ = [
    "MMError", "Plan", "mm_plan_create", "mm_destroy", "mm_coeffs", "mm_cov", "mm_corr", "mm_estimate",
    "mm_estimate_host", "mm_nyquist", "mm_plan_sync", "mm_plan_get_info", "mm_profile_enable", "mm_plan_set_graphs", "mm_plan_set_wait_limit",
    "mm_corr_pairwise",
    "mm_profile_read", "mm_status_string", "mm_version", "mm_corr_noalloc", "mm_autotune", "KERNELS", "BASES", "PRECISIONS", "STAGES",
    "Batch", "mm_batch_create", "mm_batch_destroy", "mm_batch_epps", "mm_batch_autotune", "mm_batch_coeffs",
    "mm_batch_sync", "mm_batch_get_info", "mm_batch_profile_enable", "mm_batch_profile_read",
    "Server", "mm_server_create", "mm_server_load", "mm_server_submit", "mm_server_poll", "mm_server_get_stats",
    "mm_server_destroy",
]


class MMError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        self.name = STATUS_NAMES.get(self.status, str(status))
        super().__init__(f"{where}: {self.name} ({mm_status_string(self.status)})")


def _check(st, where):
    if st != 0:
        raise MMError(st, where)


def mm_status_string(status: int) -> str:
    return _lib.load().mm_status_string(int(status)).decode()


def mm_version() -> int:
    return int(_lib.load().mm_version())


class Plan:
    """Owns an mm_plan handle plus the description it was created from."""

    def __init__(self, handle, desc: dict):
        self.handle = handle
        self.desc = desc

    @property
    def fp64(self) -> bool:
        return self.desc["prec"] == "fp64"

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                _lib.load().mm_destroy(h)
            except Exception:
                pass
            self.handle = None


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(x, dtype, name, device=True):
    torch = _torch()
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if x.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {x.dtype}")
    if device and not x.is_cuda:
        raise ValueError(f"{name} must live on the GPU")
    if not device and x.is_cuda:
        raise ValueError(f"{name} must live in host memory")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(x.data_ptr())


def mm_plan_create(D, N_max, max_events=0, tol=1e-6, kernel="es", basis="dirichlet", prec="bf16x3",
                   spread_tile=0, spread_algo="default", fft_algo="default", gram_algo="default") -> Plan:
    d = _lib.PlanDesc()
    d.D, d.N_max, d.max_events, d.tol = int(D), int(N_max), int(max_events), float(tol)
    d.kernel, d.basis, d.prec = KERNELS[kernel], BASES[basis], PRECISIONS[prec]
    d.spread_tile = int(spread_tile)
    d.spread_algo = _lib.SPREAD_ALGOS[spread_algo]
    d.fft_algo = _lib.FFT_ALGOS[fft_algo]
    d.gram_algo = _lib.GRAM_ALGOS[gram_algo]
    h = ctypes.c_void_p()
    _check(_lib.load().mm_plan_create(ctypes.byref(d), ctypes.byref(h)), "mm_plan_create")
    return Plan(h, dict(D=int(D), N_max=int(N_max), max_events=int(max_events), tol=float(tol), kernel=kernel,
                        basis=basis, prec=prec, spread_tile=int(spread_tile), spread_algo=spread_algo,
                        fft_algo=fft_algo, gram_algo=gram_algo))


def mm_destroy(plan: Plan):
    if plan.handle:
        _check(_lib.load().mm_destroy(plan.handle), "mm_destroy")
        plan.handle = None


def _coef_dtype(plan):
    torch = _torch()
    return torch.complex128 if plan.fp64 else torch.complex64


def _real_dtype(plan):
    torch = _torch()
    return torch.float64 if plan.fp64 else torch.float32


def _events(offsets, t, logp):
    torch = _torch()
    return (_dptr(offsets, torch.int64, "offsets"), _dptr(t, torch.float64, "t"),
            _dptr(logp, torch.float64, "logp"))


def _alloc_coeffs(plan, N, device):
    return _torch().empty((plan.desc["D"], N + 1), dtype=_coef_dtype(plan), device=device)


def mm_nyquist(plan, offsets, t, window=None, stream=None) -> int:
    torch = _torch()
    t0, t1 = window if window is not None else (0.0, 0.0)
    N = ctypes.c_int32()
    _check(_lib.load().mm_nyquist(plan.handle, _dptr(offsets, torch.int64, "offsets"),
                                  _dptr(t, torch.float64, "t"), float(t0), float(t1), ctypes.byref(N),
                                  _stream(stream)), "mm_nyquist")
    return int(N.value)


def mm_coeffs(plan, offsets, t, logp, N=0, window=None, out=None, stream=None):
    """F(dp_i)(k), k = 0..N, as a D x (N+1) complex tensor; N <= 0 uses the
    Nyquist cutoff (and synchronises). Returns (coeffs, N_used)."""
    if N <= 0:
        N = mm_nyquist(plan, offsets, t, window, stream)
    if out is None:
        out = _alloc_coeffs(plan, N, t.device)
    t0, t1 = window if window is not None else (0.0, 0.0)
    Nu = ctypes.c_int32()
    po, pt, pp = _events(offsets, t, logp)
    _check(_lib.load().mm_coeffs(plan.handle, po, pt, pp, int(N), float(t0), float(t1),
                                 _dptr(out, _coef_dtype(plan), "out"), ctypes.byref(Nu), _stream(stream)),
           "mm_coeffs")
    return out, int(Nu.value)


def mm_cov(plan, coeffs, N, out=None, stream=None):
    torch = _torch()
    D = plan.desc["D"]
    if out is None:
        out = torch.empty((D, D), dtype=_real_dtype(plan), device=coeffs.device)
    _check(_lib.load().mm_cov(plan.handle, _dptr(coeffs, _coef_dtype(plan), "coeffs"), int(N),
                              _dptr(out, _real_dtype(plan), "sigma"), _stream(stream)), "mm_cov")
    return out


def mm_corr(plan, coeffs, N, sigma=True, R=None, stream=None):
    """Returns (Sigma or None, R)."""
    torch = _torch()
    D = plan.desc["D"]
    dt = _real_dtype(plan)
    if R is None:
        R = torch.empty((D, D), dtype=dt, device=coeffs.device)
    S = None
    if sigma is True:
        S = torch.empty((D, D), dtype=dt, device=coeffs.device)
    elif sigma is not None and sigma is not False:
        S = sigma
    ps = _dptr(S, dt, "sigma") if S is not None else ctypes.c_void_p(0)
    _check(_lib.load().mm_corr(plan.handle, _dptr(coeffs, _coef_dtype(plan), "coeffs"), int(N), ps,
                               _dptr(R, dt, "R"), _stream(stream)), "mm_corr")
    return S, R


def mm_corr_pairwise(plan, coeffs, N_coeffs, N_per_asset, psd_repair=False, sigma=True, R=None, stream=None):
    """Sigma and R with a cutoff per pair of assets, N_ij = min(N_i, N_j)
    (Sec. 3.1), from coefficients computed at N_coeffs; psd_repair replaces
    Sigma by the nearest positive semi-definite matrix (Frobenius norm)
    before R is formed. Returns (Sigma or None, R, clipped), clipped a device
    int32 tensor holding the number of negative eigenvalues removed."""
    torch = _torch()
    D = plan.desc["D"]
    dt = _real_dtype(plan)
    if R is None:
        R = torch.empty((D, D), dtype=dt, device=coeffs.device)
    S = None
    if sigma is True:
        S = torch.empty((D, D), dtype=dt, device=coeffs.device)
    elif sigma is not None and sigma is not False:
        S = sigma
    Ns = [int(x) for x in N_per_asset]
    if len(Ns) != D:
        raise ValueError(f"mm_corr_pairwise: {len(Ns)} cutoffs for {D} assets")
    hN = (ctypes.c_int32 * D)(*Ns)
    clipped = torch.zeros(1, dtype=torch.int32, device=coeffs.device)
    ps = _dptr(S, dt, "sigma") if S is not None else ctypes.c_void_p(0)
    _check(_lib.load().mm_corr_pairwise(plan.handle, _dptr(coeffs, _coef_dtype(plan), "coeffs"), int(N_coeffs), hN,
                                        1 if psd_repair else 0, ps, _dptr(R, dt, "R"),
                                        ctypes.c_void_p(clipped.data_ptr()), _stream(stream)), "mm_corr_pairwise")
    return S, R, clipped


def mm_corr_noalloc(coeffs, N, basis="dirichlet", prec="bf16x3", sigma=True, R=None, stream=None):
    """Sigma and R from coefficients without a plan and without any device
    allocation inside the library (its scratch is a fixed device array; see
    include/mm.h). Synchronises the stream; returns (status, Sigma or None, R).
    Only D <= 128 and N <= 65535 are accepted."""
    torch = _torch()
    D = int(coeffs.shape[0])
    fp64 = prec == "fp64"
    cdt = torch.complex128 if fp64 else torch.complex64
    dt = torch.float64 if fp64 else torch.float32
    if R is None:
        R = torch.empty((D, D), dtype=dt, device=coeffs.device)
    if sigma is True:
        S = torch.empty((D, D), dtype=dt, device=coeffs.device)
    elif sigma is None or sigma is False:
        S = None
    else:
        S = sigma
    ps = _dptr(S, dt, "sigma") if S is not None else ctypes.c_void_p(0)
    st = _lib.load().mm_corr_noalloc(D, int(N), BASES[basis], PRECISIONS[prec], _dptr(coeffs, cdt, "coeffs"),
                                     ps, _dptr(R, dt, "R"), _stream(stream))
    return int(st), S, R


def mm_estimate(plan, offsets, t, logp, N, window=None, coeffs=None, sigma=True, R=None, stream=None):
    """Algorithm 3 on device tensors: returns (coeffs, Sigma or None, R, N_used).
    N must be positive here (use mm_nyquist first for the Nyquist cutoff)."""
    torch = _torch()
    if N <= 0:
        N = mm_nyquist(plan, offsets, t, window, stream)
    D = plan.desc["D"]
    dt = _real_dtype(plan)
    if coeffs is None:
        coeffs = _alloc_coeffs(plan, N, t.device)
    if R is None:
        R = torch.empty((D, D), dtype=dt, device=t.device)
    if sigma is True:
        S = torch.empty((D, D), dtype=dt, device=t.device)
    elif sigma is None or sigma is False:
        S = None
    else:
        S = sigma
    ps = _dptr(S, dt, "sigma") if S is not None else ctypes.c_void_p(0)
    t0, t1 = window if window is not None else (0.0, 0.0)
    Nu = ctypes.c_int32()
    po, pt, pp = _events(offsets, t, logp)
    _check(_lib.load().mm_estimate(plan.handle, po, pt, pp, int(N), float(t0), float(t1),
                                   _dptr(coeffs, _coef_dtype(plan), "coeffs"), ps, _dptr(R, dt, "R"),
                                   ctypes.byref(Nu), _stream(stream)), "mm_estimate")
    return coeffs, S, R, int(Nu.value)


def mm_estimate_host(plan, offsets, t, logp, N, window=None, coeffs=None, sigma=None, R=None, stream=None,
                     allow_status=()):
    """Algorithm 3 from host tensors (pinned memory for asynchronous copies);
    the library copies in and out and synchronises. Returns the status."""
    torch = _torch()
    dt = _real_dtype(plan)
    pc = _dptr(coeffs, _coef_dtype(plan), "coeffs", device=False) if coeffs is not None else ctypes.c_void_p(0)
    ps = _dptr(sigma, dt, "sigma", device=False) if sigma is not None else ctypes.c_void_p(0)
    t0, t1 = window if window is not None else (0.0, 0.0)
    Nu = ctypes.c_int32()
    st = _lib.load().mm_estimate_host(plan.handle, _dptr(offsets, torch.int64, "offsets", device=False),
                                      _dptr(t, torch.float64, "t", device=False),
                                      _dptr(logp, torch.float64, "logp", device=False), int(N), float(t0),
                                      float(t1), pc, ps, _dptr(R, dt, "R", device=False), ctypes.byref(Nu),
                                      _stream(stream))
    if st != 0 and st not in allow_status:
        raise MMError(st, "mm_estimate_host")
    return st, int(Nu.value)


def mm_autotune(plan, offsets, t, logp, N, window=None, coeffs=None, reps=5, stream=None) -> dict:
    """Time every candidate configuration of stages (a)-(c) on this data and
    keep the fastest in the plan; returns mm_plan_get_info afterwards."""
    if coeffs is None:
        coeffs = _alloc_coeffs(plan, N, t.device)
    t0, t1 = window if window is not None else (0.0, 0.0)
    po, pt, pp = _events(offsets, t, logp)
    _check(_lib.load().mm_autotune(plan.handle, po, pt, pp, int(N), float(t0), float(t1),
                                   _dptr(coeffs, _coef_dtype(plan), "coeffs"), int(reps), _stream(stream)),
           "mm_autotune")
    return mm_plan_get_info(plan)


def mm_plan_sync(plan) -> int:
    """Wait for the plan's work; returns (and clears) the device status code."""
    return int(_lib.load().mm_plan_sync(plan.handle))


def mm_plan_get_info(plan) -> dict:
    info = _lib.PlanInfo()
    _check(_lib.load().mm_plan_get_info(plan.handle, ctypes.byref(info)), "mm_plan_get_info")
    out = {k: getattr(info, k) for k, _ in _lib.PlanInfo._fields_ if k != "reserved"}
    out["fft_radix"] = list(out["fft_radix"])[: out["fft_passes"]]
    return out


def mm_profile_enable(plan, on=True):
    _check(_lib.load().mm_profile_enable(plan.handle, 1 if on else 0), "mm_profile_enable")


def mm_plan_set_graphs(plan, on=True):
    """CUDA graph replay of steady mm_estimate calls (on by default)."""
    _check(_lib.load().mm_plan_set_graphs(plan.handle, 1 if on else 0), "mm_plan_set_graphs")


def mm_plan_set_wait_limit(plan, ns=-1):
    """Limit of the contraction's device-side waits in ns (0: one
    non-blocking test; < 0: the 1 s default); a diagnostic of the
    bounded-wait path."""
    _check(_lib.load().mm_plan_set_wait_limit(plan.handle, int(ns)), "mm_plan_set_wait_limit")


def mm_profile_read(plan, reset=False) -> dict:
    ms = (ctypes.c_double * len(STAGES))()
    nl = (ctypes.c_int64 * len(STAGES))()
    _check(_lib.load().mm_profile_read(plan.handle, ms, nl, 1 if reset else 0), "mm_profile_read")
    return {s: (ms[i], nl[i]) for i, s in enumerate(STAGES)}


# --------------------------------------------------------------------------
# Batched form: replications x cutoff sweep (see include/mm.h)
# --------------------------------------------------------------------------
class Batch:
    """Owns an mm_batch handle plus the description it was created from."""

    def __init__(self, handle, desc: dict):
        self.handle = handle
        self.desc = desc

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                _lib.load().mm_batch_destroy(h)
            except Exception:
                pass
            self.handle = None


def mm_batch_create(reps, D, N_max, max_events, tol=1e-6, kernel="es", basis="dirichlet", prec="bf16x3",
                    spread_algo="default") -> Batch:
    d = _lib.BatchDesc()
    d.reps, d.D, d.N_max, d.max_events, d.tol = int(reps), int(D), int(N_max), int(max_events), float(tol)
    d.kernel, d.basis, d.prec = KERNELS[kernel], BASES[basis], PRECISIONS[prec]
    d.spread_algo = _lib.SPREAD_ALGOS[spread_algo]
    h = ctypes.c_void_p()
    _check(_lib.load().mm_batch_create(ctypes.byref(d), ctypes.byref(h)), "mm_batch_create")
    return Batch(h, dict(reps=int(reps), D=int(D), N_max=int(N_max), max_events=int(max_events), tol=float(tol),
                         kernel=kernel, basis=basis, prec=prec, spread_algo=spread_algo))


def mm_batch_destroy(batch: Batch):
    if batch.handle:
        _check(_lib.load().mm_batch_destroy(batch.handle), "mm_batch_destroy")
        batch.handle = None


def mm_batch_epps(batch, offsets, t, logp, cutoffs, sigma=True, R=None, stream=None):
    """Covariance / correlation of every problem at every cutoff (ascending).
    Returns (Sigma or None, R), each [reps, len(cutoffs), D, D] float32
    (float64 for an FP64 batch)."""
    torch = _torch()
    reps, D = batch.desc["reps"], batch.desc["D"]
    J = len(cutoffs)
    cut = (ctypes.c_int32 * J)(*[int(x) for x in cutoffs])
    dev = t.device
    dt = torch.float64 if batch.desc["prec"] == "fp64" else torch.float32
    if R is None:
        R = torch.empty((reps, J, D, D), dtype=dt, device=dev)
    if sigma is True:
        S = torch.empty((reps, J, D, D), dtype=dt, device=dev)
    elif sigma is None or sigma is False:
        S = None
    else:
        S = sigma
    ps = _dptr(S, dt, "sigma") if S is not None else ctypes.c_void_p(0)
    po, pt, pp = _events(offsets, t, logp)
    _check(_lib.load().mm_batch_epps(batch.handle, po, pt, pp, cut, J, ps, _dptr(R, dt, "R"),
                                     _stream(stream)), "mm_batch_epps")
    return S, R


def mm_batch_autotune(batch, offsets, t, logp, N, reps=3, stream=None) -> dict:
    po, pt, pp = _events(offsets, t, logp)
    _check(_lib.load().mm_batch_autotune(batch.handle, po, pt, pp, int(N), int(reps), _stream(stream)),
           "mm_batch_autotune")
    return mm_batch_get_info(batch)


def mm_batch_coeffs(batch, stream=None):
    """Copy of the last sweep's coefficients: complex64 (complex128 for an
    FP64 batch) [reps * D, N_J + 1]."""
    torch = _torch()
    ptr, ld = ctypes.c_void_p(), ctypes.c_int32()
    _check(_lib.load().mm_batch_coeffs(batch.handle, ctypes.byref(ptr), ctypes.byref(ld)), "mm_batch_coeffs")
    cdt = torch.complex128 if batch.desc["prec"] == "fp64" else torch.complex64
    out = torch.empty((batch.desc["reps"] * batch.desc["D"], ld.value), dtype=cdt, device="cuda")
    _check(_lib.load().mm_batch_copy_coeffs(batch.handle, ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "mm_batch_copy_coeffs")
    return out


def mm_batch_sync(batch) -> int:
    return int(_lib.load().mm_batch_sync(batch.handle))


def mm_batch_get_info(batch) -> dict:
    info = _lib.BatchInfo()
    _check(_lib.load().mm_batch_get_info(batch.handle, ctypes.byref(info)), "mm_batch_get_info")
    return {k: getattr(info, k) for k, _ in _lib.BatchInfo._fields_}


def mm_batch_profile_enable(batch, on=True):
    _check(_lib.load().mm_batch_profile_enable(batch.handle, 1 if on else 0), "mm_batch_profile_enable")


def mm_batch_profile_read(batch, reset=False) -> dict:
    ms = (ctypes.c_double * len(STAGES))()
    nl = (ctypes.c_int64 * len(STAGES))()
    _check(_lib.load().mm_batch_profile_read(batch.handle, ms, nl, 1 if reset else 0), "mm_batch_profile_read")
    return {s: (ms[i], nl[i]) for i, s in enumerate(STAGES)}


# --------------------------------------------------------------------------
# Serving form: request loop over a resident event store (see include/mm.h)
# --------------------------------------------------------------------------
class Server:
    """Owns an mm_server handle and the host result buffers of requests in
    flight (kept alive until their completion is polled)."""

    def __init__(self, handle, desc: dict):
        self.handle = handle
        self.desc = desc
        self.pending = {}
        self._store = None

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                _lib.load().mm_server_destroy(h)
            except Exception:
                pass
            self.handle = None


def mm_server_create(D, N_max, max_events, request_max_events=0, hbm_budget=0, max_slots=4, tol=1e-6,
                     kernel="es", basis="fejer", prec="bf16x3", cache_rows=0) -> Server:
    """cache_rows > 0 keeps that many coefficient rows (one asset over one
    window at one cutoff each) resident across requests."""
    d = _lib.ServerDesc()
    d.D, d.N_max, d.max_events, d.request_max_events = int(D), int(N_max), int(max_events), int(request_max_events)
    d.hbm_budget, d.max_slots, d.tol = int(hbm_budget), int(max_slots), float(tol)
    d.cache_rows = int(cache_rows)
    d.kernel, d.basis, d.prec = KERNELS[kernel], BASES[basis], PRECISIONS[prec]
    h = ctypes.c_void_p()
    _check(_lib.load().mm_server_create(ctypes.byref(d), ctypes.byref(h)), "mm_server_create")
    return Server(h, dict(D=int(D), N_max=int(N_max), max_events=int(max_events), prec=prec, basis=basis,
                          kernel=kernel, tol=float(tol)))


def mm_server_load(server, offsets, t, logp):
    """Upload the resident store from host numpy arrays (CSR, sorted per asset)."""
    import numpy as np
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    tt = np.ascontiguousarray(t, dtype=np.float64)
    pp = np.ascontiguousarray(logp, dtype=np.float64)
    server._store = (off, tt, pp)
    _check(_lib.load().mm_server_load(server.handle, off.ctypes.data, tt.ctypes.data, pp.ctypes.data),
           "mm_server_load")


def mm_server_submit(server, t0, t1, assets, N=0, dt=0.0, sigma=False) -> int:
    """Queue a request; returns its ticket. N > 0: that cutoff; N = 0 with
    dt > 0: Eq. (19) for dt; N = 0, dt = 0: the window's Nyquist cutoff."""
    import numpy as np
    a = np.ascontiguousarray(assets, dtype=np.int32)
    n = len(a)
    dt_ = np.float64 if server.desc["prec"] == "fp64" else np.float32
    R = np.empty((n, n), dtype=dt_)
    S = np.empty((n, n), dtype=dt_) if sigma else None
    rq = _lib.Request()
    rq.t0, rq.t1, rq.n_assets, rq.N, rq.dt_equiv = float(t0), float(t1), n, int(N), float(dt)
    rq.assets = a.ctypes.data
    rq.h_R = R.ctypes.data
    rq.h_sigma_or_null = S.ctypes.data if S is not None else None
    tk = ctypes.c_int64()
    _check(_lib.load().mm_server_submit(server.handle, ctypes.byref(rq), ctypes.byref(tk)), "mm_server_submit")
    server.pending[tk.value] = (a, R, S)
    return tk.value


def mm_server_poll(server, max_items=256, wait=0.0) -> list:
    """Completed requests: dicts with ticket, status, N, n_assets, t_submit,
    t_start, t_done (seconds) and the result arrays R (and Sigma)."""
    buf = (_lib.Completion * int(max_items))()
    n = ctypes.c_int32()
    _check(_lib.load().mm_server_poll(server.handle, buf, int(max_items), ctypes.byref(n), float(wait)),
           "mm_server_poll")
    out = []
    for i in range(n.value):
        c = buf[i]
        _, R, S = server.pending.pop(c.ticket)
        out.append(dict(ticket=c.ticket, status=c.status, N=c.N, n_assets=c.n_assets, t_submit=c.t_submit,
                        t_start=c.t_start, t_done=c.t_done, R=R, Sigma=S))
    return out


def mm_server_get_stats(server) -> dict:
    st = _lib.ServerStats()
    _check(_lib.load().mm_server_get_stats(server.handle, ctypes.byref(st)), "mm_server_get_stats")
    return {k: getattr(st, k) for k, _ in _lib.ServerStats._fields_}


def mm_server_destroy(server):
    if server.handle:
        _check(_lib.load().mm_server_destroy(server.handle), "mm_server_destroy")
        server.handle = None

