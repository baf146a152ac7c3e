"""Shared helpers for the GPU parity tests: upload seeded events, run the
library through its C ABI, and measure errors against the CPU oracle."""
import numpy as np


def to_dev(ev, dev="cuda"):
    import torch
    return (torch.from_numpy(ev.offsets).to(dev), torch.from_numpy(ev.t).to(dev),
            torch.from_numpy(ev.logp).to(dev))


def rel_l2_rows(F_gpu, F_ref):
    """Eq. (15) per asset (rows with a zero reference are compared absolutely)."""
    F_gpu = np.asarray(F_gpu, dtype=np.complex128)
    out = []
    for a, b in zip(F_gpu, F_ref):
        nb = np.linalg.norm(b)
        out.append(np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a))
    return np.array(out)


def sigma_err(S_gpu, S_ref):
    """max_ij |dSigma_ij| / sqrt(Sigma_ii Sigma_jj) (reference diagonal)."""
    S_gpu = np.asarray(S_gpu, dtype=np.float64)
    d = np.sqrt(np.abs(np.diag(S_ref)))
    sc = np.outer(d, d)
    sc[sc == 0] = 1.0
    return float(np.max(np.abs(S_gpu - S_ref) / sc))


def run(plan_kw, ev, N, window=None, dev="cuda"):
    import paper_2003_02842_gb300 as mm
    plan = mm.mm_plan_create(D=ev.D, N_max=max(N, 1), max_events=ev.n_events, **plan_kw)
    off, t, p = to_dev(ev, dev)
    F, S, R, Nu = mm.mm_estimate(plan, off, t, p, N, window=window)
    st = mm.mm_plan_sync(plan)
    out = dict(F=F.cpu().numpy(), S=S.cpu().numpy(), R=R.cpu().numpy(), N=Nu, status=st,
               info=mm.mm_plan_get_info(plan))
    mm.mm_destroy(plan)
    return out
