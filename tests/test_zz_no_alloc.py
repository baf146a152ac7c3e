"""mm_corr_noalloc: the contraction for callers that cannot allocate device
memory (its scratch is a fixed file-scope device array inside the library).

Checked through the C ABI against the plan-based mm_corr on the same
coefficients, twice in a row (the shared scratch keeps the previous call's
contents, which must not leak into the next result). This file is collected
last on purpose and also passes when run alone in a fresh process."""
import numpy as np
import pytest

from paper_2003_02842_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "bf16x3": 1e-4, "3xtf32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32", "fp64"])
@pytest.mark.parametrize("basis", ["dirichlet", "fejer"])
def test_noalloc_matches_plan_path_twice(prec, basis):
    import torch
    import paper_2003_02842_gb300 as mm
    from gpu_helpers import to_dev
    ev = synth.random_events(61, D=100, n_range=(50, 400), T=5000.0)
    N = 700
    plan = mm.mm_plan_create(D=ev.D, N_max=N, max_events=ev.n_events,
                             tol=1e-12 if prec == "fp64" else 1e-6, kernel="es", basis=basis, prec=prec)
    off, t, p = to_dev(ev)
    F, Nu = mm.mm_coeffs(plan, off, t, p, N)
    S_ref, R_ref = mm.mm_corr(plan, F, N)
    assert mm.mm_plan_sync(plan) == 0
    S_ref = S_ref.double().cpu().numpy()
    R_ref = R_ref.double().cpu().numpy()
    scale = np.sqrt(np.outer(np.diag(S_ref), np.diag(S_ref)))
    for _ in range(2):
        st, S, R = mm.mm_corr_noalloc(F, N, basis=basis, prec=prec)
        assert st == 0
        S = S.double().cpu().numpy()
        R = R.double().cpu().numpy()
        assert np.max(np.abs(S - S_ref) / scale) <= TOL[prec]
        assert np.max(np.abs(R - R_ref)) <= TOL[prec]
        assert np.all(np.diag(R) == 1.0)
    mm.mm_destroy(plan)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_2003_02842_gb300 as mm
    F = torch.zeros((129, 11), dtype=torch.complex64, device="cuda")
    st, _, _ = mm.mm_corr_noalloc(F, 10)
    assert st == 11  # MM_ERR_UNSUPPORTED
    F = torch.zeros((4, 65537), dtype=torch.complex64, device="cuda")
    st, _, _ = mm.mm_corr_noalloc(F, 65536)
    assert st == 11
