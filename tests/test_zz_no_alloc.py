"""mm_corr_noalloc: the contraction for callers that cannot allocate device
memory (its scratch is a fixed file-scope device array inside the library).

Checked through the C ABI against the plan-based mm_corr on the same
coefficients, twice in a row (the shared scratch keeps the previous call's
contents, which must not leak into the next result), at the sizes where the
fixed scratch is exactly full (D = 128 in FP64: 3 tile pairs x 16 splits of
partial tiles; N = 65535 weights), at D not a multiple of 4 (the mixed
accumulator's padded rows) and D = 1, and after a larger call. This file is
collected last on purpose and also passes when run alone in a fresh
process."""
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


def _plan_reference(F, N, basis, prec):
    import paper_2003_02842_gb300 as mm
    D = int(F.shape[0])
    plan = mm.mm_plan_create(D=D, N_max=max(N, 1), max_events=0, tol=1e-12 if prec == "fp64" else 1e-6,
                             kernel="es", basis=basis, prec=prec)
    S, R = mm.mm_corr(plan, F, N)
    assert mm.mm_plan_sync(plan) == 0
    out = S.double().cpu().numpy(), R.double().cpu().numpy()
    mm.mm_destroy(plan)
    return out


def _coefficients(seed, D, N, prec):
    import torch
    F = torch.from_numpy(synth.gram_coefficients(seed, D, N)).cuda()
    return F.to(torch.complex128) if prec == "fp64" else F


def _check(F, N, basis, prec):
    import paper_2003_02842_gb300 as mm
    S_ref, R_ref = _plan_reference(F, N, basis, prec)
    scale = np.sqrt(np.outer(np.diag(S_ref), np.diag(S_ref)))
    st, S, R = mm.mm_corr_noalloc(F, N, basis=basis, prec=prec)
    assert st == 0
    S = S.double().cpu().numpy()
    R = R.double().cpu().numpy()
    assert np.max(np.abs(S - S_ref) / scale) <= TOL[prec]
    assert np.max(np.abs(R - R_ref)) <= TOL[prec]
    assert np.all(np.diag(R) == 1.0)


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32", "fp64"])
@pytest.mark.parametrize("D", [1, 7, 128])
def test_noalloc_edge_sizes_twice(prec, D):
    F = _coefficients(5, D, 700, prec)
    for _ in range(2):
        _check(F, 700, "fejer", prec)


@pytest.mark.parametrize("prec", ["bf16x3", "fp64"])
def test_noalloc_largest_cutoff(prec):
    F = _coefficients(6, 4, 65535, prec)
    _check(F, 65535, "dirichlet", prec)


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32", "fp64"])
def test_noalloc_smaller_call_after_a_larger_one(prec):
    big = _coefficients(7, 128, 900, prec)
    small = _coefficients(8, 7, 300, prec)
    _check(big, 900, "dirichlet", prec)
    _check(small, 300, "dirichlet", prec)
    _check(big, 900, "fejer", prec)


def test_noalloc_refuses_a_capturing_stream():
    import torch
    import paper_2003_02842_gb300 as mm
    F = _coefficients(9, 8, 50, "bf16x3")
    mm.mm_corr_noalloc(F, 50)  # the first call on the device looks up the scratch
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        st, _, _ = mm.mm_corr_noalloc(F, 50, stream=s)
        g.capture_end()
    assert st == 1  # MM_ERR_INVALID_ARG: nothing was launched into the capture
    _check(F, 50, "dirichlet", "bf16x3")
