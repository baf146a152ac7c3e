"""CUDA graph replay of mm_estimate: a plan with graphs on gives, call after
call, the results of a plan with graphs off (both accumulators of the
contraction, inputs whose contents change under the same pointers, new output
pointers), and both match the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2003_02842_gb300 import synth

from gpu_helpers import sigma_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("prec,D", [("bf16x3", 12), ("bf16x3", 40), ("3xtf32", 12), ("fp64", 12)])
def test_graph_replay_matches_eager(prec, D):
    import torch
    import paper_2003_02842_gb300 as mm
    ev = synth.random_events(31, D=D, n_range=(100, 800), T=20000.0)
    N = 400
    tol = 1e-12 if prec == "fp64" else 1e-6
    plans = {g: mm.mm_plan_create(D=D, N_max=N, max_events=ev.n_events, tol=tol, kernel="es", prec=prec)
             for g in (True, False)}
    mm.mm_plan_set_graphs(plans[False], False)
    off, t, p = to_dev(ev)
    p0 = p.clone()
    rng = np.random.default_rng(5)
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    rdt = torch.float64 if prec == "fp64" else torch.float32
    outs = {g: [torch.empty((D, N + 1), dtype=cdt, device="cuda"), torch.empty((D, D), dtype=rdt, device="cuda"),
                torch.empty((D, D), dtype=rdt, device="cuda")] for g in (True, False)}
    # the same kernels on the same inputs; the mixed contraction's split-K
    # float atomics may add in another order
    lim = 1e-12 if prec == "fp64" else 1e-5
    for call in range(8):
        # new returns under the same pointer (the log-prices of every second
        # call get a random walk added)
        if call % 2:
            p.copy_(p0 + torch.from_numpy(np.cumsum(rng.normal(0, 1e-3, size=p0.numel()))).to(p0))
        else:
            p.copy_(p0)
        if call == 5:
            # new output buffers: the graph is captured again
            outs[True] = [torch.empty_like(x) for x in outs[True]]
        res = {}
        for g in (True, False):
            F, S, R = outs[g]
            mm.mm_estimate(plans[g], off, t, p, N, coeffs=F, sigma=S, R=R)
            assert mm.mm_plan_sync(plans[g]) == 0
            res[g] = [x.cpu().numpy().astype(np.complex128 if x.is_complex() else np.float64) for x in (F, S, R)]
        for a, b in zip(res[True], res[False]):
            assert np.max(np.abs(a - b)) <= lim * np.max(np.abs(b)) + 1e-300, call
        if call in (0, 3):
            ref = oracle.estimate(ev.offsets, ev.t, p.cpu().numpy(), N=N, basis="dirichlet")
            assert sigma_err(res[True][1], ref["Sigma"]) <= (1e-9 if prec == "fp64" else 1e-4)
            assert np.max(np.abs(res[True][2] - ref["R"])) <= (1e-9 if prec == "fp64" else 1e-4)
    info = mm.mm_plan_get_info(plans[True])
    assert info["graphs"] == 1 and info["graph_launches"] >= 5, info
    assert mm.mm_plan_get_info(plans[False])["graph_launches"] == 0
    for pl in plans.values():
        mm.mm_destroy(pl)


def test_no_graph_while_profiling():
    import torch
    import paper_2003_02842_gb300 as mm
    ev = synth.c2_async(2)
    N = ev.meta["N"]
    plan = mm.mm_plan_create(D=ev.D, N_max=N, max_events=ev.n_events, tol=1e-6, kernel="es", prec="bf16x3")
    off, t, p = to_dev(ev)
    F = torch.empty((ev.D, N + 1), dtype=torch.complex64, device="cuda")
    S = torch.empty((ev.D, ev.D), dtype=torch.float32, device="cuda")
    R = torch.empty_like(S)
    mm.mm_profile_enable(plan, True)
    for _ in range(3):
        mm.mm_estimate(plan, off, t, p, N, coeffs=F, sigma=S, R=R)
    torch.cuda.synchronize()
    assert mm.mm_plan_get_info(plan)["graph_launches"] == 0
    prof = mm.mm_profile_read(plan, reset=True)
    assert prof["spread"][1] == 3
    mm.mm_profile_enable(plan, False)
    for _ in range(3):
        mm.mm_estimate(plan, off, t, p, N, coeffs=F, sigma=S, R=R)
    assert mm.mm_plan_sync(plan) == 0
    assert mm.mm_plan_get_info(plan)["graph_launches"] == 3
    ref = oracle.estimate(ev.offsets, ev.t, ev.logp, N=N, basis="dirichlet")
    assert np.max(np.abs(R.cpu().numpy() - ref["R"])) <= 1e-4
    mm.mm_destroy(plan)
