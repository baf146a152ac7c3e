"""Failure detection without a GPU fault: the tensor-core contraction's
device-side waits are bounded. With the plan's wait limit set to 0 every
wait is a single non-blocking test, so the contraction gives up at its
drain (its MMAs cannot have finished the instant they are issued), lets the
MMAs it issued finish, frees its tensor memory and reports MM_ERR_TIMEOUT
through the plan's status word. The next calls on the same plan, with the
default limit, are correct: nothing is left allocated or half-written.
Nothing here faults, traps or spins without a bound."""
import numpy as np
import pytest

import oracle
from paper_2003_02842_gb300 import synth

from gpu_helpers import sigma_err, to_dev

pytestmark = pytest.mark.gpu

MM_ERR_TIMEOUT = 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("gram", ["convert", "tma"])
@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32"])
@pytest.mark.parametrize("D", [20, 100, 200])
def test_contraction_wait_gives_up_and_the_plan_recovers(prec, D, gram):
    # D = 20: the contraction's last CTA writes Sigma and R itself (the
    # in-register variant); D = 100: one output tile and the separate
    # epilogue; D = 200: several tiles. Both contraction variants: the
    # in-register one and the warp-specialised one fed by TMA (whose producer
    # and MMA threads both give up and wait for their copies and MMAs)
    import paper_2003_02842_gb300 as mm
    ev = synth.random_events(70 + D, D=D, n_range=(30, 300), T=6000.0)
    N = 400
    plan = mm.mm_plan_create(D=D, N_max=N, max_events=ev.n_events, tol=1e-6, kernel="es", basis="fejer", prec=prec,
                             gram_algo=gram)
    off, t, p = to_dev(ev)
    F, _ = mm.mm_coeffs(plan, off, t, p, N)
    assert mm.mm_plan_sync(plan) == 0
    ref = oracle.estimate(ev.offsets, ev.t, ev.logp, N=N, basis="fejer")
    for rounds in range(2):
        mm.mm_plan_set_wait_limit(plan, 0)
        mm.mm_corr(plan, F, N)
        assert mm.mm_plan_sync(plan) == MM_ERR_TIMEOUT
        assert mm.mm_plan_sync(plan) == 0  # the status word was cleared
        mm.mm_plan_set_wait_limit(plan, -1)
        for _ in range(2):  # both accumulators the calls alternate between
            S, R = mm.mm_corr(plan, F, N)
            assert mm.mm_plan_sync(plan) == 0
            assert sigma_err(S.cpu().numpy().astype(np.float64), ref["Sigma"]) <= 1e-4
            assert np.max(np.abs(R.cpu().numpy().astype(np.float64) - ref["R"])) <= 1e-4
    mm.mm_destroy(plan)


def test_timeout_through_the_graph_replayed_estimate():
    # steady mm_estimate calls replay a captured graph; a new limit is
    # re-captured, and the default afterwards gives the correct result
    import paper_2003_02842_gb300 as mm
    ev = synth.random_events(91, D=64, n_range=(30, 300), T=6000.0)
    N = 300
    plan = mm.mm_plan_create(D=64, N_max=N, max_events=ev.n_events, tol=1e-6, kernel="es", prec="bf16x3")
    off, t, p = to_dev(ev)
    for _ in range(3):
        mm.mm_estimate(plan, off, t, p, N)
    assert mm.mm_plan_sync(plan) == 0
    g0 = mm.mm_plan_get_info(plan)["graph_launches"]
    mm.mm_plan_set_wait_limit(plan, 0)
    for _ in range(2):
        mm.mm_estimate(plan, off, t, p, N)
        assert mm.mm_plan_sync(plan) == MM_ERR_TIMEOUT
    mm.mm_plan_set_wait_limit(plan, -1)
    for _ in range(3):
        F, S, R, _ = mm.mm_estimate(plan, off, t, p, N)
    assert mm.mm_plan_sync(plan) == 0
    assert mm.mm_plan_get_info(plan)["graph_launches"] > g0
    ref = oracle.estimate(ev.offsets, ev.t, ev.logp, N=N)
    assert np.max(np.abs(R.cpu().numpy().astype(np.float64) - ref["R"])) <= 1e-4
    mm.mm_destroy(plan)
