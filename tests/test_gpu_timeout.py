"""The bounded wait of the tensor-core product (failure detection without a
GPU fault): with the wait's bound set to zero polls every product gives up
at once, drains the MMAs it issued, frees its tensor memory and records the
timeout, which negf_sync reports; the same plan then solves normally."""
import numpy as np
import pytest

from gpu_parity import MIXED_TOL, band_rel_err, rel_err, to_dev
from oracle import rgf as O
from workloads import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_2605_19910_gb300 as P
    return P


def test_wait_that_runs_out_is_reported_and_the_plan_recovers(P):
    import torch
    prob = make_problem(8, b=32, w=1, n_energies=4, eta=1e-3, seed=91)
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 3, 4, precision="mixed")
    assert P.negf_plan_set_wait_limit(plan.handle, 0) == P.NEGF_OK
    with pytest.raises(P.NegfError) as ei:
        plan.solve(Hp, sL, sR, E)
    assert ei.value.status == P.NEGF_ERR_TIMEOUT
    assert P.negf_sync(plan.handle) == P.NEGF_OK          # the error word was cleared
    assert P.negf_plan_set_wait_limit(plan.handle, -1) == P.NEGF_OK
    Gb, G1 = plan.solve(Hp, sL, sR, E)                    # same plan, default bound
    Gb, G1 = Gb.cpu().numpy(), G1.cpu().numpy()
    plan.close()
    for e in range(4):
        ref = O.rgf_selected(O.system_blocks(prob, prob.energies[e]), prob.sizes, 1, first_row=True)
        assert band_rel_err(Gb[e], ref["band"], prob.sizes, 1) < MIXED_TOL
        assert rel_err(G1[e], ref["G1N"]) < MIXED_TOL
    assert P.negf_plan_set_wait_limit(None, 0) == P.NEGF_ERR_ARG
