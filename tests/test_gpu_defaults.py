"""The mixed path at the library's defaults (no product_bits): sampled
energies of every named workload within the mixed bar against the oracle,
per energy and per output kind; and the precision tuner's choice holding the
bar on the inputs it was tuned on."""
import numpy as np
import pytest

from gpu_parity import MIXED_TOL, band_rel_err, rel_err, to_dev
from oracle import rgf as O
from workloads import make_problem, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_2605_19910_gb300 as P
    return P


def _check(P, prob, idx, plan=None):
    import torch
    Hp, sL, sR, E = to_dev(prob, torch)
    nE = len(prob.energies)
    own = plan is None
    if own:
        plan = P.Plan(prob.sizes, 2 * prob.w + 1, nE, precision="mixed")
        assert P.negf_plan_product_bits(plan.handle) == P.NEGF_DEFAULT_PRODUCT_BITS
    Gb, G1 = plan.solve(Hp, sL, sR, E)
    assert not plan.info.cpu().numpy().any()
    if own:
        plan.close()
    for e in idx:
        ref = O.rgf_selected(O.system_blocks(prob, prob.energies[e]), prob.sizes, prob.w, first_row=True)
        assert band_rel_err(Gb[e].cpu().numpy(), ref["band"], prob.sizes, prob.w) < MIXED_TOL, e
        assert rel_err(G1[e].cpu().numpy(), ref["G1N"]) < MIXED_TOL, e


@pytest.mark.parametrize("name,idx", [("chain16x8", [0]), ("batched64x64", [0, 255, 511]),
                                      ("trans128x48", [0, 85, 170, 255]),
                                      ("penta256x32", [0, 256, 512, 768, 1023])])
def test_mixed_defaults_meet_the_bar(P, name, idx):
    _check(P, workload(name), idx)


def test_precision_tuner_keeps_a_width_that_meets_the_bar(P):
    import torch
    prob = make_problem(48, b=40, w=1, n_energies=96, eta=1e-6, seed=5)
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 3, 96, precision="mixed")
    bits, dev = plan.tune_precision(Hp, sL, sR, E, tol=1e-6)
    assert bits in P.TUNE_BITS + (56,)
    assert bits == P.negf_plan_product_bits(plan.handle)
    assert dev < 1e-6
    _check(P, prob, [0, 31, 47, 70, 95], plan=plan)
    plan.close()
