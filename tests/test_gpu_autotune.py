"""negf_autotune: the energy-group count it keeps is one of the timed
candidates, later calls use it, and the results stay those of the oracle."""
import pytest

from gpu_parity import FP64_TOL, MIXED_TOL, band_rel_err, to_dev
from oracle import rgf as O
from workloads import make_problem, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_2605_19910_gb300 as P
    return P


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("mixed", MIXED_TOL)])
def test_autotune_keeps_a_timed_candidate_and_results_hold(P, precision, tol):
    import torch
    prob = workload("batched64x64", n_blocks=16)
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 3, len(prob.energies), precision=precision)
    best, ms = plan.autotune(Hp, sL, sR, E)
    assert set(ms) == set(P.AUTOTUNE_GROUPS) and all(t > 0 for t in ms.values())
    # the fewest groups within 1 % of the fastest
    assert best in ms and ms[best] <= 1.01 * min(ms.values())
    assert all(ms[g] > 1.01 * min(ms.values()) for g in ms if g < best)
    assert P.negf_plan_groups(plan.handle) == best
    assert P.negf_plan_tile_cols(plan.handle) in ((512, 256) if precision == "mixed" else (512,))
    Gb, _ = plan.solve(Hp, sL, sR, E)
    plan.close()
    Gb = Gb.cpu().numpy()
    for e in (0, 200, 511):
        ref = O.rgf_selected(O.system_blocks(prob, prob.energies[e]), prob.sizes, 1)
        assert band_rel_err(Gb[e], ref["band"], prob.sizes, 1) < tol


def test_autotune_skips_counts_above_the_energies(P):
    import torch
    prob = make_problem(5, b=8, w=1, n_energies=3, eta=1e-3, seed=90)
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 3, 3)
    best, ms = plan.autotune(Hp, sL, sR, E)
    assert set(ms) == {1, 2, 3} and best in (1, 2, 3)
    plan.close()


def test_autotune_refuses_ddrgf_plans(P):
    import torch
    prob = make_problem(12, b=8, w=1, n_energies=2, eta=1e-3, seed=91, diag_shift=4.0)
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 3, 2, n_domains=2)
    with pytest.raises(P.NegfError) as ei:
        plan.autotune(Hp, sL, sR, E)
    assert ei.value.status == P.NEGF_ERR_UNSUPPORTED
    plan.close()


@pytest.mark.parametrize("cols", [256, 512])
def test_tile_widths_give_the_oracle_results(P, cols):
    """Both tensor-core N tiles negf_autotune chooses from (accumulators within
    256 or 512 TMEM columns), on blocks of 96..160 (several tiles, ragged
    last tiles) at the mixed defaults."""
    import torch
    prob = make_problem(10, b=None, size_range=(96, 160), w=1, n_energies=3, eta=1e-3, seed=95)
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 3, 3, precision="mixed")
    assert P.negf_plan_set_tile_cols(plan.handle, cols) == 0
    assert P.negf_plan_tile_cols(plan.handle) == cols
    assert P.negf_plan_set_tile_cols(plan.handle, 300) == P.NEGF_ERR_ARG
    Gb, _ = plan.solve(Hp, sL, sR, E)
    plan.close()
    Gb = Gb.cpu().numpy()
    for e in range(3):
        ref = O.rgf_selected(O.system_blocks(prob, prob.energies[e]), prob.sizes, 1)
        assert band_rel_err(Gb[e], ref["band"], prob.sizes, 1) < MIXED_TOL
