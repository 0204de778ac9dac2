"""Parity of the mixed-precision CUDA path (tcgen05 block products from exact BF16 slices,
FP64 block inversions) with the FP64 oracle, through the C-ABI: relative
Frobenius error per energy and per output kind below 1e-5."""
import pytest

from gpu_parity import MIXED_TOL
from test_gpu_rgf import run_and_compare
from workloads import make_problem, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_2605_19910_gb300 as P
    return P


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def test_mixed_chain16x8(P, torch):
    run_and_compare(P, torch, workload("chain16x8"), tol=MIXED_TOL, precision="mixed")


def test_mixed_b64_several_energies(P, torch):
    prob = make_problem(12, b=64, w=1, n_energies=8, eta=1e-6, seed=3)
    run_and_compare(P, torch, prob, tol=MIXED_TOL, precision="mixed")


def test_mixed_ragged_and_multi_tile(P, torch):
    # b = 100: two M tiles (64 + 36 rows), K in four chunks (32 + 32 + 32 + 4)
    prob = make_problem(5, b=100, w=1, n_energies=3, eta=1e-3, seed=4)
    run_and_compare(P, torch, prob, tol=MIXED_TOL, precision="mixed")
    prob = make_problem(9, b=37, w=1, n_energies=4, eta=1e-6, seed=5)
    run_and_compare(P, torch, prob, tol=MIXED_TOL, precision="mixed")


def test_mixed_variable_sizes(P, torch):
    prob = make_problem(10, b=None, size_range=(3, 70), w=1, n_energies=3, eta=1e-3, seed=6)
    run_and_compare(P, torch, prob, tol=MIXED_TOL, precision="mixed")


def test_mixed_pentadiagonal(P, torch):
    prob = make_problem(12, b=32, w=2, n_energies=4, eta=1e-6, seed=7)
    run_and_compare(P, torch, prob, tol=MIXED_TOL, precision="mixed")


def test_mixed_full_batched64x64_sampled(P, torch):
    prob = workload("batched64x64")
    run_and_compare(P, torch, prob, energies_idx=[0, 100, 255, 256, 383, 511], tol=MIXED_TOL,
                    precision="mixed")


def test_mixed_variable_sizes_many_energies(P, torch):
    prob = make_problem(14, b=None, size_range=(2, 60), w=1, n_energies=9, eta=1e-3, seed=15)
    run_and_compare(P, torch, prob, tol=MIXED_TOL, precision="mixed")


def test_mixed_nanowire_block_sizes_96_to_160(P, torch):
    prob = make_problem(6, b=None, size_range=(96, 160), w=1, n_energies=2, eta=1e-3, seed=61)
    run_and_compare(P, torch, prob, tol=MIXED_TOL, precision="mixed")


def _g1n_err(P, torch, prob, refine):
    import numpy as np
    from gpu_parity import rel_err, to_dev
    from oracle import rgf as O
    Hp, sL, sR, E = to_dev(prob, torch)
    nE = len(prob.energies)
    plan = P.Plan(prob.sizes, 2 * prob.w + 1, nE, precision="mixed", refine_steps=refine,
                  outputs=P.NEGF_OUT_G1N | P.NEGF_OUT_TRANSMISSION)
    _, G1 = plan.solve(Hp, sL, sR, E, band=False)
    T = plan.transmission(Hp, sL, sR, E).cpu().numpy()
    plan.close()
    G1 = G1.cpu().numpy()
    eg, et = 0.0, 0.0
    for e in range(nE):
        ref = O.rgf_selected(O.system_blocks(prob, prob.energies[e]), prob.sizes, prob.w, first_row=True)
        Tref = O.transmission(ref["G1N"], prob.sigma_L, prob.sigma_R)
        eg = max(eg, rel_err(G1[e], ref["G1N"]))
        et = max(et, abs(T[e] - Tref) / abs(Tref))
    return eg, et


@pytest.mark.parametrize("w,N,b", [(1, 12, 64), (1, 9, 37), (2, 10, 24)])
def test_refinement_recovers_fp64_level_g1n_and_transmission(P, torch, w, N, b):
    """One step of iterative refinement of the last block column (FP64-accurate
    residual from 56-bit tensor products, correction with the mixed factors)
    brings G_1N and T(E) from the mixed level to the FP64 level."""
    prob = make_problem(N, b=b, w=w, n_energies=6, eta=1e-6, seed=70 + N)
    e0, t0 = _g1n_err(P, torch, prob, 0)
    e1, t1 = _g1n_err(P, torch, prob, 1)
    assert e0 < MIXED_TOL and t0 < MIXED_TOL
    assert e1 < 1e-10 and t1 < 1e-10, (e0, e1, t0, t1)
    assert e1 < e0 / 100


def test_mixed_wire1024_full_size_sampled(P, torch):
    """1024 blocks with sizes uniform in {96..160} (2-CTA cluster inversions
    above 119), 128 energies, mixed precision at the default product width,
    band + G_1N: two sampled energies against the oracle (this long
    disordered wire at eta = 1e-6 has localized states, large |G|)."""
    prob = workload("wire1024")
    run_and_compare(P, torch, prob, energies_idx=[5, 97], tol=MIXED_TOL, precision="mixed")
