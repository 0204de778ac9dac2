"""Parity of the mixed-precision CUDA path (tcgen05 split-TF32 block products,
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
