"""negf_solve_noalloc: the plan-free entry point for callers that cannot
allocate device memory (for example code running under another component's
memory pool, or with a device-memory budget fixed in advance).  It must give
the same selected blocks and G_1N as negf_solve, call after call, although
every call reuses one fixed device scratch array.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

from gpu_parity import FP64_TOL, band_rel_err, rel_err, to_dev
from workloads import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_2605_19910_gb300 as P
    return P


def _planned(P, torch, prob):
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 2 * prob.w + 1, len(prob.energies))
    Gb, G1 = plan.solve(Hp, sL, sR, E)
    out = (Gb.cpu().numpy(), G1.cpu().numpy())
    plan.close()
    return out


def _noalloc(P, torch, prob):
    Hp, sL, sR, E = to_dev(prob, torch)
    nE = len(prob.energies)
    off, n = P.band_layout(prob.sizes, prob.w)
    Gb = torch.full((nE, n), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    G1 = torch.full((nE, prob.sizes[0], prob.sizes[-1]), complex(np.nan, np.nan), dtype=torch.complex128,
                    device="cuda")
    info = torch.full((nE,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    s = P.negf_solve_noalloc(prob.sizes, 2 * prob.w + 1, nE, Hp, sL, sR, 0, E, Gb, G1, info,
                             stream=stream.cuda_stream)
    assert s == P.NEGF_OK, P.negf_status_string(s)
    torch.cuda.synchronize()
    assert not info.cpu().numpy().any()
    return Gb.cpu().numpy(), G1.cpu().numpy()


def _compare(P, prob, a, b):
    for e in range(len(prob.energies)):
        ref_band = P.unpack_band(b[0][e], prob.sizes, prob.w)
        assert band_rel_err(a[0][e], ref_band, prob.sizes, prob.w) < FP64_TOL
        assert rel_err(a[1][e], b[1][e]) < FP64_TOL


def test_noalloc_matches_planned_solve_on_two_calls_in_a_row(P):
    import torch
    first = make_problem(10, b=48, w=1, n_energies=4, eta=1e-6, seed=21)
    second = make_problem(7, b=None, size_range=(5, 40), w=2, n_energies=3, eta=1e-4, seed=22)
    got1 = _noalloc(P, torch, first)        # first call on this device also sets it up
    got2 = _noalloc(P, torch, second)       # second call: the scratch holds the first call's data
    _compare(P, first, got1, _planned(P, torch, first))
    _compare(P, second, got2, _planned(P, torch, second))


def test_noalloc_rejects_sizes_beyond_its_scratch(P):
    import torch
    # 64 layers of b = 64 need ~12.6 MB of scratch per energy: 8 energies exceed 32 MiB
    nE = 8
    sizes = [64] * 64
    H = torch.zeros(P.band_layout(sizes, 1)[1], dtype=torch.complex128, device="cuda")
    sig = torch.zeros(64, 64, dtype=torch.complex128, device="cuda")
    E = torch.zeros(nE, dtype=torch.complex128, device="cuda")
    G1 = torch.zeros(nE, 64, 64, dtype=torch.complex128, device="cuda")
    info = torch.zeros(nE, dtype=torch.int32, device="cuda")
    s = P.negf_solve_noalloc(sizes, 3, nE, H, sig, sig, 0, E, None, G1, info,
                             stream=torch.cuda.current_stream().cuda_stream)
    assert s == P.NEGF_ERR_ARG
