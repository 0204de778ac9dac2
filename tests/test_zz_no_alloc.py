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


def _per_energy_sigma(prob, torch):
    """Distinct lead self-energies per energy (stride b^2): -0.5i I scaled by
    1 + 0.1 e, so that a wrong energy offset changes the result."""
    nE = len(prob.energies)
    sL = np.stack([prob.sigma_L * (1.0 + 0.1 * e) for e in range(nE)])
    sR = np.stack([prob.sigma_R * (1.0 + 0.1 * e) for e in range(nE)])
    return torch.tensor(sL, device="cuda"), torch.tensor(sR, device="cuda")


def _planned(P, torch, prob, per_energy=False):
    Hp, sL, sR, E = to_dev(prob, torch)
    if per_energy:
        sL, sR = _per_energy_sigma(prob, torch)
    plan = P.Plan(prob.sizes, 2 * prob.w + 1, len(prob.energies))
    Gb, G1 = plan.solve(Hp, sL, sR, E)
    out = (Gb.cpu().numpy(), G1.cpu().numpy())
    plan.close()
    return out


def _noalloc_buffers(P, torch, prob, per_energy=False):
    Hp, sL, sR, E = to_dev(prob, torch)
    stride = 0
    if per_energy:
        assert prob.sizes[0] == prob.sizes[-1]
        sL, sR = _per_energy_sigma(prob, torch)
        stride = prob.sizes[0] ** 2
    nE = len(prob.energies)
    off, n = P.band_layout(prob.sizes, prob.w)
    Gb = torch.full((nE, n), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    G1 = torch.full((nE, prob.sizes[0], prob.sizes[-1]), complex(np.nan, np.nan), dtype=torch.complex128,
                    device="cuda")
    info = torch.full((nE,), -7, dtype=torch.int32, device="cuda")
    return Hp, sL, sR, stride, E, Gb, G1, info


def _noalloc(P, torch, prob, per_energy=False):
    Hp, sL, sR, stride, E, Gb, G1, info = _noalloc_buffers(P, torch, prob, per_energy)
    nE = len(prob.energies)
    stream = torch.cuda.current_stream()
    s = P.negf_solve_noalloc(prob.sizes, 2 * prob.w + 1, nE, Hp, sL, sR, stride, E, Gb, G1, info,
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
                             stream=torch.cuda.current_stream().cuda_stream, outputs=P.NEGF_OUT_G1N)
    assert s == P.NEGF_ERR_ARG
    # the same descriptor with one energy fits
    s = P.negf_solve_noalloc(sizes, 3, 1, H, sig, sig, 0, E[:1], None, G1[:1], info[:1],
                             stream=torch.cuda.current_stream().cuda_stream, outputs=P.NEGF_OUT_G1N)
    assert s == P.NEGF_OK


def test_noalloc_rejects_short_sigma_stride_and_unsupported_outputs(P):
    import torch
    prob = make_problem(6, b=16, w=1, n_energies=3, eta=1e-6, seed=23)
    Hp, sL, sR, stride, E, Gb, G1, info = _noalloc_buffers(P, torch, prob, per_energy=True)
    st = torch.cuda.current_stream().cuda_stream
    args = (prob.sizes, 3, 3, Hp, sL, sR)
    # a positive stride shorter than a lead block would read past the last energy's Sigma
    for bad in (-1, 1, 16 * 16 - 1):
        assert P.negf_solve_noalloc(*args, bad, E, Gb, G1, info, stream=st) == P.NEGF_ERR_ARG
    # outputs other than the band and G_1N are not computed here
    for outputs in (P.NEGF_OUT_TRANSMISSION, P.NEGF_OUT_BAND | P.NEGF_OUT_LESSER, P.NEGF_OUT_GRAD):
        assert P.negf_solve_noalloc(*args, 0, E, Gb, G1, info, stream=st, outputs=outputs) == \
            P.NEGF_ERR_UNSUPPORTED
    # a requested output needs its buffer
    assert P.negf_solve_noalloc(*args, 0, E, None, G1, info, stream=st) == P.NEGF_ERR_ARG
    torch.cuda.synchronize()
    assert (info.cpu().numpy() == -7).all()      # nothing was launched


def test_noalloc_per_energy_sigma_matches_planned_solve(P):
    import torch
    prob = make_problem(9, b=24, w=1, n_energies=5, eta=1e-6, seed=24)
    _compare(P, prob, _noalloc(P, torch, prob, per_energy=True), _planned(P, torch, prob, per_energy=True))


def test_noalloc_allocates_no_device_memory(P):
    import torch
    prob = make_problem(12, b=32, w=1, n_energies=4, eta=1e-6, seed=25)
    Hp, sL, sR, stride, E, Gb, G1, info = _noalloc_buffers(P, torch, prob)
    st = torch.cuda.current_stream().cuda_stream

    def call():
        s = P.negf_solve_noalloc(prob.sizes, 3, 4, Hp, sL, sR, stride, E, Gb, G1, info, stream=st)
        assert s == P.NEGF_OK
        torch.cuda.synchronize()
    call()                                      # same kernels and shapes as the measured call
    free0, _ = torch.cuda.mem_get_info()
    alloc0, res0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == res0
