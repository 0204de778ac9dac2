"""Parity of the CUDA RGF path (FP64) with the oracle, through the C-ABI."""
import numpy as np
import pytest

from gpu_parity import FP64_TOL, band_rel_err, rel_err, to_dev
from oracle import rgf as O
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


def run_and_compare(P, torch, prob, energies_idx=None, per_energy_sigma=False, band=True, g1n=True,
                    tol=FP64_TOL, precision="fp64", product_bits=0):
    Hp, sL, sR, E = to_dev(prob, torch, per_energy_sigma)
    plan = P.Plan(prob.sizes, 2 * prob.w + 1, len(prob.energies), precision=precision,
                  outputs=P.NEGF_OUT_BAND | P.NEGF_OUT_G1N | P.NEGF_OUT_TRANSMISSION, product_bits=product_bits)
    Gb, G1 = plan.solve(Hp, sL, sR, E, band=band, g1n=g1n)
    T = plan.transmission(Hp, sL, sR, E)
    info = plan.info.cpu().numpy()
    plan.close()
    assert not info.any()
    idx = range(len(prob.energies)) if energies_idx is None else energies_idx
    Gb = Gb.cpu().numpy() if Gb is not None else None
    G1 = G1.cpu().numpy() if G1 is not None else None
    T = T.cpu().numpy()
    worst = 0.0
    for e in idx:
        Ee = prob.energies[e]
        ref = O.rgf_selected(O.system_blocks(prob, Ee), prob.sizes, prob.w, first_row=True)
        Tref = O.transmission(ref["G1N"], prob.sigma_L, prob.sigma_R)
        if band:
            eb = band_rel_err(Gb[e], ref["band"], prob.sizes, prob.w)
            assert eb < tol, (e, eb)
            worst = max(worst, eb)
        if g1n:
            e1 = rel_err(G1[e], ref["G1N"])
            assert e1 < tol, (e, e1)
        eT = abs(T[e] - Tref) / max(abs(Tref), 1e-300)
        assert eT < tol, (e, T[e], Tref)
    return worst


def test_config_chain16x8(P, torch):
    run_and_compare(P, torch, workload("chain16x8"))


def test_several_tiles_uniform_b64(P, torch):
    prob = make_problem(12, b=64, w=1, n_energies=8, eta=1e-6, seed=3)
    run_and_compare(P, torch, prob)


def test_ragged_tile_tail_b37(P, torch):
    prob = make_problem(9, b=37, w=1, n_energies=5, eta=1e-6, seed=4)
    run_and_compare(P, torch, prob)


def test_variable_block_sizes(P, torch):
    prob = make_problem(11, b=None, size_range=(5, 70), w=1, n_energies=3, eta=1e-3, seed=5)
    run_and_compare(P, torch, prob)


def test_pentadiagonal_n5(P, torch):
    prob = make_problem(10, b=24, w=2, n_energies=4, eta=1e-6, seed=6)
    run_and_compare(P, torch, prob)


def test_pentadiagonal_variable_sizes(P, torch):
    prob = make_problem(9, b=None, size_range=(3, 40), w=2, n_energies=3, eta=1e-3, seed=7)
    run_and_compare(P, torch, prob)


@pytest.mark.parametrize("N,b", [(1, 16), (2, 8), (20, 1), (3, 100)])
def test_degenerate_shapes(P, torch, N, b):
    prob = make_problem(N, b=b, w=1, n_energies=3, eta=1e-2, seed=N)
    run_and_compare(P, torch, prob)


def test_per_energy_sigma_stride(P, torch):
    prob = make_problem(6, b=16, w=1, n_energies=4, eta=1e-6, seed=8)
    run_and_compare(P, torch, prob, per_energy_sigma=True)


def test_g1n_only_and_band_only(P, torch):
    prob = make_problem(7, b=20, w=1, n_energies=3, eta=1e-6, seed=9)
    run_and_compare(P, torch, prob, band=False, g1n=True)
    run_and_compare(P, torch, prob, band=True, g1n=False)


def test_full_batched64x64_sampled_energies(P, torch):
    """The benchmark workload (64 blocks x b=64, 512 energies), in the launch
    configuration the benchmark times; sampled energies against the oracle."""
    prob = workload("batched64x64")
    run_and_compare(P, torch, prob, energies_idx=[0, 77, 255, 256, 400, 511])


def test_graph_replay_sees_new_inputs(P, torch):
    prob = make_problem(6, b=12, w=1, n_energies=3, eta=1e-6, seed=10)
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 3, 3)
    Gb1, _ = plan.solve(Hp, sL, sR, E)
    Gb1 = Gb1.clone()
    out_b = torch.empty_like(Gb1)
    out_1 = torch.empty(3, 12, 12, dtype=torch.complex128, device="cuda")
    plan.solve(Hp, sL, sR, E, out_band=out_b, out_g1n=out_1)
    E.add_(0.25)                                # same pointers, new contents
    plan.solve(Hp, sL, sR, E, out_band=out_b, out_g1n=out_1)   # graph replay
    plan.close()
    for e in range(3):
        Ee = prob.energies[e] + 0.25
        ref = O.rgf_selected(O.system_blocks(prob, Ee), prob.sizes, 1)
        assert band_rel_err(out_b[e].cpu().numpy(), ref["band"], prob.sizes, 1) < FP64_TOL


def test_band_offsets_match_python_layout(P, torch):
    sizes = [3, 5, 4, 2, 6]
    for band_n in (3, 5):
        plan = P.Plan(sizes, band_n, 1)
        off, n = P.band_layout(sizes, (band_n - 1) // 2)
        assert plan.band_elems == n
        for (i, j), o in off.items():
            assert P.negf_band_offset(plan.handle, j - i, i) == o
        assert P.negf_band_offset(plan.handle, (band_n + 1) // 2, 0) == -1
        assert P.negf_band_offset(plan.handle, 1, len(sizes) - 1) == -1
        plan.close()


def test_singular_block_reports_info(P, torch):
    # one layer, H = diag(1,2,3,4), no leads, E = 2 exactly: M has a zero pivot
    from workloads import Problem
    H = {(0, 0): np.diag([1.0, 2.0, 3.0, 4.0]).astype(complex)}
    z = np.zeros((4, 4), complex)
    prob = Problem(sizes=[4], w=1, H=H, sigma_L=z, sigma_R=z, energies=np.array([2.0 + 0j, 2.5 + 0j]))
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan([4], 3, 2)
    s = P.negf_solve(plan.handle, Hp, sL, sR, 0, E, None,
                     torch.empty(2, 4, 4, dtype=torch.complex128, device="cuda"), plan.info)
    assert s == P.NEGF_OK
    assert P.negf_sync(plan.handle) == P.NEGF_ERR_SINGULAR
    assert plan.info.cpu().tolist() == [1, 0]
    # the error word was cleared by negf_sync
    assert P.negf_sync(plan.handle) == P.NEGF_OK
    plan.close()


def test_nan_in_h_reports_nonfinite(P, torch):
    prob = make_problem(5, b=8, w=1, n_energies=2, eta=1e-6, seed=11)
    prob.H[(2, 2)] = prob.H[(2, 2)].copy()
    prob.H[(2, 2)][3, 3] = np.nan
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 3, 2)
    s = P.negf_solve(plan.handle, Hp, sL, sR, 0, E,
                     torch.empty(2, plan.band_elems, dtype=torch.complex128, device="cuda"), None, plan.info)
    assert s == P.NEGF_OK
    assert P.negf_sync(plan.handle) == P.NEGF_ERR_NONFINITE
    info = plan.info.cpu().tolist()
    assert all(1 <= v <= 3 for v in info), info     # layer 3 (1-based) or earlier in sweep order
    plan.close()


def test_argument_errors(P, torch):
    plan = P.Plan([4, 4], 3, 1)
    assert P.negf_solve(plan.handle, None, None, None, 0, None, None, None, None) == P.NEGF_ERR_ARG
    assert P.negf_transmission(plan.handle, None, None, None, 0, None, None, None) == P.NEGF_ERR_ARG
    plan.close()
    # a per-energy Sigma stride shorter than a lead block is rejected before any launch
    prob = make_problem(3, b=5, w=1, n_energies=2, eta=1e-2, seed=141)
    Hp, sL, sR, E = to_dev(prob, torch, per_energy_sigma=True)
    plan = P.Plan(prob.sizes, 3, 2)
    out = torch.empty(2, plan.band_elems, dtype=torch.complex128, device="cuda")
    for bad in (-1, 24):
        assert P.negf_solve(plan.handle, Hp, sL, sR, bad, E, out, None, plan.info) == P.NEGF_ERR_ARG
    assert P.negf_solve(plan.handle, Hp, sL, sR, 25, E, out, None, plan.info) == P.NEGF_OK
    assert P.negf_sync(plan.handle) == P.NEGF_OK
    plan.close()


def test_variable_sizes_many_energies_concurrent_groups(P, torch):
    # energy groups run concurrently on forked streams and sit at different
    # layers of different block sizes: the shared window slots must not overlap
    prob = make_problem(14, b=None, size_range=(2, 60), w=1, n_energies=9, eta=1e-3, seed=15)
    run_and_compare(P, torch, prob)
    prob = make_problem(12, b=None, size_range=(2, 40), w=2, n_energies=7, eta=1e-3, seed=16)
    run_and_compare(P, torch, prob)


def test_single_layer_with_distinct_leads(P, torch):
    # N = 1: Sigma_L and Sigma_R both act on the one layer and must both enter
    rng = np.random.default_rng(12)
    prob = make_problem(1, b=6, w=1, n_energies=2, eta=1e-2, seed=12)
    prob.sigma_L = -0.3j * np.eye(6) + 0.2 * rng.normal(size=(6, 6))
    prob.sigma_R = -0.7j * np.eye(6) + 0.1 * rng.normal(size=(6, 6))
    run_and_compare(P, torch, prob)


@pytest.mark.parametrize("b", [120, 127, 160])
def test_large_blocks_cluster_inversion(P, torch, b):
    # blocks above one CTA's shared memory: two-CTA cluster inversion
    prob = make_problem(3, b=b, w=1, n_energies=3, eta=1e-3, seed=b)
    run_and_compare(P, torch, prob)


def test_nanowire_block_sizes_96_to_160(P, torch):
    prob = make_problem(6, b=None, size_range=(96, 160), w=1, n_energies=2, eta=1e-3, seed=61)
    run_and_compare(P, torch, prob)


@pytest.mark.parametrize("pinned", [True, False])
def test_solve_host_matches_device_solve(P, torch, pinned):
    # negf_solve_host (host buffers in and out) gives the device call's results
    prob = make_problem(7, b=9, w=1, n_energies=5, eta=1e-3, seed=140)
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 3, 5)
    Gb, G1 = plan.solve(Hp, sL, sR, E)
    host = lambda t: t.cpu().pin_memory() if pinned else t.cpu()
    Gb_h = host(torch.zeros_like(Gb))
    G1_h = host(torch.zeros_like(G1))
    info = plan.solve_host(host(Hp), host(sL), host(sR), host(E), Gb_h, G1_h)
    assert not info.numpy().any()
    assert torch.equal(Gb_h, Gb.cpu()) and torch.equal(G1_h, G1.cpu())
    # a second call reuses the plan's device copies and the captured graph
    E2 = E.clone() + 0.1
    plan.solve_host(host(Hp), host(sL), host(sR), host(E2), Gb_h, G1_h)
    Gb2, _ = plan.solve(Hp, sL, sR, E2)
    plan.close()
    assert torch.equal(Gb_h, Gb2.cpu())
