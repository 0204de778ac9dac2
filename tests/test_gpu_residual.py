"""negf_band_residual (the a-posteriori check of a band from the band alone)
against the oracle's band_diag_residual on the same band: exact bands,
perturbed bands (where the value is known in closed form), per-energy
self-energies and the mixed path."""
import numpy as np
import pytest

from gpu_parity import to_dev
from oracle import rgf as O
from workloads import make_problem, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_2605_19910_gb300 as P
    return P


def _oracle_res(P, prob, Gb_vec, e, sL=None, sR=None):
    M = O.system_blocks(prob, prob.energies[e], sL, sR)
    band = P.unpack_band(Gb_vec, prob.sizes, prob.w)
    return O.band_diag_residual(M, prob.sizes, prob.w, band)


@pytest.mark.parametrize("w", [1, 2])
def test_residual_of_fp64_band_and_of_a_perturbed_band(P, w):
    import torch
    prob = make_problem(9, b=None, size_range=(3, 17), w=w, n_energies=3, eta=1e-3, seed=80 + w)
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 2 * w + 1, 3)
    Gb, _ = plan.solve(Hp, sL, sR, E)
    res = plan.band_residual(Hp, sL, sR, E, Gb).cpu().numpy()
    Gh = Gb.cpu().numpy()
    for e in range(3):
        assert res[e] < 1e-11
        assert abs(res[e] - _oracle_res(P, prob, Gh[e], e)) < 1e-11
    # perturb one element of every energy's band: the residual follows it
    off, _ = P.band_layout(prob.sizes, w)
    k = off[(4, 4 + w)]
    Gp = Gb.clone()
    Gp[:, k] += 1e-4
    resp = plan.band_residual(Hp, sL, sR, E, Gp).cpu().numpy()
    Gph = Gp.cpu().numpy()
    plan.close()
    for e in range(3):
        ref = _oracle_res(P, prob, Gph[e], e)
        assert ref > 1e-6
        assert abs(resp[e] - ref) < 1e-9 * ref + 1e-12


def test_residual_per_energy_sigma(P):
    import torch
    rng = np.random.default_rng(83)
    prob = make_problem(6, b=5, w=1, n_energies=4, eta=1e-3, seed=84)
    sLs = np.stack([-0.4j * np.eye(5) + 0.2 * rng.normal(size=(5, 5)) for _ in range(4)])
    sRs = np.stack([-0.6j * np.eye(5) + 0.2 * rng.normal(size=(5, 5)) for _ in range(4)])
    Hp = torch.tensor(P.pack_band(prob.H, prob.sizes, 1), device="cuda")
    sL, sR = torch.tensor(sLs, device="cuda"), torch.tensor(sRs, device="cuda")
    E = torch.tensor(prob.energies, device="cuda")
    plan = P.Plan(prob.sizes, 3, 4)
    Gb, _ = plan.solve(Hp, sL, sR, E)
    Gp = Gb.clone()
    Gp[:, 7] += 1e-4            # an element of block (1, 0)
    res = plan.band_residual(Hp, sL, sR, E, Gp).cpu().numpy()
    Gph = Gp.cpu().numpy()
    plan.close()
    for e in range(4):
        ref = _oracle_res(P, prob, Gph[e], e, sLs[e], sRs[e])
        assert abs(res[e] - ref) < 1e-9 * ref


def test_residual_ranks_fp64_and_mixed_bands(P):
    """batched64x64 at 64 energies: the mixed band's residual is well above
    the FP64 band's (a residual scales with ||M|| ||G|| times the band's
    relative error, so no absolute bound is asserted for it)."""
    import torch
    prob = workload("batched64x64", n_energies=64)
    Hp, sL, sR, E = to_dev(prob, torch)
    out = {}
    for prec in ("fp64", "mixed"):
        plan = P.Plan(prob.sizes, 3, 64, precision=prec)
        Gb, _ = plan.solve(Hp, sL, sR, E, g1n=False)
        out[prec] = plan.band_residual(Hp, sL, sR, E, Gb).cpu().numpy()
        plan.close()
    assert out["fp64"].max() < 1e-9
    assert np.median(out["mixed"]) > 10 * np.median(out["fp64"])
    assert np.isfinite(out["mixed"]).all()
