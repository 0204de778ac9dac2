"""The checkpointed adjoint (checkpoint_every = k > 0: segments of k layers
recomputed from stored Schur complements in the reverse pass) and the
mixed-precision adjoint, through the C-ABI, against the oracle's gradient and
against the plain FP64 adjoint."""
import numpy as np
import pytest

from gpu_parity import FP64_TOL, MIXED_TOL, rel_err, to_dev
from test_gpu_grad import _oracle_grad, _random_sigma
from workloads import make_problem, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_2605_19910_gb300 as P
    return P


def _grad(P, prob, weights, checkpoint_every, precision="fp64", product_bits=0):
    import torch
    Hp = torch.tensor(P.pack_band(prob.H, prob.sizes, 1), device="cuda")
    sL = torch.tensor(prob.sigma_L, device="cuda")
    sR = torch.tensor(prob.sigma_R, device="cuda")
    E = torch.tensor(prob.energies, device="cuda")
    w = torch.tensor(weights, device="cuda")
    plan = P.Plan(prob.sizes, 3, len(prob.energies), precision=precision,
                  outputs=P.NEGF_OUT_TRANSMISSION | P.NEGF_OUT_GRAD, checkpoint_every=checkpoint_every,
                  product_bits=product_bits)
    T, dH, dSL, dSR = plan.grad(Hp, sL, sR, E, w)
    ws = P.negf_workspace_bytes(plan.handle)
    plan.close()
    return T.cpu().numpy(), P.unpack_band(dH.cpu().numpy(), prob.sizes, 1), dSL.cpu().numpy(), dSR.cpu().numpy(), ws


def _band_err(got, ref):
    num = sum(np.linalg.norm(got[k] - v) ** 2 for k, v in ref.items())
    den = sum(np.linalg.norm(v) ** 2 for v in ref.values())
    return np.sqrt(num / den)


@pytest.mark.parametrize("k", [1, 2, 3, 6, 7, 50])
def test_checkpointed_grad_matches_oracle(P, k):
    # 7 layers: k = 2, 3 leave a ragged last segment; k = 7, 50 one segment
    rng = np.random.default_rng(40 + k)
    prob = make_problem(7, b=6, w=1, n_energies=5, eta=1e-3, seed=41)
    prob.sigma_L = _random_sigma(rng, 6)
    prob.sigma_R = _random_sigma(rng, 6)
    weights = rng.normal(size=5)
    T, dH, dSL, dSR, _ = _grad(P, prob, weights, k)
    gH, gL, gR, Tref = _oracle_grad(prob, weights, False)
    assert _band_err(dH, gH) < FP64_TOL
    assert rel_err(dSL, gL) < FP64_TOL
    assert rel_err(dSR, gR) < FP64_TOL
    assert rel_err(T, Tref) < FP64_TOL


@pytest.mark.parametrize("k", [1, 4])
def test_checkpointed_grad_per_energy_sigma_variable_sizes(P, k):
    rng = np.random.default_rng(50 + k)
    prob = make_problem(9, b=None, size_range=(3, 11), w=1, n_energies=4, eta=1e-3, seed=52)
    b0, bN = prob.sizes[0], prob.sizes[-1]
    prob.sigma_L = np.stack([_random_sigma(rng, b0) for _ in range(4)])
    prob.sigma_R = np.stack([_random_sigma(rng, bN) for _ in range(4)])
    weights = rng.normal(size=4)
    T, dH, dSL, dSR, _ = _grad(P, prob, weights, k)
    gH, gL, gR, Tref = _oracle_grad(prob, weights, True)
    assert _band_err(dH, gH) < FP64_TOL
    assert rel_err(dSL, gL) < FP64_TOL
    assert rel_err(dSR, gR) < FP64_TOL
    assert rel_err(T, Tref) < FP64_TOL


def test_checkpointed_grad_single_layer(P):
    rng = np.random.default_rng(60)
    prob = make_problem(1, b=5, w=1, n_energies=3, eta=1e-2, seed=61)
    prob.sigma_L = _random_sigma(rng, 5)
    prob.sigma_R = _random_sigma(rng, 5)
    weights = rng.normal(size=3)
    T, dH, dSL, dSR, _ = _grad(P, prob, weights, 1)
    gH, gL, gR, Tref = _oracle_grad(prob, weights, False)
    assert _band_err(dH, gH) < FP64_TOL
    assert rel_err(dSL, gL) < FP64_TOL
    assert rel_err(T, Tref) < FP64_TOL


def test_checkpointed_grad_config_trans128x48(P):
    """128 blocks x b = 48, 256 energies with k = 11 (about sqrt(N)): the same
    gradient as the adjoint that keeps the whole factorisation, in a fraction
    of its workspace; four weighted energies checked against the oracle."""
    prob = workload("trans128x48")
    weights = np.zeros(len(prob.energies))
    idx = [3, 90, 128, 250]
    weights[idx] = [1.0, -0.5, 2.0, 0.25]
    T0, dH0, dSL0, dSR0, ws0 = _grad(P, prob, weights, 0)
    T1, dH1, dSL1, dSR1, ws1 = _grad(P, prob, weights, 11)
    assert ws1 < 0.25 * ws0, (ws1, ws0)
    assert _band_err(dH1, dH0) < 1e-12
    assert rel_err(dSL1, dSL0) < 1e-12
    assert rel_err(T1, T0) < 1e-12
    sub = make_problem(128, b=48, w=1, n_energies=256, eta=1e-6, seed=0)
    sub.energies = prob.energies[idx]
    gH, gL, gR, Tref = _oracle_grad(sub, weights[idx], False)
    assert _band_err(dH1, gH) < FP64_TOL
    assert rel_err(dSL1, gL) < FP64_TOL
    assert rel_err(T1[idx], Tref) < FP64_TOL


def test_checkpointed_plan_serves_transmission_and_g1n(P):
    import torch
    prob = make_problem(8, b=7, w=1, n_energies=3, eta=1e-3, seed=62)
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 3, 3, outputs=P.NEGF_OUT_G1N | P.NEGF_OUT_TRANSMISSION | P.NEGF_OUT_GRAD,
                  checkpoint_every=3)
    T = plan.transmission(Hp, sL, sR, E).cpu().numpy()
    _, G1 = plan.solve(Hp, sL, sR, E, band=False, g1n=True)
    G1 = G1.cpu().numpy()
    st = P.negf_solve(plan.handle, Hp, sL, sR, 0, E,
                      torch.empty(3, plan.band_elems, dtype=torch.complex128, device="cuda"), None, plan.info)
    assert st == P.NEGF_ERR_UNSUPPORTED
    plan.close()
    from oracle import rgf as O
    for e in range(3):
        ref = O.rgf_selected(O.system_blocks(prob, prob.energies[e]), prob.sizes, 1, first_row=True)
        assert rel_err(G1[e], ref["G1N"]) < FP64_TOL
        Tref = O.transmission(ref["G1N"], prob.sigma_L, prob.sigma_R)
        assert abs(T[e] - Tref) / abs(Tref) < FP64_TOL


def test_checkpointed_autograd_function(P):
    import torch
    rng = np.random.default_rng(63)
    prob = make_problem(6, b=5, w=1, n_energies=3, eta=1e-3, seed=64)
    prob.sigma_L = _random_sigma(rng, 5)
    prob.sigma_R = _random_sigma(rng, 5)
    Hp = torch.tensor(P.pack_band(prob.H, prob.sizes, 1), device="cuda", requires_grad=True)
    sL = torch.tensor(prob.sigma_L, device="cuda", requires_grad=True)
    sR = torch.tensor(prob.sigma_R, device="cuda", requires_grad=True)
    E = torch.tensor(prob.energies, device="cuda")
    plan = P.Plan(prob.sizes, 3, 3, outputs=P.NEGF_OUT_TRANSMISSION | P.NEGF_OUT_GRAD, checkpoint_every=2)
    T = P.Transmission.apply(plan, Hp, sL, sR, E)
    weights = torch.tensor([0.3, -1.0, 2.0], device="cuda", dtype=torch.float64)
    (T * weights).sum().backward()
    plan.close()
    gH, gL, gR, Tref = _oracle_grad(prob, weights.cpu().numpy(), False)
    got = P.unpack_band(Hp.grad.cpu().numpy(), prob.sizes, 1)
    assert _band_err(got, gH) < FP64_TOL
    assert rel_err(sL.grad.cpu().numpy(), gL) < FP64_TOL
    assert rel_err(sR.grad.cpu().numpy(), gR) < FP64_TOL


@pytest.mark.parametrize("k", [0, 5])
def test_mixed_adjoint_matches_fp64_adjoint(P, k):
    """Mixed precision (tensor-core products, FP64 inverses) against the FP64
    adjoint at the mixed bar, with and without checkpoints."""
    rng = np.random.default_rng(70 + k)
    prob = make_problem(16, b=32, w=1, n_energies=8, eta=1e-3, seed=71)
    weights = rng.normal(size=8)
    T0, dH0, dSL0, dSR0, _ = _grad(P, prob, weights, 0, "fp64")
    T1, dH1, dSL1, dSR1, _ = _grad(P, prob, weights, k, "mixed")
    assert _band_err(dH1, dH0) < MIXED_TOL
    assert rel_err(dSL1, dSL0) < MIXED_TOL
    assert rel_err(dSR1, dSR0) < MIXED_TOL
    assert rel_err(T1, T0) < MIXED_TOL


def test_mixed_adjoint_config_trans128x48(P):
    """Config 4 in mixed precision: the whole 256-energy gradient against the
    FP64 adjoint (itself pinned to the oracle above)."""
    prob = workload("trans128x48")
    rng = np.random.default_rng(72)
    weights = rng.normal(size=len(prob.energies))
    T0, dH0, dSL0, _, _ = _grad(P, prob, weights, 0, "fp64")
    T1, dH1, dSL1, _, _ = _grad(P, prob, weights, 11, "mixed")
    assert _band_err(dH1, dH0) < MIXED_TOL
    assert rel_err(dSL1, dSL0) < MIXED_TOL
    assert rel_err(T1, T0) < MIXED_TOL
