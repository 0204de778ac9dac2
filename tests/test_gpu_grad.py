"""The adjoint: gradient of T(E) with respect to the band blocks of H and to
Sigma_L / Sigma_R, through the C-ABI (negf_grad) and through the
torch.autograd.Function, against the oracle's gradient (itself pinned by
central differences and by torch autograd on a dense inverse) and against
central differences of the GPU transmission."""
import numpy as np
import pytest

from gpu_parity import FP64_TOL, rel_err, to_dev
from oracle import rgf as O
from workloads import make_problem, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_2605_19910_gb300 as P
    return P


def _oracle_grad(prob, weights, per_energy_sigma):
    N = prob.n_blocks
    pairs = O.band_pairs(N, 1)
    gH = {k: np.zeros((prob.sizes[k[0]], prob.sizes[k[1]]), complex) for k in pairs}
    gL, gR, T = [], [], []
    for e, E in enumerate(prob.energies):
        sL = prob.sigma_L[e] if per_energy_sigma else prob.sigma_L
        sR = prob.sigma_R[e] if per_energy_sigma else prob.sigma_R
        M = O.system_blocks(prob, E, sL, sR)
        r = O.rgf_selected(M, prob.sizes, 1, first_row=True)
        lc = O.rgf_last_column(M, prob.sizes, 1)
        T.append(O.transmission(r["G1N"], sL, sR))
        g, a, b = O.transmission_grad(r["first_row"], lc, pairs, sL, sR, N)
        for k in pairs:
            gH[k] += weights[e] * g[k]
        gL.append(weights[e] * a)
        gR.append(weights[e] * b)
    if not per_energy_sigma:
        gL, gR = sum(gL), sum(gR)
    else:
        gL, gR = np.stack(gL), np.stack(gR)
    return gH, gL, gR, np.array(T)


def _random_sigma(rng, b, scale=0.3):
    return -0.5j * np.eye(b) + scale * (rng.normal(size=(b, b)) + 1j * rng.normal(size=(b, b))) / np.sqrt(b)


def _check(P, prob, weights, per_energy_sigma, tol=FP64_TOL):
    import torch
    Hp = torch.tensor(P.pack_band(prob.H, prob.sizes, 1), device="cuda")
    sL = torch.tensor(prob.sigma_L, device="cuda")
    sR = torch.tensor(prob.sigma_R, device="cuda")
    E = torch.tensor(prob.energies, device="cuda")
    w = torch.tensor(weights, device="cuda")
    plan = P.Plan(prob.sizes, 3, len(prob.energies), outputs=P.NEGF_OUT_TRANSMISSION | P.NEGF_OUT_GRAD)
    T, dH, dSL, dSR = plan.grad(Hp, sL, sR, E, w)
    plan.close()
    gH, gL, gR, Tref = _oracle_grad(prob, weights, per_energy_sigma)
    got = P.unpack_band(dH.cpu().numpy(), prob.sizes, 1)
    num = sum(np.linalg.norm(got[k] - v) ** 2 for k, v in gH.items())
    den = sum(np.linalg.norm(v) ** 2 for v in gH.values())
    assert np.sqrt(num / den) < tol
    assert rel_err(dSL.cpu().numpy(), gL) < tol
    assert rel_err(dSR.cpu().numpy(), gR) < tol
    assert rel_err(T.cpu().numpy(), Tref) < tol


def test_grad_shared_sigma(P):
    rng = np.random.default_rng(1)
    prob = make_problem(7, b=6, w=1, n_energies=5, eta=1e-3, seed=31)
    prob.sigma_L = _random_sigma(rng, 6)
    prob.sigma_R = _random_sigma(rng, 6)
    _check(P, prob, rng.normal(size=5), per_energy_sigma=False)


def test_grad_per_energy_sigma_variable_sizes(P):
    rng = np.random.default_rng(2)
    prob = make_problem(6, b=None, size_range=(3, 9), w=1, n_energies=4, eta=1e-3, seed=32)
    b0, bN = prob.sizes[0], prob.sizes[-1]
    prob.sigma_L = np.stack([_random_sigma(rng, b0) for _ in range(4)])
    prob.sigma_R = np.stack([_random_sigma(rng, bN) for _ in range(4)])
    _check(P, prob, rng.normal(size=4), per_energy_sigma=True)


def test_grad_one_lead_per_energy_the_other_shared(P):
    """Sigma_L given per energy, Sigma_R once for all energies: the library
    returns dSigma_L per energy and dSigma_R summed over energies itself
    (negf_grad_strided's separate output strides)."""
    import torch
    rng = np.random.default_rng(4)
    prob = make_problem(6, b=None, size_range=(3, 9), w=1, n_energies=4, eta=1e-3, seed=35)
    b0, bN = prob.sizes[0], prob.sizes[-1]
    sLs = np.stack([_random_sigma(rng, b0) for _ in range(4)])
    sR1 = _random_sigma(rng, bN)
    weights = rng.normal(size=4)
    # oracle: every energy with its own Sigma_L and the shared Sigma_R
    prob.sigma_L, prob.sigma_R = sLs, np.stack([sR1] * 4)
    gH, gL, gR, Tref = _oracle_grad(prob, weights, per_energy_sigma=True)
    Hp = torch.tensor(P.pack_band(prob.H, prob.sizes, 1), device="cuda")
    E = torch.tensor(prob.energies, device="cuda")
    plan = P.Plan(prob.sizes, 3, 4, outputs=P.NEGF_OUT_TRANSMISSION | P.NEGF_OUT_GRAD)
    T, dH, dSL, dSR = plan.grad(Hp, torch.tensor(sLs, device="cuda"), torch.tensor(sR1, device="cuda"), E,
                                torch.tensor(weights, device="cuda"))
    plan.close()
    assert tuple(dSL.shape) == (4, b0, b0) and tuple(dSR.shape) == (bN, bN)
    assert rel_err(dSL.cpu().numpy(), gL) < FP64_TOL
    assert rel_err(dSR.cpu().numpy(), gR.sum(0)) < FP64_TOL
    assert rel_err(T.cpu().numpy(), Tref) < FP64_TOL
    got = P.unpack_band(dH.cpu().numpy(), prob.sizes, 1)
    assert max(rel_err(got[k], v) for k, v in gH.items()) < 1e-10


def test_grad_single_layer(P):
    rng = np.random.default_rng(3)
    prob = make_problem(1, b=5, w=1, n_energies=3, eta=1e-2, seed=33)
    prob.sigma_L = _random_sigma(rng, 5)
    prob.sigma_R = _random_sigma(rng, 5)
    _check(P, prob, rng.normal(size=3), per_energy_sigma=False)


def test_grad_config_trans128x48_weighted_subset(P):
    """128 blocks x b = 48, 256 energies: full-size adjoint run; the loss
    weights are nonzero on four energies so the oracle sum stays small."""
    prob = workload("trans128x48")
    weights = np.zeros(len(prob.energies))
    weights[[3, 90, 128, 250]] = [1.0, -0.5, 2.0, 0.25]
    import torch
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 3, len(prob.energies), outputs=P.NEGF_OUT_TRANSMISSION | P.NEGF_OUT_GRAD)
    T, dH, dSL, dSR = plan.grad(Hp, sL, sR, E, torch.tensor(weights, device="cuda"))
    plan.close()
    sub = make_problem(128, b=48, w=1, n_energies=256, eta=1e-6, seed=0)
    sub.energies = prob.energies[[3, 90, 128, 250]]
    gH, gL, gR, Tref = _oracle_grad(sub, weights[[3, 90, 128, 250]], False)
    got = P.unpack_band(dH.cpu().numpy(), prob.sizes, 1)
    num = sum(np.linalg.norm(got[k] - v) ** 2 for k, v in gH.items())
    den = sum(np.linalg.norm(v) ** 2 for v in gH.values())
    assert np.sqrt(num / den) < FP64_TOL
    assert rel_err(dSL.cpu().numpy(), gL) < FP64_TOL
    assert rel_err(T.cpu().numpy()[[3, 90, 128, 250]], Tref) < FP64_TOL


def test_grad_matches_central_differences_of_gpu_transmission(P):
    import torch
    prob = make_problem(5, b=4, w=1, n_energies=2, eta=1e-2, seed=34)
    Hv = P.pack_band(prob.H, prob.sizes, 1)
    sL = torch.tensor(prob.sigma_L, device="cuda")
    sR = torch.tensor(prob.sigma_R, device="cuda")
    E = torch.tensor(prob.energies, device="cuda")
    w = torch.tensor([1.0, 0.7], device="cuda", dtype=torch.float64)
    plan = P.Plan(prob.sizes, 3, 2, outputs=P.NEGF_OUT_TRANSMISSION | P.NEGF_OUT_GRAD)
    _, dH, _, _ = plan.grad(torch.tensor(Hv, device="cuda"), sL, sR, E, w)
    dH = dH.cpu().numpy()
    h = 1e-6
    rng = np.random.default_rng(0)
    for idx in rng.choice(len(Hv), size=6, replace=False):
        for unit, part in [(1.0, "re"), (1j, "im")]:
            Hp, Hm = Hv.copy(), Hv.copy()
            Hp[idx] += h * unit
            Hm[idx] -= h * unit
            Tp = plan.transmission(torch.tensor(Hp, device="cuda"), sL, sR, E)
            Tm = plan.transmission(torch.tensor(Hm, device="cuda"), sL, sR, E)
            fd = float(((Tp - Tm) / (2 * h) * w).sum())
            an = dH[idx].real if part == "re" else dH[idx].imag
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (idx, part, fd, an)
    plan.close()


def test_autograd_function(P):
    import torch
    rng = np.random.default_rng(5)
    prob = make_problem(6, b=5, w=1, n_energies=3, eta=1e-3, seed=35)
    prob.sigma_L = _random_sigma(rng, 5)
    prob.sigma_R = _random_sigma(rng, 5)
    Hp = torch.tensor(P.pack_band(prob.H, prob.sizes, 1), device="cuda", requires_grad=True)
    sL = torch.tensor(prob.sigma_L, device="cuda", requires_grad=True)
    sR = torch.tensor(prob.sigma_R, device="cuda", requires_grad=True)
    E = torch.tensor(prob.energies, device="cuda")
    plan = P.Plan(prob.sizes, 3, 3, outputs=P.NEGF_OUT_TRANSMISSION | P.NEGF_OUT_GRAD)
    T = P.Transmission.apply(plan, Hp, sL, sR, E)
    weights = torch.tensor([0.3, -1.0, 2.0], device="cuda", dtype=torch.float64)
    (T * weights).sum().backward()
    plan.close()
    gH, gL, gR, Tref = _oracle_grad(prob, weights.cpu().numpy(), False)
    got = P.unpack_band(Hp.grad.cpu().numpy(), prob.sizes, 1)
    for k, v in gH.items():
        assert rel_err(got[k], v) < FP64_TOL
    assert rel_err(sL.grad.cpu().numpy(), gL) < FP64_TOL
    assert rel_err(sR.grad.cpu().numpy(), gR) < FP64_TOL
    assert rel_err(T.detach().cpu().numpy(), Tref) < FP64_TOL


def _oracle_grad_w(prob, weights, w):
    N = prob.n_blocks
    pairs = O.band_pairs(N, w)
    gH = {k: np.zeros((prob.sizes[k[0]], prob.sizes[k[1]]), complex) for k in pairs}
    gL, gR, T = [], [], []
    for e, E in enumerate(prob.energies):
        M = O.system_blocks(prob, E)
        r = O.rgf_selected(M, prob.sizes, w, first_row=True)
        lc = O.rgf_last_column(M, prob.sizes, w)
        T.append(O.transmission(r["G1N"], prob.sigma_L, prob.sigma_R))
        g, a, b = O.transmission_grad(r["first_row"], lc, pairs, prob.sigma_L, prob.sigma_R, N)
        for k in pairs:
            gH[k] += weights[e] * g[k]
        gL.append(weights[e] * a)
        gR.append(weights[e] * b)
    return gH, np.stack(gL), np.stack(gR), np.array(T)


@pytest.mark.parametrize("w,N,ck,nd", [(2, 9, 0, 1), (3, 10, 0, 1), (2, 12, 2, 1), (1, 14, 0, 3), (2, 18, 0, 2)])
def test_grad_block_ndiagonal_through_the_fused_chain(P, w, N, ck, nd):
    """n = 5 and 7 (and n = 5 checkpointed on the fused chain), and DDRGF plans
    (n = 3 and 5, whose adjoint runs on a plain RGF sub-plan): dH for every
    band block |a - b| <= w and the energy-summed dSigma_L / dSigma_R, against
    the oracle's gradient over the band."""
    import torch
    rng = np.random.default_rng(200 + 10 * w + N)
    nE = 4
    prob = make_problem(N, b=None, size_range=(3, 8), w=w, n_energies=nE, eta=1e-3, seed=201 + N)
    prob.sigma_L = _random_sigma(rng, prob.sizes[0])
    prob.sigma_R = _random_sigma(rng, prob.sizes[-1])
    weights = rng.normal(size=nE)
    Hp = torch.tensor(P.pack_band(prob.H, prob.sizes, w), device="cuda")
    sL = torch.tensor(prob.sigma_L, device="cuda")
    sR = torch.tensor(prob.sigma_R, device="cuda")
    E = torch.tensor(prob.energies, device="cuda")
    plan = P.Plan(prob.sizes, 2 * w + 1, nE, outputs=P.NEGF_OUT_TRANSMISSION | P.NEGF_OUT_GRAD,
                  checkpoint_every=ck, n_domains=nd)
    assert plan.n_domains == nd
    T, dH, dSL, dSR = plan.grad(Hp, sL, sR, E, torch.tensor(weights, device="cuda"))
    assert not plan.info.cpu().numpy().any()
    plan.close()
    gH, gL, gR, Tref = _oracle_grad_w(prob, weights, w)
    got = P.unpack_band(dH.cpu().numpy(), prob.sizes, w)
    num = sum(np.linalg.norm(got[k] - v) ** 2 for k, v in gH.items())
    den = sum(np.linalg.norm(v) ** 2 for v in gH.values())
    assert np.sqrt(num / den) < FP64_TOL
    assert rel_err(dSL.cpu().numpy(), gL.sum(0)) < FP64_TOL   # shared leads: energy-summed gradients
    assert rel_err(dSR.cpu().numpy(), gR.sum(0)) < FP64_TOL
    assert rel_err(T.cpu().numpy(), Tref) < FP64_TOL
