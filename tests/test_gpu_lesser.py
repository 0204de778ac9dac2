"""Keldysh equation G^< = G^R Sigma^< G^A on the GPU (negf_lesser) against the
oracle's dense definition and its recursion, and against the equilibrium
closed form G^< = -f (G^R - G^A) computed from the GPU's own retarded band."""
import numpy as np
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


def _sless(rng, b):
    A = rng.normal(size=(b, b)) + 1j * rng.normal(size=(b, b))
    return 1j * (A @ A.conj().T) / b


def _run(P, prob, slL, slR, diag=None, precision="fp64"):
    import torch
    Hp, sL, sR, E = to_dev(prob, torch)
    nE = len(prob.energies)
    plan = P.Plan(prob.sizes, 3, nE, precision=precision, outputs=P.NEGF_OUT_BAND | P.NEGF_OUT_LESSER)
    tl = torch.tensor(slL, device="cuda")
    tr = torch.tensor(slR, device="cuda")
    td = torch.tensor(diag, device="cuda") if diag is not None else None
    Gb, Gl = plan.lesser(Hp, sL, sR, E, tl, tr, td)
    assert not plan.info.cpu().numpy().any()
    plan.close()
    return Gb.cpu().numpy(), Gl.cpu().numpy()


def _check_vs_oracle(P, prob, Gl, slL, slR, diag, tol, idx=None):
    N = prob.n_blocks
    for e in (range(len(prob.energies)) if idx is None else idx):
        M = O.system_blocks(prob, prob.energies[e])
        sl = {}
        l_e = slL[e] if slL.ndim == 3 else slL
        r_e = slR[e] if slR.ndim == 3 else slR
        sl[0] = l_e.copy()
        sl[N - 1] = sl.get(N - 1, np.zeros_like(r_e)) + r_e
        if diag is not None:
            for i in range(N):
                sl[i] = sl.get(i, np.zeros((prob.sizes[i], prob.sizes[i]), complex)) + diag[e] * np.eye(prob.sizes[i])
        ref = O.lesser_dense(M, prob.sizes, 1, sl)
        assert band_rel_err(Gl[e], ref, prob.sizes, 1) < tol, e


def test_lesser_matches_dense_keldysh_equation(P):
    rng = np.random.default_rng(120)
    prob = make_problem(9, b=7, w=1, n_energies=4, eta=1e-3, seed=121)
    slL, slR = _sless(rng, 7), _sless(rng, 7)
    _, Gl = _run(P, prob, slL, slR)
    _check_vs_oracle(P, prob, Gl, slL, slR, None, FP64_TOL)


def test_lesser_variable_sizes_per_energy_sigma_and_diagonal_term(P):
    rng = np.random.default_rng(122)
    prob = make_problem(8, b=None, size_range=(3, 12), w=1, n_energies=3, eta=1e-3, seed=123)
    b0, bN = prob.sizes[0], prob.sizes[-1]
    slL = np.stack([_sless(rng, b0) for _ in range(3)])
    slR = np.stack([_sless(rng, bN) for _ in range(3)])
    diag = 1j * rng.uniform(0.0, 1e-2, size=3) + 0j
    _, Gl = _run(P, prob, slL, slR, diag)
    _check_vs_oracle(P, prob, Gl, slL, slR, diag, FP64_TOL)


@pytest.mark.parametrize("N", [1, 2])
def test_lesser_short_chains(P, N):
    rng = np.random.default_rng(124 + N)
    prob = make_problem(N, b=5, w=1, n_energies=2, eta=1e-2, seed=125 + N)
    slL, slR = _sless(rng, 5), _sless(rng, 5)
    _, Gl = _run(P, prob, slL, slR)
    _check_vs_oracle(P, prob, Gl, slL, slR, None, FP64_TOL)


def test_lesser_equilibrium_from_gpu_retarded_band(P):
    """All reservoirs at one occupation f: Sigma^< = i f (Gamma_L + Gamma_R + 2 eta I)
    gives G^< = -f (G^R - G^A) on the band, with G^R the GPU's own band."""
    prob = make_problem(12, b=16, w=1, n_energies=5, eta=2e-2, seed=126)
    f = 0.61
    gL, gR = O.gamma(prob.sigma_L), O.gamma(prob.sigma_R)
    diag = np.full(5, 1j * f * 2 * 2e-2, dtype=complex)
    Gb, Gl = _run(P, prob, 1j * f * gL, 1j * f * gR, diag)
    off, _ = P.band_layout(prob.sizes, 1)
    for e in range(5):
        band = P.unpack_band(Gb[e], prob.sizes, 1)
        less = P.unpack_band(Gl[e], prob.sizes, 1)
        for (a, b), v in less.items():
            expect = -f * (band[(a, b)] - band[(b, a)].conj().T)
            assert np.linalg.norm(v - expect) < 1e-10 * np.linalg.norm(expect), (e, a, b)


def test_lesser_on_mixed_plan(P):
    # retarded sweep and lesser products on the tensor cores
    rng = np.random.default_rng(127)
    prob = make_problem(10, b=32, w=1, n_energies=3, eta=1e-3, seed=128)
    slL, slR = _sless(rng, 32), _sless(rng, 32)
    _, Gl = _run(P, prob, slL, slR, precision="mixed")
    _check_vs_oracle(P, prob, Gl, slL, slR, None, MIXED_TOL)


def test_lesser_full_size_batched64x64_sampled(P):
    """64 x 64 x 512 energies, leads at different occupations (f_L = 1, f_R = 0):
    sampled energies against the oracle's recursion."""
    prob = workload("batched64x64")
    gL, gR = O.gamma(prob.sigma_L), O.gamma(prob.sigma_R)
    slL, slR = 1j * gL, 0.0 * gR
    _, Gl = _run(P, prob, slL, slR)
    for e in (0, 255, 511):
        M = O.system_blocks(prob, prob.energies[e])
        ref, _ = O.rgf_lesser(M, prob.sizes, {0: slL, 63: slR})
        assert band_rel_err(Gl[e], ref, prob.sizes, 1) < FP64_TOL, e


def test_lesser_plan_requirements(P):
    import torch
    prob = make_problem(4, b=4, w=1, n_energies=1, eta=1e-2, seed=129)
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 3, 1)   # no NEGF_OUT_LESSER
    with pytest.raises(P.NegfError) as ei:
        plan.lesser(Hp, sL, sR, E)
    assert ei.value.status == P.NEGF_ERR_ARG
    plan.close()
    # n = 5 runs on the fused chain, whose super-blocks (two layers) must invert
    with pytest.raises(P.NegfError) as ei:
        P.Plan([100] * 6, 5, 1, outputs=P.NEGF_OUT_LESSER)
    assert ei.value.status == P.NEGF_ERR_UNSUPPORTED
    P.Plan([4] * 6, 5, 1, outputs=P.NEGF_OUT_LESSER).close()


@pytest.mark.parametrize("N", [6, 9])
def test_lesser_pentadiagonal_through_the_fused_chain(P, N):
    """n = 5: G^R and G^< bands through the fused block tridiagonal chain
    (lesser_ndiag) against the oracle's dense Keldysh equation."""
    import torch
    rng = np.random.default_rng(130 + N)
    prob = make_problem(N, b=None, size_range=(3, 9), w=2, n_energies=3, eta=1e-3, seed=131 + N)
    b0, bN = prob.sizes[0], prob.sizes[-1]
    slL, slR = _sless(rng, b0), _sless(rng, bN)
    Hp, sL, sR, E = to_dev(prob, torch)
    Gb, Gl = P.lesser_ndiag(prob.sizes, 5, Hp, sL, sR, E, torch.tensor(slL, device="cuda"),
                            torch.tensor(slR, device="cuda"))
    Gb, Gl = Gb.cpu().numpy(), Gl.cpu().numpy()
    for e in range(3):
        M = O.system_blocks(prob, prob.energies[e])
        ref = O.lesser_dense(M, prob.sizes, 2, {0: slL, N - 1: slR})
        assert band_rel_err(Gl[e], ref, prob.sizes, 2) < FP64_TOL, e
        refR = O.dense_selected(M, prob.sizes, 2)["band"]
        assert band_rel_err(Gb[e], refR, prob.sizes, 2) < FP64_TOL, e


@pytest.mark.parametrize("w,N,precision", [(2, 11, "fp64"), (3, 10, "fp64"), (2, 9, "mixed")])
def test_lesser_ndiag_per_energy_leads_and_diagonal_term(P, w, N, precision):
    """n = 5 and 7 through the C-ABI (negf_lesser on the plan's fused chain),
    per-energy lead self-energies of both kinds and the per-energy diagonal
    term, FP64 and mixed, against the oracle's dense Keldysh equation and
    dense retarded band."""
    import torch
    rng = np.random.default_rng(140 + 10 * w + N)
    nE = 3
    prob = make_problem(N, b=None, size_range=(3, 8), w=w, n_energies=nE, eta=1e-3, seed=141 + N)
    b0, bN = prob.sizes[0], prob.sizes[-1]
    slL = np.stack([_sless(rng, b0) for _ in range(nE)])
    slR = np.stack([_sless(rng, bN) for _ in range(nE)])
    diag = 2e-3j * np.array([0.3, 0.5, 0.7])
    Hp, sL, sR, E = to_dev(prob, torch, per_energy_sigma=True)
    plan = P.Plan(prob.sizes, 2 * w + 1, nE, precision=precision, outputs=P.NEGF_OUT_BAND | P.NEGF_OUT_LESSER)
    Gb, Gl = plan.lesser(Hp, sL, sR, E, torch.tensor(slL, device="cuda"), torch.tensor(slR, device="cuda"),
                         torch.tensor(diag, device="cuda"))
    assert not plan.info.cpu().numpy().any()
    plan.close()
    Gb, Gl = Gb.cpu().numpy(), Gl.cpu().numpy()
    tol = FP64_TOL if precision == "fp64" else MIXED_TOL
    for e in range(nE):
        M = O.system_blocks(prob, prob.energies[e])
        sl = {i: diag[e] * np.eye(prob.sizes[i]) for i in range(N)}
        sl[0] = sl[0] + slL[e]
        sl[N - 1] = sl[N - 1] + slR[e]
        ref = O.lesser_dense(M, prob.sizes, w, sl)
        assert band_rel_err(Gl[e], ref, prob.sizes, w) < tol, e
        refR = O.dense_selected(M, prob.sizes, w)["band"]
        assert band_rel_err(Gb[e], refR, prob.sizes, w) < tol, e
