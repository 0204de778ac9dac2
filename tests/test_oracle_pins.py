"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test would fail for a plausible slip in the oracle (a dropped term, a
wrong sign, a transposed block, an off-by-one window).  None of these tests
uses the CUDA library.
"""
import numpy as np
import pytest

from oracle import rgf as O
from workloads import make_problem, random_band_matrix, uniform_chain

inv = np.linalg.inv


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------------------
# Dense reference
# ---------------------------------------------------------------------------
def test_dense_inverse_residual_and_block_placement():
    sizes = [3, 5, 2, 4]
    M = random_band_matrix(sizes, 1, seed=3, diag_shift=2.0)
    A = O.dense_from_blocks(M, sizes)
    # block (1, 2) of M sits at rows 3..7, cols 8..9 of the full matrix
    assert np.array_equal(A[3:8, 8:10], M[(1, 2)])
    assert np.array_equal(A[8:10, 3:8], M[(2, 1)])
    assert not np.any(A[0:3, 8:10])      # (0, 2) is outside the band
    G = O.dense_inverse(M, sizes)
    n = A.shape[0]
    assert np.linalg.norm(A @ G - np.eye(n)) < 1e-13 * np.linalg.cond(A)
    assert np.linalg.norm(G @ A - np.eye(n)) < 1e-13 * np.linalg.cond(A)


# ---------------------------------------------------------------------------
# Closed forms printed in the paper (Eqs. 2x2_exact_RGF and 4x4_exact_RGF)
# ---------------------------------------------------------------------------
def test_eq_2x2_exact_rgf():
    sizes = [4, 3]
    T = random_band_matrix(sizes, 1, seed=11, diag_shift=1.5)
    t22 = inv(T[(1, 1)])
    t11 = inv(T[(0, 0)] - T[(0, 1)] @ t22 @ T[(1, 0)])
    expect = {
        (0, 0): t11,
        (0, 1): -t11 @ T[(0, 1)] @ t22,
        (1, 0): -t22 @ T[(1, 0)] @ t11,
        (1, 1): t22 + t22 @ T[(1, 0)] @ t11 @ T[(0, 1)] @ t22,
    }
    d = O.dense_selected(T, sizes, 1)
    r = O.rgf_selected(T, sizes, 1)
    for k, v in expect.items():
        assert rel(d["band"][k], v) < 1e-13
        assert rel(r["band"][k], v) < 1e-13


def _paper_4x4(T):
    """Eq. 4x4_exact_RGF written out block by block."""
    t44 = inv(T[(3, 3)])
    t33 = inv(T[(2, 2)] - T[(2, 3)] @ t44 @ T[(3, 2)])
    t22 = inv(T[(1, 1)] - T[(1, 2)] @ t33 @ T[(2, 1)])
    t11 = inv(T[(0, 0)] - T[(0, 1)] @ t22 @ T[(1, 0)])
    tt11 = t11
    tt22 = t22 + t22 @ T[(1, 0)] @ tt11 @ T[(0, 1)] @ t22
    tt33 = t33 + t33 @ T[(2, 1)] @ tt22 @ T[(1, 2)] @ t33
    tt44 = t44 + t44 @ T[(3, 2)] @ tt33 @ T[(2, 3)] @ t44
    T12, T21, T23, T32, T34, T43 = T[(0, 1)], T[(1, 0)], T[(1, 2)], T[(2, 1)], T[(2, 3)], T[(3, 2)]
    return {
        (0, 0): tt11,
        (0, 1): -t11 @ T12 @ t22,
        (0, 2): t11 @ T12 @ t22 @ T23 @ t33,
        (0, 3): -t11 @ T12 @ t22 @ T23 @ t33 @ T34 @ t44,
        (1, 0): -t22 @ T21 @ t11,
        (1, 1): tt22,
        (1, 2): -tt22 @ T23 @ t33,
        (1, 3): tt22 @ T23 @ t33 @ T34 @ t44,
        (2, 0): t33 @ T32 @ t22 @ T21 @ t11,
        (2, 1): -t33 @ T32 @ tt22,
        (2, 2): tt33,
        (2, 3): -tt33 @ T34 @ t44,
        (3, 0): -t44 @ T43 @ t33 @ T32 @ t22 @ T21 @ t11,
        (3, 1): t44 @ T43 @ t33 @ T32 @ tt22,
        (3, 2): -t44 @ T43 @ tt33,
        (3, 3): tt44,
    }


@pytest.mark.parametrize("sizes", [[3, 3, 3, 3], [2, 5, 3, 4]])
def test_eq_4x4_exact_rgf(sizes):
    T = random_band_matrix(sizes, 1, seed=7, diag_shift=1.5)
    expect = _paper_4x4(T)
    full = O.dense_inverse(T, sizes)
    got = O.blocks_from_dense(full, sizes, list(expect))
    for k in expect:
        assert rel(got[k], expect[k]) < 1e-12, k
    r = O.rgf_selected(T, sizes, 1, first_row=True)
    for k, v in r["band"].items():
        assert rel(v, expect[k]) < 1e-12, k
    for j in range(4):
        assert rel(r["first_row"][(0, j)], expect[(0, j)]) < 1e-12
    lc = O.rgf_last_column(T, sizes, 1)
    for i in range(4):
        assert rel(lc[(i, 3)], expect[(i, 3)]) < 1e-12


# ---------------------------------------------------------------------------
# Brute force against the dense inverse on tiny random inputs
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("w", [1, 2, 3])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 8])
def test_rgf_equals_dense_random(w, N):
    if N <= w and N > 1:
        pytest.skip("N > w required")
    rng = np.random.default_rng(100 * w + N)
    sizes = [int(x) for x in rng.integers(1, 7, size=N)]
    M = random_band_matrix(sizes, w, seed=N + 31 * w, diag_shift=2.0)
    r = O.rgf_selected(M, sizes, w, first_row=True)
    d = O.dense_selected(M, sizes, w)
    for k in d["band"]:
        assert rel(r["band"][k], d["band"][k]) < 1e-12, k
    for k in d["first_row"]:
        assert rel(r["first_row"][k], d["first_row"][k]) < 1e-12
    lc = O.rgf_last_column(M, sizes, w)
    for k in d["last_col"]:
        assert rel(lc[k], d["last_col"][k]) < 1e-12


# ---------------------------------------------------------------------------
# Operation counts (Eqs. cost_model_RGF and cost_model_general_RGF)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("w", [1, 2, 3])
@pytest.mark.parametrize("ell", [4, 7, 12])
def test_op_counts_match_paper(w, ell):
    sizes = [2] * ell
    M = random_band_matrix(sizes, w, seed=1, diag_shift=2.0)
    ops = O.OpCount()
    O.rgf_selected(M, sizes, w, ops=ops)
    assert ops.lu == ell
    assert ops.getrs == ell * (2 * w + 1) - w * w - w
    assert ops.gemm == (3 * w * w + w) * ell - 2 * w ** 3 - 2 * w * w
    if w == 1:
        assert ops.getrs == 3 * ell - 2 and ops.gemm == 4 * (ell - 1)


# ---------------------------------------------------------------------------
# n-diagonal RGF: block fusing and the tridiagonal special case (Sec. 2.3)
# ---------------------------------------------------------------------------
def test_ndiag_equals_fused_tridiagonal():
    w = 2
    sizes = [3] * 8
    M = random_band_matrix(sizes, w, seed=9, diag_shift=2.0)
    r = O.rgf_selected(M, sizes, w)["band"]
    Mf, sf, groups = O.fuse_blocks(M, sizes, w)
    rf = O.rgf_selected(Mf, sf, 1)["band"]
    # compare every band block of the native result with the fused result
    loc = {}
    for g, grp in enumerate(groups):
        o = 0
        for i in grp:
            loc[i] = (g, o)
            o += sizes[i]
    for (a, b), blk in r.items():
        ga, oa = loc[a]
        gb, ob = loc[b]
        ref = rf[(ga, gb)][oa:oa + sizes[a], ob:ob + sizes[b]]
        assert rel(blk, ref) < 1e-12


def test_pentadiagonal_with_zero_next_coupling_equals_tridiagonal():
    sizes = [4] * 7
    M3 = random_band_matrix(sizes, 1, seed=4, diag_shift=2.0)
    M5 = dict(M3)
    for i in range(5):
        M5[(i, i + 2)] = np.zeros((4, 4), complex)
        M5[(i + 2, i)] = np.zeros((4, 4), complex)
    r3 = O.rgf_selected(M3, sizes, 1)["band"]
    r5 = O.rgf_selected(M5, sizes, 2)["band"]
    for k, v in r3.items():
        assert rel(r5[k], v) < 1e-13


# ---------------------------------------------------------------------------
# Uniform tight-binding chain with semi-infinite leads (closed form)
# ---------------------------------------------------------------------------
def chain_root(E, eps, t):
    """|z| < 1 root of t z^2 - (E - eps) z + t = 0 (Im E > 0)."""
    r = np.roots([t, -(E - eps), t])
    return r[np.argmin(np.abs(r))]


@pytest.mark.parametrize("E", [0.3 + 1e-3j, -1.7 + 1e-2j, 2.6 + 1e-3j])
def test_uniform_chain_closed_form(E):
    eps, t, b, N = 0.1, -1.0, 3, 9
    prob = uniform_chain(N, b, eps, t, [E])
    z = chain_root(E, eps, t)
    sig = t * z * np.eye(b)
    M = O.system_blocks(prob, E, sig, sig)
    r = O.rgf_selected(M, prob.sizes, 1, first_row=True)
    g0 = 1.0 / (t * (1.0 / z - z))
    for (j, k), blk in r["band"].items():
        assert rel(blk, g0 * z ** abs(j - k) * np.eye(b)) < 1e-12
    # every right-connected inverse of the sweep is the surface Green's function z/t
    Mb = O.system_blocks(prob, E, sig, sig)
    S = Mb[(N - 1, N - 1)]
    for i in range(N - 1, 0, -1):
        ti = inv(S)
        assert rel(ti, (z / t) * np.eye(b)) < 1e-12
        S = Mb[(i - 1, i - 1)] - Mb[(i - 1, i)] @ ti @ Mb[(i, i - 1)]
    assert rel(r["G1N"], g0 * z ** (N - 1) * np.eye(b)) < 1e-12


def test_uniform_chain_transmission_counts_channels():
    eps, t, b, N = 0.0, -1.0, 4, 12
    for E, expect in [(0.5 + 1e-9j, b), (-1.2 + 1e-9j, b), (2.5 + 1e-9j, 0.0)]:
        prob = uniform_chain(N, b, eps, t, [E])
        z = chain_root(E, eps, t)
        sig = t * z * np.eye(b)
        M = O.system_blocks(prob, E, sig, sig)
        r = O.rgf_selected(M, prob.sizes, 1, first_row=True)
        T = O.transmission(r["G1N"], sig, sig)
        assert abs(T - expect) < 1e-6


def test_mixed_channel_chain_counts_open_channels():
    # H_ii = U diag(eps_c) U^H: channel c is open where |E - eps_c| < 2|t|
    eps_c = [-2.5, -0.5, 0.0, 1.0, 3.0]
    t, N, E = -1.0, 10, 0.2 + 1e-9j
    prob = uniform_chain(N, 5, 0.0, t, [E], channel_energies=eps_c, seed=2)
    # lead self-energy in the channel basis, rotated back
    Hd = prob.H[(0, 0)]
    w_, U = np.linalg.eigh(Hd)
    zs = np.array([chain_root(E, e, t) for e in w_])
    sig = (U * (t * zs)) @ U.conj().T
    M = O.system_blocks(prob, E, sig, sig)
    r = O.rgf_selected(M, prob.sizes, 1, first_row=True)
    T = O.transmission(r["G1N"], sig, sig)
    n_open = sum(abs(E.real - e) < 2 * abs(t) for e in eps_c)
    assert n_open == 3
    assert abs(T - n_open) < 1e-6


# ---------------------------------------------------------------------------
# G^A = (G^R)^H and G^R - G^A = -i G^R (Gamma_L + Gamma_R + 2 eta I) G^A
# ---------------------------------------------------------------------------
def test_advanced_and_spectral_identity():
    prob = make_problem(6, b=4, w=1, energy=0.3 + 0.02j, seed=5)
    E = prob.energies[0]
    M = O.system_blocks(prob, E)
    G = O.dense_inverse(M, prob.sizes)
    # G^A: inverse of M^A = conj(E) I - H - Sigma^H
    MA = O.system_blocks(prob, np.conj(E), prob.sigma_L.conj().T, prob.sigma_R.conj().T)
    GA = O.dense_inverse(MA, prob.sizes)
    assert rel(GA, G.conj().T) < 1e-13
    n = G.shape[0]
    GamL = np.zeros((n, n), complex)
    GamR = np.zeros((n, n), complex)
    b0, bN = prob.sizes[0], prob.sizes[-1]
    GamL[:b0, :b0] = O.gamma(prob.sigma_L)
    GamR[-bN:, -bN:] = O.gamma(prob.sigma_R)
    eta = E.imag
    lhs = G - GA
    rhs = -1j * G @ (GamL + GamR + 2 * eta * np.eye(n)) @ GA
    assert rel(lhs, rhs) < 1e-12
    # without the 2 eta term the identity fails by a visible margin
    rhs_bad = -1j * G @ (GamL + GamR) @ GA
    assert rel(lhs, rhs_bad) > 1e-3


def test_spectral_identity_on_rgf_band_diagonal():
    prob = make_problem(7, b=3, w=1, energy=-0.4 + 0.0j, seed=8)
    E = prob.energies[0]
    M = O.system_blocks(prob, E)
    d = O.dense_selected(M, prob.sizes, 1)
    r = O.rgf_selected(M, prob.sizes, 1)
    G = d["full"]
    off = np.concatenate([[0], np.cumsum(prob.sizes)])
    gL, gR = O.gamma(prob.sigma_L), O.gamma(prob.sigma_R)
    for i in range(prob.n_blocks):
        Gii = r["band"][(i, i)]
        Gi1 = G[off[i]:off[i + 1], off[0]:off[1]]
        GiN = G[off[i]:off[i + 1], off[-2]:off[-1]]
        lhs = 1j * (Gii - Gii.conj().T)
        rhs = Gi1 @ gL @ Gi1.conj().T + GiN @ gR @ GiN.conj().T
        assert rel(lhs, rhs) < 1e-11


# ---------------------------------------------------------------------------
# DDRGF (Alg. 2): exact algebra, Prop. 4, and the Schur complement
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("w,N,nd", [(1, 20, 4), (1, 13, 3), (2, 24, 4), (2, 31, 3)])
def test_ddrgf_equals_dense(w, N, nd):
    rng = np.random.default_rng(N)
    sizes = [int(x) for x in rng.integers(2, 5, size=N)]
    M = random_band_matrix(sizes, w, seed=N + w, diag_shift=2.5)
    dd = O.ddrgf_selected(M, sizes, w, nd, return_parts=True)
    d = O.dense_selected(M, sizes, w)
    for k in d["band"]:
        assert rel(dd["band"][k], d["band"][k]) < 1e-11, k
    # T_S equals the dense Schur complement T11 - T12 T22^{-1} T21 on the separators
    pairs = dd["pairs"]
    D1 = [i for (_, s) in pairs for i in s]
    D2 = [i for (d2, _) in pairs for i in d2]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    idx = lambda L: np.concatenate([np.arange(off[i], off[i + 1]) for i in L])
    A = O.dense_from_blocks(M, sizes)
    i1, i2 = idx(D1), idx(D2)
    TS = A[np.ix_(i1, i1)] - A[np.ix_(i1, i2)] @ inv(A[np.ix_(i2, i2)]) @ A[np.ix_(i2, i1)]
    o1 = {}
    o = 0
    for s in D1:
        o1[s] = o
        o += sizes[s]
    for s in D1:
        for s2 in D1:
            blk = TS[o1[s]:o1[s] + sizes[s], o1[s2]:o1[s2] + sizes[s2]]
            got = dd["TS"].get((s, s2))
            if got is None:
                assert np.abs(blk).max() < 1e-12          # Prop. 4: outside the pattern
            else:
                assert rel(got, blk) < 1e-11
    # the separator part of M^{-1} is exactly T_S^{-1}
    Ginv = inv(A)
    assert rel(Ginv[np.ix_(i1, i1)], inv(TS)) < 1e-11


@pytest.mark.parametrize("w,N,nd,levels", [(1, 40, 10, (3,)), (1, 60, 15, (5, 2)), (2, 48, 8, (3,)),
                                             (1, 64, 16, (4, 2)), (2, 60, 12, (4, 2))])
def test_recursive_ddrgf_equals_dense(w, N, nd, levels):
    """Alg. 2 step 3 by DDRGF itself on the separators' chain (2 and 3
    levels, one-super-layer separators below the first level) gives the
    dense band."""
    rng = np.random.default_rng(N + 7)
    sizes = [int(x) for x in rng.integers(2, 5, size=N)]
    M = random_band_matrix(sizes, w, seed=N + 11, diag_shift=3.0)
    d = O.dense_selected(M, sizes, w)
    r = O.ddrgf_selected(M, sizes, w, nd, levels=levels)
    for k in d["band"]:
        assert rel(r["band"][k], d["band"][k]) < 1e-11, k
    # a recursion that cuts the separators' chain differently gives the same band
    r2 = O.ddrgf_selected(M, sizes, w, nd, levels=(2,))
    for k in d["band"]:
        assert rel(r2["band"][k], d["band"][k]) < 1e-11, k


def test_recursive_ddrgf_rejects_a_level_too_fine_for_its_chain():
    sizes = [3] * 20
    M = random_band_matrix(sizes, 1, seed=3, diag_shift=3.0)
    with pytest.raises(ValueError):
        O.ddrgf_selected(M, sizes, 1, 5, levels=(4,))   # 5 separators cannot hold 4 pairs of >= 2


def test_ddrgf_interface_couplings_cannot_be_dropped():
    # the "orange" next-separator couplings (Sec. 3, after Prop. 4) matter
    sizes = [3] * 16
    M = random_band_matrix(sizes, 1, seed=2, diag_shift=2.0)
    dd = O.ddrgf_selected(M, sizes, 1, 4, return_parts=True)
    seps = [s[0] for (_, s) in dd["pairs"]]
    assert np.abs(dd["TS"][(seps[0], seps[1])]).max() > 1e-3


# ---------------------------------------------------------------------------
# Transmission and gradient
# ---------------------------------------------------------------------------
def test_transmission_is_frobenius_norm_for_unit_broadening():
    prob = make_problem(8, b=5, w=1, energy=0.7 + 1e-6j, seed=1)
    E = prob.energies[0]
    r = O.rgf_selected(O.system_blocks(prob, E), prob.sizes, 1, first_row=True)
    T = O.transmission(r["G1N"], prob.sigma_L, prob.sigma_R)   # Sigma = -0.5i I -> Gamma = I
    assert np.allclose(O.gamma(prob.sigma_L), np.eye(5))
    assert abs(T - np.linalg.norm(r["G1N"]) ** 2) < 1e-12 * max(1.0, T)


def _T_of(prob, E, H=None, sL=None, sR=None):
    import copy
    p = copy.copy(prob)
    if H is not None:
        p.H = H
    sL = prob.sigma_L if sL is None else sL
    sR = prob.sigma_R if sR is None else sR
    M = O.system_blocks(p, E, sL, sR)
    r = O.rgf_selected(M, p.sizes, p.w, first_row=True)
    return O.transmission(r["G1N"], sL, sR)


def _grads(prob, E):
    M = O.system_blocks(prob, E)
    d = O.dense_selected(M, prob.sizes, 1)
    return O.transmission_grad(d["first_row"], d["last_col"], O.band_pairs(prob.n_blocks, 1),
                               prob.sigma_L, prob.sigma_R, prob.n_blocks)


def test_gradient_matches_central_differences():
    prob = make_problem(5, b=3, w=1, energy=0.4 + 0.05j, seed=6)
    rng = np.random.default_rng(0)
    sL = prob.sigma_L + 0.1 * (rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3)))
    prob.sigma_L = sL
    E = prob.energies[0]
    gH, gSL, gSR = _grads(prob, E)
    h = 1e-6
    for (a, b) in [(0, 0), (1, 2), (3, 2), (4, 4)]:
        for (r, c) in [(0, 0), (1, 2), (2, 1)]:
            for unit, part in [(1.0, "re"), (1j, "im")]:
                Hp = {k: v.copy() for k, v in prob.H.items()}
                Hm = {k: v.copy() for k, v in prob.H.items()}
                Hp[(a, b)][r, c] += h * unit
                Hm[(a, b)][r, c] -= h * unit
                fd = (_T_of(prob, E, H=Hp) - _T_of(prob, E, H=Hm)) / (2 * h)
                g = gH[(a, b)][r, c]
                an = g.real if part == "re" else g.imag
                assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (a, b, r, c, part, fd, an)
    for which, G in (("L", gSL), ("R", gSR)):
        for (r, c) in [(0, 0), (0, 2), (2, 1)]:
            for unit, part in [(1.0, "re"), (1j, "im")]:
                S = (prob.sigma_L if which == "L" else prob.sigma_R).copy()
                Sp, Sm = S.copy(), S.copy()
                Sp[r, c] += h * unit
                Sm[r, c] -= h * unit
                if which == "L":
                    fd = (_T_of(prob, E, sL=Sp) - _T_of(prob, E, sL=Sm)) / (2 * h)
                else:
                    fd = (_T_of(prob, E, sR=Sp) - _T_of(prob, E, sR=Sm)) / (2 * h)
                an = G[r, c].real if part == "re" else G[r, c].imag
                assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (which, r, c, part, fd, an)


def test_gradient_matches_torch_autograd_dense():
    torch = pytest.importorskip("torch")
    prob = make_problem(4, b=3, w=1, energy=-0.3 + 0.02j, seed=12)
    E = prob.energies[0]
    gH, gSL, gSR = _grads(prob, E)
    sizes = prob.sizes
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    n = off[-1]
    Hs = {k: torch.tensor(v, requires_grad=True) for k, v in prob.H.items()}
    sL = torch.tensor(prob.sigma_L, requires_grad=True)
    sR = torch.tensor(prob.sigma_R, requires_grad=True)
    rows = []
    for a in range(4):
        row = []
        for b in range(4):
            if (a, b) in Hs:
                row.append(Hs[(a, b)])
            else:
                row.append(torch.zeros(sizes[a], sizes[b], dtype=torch.complex128))
        rows.append(torch.cat(row, 1))
    Hfull = torch.cat(rows, 0)
    Sfull = torch.zeros(n, n, dtype=torch.complex128)
    Sfull = Sfull.index_put((torch.arange(3)[:, None], torch.arange(3)[None, :]), sL)
    Sfull = Sfull.index_put((torch.arange(n - 3, n)[:, None], torch.arange(n - 3, n)[None, :]), sR)
    M = E * torch.eye(n, dtype=torch.complex128) - Hfull - Sfull
    G = torch.linalg.inv(M)
    G1N = G[:3, n - 3:]
    gl = 1j * (sL - sL.conj().T)
    gr = 1j * (sR - sR.conj().T)
    T = torch.real(torch.trace(gl @ G1N @ gr @ G1N.conj().T))
    T.backward()
    for k, v in Hs.items():
        assert rel(gH[k], v.grad.numpy()) < 1e-10, k
    assert rel(gSL, sL.grad.numpy()) < 1e-10
    assert rel(gSR, sR.grad.numpy()) < 1e-10


def test_paper_flop_count_normaliser():
    # 4 GEMM + 1 LU + 3 GETRS per block at large N: 58.67 b^3 real flops
    f = O.rgf_flops_paper([64] * 1000, 1) / 1000 / 64 ** 3
    assert abs(f - (32 + 8 / 3 + 24)) < 0.2


@pytest.mark.parametrize("w", [1, 2])
def test_band_diag_residual_zero_for_exact_band_and_closed_form_for_a_perturbation(w):
    # exact band (dense LAPACK inverse): residual at rounding level
    prob = make_problem(7, b=None, size_range=(2, 6), w=w, n_energies=1, eta=1e-2, seed=90 + w)
    E = prob.energies[0]
    M = O.system_blocks(prob, E)
    ref = O.dense_selected(M, prob.sizes, w)["band"]
    assert O.band_diag_residual(M, prob.sizes, w, ref) < 1e-13
    nb = float(sum(prob.sizes))
    delta = 1e-3
    # G_kk += delta e_1 e_1^T enters only R_k, through M_kk's first column
    k = 3
    band = {key: v.copy() for key, v in ref.items()}
    band[(k, k)][0, 0] += delta
    expect = delta * np.linalg.norm(M[(k, k)][:, 0]) / np.sqrt(nb)
    assert abs(O.band_diag_residual(M, prob.sizes, w, band) - expect) < 1e-6 * expect
    # G_{k,k+w} += delta e_1 e_1^T enters only R_{k+w}, through M_{k+w,k}
    band = {key: v.copy() for key, v in ref.items()}
    band[(k, k + w)][0, 0] += delta
    expect = delta * np.linalg.norm(M[(k + w, k)][:, 0]) / np.sqrt(nb)
    assert abs(O.band_diag_residual(M, prob.sizes, w, band) - expect) < 1e-6 * expect


def _random_sigma_less(rng, b):
    # a layer-local lesser self-energy: i * (positive semidefinite)
    A = rng.normal(size=(b, b)) + 1j * rng.normal(size=(b, b))
    return 1j * (A @ A.conj().T) / b


@pytest.mark.parametrize("N", [1, 2, 5, 8])
def test_recursive_lesser_equals_dense_keldysh_equation(N):
    rng = np.random.default_rng(100 + N)
    prob = make_problem(N, b=None, size_range=(2, 6), w=1, n_energies=1, eta=1e-2, seed=100 + N)
    M = O.system_blocks(prob, prob.energies[0])
    sl = {0: _random_sigma_less(rng, prob.sizes[0]), N - 1: _random_sigma_less(rng, prob.sizes[-1])}
    if N > 2:
        sl[N // 2] = _random_sigma_less(rng, prob.sizes[N // 2])
    if N == 1:
        sl = {0: _random_sigma_less(rng, prob.sizes[0])}
    ref = O.lesser_dense(M, prob.sizes, 1, sl)
    got, _ = O.rgf_lesser(M, prob.sizes, sl)
    for k, v in ref.items():
        assert np.linalg.norm(got[k] - v) <= 1e-12 * max(1.0, np.linalg.norm(v)), k


def test_lesser_equilibrium_fluctuation_dissipation():
    # all reservoirs at one occupation f (leads and the eta broadening):
    # Sigma^< = i f (Gamma_L + Gamma_R + 2 eta I)  =>  G^< = -f (G^R - G^A)
    prob = make_problem(7, b=5, w=1, n_energies=1, eta=3e-2, seed=110)
    E = prob.energies[0]
    eta = E.imag
    rng = np.random.default_rng(111)
    prob.sigma_L = -0.4j * np.eye(5) + 0.1 * (rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5)))
    prob.sigma_L = 0.5 * (prob.sigma_L + prob.sigma_L.T)            # any Sigma^R with Gamma >= 0 works
    prob.sigma_R = -0.7j * np.eye(5)
    f = 0.37
    M = O.system_blocks(prob, E)
    gL, gR = O.gamma(prob.sigma_L), O.gamma(prob.sigma_R)
    sl = {i: 1j * f * 2 * eta * np.eye(5) for i in range(7)}
    sl[0] = sl[0] + 1j * f * gL
    sl[6] = sl[6] + 1j * f * gR
    GL, GR = O.rgf_lesser(M, prob.sizes, sl)
    for (a, b), v in GL.items():
        expect = -f * (GR[(a, b)] - GR[(b, a)].conj().T)
        assert np.linalg.norm(v - expect) < 1e-12 * np.linalg.norm(expect), (a, b)


def test_lesser_is_anti_hermitian_and_single_lead_form():
    # one lead: G^<_ii = i f G^R_{i1} Gamma_L (G^R_{i1})^H (first block column)
    prob = make_problem(6, b=4, w=1, n_energies=1, eta=1e-2, seed=112)
    M = O.system_blocks(prob, prob.energies[0])
    f = 0.8
    gL = O.gamma(prob.sigma_L)
    GL, _ = O.rgf_lesser(M, prob.sizes, {0: 1j * f * gL})
    G = O.dense_inverse(M, prob.sizes)
    for i in range(6):
        assert np.linalg.norm(GL[(i, i)] + GL[(i, i)].conj().T) < 1e-13 * np.linalg.norm(GL[(i, i)])
        c = G[4 * i:4 * i + 4, 0:4]
        assert np.linalg.norm(GL[(i, i)] - 1j * f * c @ gL @ c.conj().T) < 1e-12 * np.linalg.norm(GL[(i, i)])


def _golden_counts():
    import os
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_op_counts.txt")
    rows = []
    for line in open(p):
        if line.strip() and not line.startswith("#"):
            rows.append(tuple(int(x) for x in line.split()))
    return rows


@pytest.mark.parametrize("row", _golden_counts())
def test_op_counts_at_the_papers_experiment_sizes(row):
    # the oracle's counters (incremented by the LU / GETRS / GEMM calls it
    # makes) against the counts the paper prints, at its experiment sizes
    ell, w, lu, getrs, gemm = row
    sizes = [1] * ell
    M = random_band_matrix(sizes, w, seed=2, diag_shift=3.0)
    ops = O.OpCount()
    O.rgf_selected(M, sizes, w, ops=ops)
    assert (ops.lu, ops.getrs, ops.gemm) == (lu, getrs, gemm)
