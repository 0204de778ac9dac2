"""CPU complex128 oracle for block n-diagonal selected inversion (RGF / DDRGF).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module.  The CUDA library never
calls it, and it shares no code with the CUDA library: it uses numpy/scipy
(LAPACK) primitives only, in complex128.

Notation follows the paper (di Napoli, Pecchia, Ramirez-Hidalgo, "Revisiting
recursive methods for Dyson and Keldysh in NEGF: Part I"):

* Sec. 2: ``M = E I - H - Sigma^R``; the Dyson problem is ``bndiag(M^{-1})``.
* Sec. 2.2, Alg. 1 and Eqs. (2x2_exact_RGF), (4x4_exact_RGF): block
  tridiagonal RGF (upward Schur sweep, downward pass).
* Sec. 2.3, Prop. 3 and the prose after it: block n-diagonal RGF with
  half-bandwidth ``w = (n-1)/2``, cost model Eq. (cost_model_general_RGF).
* Sec. 3, Eqs. (2x2_explicit_inverse_parallel_DDRGF),
  (Schur_complement_in_parallel_DDRGF), Prop. 4 and Alg. 2: DDRGF.

Functions with no exact pin say so in their docstring ("parity unpinned");
every function here is pinned by ``tests/test_oracle_*.py``.

Layers are 0-based in code (layer ``i`` here is layer ``i+1`` in the paper).
Block matrices are dicts ``{(a, b): ndarray}`` holding the nonzero blocks.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


# --------------------------------------------------------------------------
# Operation counters (Sec. 2.2 cost model: LU, GETRS, GEMM)
# --------------------------------------------------------------------------
class OpCount:
    """Counts the three kernels of the paper's cost model (Sec. 2.2)."""

    def __init__(self):
        self.lu = 0
        self.getrs = 0
        self.gemm = 0

    def as_tuple(self):
        return (self.lu, self.getrs, self.gemm)


class _NoCount(OpCount):
    pass


def _lu(A, ops):
    ops.lu += 1
    return sla.lu_factor(A, check_finite=False)


def _getrs_left(lu, B, ops):
    """``(LU)^{-1} B`` (a GETRS)."""
    ops.getrs += 1
    return sla.lu_solve(lu, B, check_finite=False)


def _getrs_right(lu, B, ops):
    """``B (LU)^{-1}``, solved as ``(LU)^{-T} B^T`` (a GETRS)."""
    ops.getrs += 1
    return sla.lu_solve(lu, B.T, trans=1, check_finite=False).T


def _gemm(A, B, ops):
    ops.gemm += 1
    return A @ B


# --------------------------------------------------------------------------
# Step a1: assembling M = E I - H - Sigma (Sec. 2, first paragraph)
# --------------------------------------------------------------------------
def system_blocks(prob, E, sigma_L=None, sigma_R=None):
    """Band blocks of ``M(E) = E I - H - Sigma^R``.

    ``Sigma^R`` acts on the first and last layer only (lead self-energies).
    ``E`` is complex (``E_r + i eta``).
    """
    sL = prob.sigma_L if sigma_L is None else sigma_L
    sR = prob.sigma_R if sigma_R is None else sigma_R
    N = prob.n_blocks
    M = {}
    for (a, b), h in prob.H.items():
        M[(a, b)] = -h.astype(np.complex128)
        if a == b:
            M[(a, b)] = M[(a, b)] + E * np.eye(prob.sizes[a], dtype=np.complex128)
    M[(0, 0)] = M[(0, 0)] - sL
    M[(N - 1, N - 1)] = M[(N - 1, N - 1)] - sR
    return M


def dense_from_blocks(M, sizes):
    """Assemble the full matrix from its nonzero blocks."""
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    n = int(off[-1])
    A = np.zeros((n, n), dtype=np.complex128)
    for (a, b), blk in M.items():
        A[off[a]:off[a + 1], off[b]:off[b + 1]] = blk
    return A


def blocks_from_dense(G, sizes, pairs):
    """Extract the blocks ``(a, b)`` in ``pairs`` from a full matrix."""
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    return {(a, b): G[off[a]:off[a + 1], off[b]:off[b + 1]].copy() for (a, b) in pairs}


def band_pairs(N, w):
    return [(a, b) for a in range(N) for b in range(max(0, a - w), min(N, a + w + 1))]


# --------------------------------------------------------------------------
# Dense reference: the plain definition bndiag(M^{-1}) (Sec. 2)
# --------------------------------------------------------------------------
def dense_inverse(M, sizes):
    """Full ``M^{-1}`` by LAPACK LU with partial pivoting (``zgesv``)."""
    A = dense_from_blocks(M, sizes)
    return np.linalg.inv(A)


def dense_selected(M, sizes, w):
    """``bndiag(M^{-1})`` from the dense inverse, plus ``G_{1N}``, the first
    block row and the last block column (all as dicts of blocks)."""
    N = len(sizes)
    G = dense_inverse(M, sizes)
    band = blocks_from_dense(G, sizes, band_pairs(N, w))
    row = blocks_from_dense(G, sizes, [(0, j) for j in range(N)])
    col = blocks_from_dense(G, sizes, [(i, N - 1) for i in range(N)])
    return dict(band=band, G1N=row[(0, N - 1)], first_row=row, last_col=col, full=G)


# --------------------------------------------------------------------------
# Block n-diagonal RGF (Alg. 1 for w = 1; Sec. 2.3 for general w)
# --------------------------------------------------------------------------
def rgf_selected(M, sizes, w, ops=None, first_row=False):
    """``bndiag(M^{-1})`` by the recursive Green's function method.

    Upward pass (Alg. 1 upward loop; Prop. 1 / Prop. 3): layers are eliminated
    from the last one to the first.  Eliminating layer ``i`` factors
    ``S_ii`` (LU), forms the multipliers ``X_{i,c} = t_i S_{i,c}`` and
    ``Y_{c,i} = S_{c,i} t_i`` for the ``m = min(w, i)`` layers
    ``c in [i-w, i-1]`` (``2m`` GETRS), and updates the ``m x m`` trailing
    window ``S_ab -= S_ai X_ib`` (``m^2`` GEMMs), where ``t_i = S_ii^{-1}``.

    Downward pass (Alg. 1 downward loop; Eq. 2x2_exact_RGF; the prose after
    Prop. 3): ``G_11 = t_1``; for ``i = 2..N`` with ``c`` over the ``m``
    previous layers,
    ``G_{a,i} = -sum_c G_{a,c} Y_{c,i}`` and ``G_{i,b} = -sum_c X_{i,c} G_{c,b}``
    for ``a, b`` in the window (``2 m^2`` GEMMs), then
    ``G_ii = t_i - sum_c X_{i,c} G_{c,i}`` (1 GETRS, ``m`` GEMMs).

    With ``first_row=True`` the first block row ``G_{1,j}`` is also produced
    by the same downward relation restricted to row 1 (Eq. 4x4_exact_RGF:
    ``G_{1,j} = -sum_c G_{1,c} Y_{c,j}``); its last entry is ``G_{1N}``.
    These chain GEMMs are not counted in ``ops``.

    Returns ``dict(band=..., t=..., X=..., Y=..., G1N=..., first_row=...)``.
    """
    ops = _NoCount() if ops is None else ops
    N = len(sizes)
    S = {k: v.copy() for k, v in M.items()}
    lu, X, Y = {}, {}, {}
    for i in range(N - 1, -1, -1):
        lu[i] = _lu(S[(i, i)], ops)
        nb = list(range(max(0, i - w), i))
        for c in nb:
            X[(i, c)] = _getrs_left(lu[i], S[(i, c)], ops)
            Y[(c, i)] = _getrs_right(lu[i], S[(c, i)], ops)
        for a in nb:
            for b in nb:
                S[(a, b)] = S[(a, b)] - _gemm(S[(a, i)], X[(i, b)], ops)
    G = {}
    t = {}
    eye0 = np.eye(sizes[0], dtype=np.complex128)
    t[0] = _getrs_left(lu[0], eye0, ops)
    G[(0, 0)] = t[0]
    row = {(0, 0): G[(0, 0)]} if first_row else None
    for i in range(1, N):
        nb = list(range(max(0, i - w), i))
        for a in nb:
            acc = None
            for c in nb:
                p = _gemm(G[(a, c)], Y[(c, i)], ops)
                acc = p if acc is None else acc + p
            G[(a, i)] = -acc
        for b in nb:
            acc = None
            for c in nb:
                p = _gemm(X[(i, c)], G[(c, b)], ops)
                acc = p if acc is None else acc + p
            G[(i, b)] = -acc
        t[i] = _getrs_left(lu[i], np.eye(sizes[i], dtype=np.complex128), ops)
        acc = t[i]
        for c in nb:
            acc = acc - _gemm(X[(i, c)], G[(c, i)], ops)
        G[(i, i)] = acc
        if first_row and i >= 1:
            acc = None
            for c in nb:
                p = row[(0, c)] @ Y[(c, i)]
                acc = p if acc is None else acc + p
            row[(0, i)] = -acc
    out = dict(band=G, t=t, X=X, Y=Y)
    if first_row:
        out["first_row"] = row
        out["G1N"] = row[(0, N - 1)]
    return out


def reversed_transposed(M, sizes):
    """``M' = J M^T J`` with ``J`` the block reversal: ``M'_{a,b} =
    (M_{N-1-b, N-1-a})^T``.  Then ``(M')^{-1} = J (M^{-1})^T J``, so the first
    block row of ``(M')^{-1}`` is the transposed, reversed last block column of
    ``M^{-1}``."""
    N = len(sizes)
    Mr = {}
    for (a, b), blk in M.items():
        Mr[(N - 1 - b, N - 1 - a)] = blk.T.copy()
    return Mr, list(reversed(sizes))


def rgf_last_column(M, sizes, w):
    """Last block column ``G_{a,N}`` of ``M^{-1}`` from the first block row of
    the reversed-transposed system (see :func:`reversed_transposed`)."""
    N = len(sizes)
    Mr, sr = reversed_transposed(M, sizes)
    res = rgf_selected(Mr, sr, w, first_row=True)
    return {(N - 1 - j, N - 1): res["first_row"][(0, j)].T.copy() for j in range(N)}


# --------------------------------------------------------------------------
# Block fusing (Sec. 2.3, Eq. cost_model_general_RGF_fused)
# --------------------------------------------------------------------------
def fuse_blocks(M, sizes, w):
    """Group ``w`` consecutive layers into one super-layer, which turns a block
    ``(2w+1)``-diagonal matrix into a block tridiagonal one (Sec. 2.3,
    "blocks fusing").  Returns ``(Mf, sizes_f, groups)``."""
    N = len(sizes)
    groups = [list(range(g, min(N, g + w))) for g in range(0, N, w)]
    sizes_f = [sum(sizes[i] for i in g) for g in groups]
    loc = {}
    for gi, g in enumerate(groups):
        o = 0
        for i in g:
            loc[i] = (gi, o)
            o += sizes[i]
    Mf = {}
    for (a, b), blk in M.items():
        ga, oa = loc[a]
        gb, ob = loc[b]
        if (ga, gb) not in Mf:
            Mf[(ga, gb)] = np.zeros((sizes_f[ga], sizes_f[gb]), np.complex128)
        Mf[(ga, gb)][oa:oa + sizes[a], ob:ob + sizes[b]] = blk
    return Mf, sizes_f, groups


# --------------------------------------------------------------------------
# DDRGF, single level (Sec. 3, Alg. 2)
# --------------------------------------------------------------------------
def ddrgf_layout(N, n_domains, w, first_blocks=None):
    """Domain layout of Fig. parallel_RGF_domains: the chain is cut into
    ``n_domains`` consecutive (D2, D1) pairs, D2 first and D1 last, with
    ``l1 = l2 = n_domains``.  Every separator D1 has ``s1 = w`` layers.
    ``first_blocks[j]`` is the first layer of pair ``j`` (default: equal
    split).  Returns a list of ``(d2_layers, d1_layers)``."""
    if first_blocks is None:
        first_blocks = [round(j * N / n_domains) for j in range(n_domains)]
    bounds = list(first_blocks) + [N]
    pairs = []
    for j in range(n_domains):
        lo, hi = bounds[j], bounds[j + 1]
        if hi - lo < w + 1:
            raise ValueError("domain too small for the separator width")
        pairs.append((list(range(lo, hi - w)), list(range(hi - w, hi))))
    return pairs


def ddrgf_selected(M, sizes, w, n_domains, first_blocks=None, return_parts=False, levels=()):
    """``bndiag(M^{-1})`` by DDRGF (Alg. 2), single level or recursive.

    Reordering ``T_hat = R T R^T`` (Eq. T_hat_overall_structure) puts the
    separator layers (D1) first and the interior sub-domain layers (D2)
    second.  Then, following Alg. 2:

    1. per sub-domain ``j`` of D2: ``X^(j) = (T_hat_22)_jj^{-1}`` (here by a
       dense inverse of the sub-domain; only its band and its first and last
       ``w`` block rows and columns are used, Sec. 3 "Data dependencies");
    2. ``T_S = T_hat_11 - T_hat_12 T_hat_22^{-1} T_hat_21``
       (Eq. Schur_complement_in_parallel_DDRGF);
    3. ``bndiag(T_S^{-1})`` on the separators grouped into super-layers
       (block tridiagonal at the sub-domain level, Prop. 4): by RGF, or, when
       ``levels`` is not empty, by DDRGF itself (Alg. 2 step 3, "recursive
       DDRGF"): the super-layer chain of ``T_S`` is cut into ``levels[0]``
       pairs of one-super-layer separators (``s_1 = 1``) and the next level
       uses ``levels[1:]``;
    4. the four parts of Eq. 2x2_explicit_inverse_parallel_DDRGF restricted
       to the band: ``G_11 = T_S^{-1}``, ``G_12 = -T_S^{-1} T_12 X``,
       ``G_21 = -X T_21 T_S^{-1}``, ``G_22 = X + X T_21 T_S^{-1} T_12 X``;
    5. inverse reordering (blocks are kept under their original layer labels).
    """
    N = len(sizes)
    pairs = ddrgf_layout(N, n_domains, w, first_blocks)
    D1 = [i for (_, sep) in pairs for i in sep]
    D2doms = [d for (d, _) in pairs]
    in_D1 = set(D1)

    def Mb(a, b):
        return M.get((a, b))

    # Step 1: per-domain inverses (dense inverse of the sub-domain matrix).
    Xs = []
    for dom in D2doms:
        sub = {(a - dom[0], b - dom[0]): M[(a, b)] for a in dom for b in dom if (a, b) in M}
        Gd = dense_inverse(sub, [sizes[i] for i in dom])
        off = np.concatenate([[0], np.cumsum([sizes[i] for i in dom])]).astype(int)
        X = {}
        for ia, a in enumerate(dom):
            for ib, b in enumerate(dom):
                X[(a, b)] = Gd[off[ia]:off[ia + 1], off[ib]:off[ib + 1]]
        Xs.append(X)
    dom_of = {}
    for j, dom in enumerate(D2doms):
        for i in dom:
            dom_of[i] = j

    # Step 2: T_S on the separator layers.
    TS = {}
    for s in D1:
        for s2 in D1:
            acc = None
            if (s, s2) in M:
                acc = M[(s, s2)].copy()
            for j, dom in enumerate(D2doms):
                X = Xs[j]
                cs = [c for c in dom if (s, c) in M]
                ds = [d for d in dom if (d, s2) in M]
                for c in cs:
                    for d in ds:
                        term = M[(s, c)] @ X[(c, d)] @ M[(d, s2)]
                        acc = -term if acc is None else acc - term
            if acc is not None:
                TS[(s, s2)] = acc

    # Step 3: bndiag(T_S^{-1}) at super-layer level (one super-layer per
    # separator) by block tridiagonal RGF.
    seps = [sep for (_, sep) in pairs]
    sp_sizes = [sum(sizes[i] for i in sep) for sep in seps]
    loc = {}
    for g, sep in enumerate(seps):
        o = 0
        for i in sep:
            loc[i] = (g, o)
            o += sizes[i]
    TSf = {}
    for (a, b), blk in TS.items():
        ga, oa = loc[a]
        gb, ob = loc[b]
        if abs(ga - gb) > 1:
            raise AssertionError("T_S is not block tridiagonal at separator level")
        if (ga, gb) not in TSf:
            TSf[(ga, gb)] = np.zeros((sp_sizes[ga], sp_sizes[gb]), np.complex128)
        TSf[(ga, gb)][oa:oa + sizes[a], ob:ob + sizes[b]] = blk
    for g in range(len(seps)):
        for h in (g - 1, g + 1):
            if 0 <= h < len(seps) and (g, h) not in TSf:
                TSf[(g, h)] = np.zeros((sp_sizes[g], sp_sizes[h]), np.complex128)
    if levels:
        GS_f = ddrgf_selected(TSf, sp_sizes, 1, levels[0], levels=tuple(levels[1:]))["band"]
    else:
        GS_f = rgf_selected(TSf, sp_sizes, 1)["band"]

    def GS(s, s2):
        ga, oa = loc[s]
        gb, ob = loc[s2]
        blk = GS_f.get((ga, gb))
        if blk is None:
            return None
        return blk[oa:oa + sizes[s], ob:ob + sizes[s2]]

    # Step 4: stitching, restricted to the band of the original ordering.
    G = {}
    for (a, b) in band_pairs(N, w):
        if a in in_D1 and b in in_D1:
            G[(a, b)] = GS(a, b).copy()
            continue
        if a not in in_D1 and b in in_D1:
            # G_21 = -X T_21 T_S^{-1}
            X = Xs[dom_of[a]]
            acc = np.zeros((sizes[a], sizes[b]), np.complex128)
            for (c, s), m in M.items():
                if c not in in_D1 and s in in_D1 and dom_of[c] == dom_of[a]:
                    g = GS(s, b)
                    if g is not None:
                        acc -= X[(a, c)] @ m @ g
            G[(a, b)] = acc
            continue
        if a in in_D1 and b not in in_D1:
            # G_12 = -T_S^{-1} T_12 X
            X = Xs[dom_of[b]]
            acc = np.zeros((sizes[a], sizes[b]), np.complex128)
            for (s, c), m in M.items():
                if s in in_D1 and c not in in_D1 and dom_of[c] == dom_of[b]:
                    g = GS(a, s)
                    if g is not None:
                        acc -= g @ m @ X[(c, b)]
            G[(a, b)] = acc
            continue
        # both in D2: same sub-domain when |a-b| <= w (separators are w wide)
        ja, jb = dom_of[a], dom_of[b]
        assert ja == jb
        X = Xs[ja]
        acc = X[(a, b)].copy()
        lefts = [(c, s, m) for (c, s), m in M.items()
                 if c not in in_D1 and dom_of[c] == ja and s in in_D1]
        rights = [(s, d, m) for (s, d), m in M.items()
                  if d not in in_D1 and dom_of[d] == ja and s in in_D1]
        for (c, s, m1) in lefts:
            W = X[(a, c)] @ m1
            for (s2, d, m2) in rights:
                g = GS(s, s2)
                if g is not None:
                    acc += W @ g @ m2 @ X[(d, b)]
        G[(a, b)] = acc
    if return_parts:
        return dict(band=G, TS=TS, pairs=pairs, X=Xs)
    return dict(band=G)


# --------------------------------------------------------------------------
# Transmission and its gradient (not in the paper; standard NEGF definitions)
# --------------------------------------------------------------------------
def gamma(sigma):
    """Broadening ``Gamma = i (Sigma - Sigma^H)``."""
    return 1j * (sigma - sigma.conj().T)


def transmission(G1N, sigma_L, sigma_R):
    """``T(E) = Tr[Gamma_L G_1N Gamma_R G_1N^H]`` (real up to rounding)."""
    gL, gR = gamma(sigma_L), gamma(sigma_R)
    return float(np.real(np.trace(gL @ G1N @ gR @ G1N.conj().T)))


def transmission_grad(first_row, last_col, band_pairs_list, sigma_L, sigma_R, N):
    """Gradient of ``T`` with respect to the band blocks of ``H`` and to the
    lead self-energies, in PyTorch's convention for a real function of complex
    inputs (``dT/dRe z + i dT/dIm z``).

    From ``dG = G dH G`` (``dM = -dH``):
    ``dT = 2 Re sum_ab Tr[X_ab dH_ab]`` with
    ``X_ab = G_{b,N} Gamma_R G_{1N}^H Gamma_L G_{1,a}``, so
    ``grad H_ab = 2 X_ab^H``.  ``Sigma_L`` also enters ``Gamma_L``:
    ``grad Sigma_L = 2 (X_11^H - i A)`` with ``A = G_1N Gamma_R G_1N^H``, and
    ``grad Sigma_R = 2 (X_NN^H - i B)`` with ``B = G_1N^H Gamma_L G_1N``.
    """
    gL, gR = gamma(sigma_L), gamma(sigma_R)
    G1N = first_row[(0, N - 1)]
    core = gR @ G1N.conj().T @ gL          # Gamma_R G_1N^H Gamma_L
    grads = {}
    for (a, b) in band_pairs_list:
        Xab = last_col[(b, N - 1)] @ core @ first_row[(0, a)]
        grads[(a, b)] = 2.0 * Xab.conj().T
    A = G1N @ gR @ G1N.conj().T
    B = G1N.conj().T @ gL @ G1N
    X11 = last_col[(0, N - 1)] @ core @ first_row[(0, 0)]
    XNN = last_col[(N - 1, N - 1)] @ core @ first_row[(0, N - 1)]
    gSL = 2.0 * (X11.conj().T - 1j * A)
    gSR = 2.0 * (XNN.conj().T - 1j * B)
    return grads, gSL, gSR


# --------------------------------------------------------------------------
# Convenience drivers over a Problem and an energy grid
# --------------------------------------------------------------------------
def solve_problem(prob, energies=None, method="rgf", n_domains=None, want=("band",)):
    """Run the oracle for every energy.  Returns a list of per-energy dicts
    with keys among ``band`` (dict of blocks), ``G1N``, ``T``."""
    Es = prob.energies if energies is None else energies
    out = []
    N = prob.n_blocks
    for E in Es:
        M = system_blocks(prob, E)
        if method == "rgf":
            r = rgf_selected(M, prob.sizes, prob.w, first_row=True)
        elif method == "dense":
            r = dense_selected(M, prob.sizes, prob.w)
        elif method == "ddrgf":
            r = ddrgf_selected(M, prob.sizes, prob.w, n_domains)
            r2 = rgf_selected(M, prob.sizes, prob.w, first_row=True)
            r["G1N"] = r2["G1N"]
        else:
            raise ValueError(method)
        res = {}
        if "band" in want:
            res["band"] = r["band"]
        res["G1N"] = r["G1N"]
        res["T"] = transmission(r["G1N"], prob.sigma_L, prob.sigma_R)
        out.append(res)
    return out


def rgf_flops_paper(sizes, w):
    """The paper's operation count (Sec. 2.2 / 2.3 cost model) converted to
    real flops with complex LU = 8/3 b^3, GETRS (b right-hand sides) = 8 b^3,
    GEMM = 8 b^3 (App. A), for a uniform block size ``b``."""
    N = len(sizes)
    b = float(np.mean(sizes))
    lu = N
    getrs = N * (2 * w + 1) - w * w - w
    gemm = (3 * w * w + w) * N - 2 * w ** 3 - 2 * w * w
    return (lu * 8.0 / 3.0 + getrs * 8.0 + gemm * 8.0) * b ** 3


def band_diag_residual(M, sizes, w, band):
    """A-posteriori check of a band of G = M^{-1} from band blocks alone: the
    diagonal blocks of M G - I, R_i = sum_{|c - i| <= w} M_{i,c} G_{c,i} - I
    (every block of M in row i meets only band blocks of G in column i), as
    ``sqrt(sum_i ||R_i||_F^2 / sum_i b_i)``.  Zero for the exact band."""
    N = len(sizes)
    num = 0.0
    for i in range(N):
        R = -np.eye(sizes[i], dtype=np.complex128)
        for c in range(max(0, i - w), min(N - 1, i + w) + 1):
            R = R + M[(i, c)] @ band[(c, i)]
        num += float(np.sum(np.abs(R) ** 2))
    return float(np.sqrt(num / float(sum(sizes))))


# --------------------------------------------------------------------------
# Keldysh equation G^< = G^R Sigma^< G^A (Sec. 1; the recursive solver is
# future work in the paper, Sec. 5)
# --------------------------------------------------------------------------
def lesser_dense(M, sizes, w, sigma_less):
    """The band of ``G^< = G^R Sigma^< G^A`` by its definition: ``G^R = M^{-1}``
    (dense LAPACK inverse), ``G^A = (G^R)^H`` and a layer-local lesser
    self-energy ``sigma_less = {layer: block}``.  Returns ``{(a, b): block}``
    for ``|a - b| <= w``."""
    N = len(sizes)
    G = dense_inverse(M, sizes)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    S = np.zeros_like(G)
    for i, blk in sigma_less.items():
        S[off[i]:off[i + 1], off[i]:off[i + 1]] = blk
    L = G @ S @ G.conj().T
    return blocks_from_dense(L, sizes, band_pairs(N, w))


def rgf_lesser(M, sizes, sigma_less):
    """Selected blocks of ``G^<`` for a block tridiagonal ``M`` by recursion
    over the factorisation of the upward sweep (Alg. 1; Eq.
    2x2_UDL_factorization applied layer by layer): ``M = U D L`` with
    ``U_{i,i+1} = M_{i,i+1} t_{i+1}``, ``D = diag(S_i)``,
    ``L_{i+1,i} = t_{i+1} M_{i+1,i}``, so that ``G^< = L^{-1} D^{-1} U^{-1}
    Sigma^< U^{-H} D^{-H} L^{-H}``.  With ``Q = U^{-1} Sigma^< U^{-H}``:

    * upward, ``i = N..1``: ``Q_ii = Sigma^<_i + M_{i,i+1} g^<_{i+1}
      M_{i,i+1}^H``, ``W_i = Q_ii t_i^H``, ``g^<_i = t_i W_i`` (the
      right-connected lesser function);
    * downward, ``G^<_11 = g^<_1`` and for ``i = 2..N``, with
      ``X_{i,i-1} = t_i M_{i,i-1}`` and ``A_i = G^R_{i-1,i} W_i``:
      ``G^<_{i,i-1} = -A_i^H - X_{i,i-1} G^<_{i-1,i-1}``,
      ``G^<_{i-1,i} = -(G^<_{i,i-1})^H``,
      ``G^<_ii = g^<_i - X_{i,i-1} A_i - G^<_{i,i-1} X_{i,i-1}^H``.

    The cross term uses ``(L^{-1} D^{-1} U^{-1})_{i-1,i} = G^R_{i-1,i}`` and
    the anti-Hermiticity of ``Sigma^<``.  Returns ``(lesser band, retarded
    band)`` (block tridiagonal only)."""
    N = len(sizes)
    r = rgf_selected(M, sizes, 1)
    GR = r["band"]
    t = [None] * N
    S = M[(N - 1, N - 1)].copy()
    for i in range(N - 1, -1, -1):
        t[i] = np.linalg.inv(S)
        if i > 0:
            S = M[(i - 1, i - 1)] - M[(i - 1, i)] @ t[i] @ M[(i, i - 1)]
    Wm = [None] * N
    gl = [None] * N
    for i in range(N - 1, -1, -1):
        Q = sigma_less.get(i, np.zeros((sizes[i], sizes[i]), complex)).astype(complex)
        if i < N - 1:
            Q = Q + M[(i, i + 1)] @ gl[i + 1] @ M[(i, i + 1)].conj().T
        Wm[i] = Q @ t[i].conj().T
        gl[i] = t[i] @ Wm[i]
    GL = {(0, 0): gl[0]}
    for i in range(1, N):
        X = t[i] @ M[(i, i - 1)]
        A = GR[(i - 1, i)] @ Wm[i]
        low = -A.conj().T - X @ GL[(i - 1, i - 1)]
        GL[(i, i - 1)] = low
        GL[(i - 1, i)] = -low.conj().T
        GL[(i, i)] = gl[i] - X @ A - low @ X.conj().T
    return GL, GR
