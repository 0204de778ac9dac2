"""Seeded synthetic inputs for the NEGF selected-inversion path.

This module is shared by the oracle (``oracle/``) and the CUDA path's tests and
benchmark.  It only draws random numbers and lays out the problem description;
it performs none of the method's arithmetic (no Schur complements, no
inversions, no products of blocks).

Problem statement (Sec. 2, first paragraph): the matrix to invert is
``M = E I - H - Sigma^R`` where ``H`` is block n-diagonal over ``N`` principal
layers with half-bandwidth ``w = (n-1)/2`` (Sec. 2.3, Prop. 3).  The paper only
says its matrices are "diagonally-dominant synthetic matrices with underlying
random data" (Sec. 4.1); the recipe below replaces that:

* ``CN(0, 1/b)``: real and imaginary parts each ``N(0, 1/(2b))``.
* Draw order from one ``numpy.random.default_rng(seed)`` (PCG64): block sizes
  (only when they are drawn, ``rng.integers(lo, hi + 1)`` per layer), then the
  matrices ``A_i`` of every diagonal block, then the nearest-neighbour noise
  ``C_i`` for ``i = 1..N-1``, then the next-nearest noise ``D_i`` for
  ``i = 1..N-2`` (only when ``w >= 2``).
* ``H_ii = (A_i + A_i^H) / 2``; ``H_{i,i+1} = I + 0.1 C_i`` (``I`` is the
  rectangular identity when ``b_i != b_{i+1}``; the variance uses the row
  block size); ``H_{i+1,i} = H_{i,i+1}^H``; ``H_{i,i+2} = 0.3 D_i`` and
  ``H_{i+2,i} = H_{i,i+2}^H``.
* Lead self-energies ``Sigma_L = Sigma_R = -0.5i I`` on layers 1 and N only.
* Energies ``linspace(-2, 2, n_E) + i eta`` (or one given energy).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np


@dataclass
class Problem:
    """A block n-diagonal Hamiltonian with lead self-energies and energies.

    ``H[(i, j)]`` (0-based layers, ``|i - j| <= w``) is the dense block
    ``H_{ij}`` of shape ``(sizes[i], sizes[j])``, complex128.
    ``sigma_L`` / ``sigma_R`` are ``(b_1, b_1)`` / ``(b_N, b_N)`` complex128.
    ``energies`` is a complex128 vector (``E_r + i eta``).
    """
    sizes: list
    w: int
    H: dict
    sigma_L: np.ndarray
    sigma_R: np.ndarray
    energies: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_blocks(self) -> int:
        return len(self.sizes)


def cn(rng, shape, var):
    """Circular complex normal with total variance ``var``."""
    s = np.sqrt(var / 2.0)
    re = rng.normal(0.0, s, size=shape)
    im = rng.normal(0.0, s, size=shape)
    return re + 1j * im


def rect_identity(m, n):
    return np.eye(m, n, dtype=np.complex128)


def make_problem(n_blocks, b=None, w=1, n_energies=1, eta=1e-6, seed=0,
                 energy=None, size_range=None, coupling_noise=0.1,
                 next_coupling=0.3, sigma=-0.5j, diag_shift=0.0):
    """Build one synthetic nanowire-shaped problem.

    ``b``: uniform block size, or ``None`` with ``size_range=(lo, hi)`` for
    sizes drawn uniformly from ``{lo..hi}``.  ``energy``: a single complex
    energy (overrides the grid).  Returns a :class:`Problem`.
    """
    rng = np.random.default_rng(seed)
    if b is None:
        lo, hi = size_range
        sizes = [int(x) for x in rng.integers(lo, hi + 1, size=n_blocks)]
    else:
        sizes = [int(b)] * n_blocks
    N = n_blocks
    H = {}
    for i in range(N):
        A = cn(rng, (sizes[i], sizes[i]), 1.0 / sizes[i])
        H[(i, i)] = (A + A.conj().T) / 2.0 + diag_shift * np.eye(sizes[i])
    for i in range(N - 1):
        C = cn(rng, (sizes[i], sizes[i + 1]), 1.0 / sizes[i])
        H[(i, i + 1)] = rect_identity(sizes[i], sizes[i + 1]) + coupling_noise * C
        H[(i + 1, i)] = H[(i, i + 1)].conj().T.copy()
    if w >= 2:
        for i in range(N - 2):
            D = cn(rng, (sizes[i], sizes[i + 2]), 1.0 / sizes[i])
            H[(i, i + 2)] = next_coupling * D
            H[(i + 2, i)] = H[(i, i + 2)].conj().T.copy()
    for d in range(3, w + 1):   # wider bands: zero blocks keep the pattern complete
        for i in range(N - d):
            H[(i, i + d)] = np.zeros((sizes[i], sizes[i + d]), np.complex128)
            H[(i + d, i)] = np.zeros((sizes[i + d], sizes[i]), np.complex128)
    sigma_L = sigma * np.eye(sizes[0], dtype=np.complex128)
    sigma_R = sigma * np.eye(sizes[-1], dtype=np.complex128)
    if energy is not None:
        energies = np.array([complex(energy)], dtype=np.complex128)
    else:
        energies = (np.linspace(-2.0, 2.0, n_energies) + 1j * eta).astype(np.complex128)
    return Problem(sizes=sizes, w=w, H=H, sigma_L=sigma_L, sigma_R=sigma_R,
                   energies=energies, meta=dict(seed=seed, eta=eta))


def random_band_matrix(sizes, w, seed=0, diag_shift=0.0):
    """A general (non-Hermitian) block n-diagonal matrix ``M`` as a dict of
    blocks, for testing the inversion algorithms on inputs without the
    Hermitian structure of ``H``.  ``diag_shift`` adds ``shift * I`` to each
    diagonal block."""
    rng = np.random.default_rng(seed)
    N = len(sizes)
    M = {}
    for i in range(N):
        for j in range(max(0, i - w), min(N, i + w + 1)):
            M[(i, j)] = cn(rng, (sizes[i], sizes[j]), 1.0 / sizes[i])
            if i == j and diag_shift:
                M[(i, j)] = M[(i, j)] + diag_shift * np.eye(sizes[i])
    return M


def uniform_chain(n_blocks, b, eps, t, energies, channel_energies=None, seed=0):
    """Uniform 1D tight-binding chain: ``H_ii = eps I`` (or ``U diag(eps_c) U^H``
    for ``channel_energies``), ``H_{i,i+-1} = t I``; lead self-energies are left
    to the caller (zero here)."""
    sizes = [b] * n_blocks
    if channel_energies is None:
        Hd = eps * np.eye(b, dtype=np.complex128)
    else:
        rng = np.random.default_rng(seed)
        Q, _ = np.linalg.qr(cn(rng, (b, b), 1.0))
        Hd = (Q * np.asarray(channel_energies)) @ Q.conj().T
    H = {}
    for i in range(n_blocks):
        H[(i, i)] = Hd.copy()
    for i in range(n_blocks - 1):
        H[(i, i + 1)] = t * np.eye(b, dtype=np.complex128)
        H[(i + 1, i)] = t * np.eye(b, dtype=np.complex128)
    z = np.zeros((b, b), np.complex128)
    return Problem(sizes=sizes, w=1, H=H, sigma_L=z.copy(), sigma_R=z.copy(),
                   energies=np.asarray(energies, np.complex128))


# Named workloads (sizes as the method's benchmark cases use them).
def workload(name, **over):
    """Named synthetic workloads.

    * ``chain16x8``: plain RGF, 16 blocks x b=8, one energy 0.1+1e-6i.
    * ``batched64x64``: 64 blocks x b=64, 512 energies in [-2, 2], eta=1e-6.
    * ``penta256x32``: n=5, 256 blocks x b=32, 1024 energies, 8 DDRGF domains.
    * ``trans128x48``: 128 blocks x b=48, 256 energies (transmission + adjoint).
    * ``wire1024``: 1024 blocks, b uniform in {96..160}, 128 energies, 32 domains.
    """
    table = {
        "chain16x8": dict(n_blocks=16, b=8, w=1, energy=0.1 + 1e-6j),
        "batched64x64": dict(n_blocks=64, b=64, w=1, n_energies=512, eta=1e-6),
        "penta256x32": dict(n_blocks=256, b=32, w=2, n_energies=1024, eta=1e-6),
        "trans128x48": dict(n_blocks=128, b=48, w=1, n_energies=256, eta=1e-6),
        "wire1024": dict(n_blocks=1024, b=None, size_range=(96, 160), w=1,
                         n_energies=128, eta=1e-6),
    }
    kw = dict(table[name])
    kw.update(over)
    return make_problem(**kw)
