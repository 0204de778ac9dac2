"""Host layout helpers of the n-diagonal Keldysh route (pure block copies, no
arithmetic): fuse_band / unfuse_band against the oracle's block fusing
(Sec. 2.3), on CPU tensors."""
import numpy as np
import pytest

from oracle import rgf as O
from workloads import make_problem


@pytest.mark.parametrize("N,w", [(7, 2), (8, 2), (3, 2), (10, 3), (5, 1)])
def test_fuse_band_matches_oracle_fusing_and_round_trips(N, w):
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2605_19910_gb300 as P
    prob = make_problem(N, b=None, size_range=(2, 6), w=w, n_energies=1, eta=1e-2, seed=10 * N + w)
    vec = torch.tensor(P.pack_band(prob.H, prob.sizes, w))
    fvec, fs = P.fuse_band(vec, prob.sizes, w)
    Mf, fsz, _ = O.fuse_blocks({k: np.asarray(v) for k, v in prob.H.items()}, prob.sizes, w)
    assert fs == fsz
    got = P.unpack_band(fvec.numpy(), fs, 1)
    for k, v in got.items():
        ref = Mf.get(k)
        if ref is None:
            assert not np.abs(v).any(), k
        else:
            assert np.array_equal(v, ref), k
    back = P.unfuse_band(fvec, prob.sizes, w)
    assert torch.equal(back, vec)
    # a batch of bands (energies first) round-trips too
    stack = torch.stack([vec, 2 * vec, -vec])
    fb, _ = P.fuse_band(stack, prob.sizes, w)
    assert torch.equal(P.unfuse_band(fb, prob.sizes, w), stack)
