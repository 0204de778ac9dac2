"""Energies in several workspace chunks (NEGF_WORKSPACE_GB caps the plan's
workspace): every path gives the results of a single-chunk plan."""
import os

import numpy as np
import pytest

from gpu_parity import to_dev
from workloads import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_2605_19910_gb300 as P
    return P


def _plan(P, small, *args, **kw):
    if small:
        os.environ["NEGF_WORKSPACE_GB"] = "1e-9"      # one energy per chunk
    try:
        return P.Plan(*args, **kw)
    finally:
        os.environ.pop("NEGF_WORKSPACE_GB", None)


def _close(a, b, tol):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.linalg.norm(a - b) <= tol * max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("precision,refine", [("fp64", 0), ("mixed", 1)])
def test_solve_and_transmission_in_chunks(P, precision, refine):
    import torch
    prob = make_problem(6, b=12, w=1, n_energies=5, eta=1e-3, seed=150)
    Hp, sL, sR, E = to_dev(prob, torch)
    res = []
    for small in (False, True):
        plan = _plan(P, small, prob.sizes, 3, 5, precision=precision, refine_steps=refine,
                     outputs=P.NEGF_OUT_BAND | P.NEGF_OUT_G1N | P.NEGF_OUT_TRANSMISSION)
        Gb, G1 = plan.solve(Hp, sL, sR, E)
        T = plan.transmission(Hp, sL, sR, E)
        res.append((Gb.clone(), G1.clone(), T.clone(), P.negf_workspace_bytes(plan.handle)))
        plan.close()
    assert res[1][3] < res[0][3]
    for k in range(3):
        assert _close(res[1][k], res[0][k], 1e-14)


@pytest.mark.parametrize("ck", [0, 2])
def test_gradient_in_chunks(P, ck):
    import torch
    prob = make_problem(7, b=6, w=1, n_energies=4, eta=1e-3, seed=151)
    Hp, sL, sR, E = to_dev(prob, torch)
    w = torch.tensor([0.5, -1.0, 2.0, 0.25], dtype=torch.float64, device="cuda")
    res = []
    for small in (False, True):
        plan = _plan(P, small, prob.sizes, 3, 4, outputs=P.NEGF_OUT_TRANSMISSION | P.NEGF_OUT_GRAD,
                     checkpoint_every=ck)
        T, dH, dSL, dSR = plan.grad(Hp, sL, sR, E, w)
        res.append((T.clone(), dH.clone(), dSL.clone(), dSR.clone()))
        plan.close()
    for k in range(4):
        assert _close(res[1][k], res[0][k], 1e-13)


def test_lesser_and_ddrgf_in_chunks(P):
    import torch
    prob = make_problem(12, b=8, w=1, n_energies=3, eta=1e-3, seed=152, diag_shift=4.0)
    Hp, sL, sR, E = to_dev(prob, torch)
    sl = 1j * torch.eye(8, dtype=torch.complex128, device="cuda")
    out = []
    for small in (False, True):
        lp = _plan(P, small, prob.sizes, 3, 3, outputs=P.NEGF_OUT_BAND | P.NEGF_OUT_LESSER)
        Gb, Gl = lp.lesser(Hp, sL, sR, E, sl, 0 * sl)
        lp.close()
        dp = _plan(P, small, prob.sizes, 3, 3, n_domains=3)
        Gd, _ = dp.solve(Hp, sL, sR, E)
        dp.close()
        out.append((Gb.clone(), Gl.clone(), Gd.clone()))
    for k in range(3):
        assert _close(out[1][k], out[0][k], 1e-13)
