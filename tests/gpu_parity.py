"""Shared helpers of the GPU parity tests: run the CUDA path through the C-ABI
binding and compare with the oracle, per energy and per output kind, by the
relative Frobenius error ||X_gpu - X_ref||_F / ||X_ref||_F."""
import numpy as np

FP64_TOL = 1e-11      # relative Frobenius error per result, FP64 path
MIXED_TOL = 1e-5      # relative Frobenius error per result, mixed path


def to_dev(prob, torch, per_energy_sigma=False):
    import paper_2605_19910_gb300 as P
    Hp = torch.tensor(P.pack_band(prob.H, prob.sizes, prob.w), device="cuda")
    if per_energy_sigma:
        nE = len(prob.energies)
        sL = torch.tensor(np.stack([prob.sigma_L] * nE), device="cuda")
        sR = torch.tensor(np.stack([prob.sigma_R] * nE), device="cuda")
    else:
        sL = torch.tensor(prob.sigma_L, device="cuda")
        sR = torch.tensor(prob.sigma_R, device="cuda")
    E = torch.tensor(prob.energies, device="cuda")
    return Hp, sL, sR, E


def band_rel_err(got_vec, ref_band, sizes, w):
    import paper_2605_19910_gb300 as P
    got = P.unpack_band(got_vec, sizes, w)
    num = sum(np.linalg.norm(got[k] - v) ** 2 for k, v in ref_band.items())
    den = sum(np.linalg.norm(v) ** 2 for v in ref_band.values())
    return float(np.sqrt(num / den))


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
