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


# A block whose norm is below this fraction of the band's root-mean-square
# block norm is measured against that floor instead of its own norm (the
# absolute floor of the per-result error definition, for blocks that are
# nearly zero).
BLOCK_FLOOR = 1e-3


def band_rel_err(got_vec, ref_band, sizes, w):
    """max(pooled, per-block) relative error of one energy's band: the pooled
    ratio sqrt(sum_k ||dG_k||^2 / sum_k ||G_k||^2) and, so that a wrong
    small-norm block cannot hide under the large ones, the largest
    ||dG_k||_F / max(||G_k||_F, BLOCK_FLOOR * rms_k ||G_k||_F) over blocks."""
    import paper_2605_19910_gb300 as P
    got = P.unpack_band(got_vec, sizes, w)
    d2 = {k: np.linalg.norm(got[k] - v) ** 2 for k, v in ref_band.items()}
    n2 = {k: np.linalg.norm(v) ** 2 for k, v in ref_band.items()}
    pooled = float(np.sqrt(sum(d2.values()) / sum(n2.values())))
    floor = BLOCK_FLOOR * np.sqrt(sum(n2.values()) / len(n2))
    per_block = max(float(np.sqrt(d2[k]) / max(np.sqrt(n2[k]), floor, 1e-300)) for k in d2)
    return max(pooled, per_block)


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
