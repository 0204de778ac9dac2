#!/usr/bin/env python
"""Benchmark: selected-G^R energies x blocks per second on one GB300.

A step is one full selected inversion (upward Schur sweep, per-block
inversions, downward pass; on the mixed path G_1N from the last block column
after one step of iterative refinement) of the synthetic nanowire workload
"batched64x64": 64 blocks of b = 64, block tridiagonal, 512 energies in
[-2, 2] with eta = 1e-6, all energies in one call.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference    # the CPU oracle on the host cores

Under torchrun (N > 1) the job is one energy list of N x 512 energies in
[-2, 2]; rank r solves its contiguous share of it on its own GPU (weak
scaling: fixed work per GPU, every energy solved once, no collective on the
data path); rank 0 prints the line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "batched64x64"
METRIC = "selected-G^R energies x blocks / s"
UNIT = "energy-blocks/s"

# DRAM traffic per unit (one block inversion, one block product) of the
# dominant kernel from ncu captures, valid only while the kernel source is the
# one captured (the summaries and their commands are under profiles/)
NCU_TRAFFIC = {
    # two captured 2048-inversion launches, averaged
    ("zinv_gj_kernel", 64): {
        "bytes_per_unit": ((134.351616e6 + 77.448192e6) + (134.380288e6 + 75.228672e6)) / 2 / 2048,
        "unit": "inversion",
        "src": "paper_2605_19910_gb300/csrc/negf_inv.cu",
        "sha256": "09462f341c3b6e95daf7b0464414920056a154025187f824da62513ee57447b6",
    },
    # two captured 2048-product launches at 35 bits (one with a shared
    # coupling-block operand, one with two per-energy operands), averaged
    ("zgemm_tc_kernel", 64): {
        "bytes_per_unit": ((269.672192e6 + 98.240256e6) + (408.351232e6 + 102.905088e6)) / 2 / 2048,
        "unit": "block product",
        "src": "paper_2605_19910_gb300/csrc/negf_gemm_tc.cu",
        "sha256": "c97b4531aab19d8158d8640c74a7636a480541313ce7445c473f7c1193ed61cc",
    },
}

# Largest per-energy deviation from a 56-bit solve that negf_tune_precision
# accepts: a quarter of the mixed path's 1e-5 bar (the 56-bit solve is
# accurate to ~1e-10 here, so the deviation is the error itself)
TUNE_TOL = 2.5e-6

# Nominal GB300 FP64 rate at the 2070 MHz maximum SM clock (context only: the
# roofline of the FP64 kernels is taken against the rates negf_fp64_peak
# measures in this run, DFMA for the inversion, DMMA for the FP64 product)
FP64_NOMINAL_TFLOPS = 1.25


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-fp64-side", action="store_true",
                    help="skip the side measurement of the FP64 path")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-energies", type=int, default=512,
                    help="energies of the bounded CPU-oracle sample")
    ap.add_argument("--n-blocks", type=int, default=None, help="override the workload's block count")
    ap.add_argument("--n-energies", type=int, default=None, help="override the workload's energy count")
    ap.add_argument("--block-size", type=int, default=None, help="override the workload's block size")
    ap.add_argument("--product-bits", type=int, default=None,
                    help="bits of the tensor-core block products on the mixed path "
                         "(default: the library's default, narrowed by negf_tune_precision)")
    ap.add_argument("--no-tune-precision", action="store_true",
                    help="keep the plan's product width instead of negf_tune_precision's choice")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the plan's default energy-group count instead of negf_autotune's choice")
    ap.add_argument("--no-grad-side", action="store_true",
                    help="skip the side measurement of the adjoint (gradient) path")
    ap.add_argument("--no-lesser-side", action="store_true",
                    help="skip the side measurement of the Keldysh (G^<) path")
    ap.add_argument("--refine-steps", type=int, default=1,
                    help="refinement steps of the mixed plan's G_1N (the benchmark configuration has one)")
    ap.add_argument("--no-ddrgf-side", action="store_true",
                    help="skip the side measurement of DDRGF levels on a few-energy long chain")
    ap.add_argument("--n-domains", type=int, default=1,
                    help="DDRGF (D2, D1) pairs of the timed plan (1 = plain RGF, 0 = the cost model's choice)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# CPU oracle leg (the only place besides tests and smoke that runs oracle/)
# ---------------------------------------------------------------------------
def _oracle_worker(args):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    name, idx = args
    from oracle import rgf as O
    from workloads import workload
    prob = workload(name)
    t0 = time.perf_counter()
    for e in idx:
        E = prob.energies[e]
        O.rgf_selected(O.system_blocks(prob, E), prob.sizes, prob.w, first_row=True)
    return time.perf_counter() - t0


def oracle_sample(name, n_energies, pool, cores):
    from workloads import workload
    prob = workload(name)
    nE = len(prob.energies)
    n = min(n_energies, nE)
    picks = [int(round(i * (nE - 1) / max(n - 1, 1))) for i in range(n)]
    chunks = [picks[i::cores] for i in range(cores)]
    chunks = [c for c in chunks if c]
    t0 = time.perf_counter()
    pool.map(_oracle_worker, [(name, c) for c in chunks])
    wall = time.perf_counter() - t0
    units = n * prob.n_blocks
    return dict(value=units / wall, unit=UNIT, cores=len(chunks), kind="oracle",
                sample=f"{n} of {nE} energies x all {prob.n_blocks} blocks of {name} "
                       f"(oracle sequential RGF, complex128, numpy/LAPACK), {wall:.2f} s wall"), wall


def make_pool(cores):
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    ctx = mp.get_context("spawn")
    return ctx.Pool(cores)


# ---------------------------------------------------------------------------
# clocks sampler
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to NEGF_CLOCKS_DIR (default: the system temp dir);
        # the JSON line carries their summary
        import tempfile
        out_dir = os.environ.get("NEGF_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"negf_clocks_rank{index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
# ---------------------------------------------------------------------------
# multi-rank host logic (replicas over energies; no collective on the data path)
# ---------------------------------------------------------------------------
def job_energies(prob_energies, world):
    """The job's energy list for an N-rank run: N times the workload's count
    of energies over the same interval with the same eta (one problem whose
    energies are split over the ranks; N = 1 gives the workload's list)."""
    import numpy as np
    if world <= 1:
        return prob_energies
    n = len(prob_energies) * world
    re = prob_energies.real
    return (np.linspace(re.min(), re.max(), n) + 1j * prob_energies.imag[0]).astype(np.complex128)


def rank_energies(energies, rank, world):
    """Rank r's contiguous share of the job's energy list (energy_shard of the
    binding: the shares of all ranks concatenate to the list)."""
    import paper_2605_19910_gb300 as P
    lo, hi = P.energy_shard(len(energies), rank, world)
    return energies[lo:hi]


def max_over_ranks(ms, dist, device):
    """The slowest rank's time: the job ends when the last replica does."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, n_energies, n_blocks, ms):
    """Whole-job energy-blocks per second over all ranks: ``n_energies`` is
    one rank's share, each of the ``world`` ranks solves a disjoint share of
    the job's energy list, so every energy counts once."""
    return world * n_energies * n_blocks / (ms * 1e-3)


def measure_fp64_peaks(P, local_rank, stream):
    """FP64 FMA and FP64 MMA rates of this GPU (negf_fp64_peak: one kernel of
    independent dependency chains per kind, CUDA-event timed), each run for
    about 0.3 s after a short calibration, with the SM clock sampled during
    the runs; plus both kinds side by side (whether they share one unit)."""
    out = {}
    clocks = Clocks(local_rank)
    clocks.start()
    for key, kind in (("dfma_tflops", P.NEGF_PEAK_DFMA), ("dmma_tflops", P.NEGF_PEAK_DMMA),
                      ("dfma_plus_dmma_tflops", P.NEGF_PEAK_BOTH)):
        _, ms0 = P.negf_fp64_peak(kind, 2000, stream.cuda_stream)
        iters = max(2000, int(2000 * 300.0 / max(ms0, 1e-3)))
        best = 0.0
        for _ in range(3):
            tf, _ = P.negf_fp64_peak(kind, iters, stream.cuda_stream)
            best = max(best, tf)
        out[key] = best
    out["clocks"] = clocks.stop()
    out["how"] = ("negf_fp64_peak: 4 x 256-thread CTAs per SM, 8 independent chains per thread (DFMA) or "
                  "warp (DMMA m8n8k4), ~0.3 s per run, best of 3")
    return out


def _overrides(a):
    over = {}
    if a.n_blocks:
        over["n_blocks"] = a.n_blocks
    if a.n_energies:
        over["n_energies"] = a.n_energies
    if a.block_size:
        over["b"] = a.block_size
    return over


def run_ours(a, rank, world, local_rank):
    import numpy as np
    cores = os.cpu_count() or 1
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2605_19910_gb300 as P
    from workloads import make_problem, workload

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prob = workload(a.workload, **_overrides(a))
    prob.energies = rank_energies(job_energies(prob.energies, world), rank, world)
    N, nE = prob.n_blocks, len(prob.energies)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    Hh = torch.tensor(P.pack_band(prob.H, prob.sizes, prob.w)).pin_memory()
    sLh = torch.tensor(prob.sigma_L).pin_memory()
    sRh = torch.tensor(prob.sigma_R).pin_memory()
    Eh = torch.tensor(prob.energies).pin_memory()
    H, sL, sR, E = (x.to(dev) for x in (Hh, sLh, sRh, Eh))
    outputs = P.NEGF_OUT_BAND | P.NEGF_OUT_G1N | P.NEGF_OUT_TRANSMISSION
    bits = a.product_bits if (a.product_bits is not None and a.precision == "mixed") else 0
    refine = a.refine_steps if a.precision == "mixed" else 0
    plan = P.Plan(prob.sizes, 2 * prob.w + 1, nE, precision=a.precision, outputs=outputs, product_bits=bits,
                  refine_steps=refine, n_domains=a.n_domains)
    dd_plan = plan.n_domains > 1
    if dd_plan:
        refine = 0   # DDRGF plans take G_1N through the separators
    Gb = torch.empty(nE, plan.band_elems, dtype=torch.complex128, device=dev)
    G1 = torch.empty(nE, prob.sizes[0], prob.sizes[-1], dtype=torch.complex128, device=dev)

    def step():
        plan.solve(H, sL, sR, E, out_band=Gb, out_g1n=G1, sync=False)

    # product width: the narrowest whose results stay within TUNE_TOL of a
    # 56-bit solve of these inputs at every energy (negf_tune_precision; untimed)
    prec_tune = None
    if a.precision == "mixed" and a.product_bits is None and not a.no_tune_precision:
        tb, tdev = plan.tune_precision(H, sL, sR, E, tol=TUNE_TOL)
        prec_tune = {"product_bits": tb, "max_rel_deviation_from_56_bit": tdev, "tol": TUNE_TOL,
                     "candidates": list(P.TUNE_BITS)}
        bits = tb
    # energy-group autotuner on these inputs (untimed, before the warm-up)
    tune = None
    if not a.no_autotune and not dd_plan:   # DDRGF plans keep fixed stream sets
        best, tms = plan.autotune(H, sL, sR, E, out_band=Gb, out_g1n=G1)
        tune = {"energy_groups": best, "ms_per_solve_by_groups": {str(k): v for k, v in tms.items()},
                "tensor_core_tile_tmem_cols": P.negf_plan_tile_cols(plan.handle)}
    groups = P.negf_plan_groups(plan.handle)

    # per-kernel profile of one extra step (CUDA events around every launch on
    # its stream) with the plan set to one energy group, so that concurrent
    # launches of the groups do not inflate each other's durations (same
    # chunking, hence the same launch shapes, as the timed plan)
    if not dd_plan:
        P.negf_plan_set_groups(plan.handle, 1)
    P.negf_profile_enable(plan.handle, 1)
    for _ in range(2):                  # the second of two profiled steps
        plan.solve(H, sL, sR, E, out_band=Gb, out_g1n=G1, sync=False)
        prof_iss = P.negf_profile_read_issued(plan.handle)
    prof = {k: (v[0], v[1], v[3]) for k, v in prof_iss.items()}
    P.negf_profile_enable(plan.handle, 0)
    plan.sync()
    if not dd_plan:
        P.negf_plan_set_groups(plan.handle, groups)
    P.negf_profile_enable(plan.handle, 1)
    step()
    launches_per_step = int(sum(v[2] for v in P.negf_profile_read(plan.handle).values()))
    P.negf_profile_enable(plan.handle, 0)
    plan.sync()

    for _ in range(a.warmup):
        step()
    plan.sync()

    clocks = Clocks(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(a.steps):
        step()
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    st = plan.sync  # raises on any device-reported error
    st()
    ms = max_over_ranks(t_start.elapsed_time(t_end) / a.steps, dist, dev)
    value = job_throughput(world, nE, N, ms)

    # end to end through the public API, right after the timed solves (before
    # the host-side checks below): pinned host inputs -> device, solve,
    # selected blocks and G_1N back to pinned host memory, every step
    e2e = None
    if not a.no_e2e:
        # end to end through the C-ABI call with host buffers (negf_solve_host):
        # pinned host inputs copied in, the solve, the selected blocks and
        # G_1N copied back to pinned host memory, every step; the call
        # returns when the outputs are in host memory
        Gb_h = torch.empty(Gb.shape, dtype=Gb.dtype).pin_memory()
        G1_h = torch.empty(G1.shape, dtype=G1.dtype).pin_memory()
        info_h = torch.zeros(nE, dtype=torch.int32).pin_memory()

        def e2e_step():
            plan.solve_host(Hh, sLh, sRh, Eh, Gb_h, G1_h, info_h)

        # context: a plain device-to-host copy of the band into the same
        # page-locked buffer (the copy the call overlaps with its solve)
        torch.cuda.synchronize()
        tc0 = time.perf_counter()
        Gb_h.copy_(Gb, non_blocking=True)
        torch.cuda.synchronize()
        d2h_gbps = Gb.numel() * Gb.element_size() / (time.perf_counter() - tc0) / 1e9

        e2e_step()
        k2 = max(1, min(a.steps, 5))
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_ms = []
        for _ in range(k2):
            t1 = time.perf_counter()
            e2e_step()
            e2e_ms.append((time.perf_counter() - t1) * 1e3)
        ms2 = max_over_ranks((time.perf_counter() - t0) * 1e3 / k2, dist, dev)
        h2d = sum(x.numel() * x.element_size() for x in (Hh, sLh, sRh, Eh))
        d2h = (Gb_h.numel() * Gb_h.element_size() + G1_h.numel() * G1_h.element_size() +
               info_h.numel() * info_h.element_size())
        e2e = {"value": job_throughput(world, nE, N, ms2), "unit": UNIT, "ms_per_step": ms2,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "call": "negf_solve_host",
               "timer": "host wall clock around the synchronous call",
               "plain_d2h_copy_gbps": d2h_gbps, "ms_per_call": [round(t, 2) for t in e2e_ms],
               "ms_per_call_median": float(np.median(e2e_ms)),
               "note": "value from the mean call time; ms_per_call lists every call (on some runs an "
                       "occasional call takes ~2x, cause not identified); plain_d2h_copy_gbps: this "
                       "run's plain copy rate of the band, the copy the call overlaps with its solve"}
        del Gb_h, G1_h

    fp64 = measure_fp64_peaks(P, local_rank, stream)

    # sampled parity against the oracle (two energies) for the rel-err report:
    # the band and G_1N (from the refined last column when refine_steps = 1)
    rel = None
    if rank == 0:
        from oracle import rgf as O
        errs, errs1 = [], []
        for e in (0, nE // 2):
            ref = O.rgf_selected(O.system_blocks(prob, prob.energies[e]), prob.sizes, prob.w, first_row=True)
            got = P.unpack_band(Gb[e].cpu().numpy(), prob.sizes, prob.w)
            num = sum(np.linalg.norm(got[k] - v) ** 2 for k, v in ref["band"].items())
            den = sum(np.linalg.norm(v) ** 2 for v in ref["band"].values())
            errs.append(float(np.sqrt(num / den)))
            g1 = G1[e].cpu().numpy()
            errs1.append(float(np.linalg.norm(g1 - ref["G1N"]) / np.linalg.norm(ref["G1N"])))
        rel = {"band": max(errs), "G1N": max(errs1), "energies": [0, nE // 2],
               "G1N_refined": bool(refine)}

    # a-posteriori check of every energy's band from the band alone:
    # sqrt(sum_i ||(M G)_ii - I||_F^2 / sum_i b_i) (negf_band_residual)
    res = plan.band_residual(H, sL, sR, E, Gb).cpu().numpy()
    band_residual = {"median": float(np.median(res)), "max": float(res.max()), "energies": int(nE)}

    # roofline of the dominant kernel (from the profiled step)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    src = "MEASURED_PEAKS" if "bf16_tflops_sustained" in peaks else "fallback"
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    dfma_peak, dmma_peak = fp64["dfma_tflops"], fp64["dmma_tflops"]
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    name, (dms, dfl, dln) = dom
    achieved = dfl / (dms * 1e-3) / 1e12 if dms > 0 else 0.0
    if name == "zgemm_f64_kernel":
        bound, peak = "tensor", dmma_peak
        psrc = "of measured: FP64 MMA (mma.sync m8n8k4) loop of negf_fp64_peak in this run"
    elif name == "zgemm_tc_kernel":
        # useful complex-product flops against the BF16 tensor peak: the exact
        # slicing issues several BF16 products per useful one and the kernel
        # is bound by its integer slicing / combination work (profiles/)
        bound, peak = "tensor", bf16
        psrc = f"of measured: {src} bf16 sustained (useful flops of exact-slice emulated products)"
    else:
        bound, peak = "alu", dfma_peak
        psrc = "of measured: FP64 FMA loop of negf_fp64_peak in this run (DFMA pipe)"
    # the flops the units execute (the library's count per launch): the 3M
    # FP64 product issues 6 m n k of the 8 m n k counted; the exact-slice
    # product issues L (L + 1) / 2 BF16 slice products per useful one
    issued = None
    if name in ("zgemm_f64_kernel", "zgemm_tc_kernel") and dms > 0:
        ia = prof_iss[name][2] / (dms * 1e-3) / 1e12
        issued = {"achieved": ia, "frac": ia / peak,
                  "per_useful_flop": prof_iss[name][2] / dfl if dfl > 0 else None}
    traffic = None
    uniform_b = prob.sizes[0] if len(set(prob.sizes)) == 1 else None
    t = NCU_TRAFFIC.get((name, uniform_b))
    if t is not None:
        import hashlib
        with open(os.path.join(ROOT, t["src"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() == t["sha256"]:
                # units per launch: one per energy of the single-group step's
                # launches (a layer's inversions, or one block product)
                traffic = t["bytes_per_unit"] * (N * nE / dln if t["unit"] == "inversion" else nE)
    roof = {"kernel": name, "bound": bound,
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "peak_source": psrc,
            "traffic_note": "ncu dram bytes read + written per launch (captured launches, scaled per unit) against "
                            "the algorithmic 2 x 16 b^2 bytes per inversion / up to 4 x 16 b^2 per block product "
                            "(A, B, C1 in, C out; a shared coupling-block operand is read once per launch)",
            "flop_count": "the method's 8 m n k per complex product / 8 b^3 per inversion",
            "kernel_share": dms / sum(v[0] for v in prof.values()),
            "launches_per_step": int(dln), "nominal_fp64_tflops": FP64_NOMINAL_TFLOPS}
    if issued:
        roof["issued"] = issued

    # composite roofline of the mixed path (FP64 inversions at the FP64 rate,
    # block products at the BF16 tensor peak, useful flops only)
    composite = None
    if a.precision == "mixed":
        f64 = prof["zinv_gj_kernel"][1]
        fdm = prof["zgemm_f64_kernel"][1]
        flow = prof["zgemm_tc_kernel"][1]
        t_roof = f64 / (dfma_peak * 1e12) + fdm / (dmma_peak * 1e12) + flow / (bf16 * 1e12)
        composite = {"t_roof_ms": t_roof * 1e3, "t_measured_ms": ms, "frac": t_roof * 1e3 / ms,
                     "fp64_inverse_flops": f64, "fp64_product_flops": fdm, "tensor_product_flops": flow,
                     "peaks": {"fp64_alu_tflops": dfma_peak, "fp64_dmma_tflops": dmma_peak,
                               "bf16_tflops": bf16, "source": "FP64: negf_fp64_peak in this run; "
                                                             "bf16: MEASURED_PEAKS sustained"}}

    # every kernel of the single-group profiled step: time, launches, share
    # and useful flops per second (the method's count)
    tot_ms = sum(v[0] for v in prof.values())
    kernels = {k: {"ms": v[0], "launches": int(v[2]), "share": v[0] / tot_ms if tot_ms > 0 else 0.0,
                   "tflops": (v[1] / (v[0] * 1e-3) / 1e12) if v[0] > 0 else 0.0}
               for k, v in prof.items() if v[2] > 0}
    if "zinv_gj_kernel" in kernels:
        kernels["zinv_gj_kernel"]["of_measured_dfma"] = kernels["zinv_gj_kernel"]["tflops"] / dfma_peak
    if "zgemm_f64_kernel" in kernels:
        kernels["zgemm_f64_kernel"]["of_measured_dmma"] = kernels["zgemm_f64_kernel"]["tflops"] / dmma_peak

    from oracle.rgf import rgf_flops_paper
    flops_step = rgf_flops_paper(prob.sizes, prob.w) * nE
    ws_gb = P.negf_workspace_bytes(plan.handle) / 1e9
    plan_domains = plan.n_domains
    plan_bits = P.negf_plan_product_bits(plan.handle)
    plan.close()

    # side measurement: the plain FP64 path on the same inputs (for the
    # mixed-over-FP64 speedup)
    fp64_side = None
    if a.precision == "mixed" and not a.no_fp64_side:
        fplan = P.Plan(prob.sizes, 2 * prob.w + 1, nE, precision="fp64", outputs=outputs)
        fplan.solve(H, sL, sR, E, out_band=Gb, out_g1n=G1, sync=False)
        fplan.sync()
        k3 = max(1, min(a.steps, 3))
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(k3):
            fplan.solve(H, sL, sR, E, out_band=Gb, out_g1n=G1, sync=False)
        f1.record(stream)
        torch.cuda.synchronize()
        fplan.sync()
        fplan.close()
        fms = f0.elapsed_time(f1) / k3
        fp64_side = {"ms_per_step": fms, "value": job_throughput(world, nE, N, fms), "steps": k3,
                     "mixed_speedup": fms / ms}

    # side measurement: the Keldysh path (negf_lesser: retarded sweep + the
    # lesser recursion, FP64 lesser products) with the left lead occupied and
    # the right one empty, when a second band output fits comfortably
    lesser_side = None
    band_bytes = Gb.numel() * Gb.element_size()
    if not a.no_lesser_side and prob.w == 1 and band_bytes < 16e9:
        lplan = P.Plan(prob.sizes, 3, nE, precision=a.precision, outputs=P.NEGF_OUT_BAND | P.NEGF_OUT_LESSER,
                       product_bits=bits)
        GL = torch.empty_like(Gb)
        gamL = 1j * (sL - sL.conj().transpose(-1, -2))
        slL = 1j * gamL
        slR = torch.zeros_like(sR)
        lplan.lesser(H, sL, sR, E, slL, slR, out_band=Gb, out_less=GL, sync=False)
        lplan.sync()
        k3 = max(1, min(a.steps, 3))
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        for _ in range(k3):
            lplan.lesser(H, sL, sR, E, slL, slR, out_band=Gb, out_less=GL, sync=False)
        l1.record(stream)
        torch.cuda.synchronize()
        lplan.sync()
        lplan.close()
        lms = l0.elapsed_time(l1) / k3
        lrel = None
        if rank == 0:
            from oracle import rgf as O
            e = nE // 2
            ref, _ = O.rgf_lesser(O.system_blocks(prob, prob.energies[e]), prob.sizes,
                                  {0: 1j * O.gamma(prob.sigma_L), N - 1: np.zeros_like(prob.sigma_R)})
            got = P.unpack_band(GL[e].cpu().numpy(), prob.sizes, 1)
            num = sum(np.linalg.norm(got[k] - v) ** 2 for k, v in ref.items())
            den = sum(np.linalg.norm(v) ** 2 for v in ref.values())
            lrel = float(np.sqrt(num / den))
        del GL
        lesser_side = {"ms_per_step": lms, "value": job_throughput(world, nE, N, lms), "steps": k3,
                       "outputs": "retarded band + lesser band per energy", "rel_err_vs_oracle_sampled": lrel}

    # side measurement: the adjoint (negf_grad: T(E) and dT-weighted gradients
    # with respect to the band of H and to Sigma_L / Sigma_R), full and
    # checkpointed every ~sqrt(N) layers
    grad_side = None
    if not a.no_grad_side and prob.w == 1:
        grad_side = {}
        wts = torch.linspace(-1.0, 1.0, nE, dtype=torch.float64, device=dev)
        for ck in (0, max(1, int(round(N ** 0.5)))):
            gplan = P.Plan(prob.sizes, 3, nE, precision=a.precision, product_bits=bits,
                           outputs=P.NEGF_OUT_TRANSMISSION | P.NEGF_OUT_GRAD, checkpoint_every=ck)
            gplan.grad(H, sL, sR, E, wts)
            k3 = max(1, min(a.steps, 3))
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            for _ in range(k3):
                gplan.grad(H, sL, sR, E, wts, sync=False)
            g1.record(stream)
            torch.cuda.synchronize()
            gplan.sync()
            gws = P.negf_workspace_bytes(gplan.handle) / 1e9
            gplan.close()
            gms = g0.elapsed_time(g1) / k3
            grad_side["checkpoint_every_%d" % ck] = {"ms_per_step": gms, "value": job_throughput(world, nE, N, gms),
                                                     "workspace_gb": gws, "steps": k3}

    # side measurement: one energy on a long chain (1024 x 64, diagonally
    # dominant, eta = 1e-3), where the GPU is not filled by energies: plain
    # RGF, single-level DDRGF with the cost model's pair count, and the cost
    # model's recursive choice (negf_ddrgf_model with the measured r_inv)
    ddrgf_side = None
    if not a.no_ddrgf_side and rank == 0:
        dprob = make_problem(1024, b=64, w=1, n_energies=1, eta=1e-3, seed=3, diag_shift=4.0)
        dH = torch.tensor(P.pack_band(dprob.H, dprob.sizes, 1), device=dev)
        dsL, dsR = torch.tensor(dprob.sigma_L, device=dev), torch.tensor(dprob.sigma_R, device=dev)
        dE = torch.tensor(dprob.energies, device=dev)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        r_inv = P.negf_measure_r_inv(64, 1)
        nd, levels, c_rgf, c_dd = P.negf_ddrgf_model(dprob.sizes, 3, 1, sms, r_inv)
        ref_band = None
        ddrgf_side = {"chain": "1024 x 64, 1 energy, eta 1e-3, diagonally dominant", "r_inv": r_inv,
                      "model": {"n_domains": nd, "levels": levels, "cost_rgf": c_rgf, "cost_ddrgf": c_dd}}
        for label, kw in (("rgf", dict(n_domains=1)), ("ddrgf_1_level", dict(n_domains=max(nd, 2))),
                          ("ddrgf_model", dict(n_domains=max(nd, 2), interface_levels=tuple(levels)))):
            dplan = P.Plan(dprob.sizes, 3, 1, outputs=P.NEGF_OUT_BAND | P.NEGF_OUT_G1N, **kw)
            db, _ = dplan.solve(dH, dsL, dsR, dE)
            for _ in range(2):
                dplan.solve(dH, dsL, dsR, dE, out_band=db, sync=False)
            dplan.sync()
            d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            d0.record(stream)
            for _ in range(5):
                dplan.solve(dH, dsL, dsR, dE, out_band=db, sync=False)
            d1.record(stream)
            torch.cuda.synchronize()
            dplan.sync()
            dplan.close()
            if ref_band is None:
                ref_band = db.clone()
                dev_ = 0.0
            else:
                dev_ = float(torch.linalg.norm(db - ref_band) / torch.linalg.norm(ref_band))
            ddrgf_side[label] = {"ms": d0.elapsed_time(d1) / 5, "rel_dev_from_rgf": dev_}
        del dH, ref_band

    # the CPU oracle baseline, after every GPU timing (spawned worker
    # processes, so no CUDA state is forked; none exist while the GPU is timed)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        pool = make_pool(cores)
        cpu, _ = oracle_sample(a.workload, a.cpu_energies, pool, cores)
        pool.close()

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if a.precision == "fp64" else
                     f"mixed: exact bf16-slice tensor products ({plan_bits} bit), f64 inverses",
            "data": "synthetic",
            "config": {"workload": a.workload, "n_blocks": N, "block_size": prob.sizes[0], "band_n": 2 * prob.w + 1,
                       "n_energies": nE, "eta": 1e-6, "precision": a.precision,
                       "product_bits": plan_bits if a.precision == "mixed" else None,
                       "refine_steps": refine,
                       "outputs": "band + G_1N per energy" + (" (G_1N from the refined last block column)"
                                                              if refine else ""),
                       "l2": "no flush: each step writes %.1f GB of selected blocks and %.1f GB of sweep "
                             "workspace, both far above the 129 MB L2" % (Gb.numel() * 16 / 1e9, ws_gb),
                       "parallelism": f"replicas x{world} (energies)",
                       "energy_groups": groups,
                       "n_domains": plan_domains,
                       "hbm_footprint_gb": {"outputs": Gb.numel() * 16 / 1e9 + G1.numel() * 16 / 1e9,
                                            "workspace": ws_gb}},
            "autotune": tune,
            "precision_tuning": prec_tune,
            "effective_tflops_paper_count": flops_step / (ms * 1e-3) / 1e12 * world,
            "rel_err_vs_oracle_sampled": rel,
            "band_residual": band_residual,
            "roofline": roof,
            "composite_roofline": composite,
            "kernels_single_group_step": kernels,
            "fp64_peaks_measured": fp64,
            "fp64_path": fp64_side,
            "lesser_path": lesser_side,
            "grad_path": grad_side,
            "ddrgf_levels": ddrgf_side,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": launches_per_step * a.steps,
        }
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle, on the host cores
# ---------------------------------------------------------------------------
def run_reference(a, rank, world):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    pool = make_pool(cores)
    from workloads import workload
    prob = workload(a.workload)
    n = min(a.cpu_energies, 16 * cores)
    for _ in range(a.warmup):
        oracle_sample(a.workload, min(n, cores), pool, cores)
    vals, walls = [], []
    cpu = None
    for _ in range(a.steps):
        cpu, wall = oracle_sample(a.workload, n, pool, cores)
        vals.append(cpu["value"])
        walls.append(wall)
    pool.close()
    v = statistics.median(vals)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": statistics.median(walls) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": a.workload, "n_blocks": prob.n_blocks, "block_size": prob.sizes[0],
                      "n_energies": len(prob.energies), "sample_energies_per_step": n},
           "cpu_baseline": dict(cpu, value=v),
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    a = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
    else:
        run_ours(a, rank, world, local_rank)


if __name__ == "__main__":
    main()
