"""Python binding of libnegf.so: GB300 selected inversion of G^R(E) = (E I - H - Sigma)^{-1}.

The functions named ``negf_*`` mirror the C-ABI in ``include/negf.h`` one to
one and only marshal arguments (device pointers from torch tensors, the
current CUDA stream).  Every step of the computation runs in the library's
CUDA kernels; there is no CPU or PyTorch fallback: if ``libnegf.so`` is
missing or fails to load, importing this package raises.

Higher-level helpers: :func:`band_layout` / :func:`pack_band` /
:func:`unpack_band` (host-side layout of band-packed block matrices),
:class:`Plan` (a plan bound to torch tensors), and :class:`Transmission`
(a ``torch.autograd.Function`` whose backward is the library's adjoint).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnegf.so")

NEGF_OK = 0
NEGF_ERR_ARG = 1
NEGF_ERR_SINGULAR = 2
NEGF_ERR_NONFINITE = 3
NEGF_ERR_NOMEM = 4
NEGF_ERR_CUDA = 5
NEGF_ERR_TIMEOUT = 6
NEGF_ERR_UNSUPPORTED = 7

NEGF_FP64 = 0
NEGF_MIXED = 1

NEGF_OUT_BAND = 1
NEGF_OUT_G1N = 2
NEGF_OUT_TRANSMISSION = 4
NEGF_OUT_GRAD = 8
NEGF_OUT_LESSER = 16

NEGF_MAX_BLOCK = 160
NEGF_DEFAULT_PRODUCT_BITS = 48
TUNE_BITS = (32, 35, 42, 48)   # the candidates of negf_tune_precision, in its order

NEGF_PROF_INV = 0
NEGF_PROF_GEMM_F64 = 1
NEGF_PROF_GEMM_TC = 2
NEGF_PROF_MISC = 3
NEGF_PROF_KINDS = 4
PROF_NAMES = ["zinv_gj_kernel", "zgemm_f64_kernel", "zgemm_tc_kernel", "misc"]

EXPORTED = [
    "negf_plan", "negf_workspace_bytes", "negf_band_offset", "negf_band_elems", "negf_solve",
    "negf_plan_n_domains", "negf_auto_domains", "negf_band_residual", "negf_autotune", "negf_plan_groups",
    "negf_plan_set_groups", "negf_lesser", "negf_solve_host",
    "negf_transmission", "negf_grad", "negf_sync", "negf_destroy", "negf_status_string",
    "negf_profile_enable", "negf_profile_read", "negf_profile_read_issued", "negf_last_cuda_error", "negf_solve_noalloc",
    "negf_fp64_peak", "negf_plan_set_wait_limit", "negf_grad_strided", "negf_tune_precision",
    "negf_plan_product_bits", "negf_plan_levels", "negf_ddrgf_model", "negf_measure_r_inv",
    "negf_plan_tile_cols", "negf_plan_set_tile_cols",
]

NEGF_NOALLOC_SCRATCH_BYTES = 32 << 20
NEGF_PEAK_DFMA = 0
NEGF_PEAK_DMMA = 1
NEGF_PEAK_BOTH = 2
AUTOTUNE_GROUPS = (1, 2, 3, 4, 6, 8)   # the candidates of negf_autotune, in its order


class NegfError(RuntimeError):
    """A negf_status other than NEGF_OK, with the CUDA error text for NEGF_ERR_CUDA."""

    def __init__(self, status, where=""):
        self.status = int(status)
        extra = ""
        if self.status == NEGF_ERR_CUDA:
            extra = f" [{_lib.negf_last_cuda_error().decode()}]"
        super().__init__(f"{where}: {negf_status_string(status)} ({status}){extra}")


class negf_desc(ctypes.Structure):
    """The plan descriptor of include/negf.h (same fields, same order)."""

    _fields_ = [
        ("n_blocks", ctypes.c_int32),
        ("block_sizes", ctypes.POINTER(ctypes.c_int32)),
        ("band_n", ctypes.c_int32),
        ("n_energies", ctypes.c_int32),
        ("n_domains", ctypes.c_int32),
        ("domain_first_block", ctypes.POINTER(ctypes.c_int32)),
        ("precision", ctypes.c_int32),
        ("refine_steps", ctypes.c_int32),
        ("outputs", ctypes.c_int32),
        ("checkpoint_every", ctypes.c_int32),
        ("product_bits", ctypes.c_int32),
        ("n_levels", ctypes.c_int32),
        ("level_domains", ctypes.POINTER(ctypes.c_int32)),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libnegf.so not found at {LIB_PATH}; build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, st = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int
    lib.negf_plan.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(negf_desc), vp]
    lib.negf_plan.restype = st
    lib.negf_workspace_bytes.argtypes = [vp]
    lib.negf_workspace_bytes.restype = ctypes.c_size_t
    lib.negf_band_offset.argtypes = [vp, i32, i32]
    lib.negf_band_offset.restype = i64
    lib.negf_band_elems.argtypes = [vp]
    lib.negf_band_elems.restype = i64
    lib.negf_solve.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp]
    lib.negf_solve.restype = st
    lib.negf_transmission.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp]
    lib.negf_transmission.restype = st
    lib.negf_grad.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp]
    lib.negf_grad.restype = st
    lib.negf_sync.argtypes = [vp]
    lib.negf_sync.restype = st
    lib.negf_destroy.argtypes = [vp]
    lib.negf_destroy.restype = None
    lib.negf_profile_enable.argtypes = [vp, i32]
    lib.negf_profile_enable.restype = st
    dp = ctypes.POINTER(ctypes.c_double)
    lp = ctypes.POINTER(ctypes.c_int64)
    lib.negf_profile_read.argtypes = [vp, dp, dp, lp]
    lib.negf_profile_read.restype = i32
    lib.negf_profile_read_issued.argtypes = [vp, dp, dp, dp, lp]
    lib.negf_profile_read_issued.restype = i32
    lib.negf_solve_noalloc.argtypes = [ctypes.POINTER(negf_desc), vp, vp, vp, i64, vp, vp, vp, vp, vp]
    lib.negf_solve_noalloc.restype = st
    lib.negf_last_cuda_error.argtypes = []
    lib.negf_last_cuda_error.restype = ctypes.c_char_p
    lib.negf_status_string.argtypes = [st]
    lib.negf_status_string.restype = ctypes.c_char_p
    lib.negf_autotune.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp, i32, ctypes.POINTER(i32),
                                  ctypes.POINTER(ctypes.c_double)]
    lib.negf_autotune.restype = st
    lib.negf_plan_groups.argtypes = [vp]
    lib.negf_plan_groups.restype = i32
    lib.negf_plan_tile_cols.argtypes = [vp]
    lib.negf_plan_tile_cols.restype = i32
    lib.negf_plan_set_tile_cols.argtypes = [vp, i32]
    lib.negf_plan_set_tile_cols.restype = ctypes.c_int
    lib.negf_plan_set_groups.argtypes = [vp, i32]
    lib.negf_plan_set_groups.restype = st
    lib.negf_solve_host.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp]
    lib.negf_solve_host.restype = st
    lib.negf_lesser.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, i64, vp, vp, vp, vp]
    lib.negf_lesser.restype = st
    lib.negf_band_residual.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp]
    lib.negf_band_residual.restype = st
    lib.negf_plan_n_domains.argtypes = [vp]
    lib.negf_plan_n_domains.restype = i32
    lib.negf_auto_domains.argtypes = [i32, ctypes.POINTER(i32), i32, i32, i32]
    lib.negf_auto_domains.restype = i32
    lib.negf_fp64_peak.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
    lib.negf_fp64_peak.restype = st
    lib.negf_plan_set_wait_limit.argtypes = [vp, i64]
    lib.negf_plan_set_wait_limit.restype = st
    lib.negf_grad_strided.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, i64, vp, i64, vp]
    lib.negf_grad_strided.restype = st
    lib.negf_tune_precision.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, ctypes.c_double,
                                        ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]
    lib.negf_tune_precision.restype = st
    lib.negf_plan_product_bits.argtypes = [vp]
    lib.negf_plan_product_bits.restype = i32
    lib.negf_plan_levels.argtypes = [vp, ctypes.POINTER(i32), i32]
    lib.negf_plan_levels.restype = i32
    lib.negf_ddrgf_model.argtypes = [i32, ctypes.POINTER(i32), i32, i32, i32, ctypes.c_double, i32,
                                     ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
    lib.negf_ddrgf_model.restype = i32
    lib.negf_measure_r_inv.argtypes = [i32, i32, i32, ctypes.POINTER(ctypes.c_double), vp]
    lib.negf_measure_r_inv.restype = st
    return lib


_lib = _load()


def lib():
    """The loaded libnegf.so (ctypes handle)."""
    return _lib


# ---------------------------------------------------------------------------
# C-ABI mirror (argument marshalling only)
# ---------------------------------------------------------------------------
def negf_status_string(status):
    """``negf_status_string`` of include/negf.h (argument marshalling only)."""
    return _lib.negf_status_string(int(status)).decode()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def negf_plan(block_sizes, band_n=3, n_energies=1, n_domains=1, domain_first_block=None,
              precision=NEGF_FP64, refine_steps=0, outputs=NEGF_OUT_BAND | NEGF_OUT_G1N,
              checkpoint_every=0, stream=None, product_bits=0, interface_levels=()):
    """Create a plan; returns an opaque handle (int).  Raises NegfError.
    ``interface_levels``: the pair counts of the recursive interface levels
    (negf_desc.level_domains)."""
    sizes = (ctypes.c_int32 * len(block_sizes))(*[int(b) for b in block_sizes])
    d = negf_desc()
    d.n_blocks = len(block_sizes)
    d.block_sizes = sizes
    d.band_n = band_n
    d.n_energies = n_energies
    d.n_domains = n_domains
    if domain_first_block is not None:
        dfb = (ctypes.c_int32 * len(domain_first_block))(*[int(x) for x in domain_first_block])
        d.domain_first_block = dfb
    d.precision = precision
    d.refine_steps = refine_steps
    d.outputs = outputs
    d.checkpoint_every = checkpoint_every
    d.product_bits = product_bits
    if interface_levels:
        lv = (ctypes.c_int32 * len(interface_levels))(*[int(x) for x in interface_levels])
        d.n_levels = len(interface_levels)
        d.level_domains = lv
    h = ctypes.c_void_p()
    s = _lib.negf_plan(ctypes.byref(h), ctypes.byref(d), stream)
    if s != NEGF_OK:
        raise NegfError(s, "negf_plan")
    return h.value


def negf_solve_noalloc(block_sizes, band_n, n_energies, H, sigma_L, sigma_R, sigma_E_stride, E, G_band, G_1N,
                       info, stream=None, outputs=NEGF_OUT_BAND | NEGF_OUT_G1N):
    """negf_solve without a plan and without any device allocation (scratch in
    a fixed device array of NEGF_NOALLOC_SCRATCH_BYTES).  Returns the status."""
    sizes = (ctypes.c_int32 * len(block_sizes))(*[int(b) for b in block_sizes])
    d = negf_desc()
    d.n_blocks = len(block_sizes)
    d.block_sizes = sizes
    d.band_n = band_n
    d.n_energies = n_energies
    d.n_domains = 1
    d.precision = NEGF_FP64
    d.refine_steps = 0
    d.outputs = outputs
    d.checkpoint_every = 0
    d.product_bits = 0
    return _lib.negf_solve_noalloc(ctypes.byref(d), _ptr(H), _ptr(sigma_L), _ptr(sigma_R), int(sigma_E_stride),
                                   _ptr(E), _ptr(G_band), _ptr(G_1N), _ptr(info), stream)


def negf_fp64_peak(kind, iters, stream=None):
    """``negf_fp64_peak`` of include/negf.h: returns ``(TFLOP/s, ms)``; raises NegfError."""
    tf = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    s = _lib.negf_fp64_peak(int(kind), int(iters), ctypes.byref(tf), ctypes.byref(ms), stream)
    if s != NEGF_OK:
        raise NegfError(s, "negf_fp64_peak")
    return tf.value, ms.value


def energy_shard(n_energies, rank, world):
    """Contiguous share ``[lo, hi)`` of an energy list of ``n_energies`` for
    rank ``rank`` of ``world`` (energies are independent problems, so ranks
    need no exchange); the shares of ranks 0..world-1 concatenate to the whole
    list, their sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    return (int(n_energies) * rank) // world, (int(n_energies) * (rank + 1)) // world


def negf_workspace_bytes(plan):
    """``negf_workspace_bytes`` of include/negf.h (argument marshalling only)."""
    return int(_lib.negf_workspace_bytes(plan))


def negf_solve_host(plan, H, sigma_L, sigma_R, sigma_E_stride, E, G_band, G_1N, info):
    """``negf_solve_host`` of include/negf.h (argument marshalling only)."""
    return _lib.negf_solve_host(plan, _ptr(H), _ptr(sigma_L), _ptr(sigma_R), int(sigma_E_stride), _ptr(E),
                                _ptr(G_band), _ptr(G_1N), _ptr(info))


def negf_lesser(plan, H, sigma_L, sigma_R, sigma_E_stride, E, sigma_less_L, sigma_less_R, sless_stride,
                less_diag, G_band, G_less, info):
    """``negf_lesser`` of include/negf.h (argument marshalling only)."""
    return _lib.negf_lesser(plan, _ptr(H), _ptr(sigma_L), _ptr(sigma_R), int(sigma_E_stride), _ptr(E),
                            _ptr(sigma_less_L), _ptr(sigma_less_R), int(sless_stride), _ptr(less_diag),
                            _ptr(G_band), _ptr(G_less), _ptr(info))


def negf_band_residual(plan, H, sigma_L, sigma_R, sigma_E_stride, E, G_band, res):
    """``negf_band_residual`` of include/negf.h (argument marshalling only)."""
    return _lib.negf_band_residual(plan, _ptr(H), _ptr(sigma_L), _ptr(sigma_R), int(sigma_E_stride), _ptr(E),
                                   _ptr(G_band), _ptr(res))


def negf_autotune(plan, H, sigma_L, sigma_R, sigma_E_stride, E, G_band, G_1N, info, reps=2):
    """Returns ``(status, best_groups, [ms per candidate of AUTOTUNE_GROUPS])``."""
    best = ctypes.c_int32(0)
    ms = (ctypes.c_double * len(AUTOTUNE_GROUPS))()
    st = _lib.negf_autotune(plan, _ptr(H), _ptr(sigma_L), _ptr(sigma_R), int(sigma_E_stride), _ptr(E),
                            _ptr(G_band), _ptr(G_1N), _ptr(info), int(reps), ctypes.byref(best), ms)
    return st, int(best.value), list(ms)


def negf_tune_precision(plan, H, sigma_L, sigma_R, sigma_E_stride, E, G_band, G_1N, info, G_band_ref, G_1N_ref,
                        tol):
    """``negf_tune_precision`` of include/negf.h: returns ``(status, bits, deviation)``."""
    bits = ctypes.c_int32(0)
    dev = ctypes.c_double(0.0)
    st = _lib.negf_tune_precision(plan, _ptr(H), _ptr(sigma_L), _ptr(sigma_R), int(sigma_E_stride), _ptr(E),
                                  _ptr(G_band), _ptr(G_1N), _ptr(info), _ptr(G_band_ref), _ptr(G_1N_ref),
                                  float(tol), ctypes.byref(bits), ctypes.byref(dev))
    return st, int(bits.value), float(dev.value)


def negf_plan_product_bits(plan):
    """``negf_plan_product_bits`` of include/negf.h (argument marshalling only)."""
    return int(_lib.negf_plan_product_bits(plan))


def negf_plan_levels(plan):
    """``negf_plan_levels`` of include/negf.h: the interface levels' pair counts (list)."""
    buf = (ctypes.c_int32 * 16)()
    n = int(_lib.negf_plan_levels(plan, buf, 16))
    return [int(buf[k]) for k in range(max(0, n))]


def negf_ddrgf_model(block_sizes, band_n, n_energies, sm_count, r_inv, max_levels=4):
    """``negf_ddrgf_model`` of include/negf.h: returns ``(n_domains, levels, cost_rgf, cost_ddrgf)``."""
    sizes = (ctypes.c_int32 * len(block_sizes))(*[int(b) for b in block_sizes])
    lv = (ctypes.c_int32 * max(1, max_levels))()
    nl = ctypes.c_int32(0)
    cr, cd = ctypes.c_double(0.0), ctypes.c_double(0.0)
    nd = int(_lib.negf_ddrgf_model(len(block_sizes), sizes, int(band_n), int(n_energies), int(sm_count),
                                   float(r_inv), int(max_levels), lv, ctypes.byref(nl), ctypes.byref(cr),
                                   ctypes.byref(cd)))
    return nd, [int(lv[k]) for k in range(nl.value)], cr.value, cd.value


def negf_measure_r_inv(b, batch, precision=NEGF_FP64, stream=None):
    """``negf_measure_r_inv`` of include/negf.h: returns r_inv; raises NegfError."""
    r = ctypes.c_double(0.0)
    s = _lib.negf_measure_r_inv(int(b), int(batch), int(precision), ctypes.byref(r), stream)
    if s != NEGF_OK:
        raise NegfError(s, "negf_measure_r_inv")
    return r.value


def negf_plan_groups(plan):
    """``negf_plan_groups`` of include/negf.h (argument marshalling only)."""
    return int(_lib.negf_plan_groups(plan))


def negf_plan_tile_cols(plan):
    """``negf_plan_tile_cols`` of include/negf.h (argument marshalling only)."""
    return int(_lib.negf_plan_tile_cols(plan))


def negf_plan_set_tile_cols(plan, cols):
    """``negf_plan_set_tile_cols`` of include/negf.h (argument marshalling only)."""
    return int(_lib.negf_plan_set_tile_cols(plan, cols))


def negf_plan_set_groups(plan, groups):
    """``negf_plan_set_groups`` of include/negf.h (argument marshalling only)."""
    return _lib.negf_plan_set_groups(plan, int(groups))


def negf_plan_set_wait_limit(plan, polls):
    """``negf_plan_set_wait_limit`` of include/negf.h (argument marshalling only)."""
    return _lib.negf_plan_set_wait_limit(plan, int(polls))


def negf_plan_n_domains(plan):
    """``negf_plan_n_domains`` of include/negf.h (argument marshalling only)."""
    return int(_lib.negf_plan_n_domains(plan))


def negf_auto_domains(block_sizes, band_n, n_energies, sm_count):
    """``negf_auto_domains`` of include/negf.h (argument marshalling only)."""
    sizes = (ctypes.c_int32 * len(block_sizes))(*[int(b) for b in block_sizes])
    return int(_lib.negf_auto_domains(len(block_sizes), sizes, int(band_n), int(n_energies), int(sm_count)))


def negf_band_offset(plan, d, i):
    """``negf_band_offset`` of include/negf.h (argument marshalling only)."""
    return int(_lib.negf_band_offset(plan, d, i))


def negf_band_elems(plan):
    """``negf_band_elems`` of include/negf.h (argument marshalling only)."""
    return int(_lib.negf_band_elems(plan))


def negf_solve(plan, H, sigma_L, sigma_R, sigma_E_stride, E, G_band, G_1N, info):
    """``negf_solve`` of include/negf.h (argument marshalling only)."""
    return _lib.negf_solve(plan, _ptr(H), _ptr(sigma_L), _ptr(sigma_R), int(sigma_E_stride), _ptr(E),
                           _ptr(G_band), _ptr(G_1N), _ptr(info))


def negf_transmission(plan, H, sigma_L, sigma_R, sigma_E_stride, E, T, info):
    """``negf_transmission`` of include/negf.h (argument marshalling only)."""
    return _lib.negf_transmission(plan, _ptr(H), _ptr(sigma_L), _ptr(sigma_R), int(sigma_E_stride),
                                  _ptr(E), _ptr(T), _ptr(info))


def negf_grad(plan, H, sigma_L, sigma_R, sigma_E_stride, E, dL_dT, T, dH, dSigma_L, dSigma_R, info):
    """``negf_grad`` of include/negf.h (argument marshalling only)."""
    return _lib.negf_grad(plan, _ptr(H), _ptr(sigma_L), _ptr(sigma_R), int(sigma_E_stride), _ptr(E),
                          _ptr(dL_dT), _ptr(T), _ptr(dH), _ptr(dSigma_L), _ptr(dSigma_R), _ptr(info))


def negf_grad_strided(plan, H, sigma_L, sigma_R, sigma_E_stride, E, dL_dT, T, dH, dSigma_L, dSigma_L_stride,
                      dSigma_R, dSigma_R_stride, info):
    """``negf_grad_strided`` of include/negf.h (argument marshalling only)."""
    return _lib.negf_grad_strided(plan, _ptr(H), _ptr(sigma_L), _ptr(sigma_R), int(sigma_E_stride), _ptr(E),
                                  _ptr(dL_dT), _ptr(T), _ptr(dH), _ptr(dSigma_L), int(dSigma_L_stride),
                                  _ptr(dSigma_R), int(dSigma_R_stride), _ptr(info))


def negf_sync(plan):
    """``negf_sync`` of include/negf.h (argument marshalling only)."""
    return _lib.negf_sync(plan)


def negf_destroy(plan):
    """``negf_destroy`` of include/negf.h (argument marshalling only)."""
    _lib.negf_destroy(plan)


def negf_profile_enable(plan, on):
    """``negf_profile_enable`` of include/negf.h (argument marshalling only)."""
    return _lib.negf_profile_enable(plan, int(bool(on)))


def negf_profile_read(plan):
    """Returns ``{kind_name: (ms, flops, launches)}`` for the calls made since
    profiling was enabled (or since the previous read)."""
    ms = (ctypes.c_double * NEGF_PROF_KINDS)()
    fl = (ctypes.c_double * NEGF_PROF_KINDS)()
    ln = (ctypes.c_int64 * NEGF_PROF_KINDS)()
    n = _lib.negf_profile_read(plan, ms, fl, ln)
    if n < 0:
        raise NegfError(NEGF_ERR_CUDA, "negf_profile_read")
    return {PROF_NAMES[k]: (ms[k], fl[k], ln[k]) for k in range(n)}


def negf_profile_read_issued(plan):
    """Returns ``{kind_name: (ms, flops, issued_flops, launches)}``: the read
    of ``negf_profile_read`` with the flops the units execute per kind."""
    ms = (ctypes.c_double * NEGF_PROF_KINDS)()
    fl = (ctypes.c_double * NEGF_PROF_KINDS)()
    iss = (ctypes.c_double * NEGF_PROF_KINDS)()
    ln = (ctypes.c_int64 * NEGF_PROF_KINDS)()
    n = _lib.negf_profile_read_issued(plan, ms, fl, iss, ln)
    if n < 0:
        raise NegfError(NEGF_ERR_CUDA, "negf_profile_read_issued")
    return {PROF_NAMES[k]: (ms[k], fl[k], iss[k], ln[k]) for k in range(n)}


# ---------------------------------------------------------------------------
# Host-side layout helpers (no arithmetic of the method)
# ---------------------------------------------------------------------------
def band_layout(sizes, w):
    """Offsets of the band-packed layout of include/negf.h: blocks (i, i+d)
    for d = -w..w (outer), i = 0..N-1 (inner), existing blocks only.
    Returns ``(offsets dict {(i, j): offset}, total elements)``."""
    N = len(sizes)
    off = {}
    o = 0
    for d in range(-w, w + 1):
        for i in range(N):
            j = i + d
            if 0 <= j < N:
                off[(i, j)] = o
                o += sizes[i] * sizes[j]
    return off, o


def pack_band(blocks, sizes, w, dtype=np.complex128):
    """Pack a dict ``{(i, j): block}`` into one band-packed vector."""
    off, n = band_layout(sizes, w)
    out = np.zeros(n, dtype=dtype)
    for (i, j), o in off.items():
        blk = blocks.get((i, j))
        if blk is not None:
            out[o:o + sizes[i] * sizes[j]] = np.asarray(blk, dtype=dtype).reshape(-1)
    return out


def unpack_band(vec, sizes, w):
    """Inverse of :func:`pack_band` (views into ``vec``)."""
    off, _ = band_layout(sizes, w)
    return {(i, j): vec[o:o + sizes[i] * sizes[j]].reshape(sizes[i], sizes[j]) for (i, j), o in off.items()}


def fused_sizes(sizes, w):
    """Super-block sizes of the block tridiagonal form of a block n-diagonal
    chain (Sec. 2.3, block fusing): super-layer J holds layers
    [J w, (J + 1) w) (the last one may hold fewer)."""
    return [int(sum(sizes[j:j + w])) for j in range(0, len(sizes), w)]


def _fuse_maps(sizes, w):
    off, _ = band_layout(sizes, w)
    fs = fused_sizes(sizes, w)
    foff, fn = band_layout(fs, 1)
    start = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    fstart = np.concatenate([[0], np.cumsum(fs)]).astype(int)
    maps = []   # (src offset, rows, cols, fused offset, fused rows, fused cols, row0, col0)
    for (a, b), o in off.items():
        J, K = a // w, b // w
        maps.append((o, sizes[a], sizes[b], foff[(J, K)], fs[J], fs[K],
                     int(start[a] - fstart[J]), int(start[b] - fstart[K])))
    return fs, fn, maps


def fuse_band(band, sizes, w):
    """Band-packed blocks of an n-diagonal chain (``band``: [..., band_elems]
    torch tensor) re-laid out as the band of its fused block tridiagonal
    form (block copies; zero where the fused form has no original block).
    Returns ``(fused band [..., fused_elems], fused sizes)``."""
    torch = __import__("torch")
    fs, fn, maps = _fuse_maps(sizes, w)
    lead = band.shape[:-1]
    out = torch.zeros(*lead, fn, dtype=band.dtype, device=band.device)
    for o, r, c, fo, fr, fc, r0, c0 in maps:
        fblk = out[..., fo:fo + fr * fc].view(*lead, fr, fc)
        fblk[..., r0:r0 + r, c0:c0 + c] = band[..., o:o + r * c].view(*lead, r, c)
    return out, fs


def unfuse_band(fband, sizes, w):
    """Inverse of :func:`fuse_band` restricted to the original band: the
    blocks ``(a, b)``, ``|a - b| <= w``, cut out of the fused band."""
    torch = __import__("torch")
    fs, fn, maps = _fuse_maps(sizes, w)
    _, n = band_layout(sizes, w)
    lead = fband.shape[:-1]
    out = torch.empty(*lead, n, dtype=fband.dtype, device=fband.device)
    for o, r, c, fo, fr, fc, r0, c0 in maps:
        fblk = fband[..., fo:fo + fr * fc].view(*lead, fr, fc)
        out[..., o:o + r * c].view(*lead, r, c).copy_(fblk[..., r0:r0 + r, c0:c0 + c])
    return out


def lesser_ndiag(sizes, band_n, H, sigma_L, sigma_R, E, sigma_less_L=None, sigma_less_R=None, less_diag=None,
                 precision="fp64", product_bits=0):
    """Keldysh ``G^<`` (and ``G^R``) bands of a block n-diagonal chain:
    ``negf_lesser`` on a plan of ``band_n`` diagonals, which for ``band_n >= 5``
    runs through the fused block tridiagonal form inside the library
    (``fuse_band`` / ``unfuse_band`` restate its layout in Python).  ``H``:
    band-packed torch CUDA tensor; ``sigma_*``: one matrix each (shared by all
    energies).  Returns ``(G_band, G_less)`` in the original band packing."""
    plan = Plan(sizes, band_n, len(E), precision=precision, outputs=NEGF_OUT_BAND | NEGF_OUT_LESSER,
                product_bits=product_bits)
    try:
        return plan.lesser(H, sigma_L, sigma_R, E, sigma_less_L, sigma_less_R, less_diag)
    finally:
        plan.close()


# ---------------------------------------------------------------------------
# Plan bound to torch tensors
# ---------------------------------------------------------------------------
class Plan:
    """A negf plan whose calls take and return torch CUDA tensors.

    ``sizes``: block sizes; ``band_n``: 3 or 5; ``n_energies``; ``precision``:
    ``"fp64"`` or ``"mixed"``; ``outputs``: NEGF_OUT_* mask.  The plan is bound
    to the torch CUDA stream current at construction.
    """

    def __init__(self, sizes, band_n=3, n_energies=1, n_domains=1, domain_first_block=None,
                 precision="fp64", refine_steps=0, outputs=NEGF_OUT_BAND | NEGF_OUT_G1N,
                 checkpoint_every=0, stream=None, product_bits=0, interface_levels=()):
        import torch
        self.torch = torch
        self.sizes = [int(b) for b in sizes]
        self.w = (band_n - 1) // 2
        self.band_n = band_n
        self.n_energies = int(n_energies)
        # The plan runs on a stream of its own (graph capture needs a created
        # stream); every call orders itself after the caller's current stream
        # and makes the caller's stream wait for it.
        self.stream = stream if stream is not None else torch.cuda.Stream()
        prec = {"fp64": NEGF_FP64, "mixed": NEGF_MIXED}[precision] if isinstance(precision, str) else precision
        self.handle = negf_plan(self.sizes, band_n, self.n_energies, n_domains, domain_first_block, prec,
                                refine_steps, outputs, checkpoint_every, self.stream.cuda_stream, product_bits,
                                interface_levels)
        self.band_elems = negf_band_elems(self.handle)
        self.n_domains = negf_plan_n_domains(self.handle)   # the choice made for n_domains = 0
        self.info = torch.zeros(self.n_energies, dtype=torch.int32, device="cuda")

    def close(self):
        """Destroy the plan (negf_destroy); idempotent."""
        if getattr(self, "handle", None):
            negf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status, where):
        if status != NEGF_OK:
            raise NegfError(status, where)

    def _enter(self):
        self.stream.wait_stream(self.torch.cuda.current_stream())

    def _leave(self):
        self.torch.cuda.current_stream().wait_stream(self.stream)

    def sync(self):
        """Wait for the plan's stream and raise on a device-reported error (negf_sync)."""
        s = negf_sync(self.handle)
        if s != NEGF_OK:
            raise NegfError(s, "negf_sync")

    def _sigmas(self, sigma_L, sigma_R):
        """Marshal the lead self-energies into the C-ABI form: one matrix each
        (stride 0) or per-energy stacks sharing one element stride.  When
        b_1 != b_N, per-energy stacks are copied into buffers padded to the
        larger block.  Returns (sigma_L, sigma_R, stride)."""
        if sigma_L.dim() == 2 and sigma_R.dim() == 2:
            return sigma_L.contiguous(), sigma_R.contiguous(), 0
        torch = self.torch
        nE = self.n_energies
        b0, bN = self.sizes[0], self.sizes[-1]
        if sigma_L.dim() == 2:
            sigma_L = sigma_L.expand(nE, b0, b0)
        if sigma_R.dim() == 2:
            sigma_R = sigma_R.expand(nE, bN, bN)
        stride = max(b0, bN) ** 2
        if b0 == bN:
            return sigma_L.contiguous(), sigma_R.contiguous(), stride
        pl = torch.zeros(nE, stride, dtype=sigma_L.dtype, device=sigma_L.device)
        pr = torch.zeros(nE, stride, dtype=sigma_R.dtype, device=sigma_R.device)
        pl[:, :b0 * b0] = sigma_L.reshape(nE, -1)
        pr[:, :bN * bN] = sigma_R.reshape(nE, -1)
        return pl, pr, stride

    def _unpad(self, buf, b, stride):
        if stride == 0:
            return buf.reshape(b, b)
        return buf.reshape(self.n_energies, stride)[:, :b * b].reshape(self.n_energies, b, b)

    def solve(self, H, sigma_L, sigma_R, E, band=True, g1n=True, out_band=None, out_g1n=None, sync=True):
        """Returns ``(G_band [n_E, band_elems] or None, G_1N [n_E, b1, bN] or None)``."""
        torch = self.torch
        nE = self.n_energies
        b0, bN = self.sizes[0], self.sizes[-1]
        Gb = out_band if out_band is not None else (
            torch.empty(nE, self.band_elems, dtype=torch.complex128, device="cuda") if band else None)
        G1 = out_g1n if out_g1n is not None else (
            torch.empty(nE, b0, bN, dtype=torch.complex128, device="cuda") if g1n else None)
        sigma_L, sigma_R, stride = self._sigmas(sigma_L, sigma_R)
        self._enter()
        st = negf_solve(self.handle, H, sigma_L, sigma_R, stride, E, Gb, G1, self.info)
        self._leave()
        self._check(st, "negf_solve")
        if sync:
            self.sync()
        return Gb, G1

    def solve_host(self, H, sigma_L, sigma_R, E, out_band, out_g1n=None, info=None):
        """negf_solve_host: every tensor in host memory (page-locked for full
        speed); returns the device status after the outputs have landed."""
        if sigma_L.dim() == 3 or sigma_R.dim() == 3:
            raise ValueError("solve_host takes one Sigma_L / Sigma_R for all energies")
        info = info if info is not None else self.torch.zeros(self.n_energies, dtype=self.torch.int32).pin_memory()
        st = negf_solve_host(self.handle, H, sigma_L, sigma_R, 0, E, out_band, out_g1n, info)
        self._check(st, "negf_solve_host")
        return info

    def autotune(self, H, sigma_L, sigma_R, E, out_band=None, out_g1n=None, reps=2):
        """Times the solve schedule with 1, 2, 3, 4, 6, 8 energy groups on these
        inputs and keeps the fastest (negf_autotune).  Returns
        ``(best_groups, {groups: ms})``."""
        torch = self.torch
        nE = self.n_energies
        b0, bN = self.sizes[0], self.sizes[-1]
        Gb = out_band if out_band is not None else torch.empty(nE, self.band_elems, dtype=torch.complex128,
                                                               device="cuda")
        G1 = out_g1n if out_g1n is not None else torch.empty(nE, b0, bN, dtype=torch.complex128, device="cuda")
        sigma_L, sigma_R, stride = self._sigmas(sigma_L, sigma_R)
        self._enter()
        st, best, ms = negf_autotune(self.handle, H, sigma_L, sigma_R, stride, E, Gb, G1, self.info, reps)
        self._leave()
        self._check(st, "negf_autotune")
        self.sync()
        return best, {g: t for g, t in zip(AUTOTUNE_GROUPS, ms) if t >= 0}

    def tune_precision(self, H, sigma_L, sigma_R, E, tol=1e-6, band=True, g1n=True):
        """Keeps the narrowest product width whose results stay within ``tol``
        of a 56-bit solve of these inputs (negf_tune_precision).  Returns
        ``(bits, deviation)``."""
        torch = self.torch
        nE = self.n_energies
        b0, bN = self.sizes[0], self.sizes[-1]
        mk = lambda *shape: torch.empty(*shape, dtype=torch.complex128, device="cuda")
        Gb, Gr = (mk(nE, self.band_elems), mk(nE, self.band_elems)) if band else (None, None)
        G1, G1r = (mk(nE, b0, bN), mk(nE, b0, bN)) if g1n else (None, None)
        sigma_L, sigma_R, stride = self._sigmas(sigma_L, sigma_R)
        self._enter()
        st, bits, dev = negf_tune_precision(self.handle, H, sigma_L, sigma_R, stride, E, Gb, G1, self.info, Gr, G1r,
                                            tol)
        self._leave()
        self._check(st, "negf_tune_precision")
        return bits, dev

    def lesser(self, H, sigma_L, sigma_R, E, sigma_less_L=None, sigma_less_R=None, less_diag=None,
               out_band=None, out_less=None, sync=True):
        """Selected blocks of ``G^< = G^R Sigma^< G^A`` (negf_lesser).  Returns
        ``(G_band, G_less)``, both ``[n_E, band_elems]``."""
        torch = self.torch
        nE = self.n_energies
        Gb = out_band if out_band is not None else torch.empty(nE, self.band_elems, dtype=torch.complex128,
                                                               device="cuda")
        Gl = out_less if out_less is not None else torch.empty(nE, self.band_elems, dtype=torch.complex128,
                                                               device="cuda")
        sigma_L, sigma_R, stride = self._sigmas(sigma_L, sigma_R)
        sls = 0
        if sigma_less_L is not None or sigma_less_R is not None:
            b0, bN = self.sizes[0], self.sizes[-1]
            zl = sigma_less_L if sigma_less_L is not None else torch.zeros(b0, b0, dtype=torch.complex128, device="cuda")
            zr = sigma_less_R if sigma_less_R is not None else torch.zeros(bN, bN, dtype=torch.complex128, device="cuda")
            sigma_less_L, sigma_less_R, sls = self._sigmas(zl, zr)
        self._enter()
        st = negf_lesser(self.handle, H, sigma_L, sigma_R, stride, E, sigma_less_L, sigma_less_R, sls,
                         less_diag, Gb, Gl, self.info)
        self._leave()
        self._check(st, "negf_lesser")
        if sync:
            self.sync()
        return Gb, Gl

    def band_residual(self, H, sigma_L, sigma_R, E, G_band, sync=True):
        """Per-energy ``sqrt(sum_i ||(M G)_ii - I||_F^2 / sum_i b_i)`` of a band
        (negf_band_residual)."""
        torch = self.torch
        res = torch.empty(self.n_energies, dtype=torch.float64, device="cuda")
        sigma_L, sigma_R, stride = self._sigmas(sigma_L, sigma_R)
        self._enter()
        st = negf_band_residual(self.handle, H, sigma_L, sigma_R, stride, E, G_band, res)
        self._leave()
        self._check(st, "negf_band_residual")
        if sync:
            self.sync()
        return res

    def transmission(self, H, sigma_L, sigma_R, E, out=None, sync=True):
        """``T(E)`` per energy (negf_transmission); returns a float64 tensor ``[n_E]``."""
        torch = self.torch
        T = out if out is not None else torch.empty(self.n_energies, dtype=torch.float64, device="cuda")
        sigma_L, sigma_R, stride = self._sigmas(sigma_L, sigma_R)
        self._enter()
        st = negf_transmission(self.handle, H, sigma_L, sigma_R, stride, E, T, self.info)
        self._leave()
        self._check(st, "negf_transmission")
        if sync:
            self.sync()
        return T

    def grad(self, H, sigma_L, sigma_R, E, dL_dT, sync=True):
        """Returns ``(T, dH, dSigma_L, dSigma_R)``; each self-energy gradient
        has the shape of its input (a Sigma given once for all energies gets
        the energy-summed gradient, computed by the library)."""
        torch = self.torch
        nE = self.n_energies
        T = torch.empty(nE, dtype=torch.float64, device="cuda")
        dH = torch.empty(self.band_elems, dtype=torch.complex128, device="cuda")
        per = (sigma_L.dim() == 3, sigma_R.dim() == 3)
        sigma_L, sigma_R, stride = self._sigmas(sigma_L, sigma_R)
        b = (self.sizes[0], self.sizes[-1])
        outs, ostr = [], []
        for side in range(2):
            if per[side]:
                outs.append(torch.empty(nE, stride, dtype=torch.complex128, device="cuda"))
                ostr.append(stride)
            else:
                outs.append(torch.empty(b[side], b[side], dtype=torch.complex128, device="cuda"))
                ostr.append(0)
        dL = dL_dT.contiguous()
        self._enter()
        st = negf_grad_strided(self.handle, H, sigma_L, sigma_R, stride, E, dL, T, dH, outs[0], ostr[0], outs[1],
                               ostr[1], self.info)
        self._leave()
        self._check(st, "negf_grad_strided")
        if sync:
            self.sync()
        dSL = self._unpad(outs[0], b[0], ostr[0])
        dSR = self._unpad(outs[1], b[1], ostr[1])
        return T, dH, dSL, dSR


def _autograd():
    import torch

    class Transmission(torch.autograd.Function):
        """``T(E) = Tr[Gamma_L G_1N Gamma_R G_1N^H]`` with the library's adjoint
        as backward.  ``Transmission.apply(plan, H, sigma_L, sigma_R, E)``: the
        plan must have been created with ``NEGF_OUT_GRAD``."""

        @staticmethod
        def forward(ctx, plan, H, sigma_L, sigma_R, E):
            """T(E) for the given inputs; saves them for the adjoint."""
            ctx.plan = plan
            ctx.save_for_backward(H, sigma_L, sigma_R, E)
            return plan.transmission(H, sigma_L, sigma_R, E)

        @staticmethod
        def backward(ctx, gT):
            """The library's adjoint (negf_grad) with the incoming dL/dT as energy weights."""
            H, sL, sR, E = ctx.saved_tensors
            _, dH, dSL, dSR = ctx.plan.grad(H, sL, sR, E, gT.to(torch.float64))
            return None, dH, dSL, dSR, None

    return Transmission


def __getattr__(name):
    if name == "Transmission":
        return _autograd()
    raise AttributeError(name)
