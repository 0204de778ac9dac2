"""The C-ABI library builds, loads and exports every entry point that
include/negf.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "negf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(negf_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_expected_entry_points():
    names = _header_functions()
    for n in ["negf_plan", "negf_solve", "negf_transmission", "negf_grad", "negf_sync", "negf_destroy",
              "negf_band_offset", "negf_band_elems", "negf_workspace_bytes", "negf_status_string"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2605_19910_gb300", "libnegf.so"))
    for n in _header_functions():
        assert hasattr(lib, n), n


def test_status_strings_and_null_handling():
    import paper_2605_19910_gb300 as P
    assert P.negf_status_string(P.NEGF_OK) == "NEGF_OK"
    assert "singular" in P.negf_status_string(P.NEGF_ERR_SINGULAR).lower()
    # NULL plan handles are rejected without touching a device
    assert P.lib().negf_band_elems(None) == -1
    assert P.lib().negf_band_offset(None, 0, 0) == -1
    assert P.lib().negf_workspace_bytes(None) == 0
    assert P.negf_sync(None) == P.NEGF_ERR_ARG
    assert P.lib().negf_profile_read(None, None, None, None) == -1
    assert P.lib().negf_profile_read_issued(None, None, None, None, None) == -1
    P.negf_destroy(None)


def test_invalid_descriptors_are_rejected_before_any_launch():
    import paper_2605_19910_gb300 as P
    bad = [dict(block_sizes=[4, 4], band_n=4), dict(block_sizes=[4, 0]), dict(block_sizes=[4, 4], n_energies=0),
           dict(block_sizes=[4, 4], band_n=5), dict(block_sizes=[4, 200]), dict(block_sizes=[4, 4], precision=7),
           dict(block_sizes=[4, 4], outputs=64), dict(block_sizes=[4, 4], refine_steps=3),
           dict(block_sizes=[4, 4], checkpoint_every=-1), dict(block_sizes=[4, 4], product_bits=99),
           dict(block_sizes=[4] * 8, n_domains=-1), dict(block_sizes=[4] * 8, n_domains=0, domain_first_block=[0])]
    for kw in bad:
        with pytest.raises(P.NegfError) as ei:
            P.negf_plan(**kw)
        assert ei.value.status == P.NEGF_ERR_ARG, kw


def test_band_layout_matches_header_convention():
    import paper_2605_19910_gb300 as P
    off, n = P.band_layout([2, 3, 4], 1)
    # d = -1 first: (1,0), (2,1); then d = 0: (0,0),(1,1),(2,2); then d = +1: (0,1),(1,2)
    order = sorted(off, key=lambda k: off[k])
    assert order == [(1, 0), (2, 1), (0, 0), (1, 1), (2, 2), (0, 1), (1, 2)]
    assert n == 3 * 2 + 4 * 3 + 4 + 9 + 16 + 2 * 3 + 3 * 4
