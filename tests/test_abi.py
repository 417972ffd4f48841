"""The C-ABI library builds, loads, and exports every entry point declared in
include/chfsi.h (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

from paper_1206_3768_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "chfsi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(chfsi_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("chfsi_create", "chfsi_solve_sequence", "chfsi_solve_next", "chfsi_destroy",
                     "chfsi_filter", "chfsi_orthonormalize", "chfsi_rayleigh_ritz",
                     "chfsi_residuals", "chfsi_cholesky", "chfsi_reduce", "chfsi_lanczos",
                     "chfsi_degrees", "chfsi_heev", "chfsi_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    for n in _declared():
        assert n in binding._SIGS, n
        assert hasattr(binding, n) or n == "chfsi_default_opts", n


def test_default_options_follow_table3():
    binding.load()
    o = binding.default_opts()
    # Table 3 (ChFSI column): degree 25 (upper end of the adaptive range), lanczos-iter >= 10.
    assert o.deg_max == 25
    assert o.lanczos_k_warm == 10
    assert o.lanczos_k_cold <= 3 * 40  # within "10 : 3 x blk" for any blk >= 14


def test_create_rejects_bad_sizes_without_touching_the_gpu():
    lib = binding.load()
    ctx = ctypes.c_void_p()
    assert lib.chfsi_create(ctypes.byref(ctx), 0, 10, None) == binding.CHFSI_EINVAL
    assert lib.chfsi_create(ctypes.byref(ctx), 10, 20, None) == binding.CHFSI_EINVAL
    assert lib.chfsi_create(None, 10, 5, None) == binding.CHFSI_EINVAL
