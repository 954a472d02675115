"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/rccsdt.h declares (no compute calls here)."""
import ctypes
import os
import re

from ._helpers import ROOT


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rccsdt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rccsdt_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rccsdt_create", "rccsdt_set_hamiltonian", "rccsdt_set_amplitudes",
                     "rccsdt_build_intermediates", "rccsdt_residual", "rccsdt_postprocess",
                     "rccsdt_update", "rccsdt_energy", "rccsdt_iterate", "rccsdt_solve", "rccsdt_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2607_00981_gb300.build import build
    lib = ctypes.CDLL(build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_iteration_fma_matches_the_operation_count():
    from oracle import opcount
    from paper_2607_00981_gb300.build import build
    lib = ctypes.CDLL(build())
    lib.rccsdt_iteration_fma.restype = ctypes.c_double
    lib.rccsdt_iteration_fma.argtypes = [ctypes.c_int, ctypes.c_int]
    for o, v in [(3, 12), (8, 80), (16, 160)]:
        assert lib.rccsdt_iteration_fma(o, v) == opcount.compact_fma(o, v)
