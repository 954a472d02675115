"""Converged energies on the GPU against the oracle's stored values.

tests/golden/energies.json is written by tests/golden/make_golden.py, which calls
only the FP64 oracle.  FP64 must agree to 1e-10 Eh; the split modes (split
iterations, then FP64 refinement; T3 kept in FP32) to 1e-6 Eh.
"""
import json
import os

import pytest

from paper_2607_00981_gb300 import binding as B
from paper_2607_00981_gb300.synth import workload

from ._helpers import gpu_lib

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "energies.json")


def _golden(name):
    if not os.path.exists(GOLDEN):
        pytest.skip("golden energies not generated")
    data = json.load(open(GOLDEN))
    if name not in data:
        pytest.skip(f"no golden energy for {name}")
    return data[name]["energy"]


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol_e,tol_r", [(B.FP64, 1e-10, 1e-10), (B.SPLIT_BF16X3, 1e-6, 1e-8),
                                              (B.SPLIT_TF32X3, 1e-6, 1e-8)], ids=["fp64", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("f64_tc", [0, 1], ids=["fp64-units", "fp64-tensor-cores"])
def test_converged_energy_o6v48w(prec, tol_e, tol_r, f64_tc):
    """FP64 contractions on the FP64 units or on the tensor cores (digit planes; for
    split contexts those are the final iterations)."""
    E0 = _golden("o6v48w")
    inst = workload("o6v48w")
    ctx = B.Context(gpu_lib(), inst.o, inst.v, inst.naux, precision=prec, tol=tol_r, max_iter=300, f64_tc=f64_tc)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.init_mp2()
    E, it, nrm, conv = ctx.solve()
    ctx.close()
    assert conv, (it, nrm)
    assert abs(E - E0) < tol_e, (E, E0)
