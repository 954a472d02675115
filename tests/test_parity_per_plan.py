"""Element-by-element parity of the per-plan engine (the one the o = 16, v = 160
workload runs) with the FP64 oracle at a size where its launch shapes are those of
the large workload: o = 8, v = 48 (120 stored blocks), the pp-ladder cut into two
block ranges (100 + 20 blocks, options.pp_unit_bytes), so that

* the first range's sum and difference GEMMs have 150-190 output tiles (more than
  one persistent wave) and run without split-K, the exchanged-operand view through
  the column-mirror epilogue on 256-wide tiles;
* the second range's GEMMs are short (40 tiles) and take the split-K path;
* the ring, hh-ladder and T2 terms run one launch unit per occupied pair.

Inputs carry full 53-bit mantissas (T3 rounds when stored in FP32).  Bars,
relative to the largest residual element: 3xBF16 5e-5; FP64 on the FP64 units
(DFMA) 1e-11; FP64 with its large contractions on the tensor cores (digit planes)
5e-10.  The digit-plane engine is exact to about 2^-38 of the operands' row and
column maxima per product; over K = v^2 = 2304 terms of full-precision operands
that is 2^-38 sqrt(K) ~ 2e-10 of a typical element (1.1e-10 measured), so its bar
is set from that bound rather than from the DFMA path's.
"""
import numpy as np
import pytest

from oracle import compact as oc
from paper_2607_00981_gb300 import binding as B
from paper_2607_00981_gb300.synth import make_instance, random_amplitudes_compact

from ._helpers import gpu_lib

O, V, NAUX = 8, 48, 224
PP_UNIT_BLOCKS = 100
# one stored block's T panel in the pp-ladder: v rows of round_up(v^2, 64) doubles
PP_UNIT_BYTES = PP_UNIT_BLOCKS * V * ((V * V + 63) // 64 * 64) * 8


@pytest.fixture(scope="module")
def case():
    inst = make_instance(O, V, NAUX, seed=48)
    t1, t2, t3c = random_amplitudes_compact(O, V, seed=49)
    R1, R2, R3 = oc.residuals_compact(inst.L, inst.fock_diag, t1, t2, t3c)
    return inst, (t1, t2, t3c), (R1, R2, oc.postprocess(R3, O))


@pytest.mark.gpu
@pytest.mark.parametrize("prec,f64_tc,tol", [(B.SPLIT_BF16X3, 0, 5e-5), (B.FP64, 0, 1e-11), (B.FP64, 1, 5e-10)],
                         ids=["bf16x3", "fp64-units", "fp64-tensor-cores"])
def test_per_plan_engine_at_mid_size(case, prec, f64_tc, tol):
    inst, (t1, t2, t3c), (R1, R2, P3) = case
    ctx = B.Context(gpu_lib(), O, V, NAUX, precision=prec, f64_tc=f64_tc, grouped_bytes=0,
                    pp_unit_bytes=PP_UNIT_BYTES)
    assert ctx.engine_info()["grouped"] == 0
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(t1, t2, t3c)
    ctx.build_intermediates()
    ctx.enable_timing(True)
    ctx.residual()
    st = ctx.step_times()
    ctx.enable_timing(False)
    # two block ranges x three views x (sum, difference) GEMMs
    assert int(st[10]) == 2 * 3 * 2
    norms = ctx.postprocess()
    r1, r2, r3 = ctx.residuals()
    scale = max(1.0, np.abs(P3).max())
    assert np.abs(r1 - R1).max() / scale < tol
    assert np.abs(r2 - R2).max() / scale < tol
    assert np.abs(oc.postprocess(r3, O) - P3).max() / scale < tol
    ref = oc.residual_norm(R1, R2, P3, O)
    assert abs(norms[3] - ref) < tol * max(1.0, ref)
    ctx.close()
