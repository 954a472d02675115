"""Failure detection without faulting a GPU.

* A short watchdog budget makes the tensor-core GEMMs' pipeline waits run out: the
  kernels set the context's status flag, retire their own copies and MMAs (those
  drains wait at least about a second whatever the budget), free TMEM and return;
  the call reports RCCSDT_ERR_TIMEOUT and a fresh context in the same process then
  gives the oracle's residual.  Engines: 3xBF16 per-plan and grouped
  (k_gemm_tc), FP64 on the tensor cores through digit planes (k_gemm_f64e).
* A NaN in the caller's amplitudes is reported as RCCSDT_ERR_NONFINITE (host
  simulation and GPU), and the context is usable again after new amplitudes.
"""
import numpy as np
import pytest

from oracle import compact as oc
from paper_2607_00981_gb300 import binding as B
from paper_2607_00981_gb300.synth import make_instance, random_amplitudes

from ._helpers import gpu_lib, hostsim_lib

BACKENDS = [pytest.param("hostsim", id="hostsim"), pytest.param("gpu", id="gpu", marks=pytest.mark.gpu)]
ENGINES = {"bf16x3-per-plan": dict(precision=B.SPLIT_BF16X3, grouped_bytes=0),
           "bf16x3-grouped": dict(precision=B.SPLIT_BF16X3),
           "fp64-tensor-cores": dict(precision=B.FP64, f64_tc=2)}


def _residual_error(ctx, inst, t1, t2, t3c, o):
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(t1, t2, t3c)
    ctx.build_intermediates()
    ctx.residual()
    ctx.postprocess()
    r1, r2, r3 = ctx.residuals()
    R1, R2, R3 = oc.residuals_compact(inst.L, inst.fock_diag, t1, t2, t3c)
    scale = max(1.0, np.abs(R3).max())
    return max(np.abs(r1 - R1).max(), np.abs(r2 - R2).max(),
               np.abs(oc.postprocess(r3, o) - oc.postprocess(R3, o)).max()) / scale


@pytest.mark.gpu
@pytest.mark.parametrize("engine", list(ENGINES))
def test_short_watchdog_reports_timeout_then_a_fresh_context_is_exact(engine):
    lib = gpu_lib()
    o, v, naux = 3, 20, 24
    inst = make_instance(o, v, naux, seed=2)
    t1, t2, t3 = random_amplitudes(o, v, seed=3)
    t3c = oc.pack(t3)
    opts = ENGINES[engine]
    ctx = B.Context(lib, o, v, naux, watchdog_cycles=1, **opts)   # raised to the 64-cycle minimum
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(t1, t2, t3c)
    with pytest.raises(B.RccsdtError) as ei:
        ctx.build_intermediates()
        ctx.residual()
    assert ei.value.status == B.ERR_TIMEOUT
    ctx.close()
    ctx = B.Context(lib, o, v, naux, **opts)
    tol = 1e-10 if opts["precision"] == B.FP64 else 5e-5
    assert _residual_error(ctx, inst, t1, t2, t3c, o) < tol
    ctx.close()


@pytest.mark.parametrize("kind", BACKENDS)
@pytest.mark.parametrize("prec", [B.FP64, B.SPLIT_BF16X3], ids=["fp64", "bf16x3"])
def test_nan_amplitude_is_reported_as_nonfinite(kind, prec):
    lib = gpu_lib() if kind == "gpu" else hostsim_lib()
    o, v, naux = 3, 6, 12
    inst = make_instance(o, v, naux, seed=8)
    t1, t2, t3 = random_amplitudes(o, v, seed=9)
    t3c = oc.pack(t3)
    bad = t1.copy()
    bad[1, 2] = np.nan
    ctx = B.Context(lib, o, v, naux, precision=prec)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(bad, t2, t3c)
    with pytest.raises(B.RccsdtError) as ei:
        ctx.iterate()
    assert ei.value.status == B.ERR_NONFINITE
    with pytest.raises(B.RccsdtError) as ei:
        ctx.energy()
    assert ei.value.status == B.ERR_NONFINITE
    # new amplitudes: the same context evaluates the oracle's residual
    tol = 1e-11 if prec == B.FP64 else 5e-5
    assert _residual_error(ctx, inst, t1, t2, t3c, o) < tol
    ctx.close()


def test_negative_watchdog_is_rejected():
    lib = hostsim_lib()
    with pytest.raises(B.RccsdtError) as ei:
        B.Context(lib, 2, 3, 4, watchdog_cycles=-5)
    assert ei.value.status == B.ERR_ARG
