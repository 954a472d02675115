"""Split-precision (3xBF16, 3xTF32) residuals against the FP64 oracle.

The large contractions run as hi*hi + hi*lo + lo*hi products with FP32
accumulation (tcgen05 on the GPU; FP32 emulation in the host simulation), T3 is
stored in FP32.  Bars, relative to the largest residual element: 3xBF16 keeps
about 16 bits per product, so 5e-5; 3xTF32 about 21 bits, so 5e-6.
"""
import numpy as np
import pytest

from oracle import compact as oc
from paper_2607_00981_gb300 import binding as B
from paper_2607_00981_gb300.synth import make_instance, random_amplitudes

from ._helpers import gpu_lib, hostsim_lib

BACKENDS = [pytest.param("hostsim", id="hostsim"), pytest.param("gpu", id="gpu", marks=pytest.mark.gpu)]
TOL = {B.SPLIT_BF16X3: 5e-5, B.SPLIT_TF32X3: 5e-6}


@pytest.mark.parametrize("kind", BACKENDS)
@pytest.mark.parametrize("prec", [B.SPLIT_BF16X3, B.SPLIT_TF32X3], ids=["bf16x3", "tf32x3"])
@pytest.mark.parametrize("o,v,naux", [(3, 12, 40), (4, 9, 16), (2, 21, 12)])
@pytest.mark.parametrize("grouped", [1, 0], ids=["grouped", "per-plan"])
def test_split_residual_matches_oracle(kind, prec, o, v, naux, grouped):
    """Both engines: the grouped residual (one grouped GEMM, output-stationary
    reduction) and the per-plan path (shared panels, two-phase scatter)."""
    lib = gpu_lib() if kind == "gpu" else hostsim_lib()
    inst = make_instance(o, v, naux, seed=o + v)
    t1, t2, t3 = random_amplitudes(o, v, seed=2 * v + o)
    t3c = oc.pack(t3)
    ctx = B.Context(lib, o, v, naux, precision=prec, grouped_bytes=(8 << 30) if grouped else 0)
    assert ctx.engine_info()["grouped"] == grouped
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(t1, t2, t3c)
    ctx.build_intermediates()
    ctx.residual()
    norms = ctx.postprocess()
    r1, r2, r3 = ctx.residuals()
    R1, R2, R3 = oc.residuals_compact(inst.L, inst.fock_diag, t1, t2, t3c)
    scale = max(1.0, np.abs(R3).max())
    tol = TOL[prec]
    assert np.abs(r1 - R1).max() / scale < tol
    assert np.abs(r2 - R2).max() / scale < tol
    assert np.abs(oc.postprocess(r3, o) - oc.postprocess(R3, o)).max() / scale < tol
    ref = oc.residual_norm(R1, R2, oc.postprocess(R3, o), o)
    assert abs(norms[3] - ref) < tol * max(1.0, ref)
    ctx.close()


@pytest.mark.parametrize("kind", BACKENDS)
@pytest.mark.parametrize("o,v,naux", [(3, 12, 40), (4, 9, 16)])
def test_split_step_iii_one_z_at_a_time(kind, o, v, naux):
    """Step (iii) on one z per batch (the S panel of the first contraction is then
    the second's; the second and third share one GEMM with stacked A operands)."""
    lib = gpu_lib() if kind == "gpu" else hostsim_lib()
    inst = make_instance(o, v, naux, seed=o + 2 * v)
    t1, t2, t3 = random_amplitudes(o, v, seed=v + o)
    t3c = oc.pack(t3)
    ctx = B.Context(lib, o, v, naux, precision=B.SPLIT_BF16X3, unpack_bytes=1)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(t1, t2, t3c)
    ctx.build_intermediates()
    ctx.residual()
    ctx.postprocess()
    r1, r2, r3 = ctx.residuals()
    R1, R2, R3 = oc.residuals_compact(inst.L, inst.fock_diag, t1, t2, t3c)
    scale = max(1.0, np.abs(R3).max())
    tol = TOL[B.SPLIT_BF16X3]
    assert np.abs(r1 - R1).max() / scale < tol
    assert np.abs(r2 - R2).max() / scale < tol
    assert np.abs(oc.postprocess(r3, o) - oc.postprocess(R3, o)).max() / scale < tol
    ctx.close()


@pytest.mark.parametrize("kind", BACKENDS)
@pytest.mark.parametrize("prec", [B.SPLIT_BF16X3, B.SPLIT_TF32X3], ids=["bf16x3", "tf32x3"])
@pytest.mark.parametrize("f64_tc", [0, 2], ids=["fp64-units", "fp64-tensor-cores"])
def test_split_solve_refines_to_fp64_energy(kind, prec, f64_tc):
    """Split iterations, then FP64 refinement (on the FP64 units, or on the tensor
    cores through digit planes): converged energy within 1e-6 Eh (the target) of the
    FP64 oracle's, at a weakly coupled o=3, v=8 instance."""
    lib = gpu_lib() if kind == "gpu" else hostsim_lib()
    o, v, naux = 3, 8, 20
    inst = make_instance(o, v, naux, seed=11, scale=0.2)
    E0 = oc.solve_compact(inst.L, inst.fock_diag, o, tol=1e-10, max_iter=300)[0]
    ctx = B.Context(lib, o, v, naux, precision=prec, tol=1e-8, max_iter=300, f64_tc=f64_tc)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.init_mp2()
    E, it, nrm, conv = ctx.solve()
    assert conv
    assert abs(E - E0) < 1e-6
    ctx.close()


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [None, 0, 1, 2, 3, 4, 5], ids=["tuned", "c0", "c1", "c2", "c3", "c4", "c5"])
def test_grouped_launch_shapes_match_oracle(shape):
    """Every launch shape of the grouped GEMM (256/128-wide tiles, problem orders,
    grids), and the one the autotuner picks, gives the oracle's residual."""
    lib = gpu_lib()
    o, v, naux = 3, 21, 30
    inst = make_instance(o, v, naux, seed=5)
    t1, t2, t3 = random_amplitudes(o, v, seed=9)
    t3c = oc.pack(t3)
    ctx = B.Context(lib, o, v, naux, precision=B.SPLIT_BF16X3, autotune=1 if shape is None else 2 + shape)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(t1, t2, t3c)
    ctx.build_intermediates()
    ctx.residual()
    ctx.postprocess()
    info = ctx.engine_info()
    assert info["grouped"] == 1 and info["tuned"] == 1
    if shape is not None:
        assert info["bn"] == (128 if shape in (2, 3, 5) else 256)
    r1, r2, r3 = ctx.residuals()
    R1, R2, R3 = oc.residuals_compact(inst.L, inst.fock_diag, t1, t2, t3c)
    scale = max(1.0, np.abs(R3).max())
    assert np.abs(oc.postprocess(r3, o) - oc.postprocess(R3, o)).max() / scale < TOL[B.SPLIT_BF16X3]
    assert np.abs(r2 - R2).max() / scale < TOL[B.SPLIT_BF16X3]
    ctx.close()


@pytest.mark.gpu
def test_t3_round_trip_through_pinned_and_pageable_host_memory():
    """An FP32-storage context reads and writes T3 in place when the caller's
    buffer is pinned host memory (or device memory) and through staging copies
    when it is pageable: all three give the same FP32-rounded amplitudes."""
    torch = pytest.importorskip("torch")
    lib = gpu_lib()
    o, v, naux = 3, 10, 24
    inst = make_instance(o, v, naux, seed=4)
    t1, t2, t3 = random_amplitudes(o, v, seed=5)
    t3c = np.ascontiguousarray(oc.pack(t3))
    ctx = B.Context(lib, o, v, naux, precision=B.SPLIT_BF16X3)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    want = t3c.astype(np.float32).astype(np.float64)
    outs = []
    for kind in ("pageable", "pinned", "device"):
        if kind == "pageable":
            src, dst = t3c, np.zeros_like(t3c)
        elif kind == "pinned":
            src = torch.from_numpy(t3c.copy()).pin_memory()
            dst = torch.zeros(t3c.shape, dtype=torch.float64).pin_memory()
        else:
            src = torch.from_numpy(t3c).cuda()
            dst = torch.zeros(t3c.shape, dtype=torch.float64, device="cuda")
        ctx.set_amplitudes(t1, t2, src)
        ctx.get_amplitudes(None, None, dst)
        got = dst if isinstance(dst, np.ndarray) else dst.cpu().numpy()
        assert np.array_equal(got, want), kind
        outs.append(got)
    ctx.close()


@pytest.mark.gpu
def test_t3_exchange_in_fp32_storage():
    """rccsdt_set/get_amplitudes_t3f32 move T3 in the split modes' FP32 storage as it
    is (pageable, pinned or device buffers), agree with the float64 calls on the same
    amplitudes (same residual norms), and are refused by an FP64 context."""
    torch = pytest.importorskip("torch")
    lib = gpu_lib()
    o, v, naux = 3, 10, 24
    inst = make_instance(o, v, naux, seed=4)
    t1, t2, t3 = random_amplitudes(o, v, seed=5)
    t3c = np.ascontiguousarray(oc.pack(t3))
    t3f = t3c.astype(np.float32)
    ctx = B.Context(lib, o, v, naux, precision=B.SPLIT_BF16X3)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    for kind in ("pageable", "pinned", "device"):
        if kind == "pageable":
            src, dst = t3f, np.zeros_like(t3f)
        elif kind == "pinned":
            src = torch.from_numpy(t3f.copy()).pin_memory()
            dst = torch.zeros(t3f.shape, dtype=torch.float32).pin_memory()
        else:
            src = torch.from_numpy(t3f).cuda()
            dst = torch.zeros(t3f.shape, dtype=torch.float32, device="cuda")
        ctx.set_amplitudes_t3f32(t1, t2, src)
        g1, g2 = np.zeros_like(t1), np.zeros_like(t2)
        ctx.get_amplitudes_t3f32(g1, g2, dst)
        got = dst if isinstance(dst, np.ndarray) else dst.cpu().numpy()
        assert np.array_equal(got, t3f), kind
        assert np.array_equal(g1, t1) and np.array_equal(g2, t2)
    # the same iteration from either entry point
    ctx.set_amplitudes_t3f32(t1, t2, t3f)
    e32, n32 = ctx.iterate()
    ctx.set_amplitudes(t1, t2, t3c)
    e64, n64 = ctx.iterate()
    assert e32 == e64 and np.array_equal(n32, n64)
    ctx.close()
    c64 = B.Context(lib, o, v, naux, precision=B.FP64)
    with pytest.raises(B.RccsdtError) as ei:
        c64.set_amplitudes_t3f32(t1, t2, t3f)
    assert ei.value.status == B.ERR_ARG
    with pytest.raises(ValueError):
        c64.set_amplitudes_t3f32(t1, t2, t3c)  # float64 array for the FP32 call
    c64.close()
