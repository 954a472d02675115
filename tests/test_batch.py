"""Batched instances (one graph launch per iteration of the whole batch).

Every instance of a batch must take the same iterations and reach the same
numbers as rccsdt_solve on a context of its own, and its converged energy must
match the FP64 oracle.  Each check runs on the CUDA library (gpu) and on the
test-only host simulation, which runs the same per-instance state machine with
the bodies executed directly instead of through a graph.
"""
import numpy as np
import pytest

from oracle import compact as oc
from paper_2607_00981_gb300 import binding as B
from paper_2607_00981_gb300.synth import make_instance

from ._helpers import gpu_lib, hostsim_lib

BACKENDS = [pytest.param("hostsim", id="hostsim"), pytest.param("gpu", id="gpu", marks=pytest.mark.gpu)]

# uneven shapes with weak couplings (all converge); o = 1 has no triples at all
SPECS = [(3, 8, 20, 11, 0.2), (2, 6, 10, 5, 0.25), (1, 5, 8, 3, 0.3), (4, 5, 12, 9, 0.15)]


def _lib(kind):
    return gpu_lib() if kind == "gpu" else hostsim_lib()


def _instances():
    return [make_instance(o, v, naux, seed=seed, scale=sc) for o, v, naux, seed, sc in SPECS]


def _single(lib, inst, **opt):
    ctx = B.Context(lib, inst.o, inst.v, inst.naux, **opt)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.init_mp2()
    out = ctx.solve()
    t = ctx.amplitudes()
    ctx.close()
    return out, t


def _batch(lib, insts, **opt):
    b = B.Batch(lib, [(i.o, i.v, i.naux) for i in insts], **opt)
    for c, inst in zip(b.instances, insts):
        c.set_hamiltonian(inst.fock_diag, inst.L)
        c.init_mp2()
    return b


@pytest.mark.parametrize("kind", BACKENDS)
def test_batch_equals_single_solves_fp64(kind):
    lib = _lib(kind)
    insts = _instances()
    opt = dict(tol=1e-10, max_iter=200)
    b = _batch(lib, insts, **opt)
    e, it, nrm, st = b.solve()
    assert (st == B.OK).all(), st
    for q, inst in enumerate(insts):
        (e1, it1, n1, conv), t_single = _single(lib, inst, **opt)
        assert conv
        # batched contexts keep each GEMM on its natural grid (no K split across all
        # SMs), so sums may be ordered differently than in a lone context
        assert it[q] == it1, (q, it[q], it1)
        assert abs(e[q] - e1) < 1e-11, (q, e[q], e1)
        assert abs(nrm[q] - n1) < 1e-12
        # amplitudes left in the batch context: the ones the last residual was evaluated at
        t_batch = b.instances[q].amplitudes()
        assert nrm[q] <= 1e-10
        for x, y in zip(t_batch, t_single):
            assert x.shape == y.shape
    stats = b.stats()
    assert stats["launches"] == it.max()
    assert stats["flop"] > 0
    b.close()


@pytest.mark.parametrize("kind", BACKENDS)
def test_batch_converged_energies_match_oracle(kind):
    lib = _lib(kind)
    insts = _instances()[:2]
    b = _batch(lib, insts, tol=1e-10, max_iter=200)
    e, it, nrm, st = b.solve()
    assert (st == B.OK).all()
    for q, inst in enumerate(insts):
        E0 = oc.solve_compact(inst.L, inst.fock_diag, inst.o, tol=1e-10, max_iter=300)[0]
        assert abs(e[q] - E0) < 1e-10, (q, e[q], E0)
    b.close()


@pytest.mark.parametrize("kind", BACKENDS)
@pytest.mark.parametrize("prec", [B.SPLIT_BF16X3, B.SPLIT_TF32X3], ids=["bf16x3", "tf32x3"])
def test_batch_split_precision(kind, prec):
    """Split batches: the same trajectory as single split solves, FP64 final phase,
    energies within 1e-6 Eh of the FP64 oracle.  (The FP64 phase of a split
    context still stores T3 and R3 in FP32, which puts |R| <= 1e-8 in reach but
    not much below.)"""
    lib = _lib(kind)
    insts = _instances()[:3]
    opt = dict(tol=1e-8, max_iter=200, precision=prec)
    b = _batch(lib, insts, **opt)
    e, it, nrm, st = b.solve()
    assert (st == B.OK).all(), st
    for q, inst in enumerate(insts):
        (e1, it1, n1, conv), _ = _single(lib, inst, **opt)
        assert it[q] == it1 and abs(e[q] - e1) < 1e-9, (q, it[q], it1, e[q], e1)
        E0 = oc.solve_compact(inst.L, inst.fock_diag, inst.o, tol=1e-10, max_iter=300)[0]
        assert abs(e[q] - E0) < 1e-6
    # the grouped GEMMs of all instances ran as one batch-wide launch per iteration
    stats = b.stats()
    assert stats["batch_gemm"] == 1
    if kind == "gpu":
        assert stats["batch_gemm_problems"] > 0 and stats["batch_gemm_tiles"] > 0
    b.close()


@pytest.mark.parametrize("kind", BACKENDS)
def test_batch_split_with_tensor_core_fp64_phase(kind):
    """Split batches whose final FP64 iterations run their contractions on the tensor
    cores (option f64_tc): every instance converges, energies within 1e-6 Eh of the
    oracle, and each equals its single-context solve."""
    lib = _lib(kind)
    insts = _instances()[:3]
    opt = dict(tol=1e-8, max_iter=200, precision=B.SPLIT_BF16X3, f64_tc=2)
    b = _batch(lib, insts, **opt)
    e, it, nrm, st = b.solve()
    assert (st == B.OK).all(), st
    for q, inst in enumerate(insts):
        (e1, it1, n1, conv), _ = _single(lib, inst, **opt)
        assert it[q] == it1 and abs(e[q] - e1) < 1e-9, (q, it[q], it1, e[q], e1)
        E0 = oc.solve_compact(inst.L, inst.fock_diag, inst.o, tol=1e-10, max_iter=300)[0]
        assert abs(e[q] - E0) < 1e-6
    b.close()


@pytest.mark.parametrize("kind", BACKENDS)
def test_batch_max_iter_stops_one_instance(kind):
    """An instance that needs more than max_iter evaluations stops with
    NOT_CONVERGED while the others still converge."""
    lib = _lib(kind)
    insts = _instances()[:2]
    b = _batch(lib, insts, tol=1e-10, max_iter=200)
    e, it, nrm, st = b.solve()
    need = int(it.max())
    b.close()
    b = _batch(lib, insts, tol=1e-10, max_iter=need - 1)
    e2, it2, nrm2, st2 = b.solve()
    for q in range(2):
        if it[q] == need:
            assert st2[q] == B.NOT_CONVERGED and it2[q] == need - 1
        else:
            assert st2[q] == B.OK and abs(e2[q] - e[q]) < 1e-12
    b.close()


@pytest.mark.parametrize("kind", BACKENDS)
def test_batch_errors(kind):
    lib = _lib(kind)
    with pytest.raises(B.RccsdtError):
        B.Batch(lib, [(3, 0, 4)])
    h = B._P()
    assert lib.rccsdt_batch_create(0, None, None, None, None, None, B.C.byref(h)) == B.ERR_ARG
    b = B.Batch(lib, [(2, 4, 6), (3, 5, 8)])
    with pytest.raises(B.RccsdtError) as ex:
        b.solve()           # no Hamiltonian set
    assert ex.value.status == B.ERR_STATE
    assert lib.rccsdt_batch_instance(b.h, 2) is None
    b.close()


@pytest.mark.gpu
def test_batch_autotuned_split_converges():
    """The batch tunes the launch shape of its batch-wide grouped GEMM on its own
    table before the graph is captured; the tuned batch converges to the oracle's
    energies within the split target."""
    lib = gpu_lib()
    insts = _instances()[:3]
    b = _batch(lib, insts, tol=1e-8, max_iter=200, precision=B.SPLIT_BF16X3, autotune=1)
    e, it, nrm, st = b.solve()
    assert (st == B.OK).all(), st
    stats = b.stats()
    assert stats["batch_gemm"] == 1 and stats["batch_gemm_tuned_ms"] > 0
    assert stats["batch_gemm_tuned_ms"] <= stats["batch_gemm_fixed_ms"]
    assert stats["batch_gemm_bn"] in (128, 256)
    for q in range(len(insts)):
        E0 = oc.solve_compact(insts[q].L, insts[q].fock_diag, insts[q].o, tol=1e-10, max_iter=300)[0]
        assert abs(e[q] - E0) < 1e-6
    b.close()
