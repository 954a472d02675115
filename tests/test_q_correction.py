"""RCCSDT(Q) energy correction on the GPU (ABC-based algorithm, Sec. II.E.2) against
the FP64 oracle of the (Q) appendix (``oracle.q_correction``, itself pinned to the
spin-orbital CCSDT(Q) energy by brute force in determinant space).

* The one-time transposition of compact T3 to the virtual-triangular layout is pure
  data movement: bit for bit against the oracle's, FP64 and FP32 storage.
* E_(Q) at seeded amplitudes with full 53-bit mantissas (the expression is defined
  for any amplitudes with the column symmetries): FP64 within 1e-10 relative;
  FP32 arithmetic within 1e-5 relative (its error is stated by the test).
* o = 1: no quadruple excitation exists, the energy vanishes.
"""
import numpy as np
import pytest

from oracle import compact as oc
from oracle import q_correction as oq
from paper_2607_00981_gb300 import binding as B
from paper_2607_00981_gb300.synth import make_instance, random_amplitudes

from ._helpers import gpu_lib

SHAPES = [(2, 9, 12), (3, 20, 24), (4, 12, 16), (5, 8, 14)]


def _ctx(o, v, naux, prec=B.FP64):
    inst = make_instance(o, v, naux, seed=o + v)
    t1, t2, t3 = random_amplitudes(o, v, seed=3 * o + v)
    ctx = B.Context(gpu_lib(), o, v, naux, precision=prec)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(t1, t2, oc.pack(t3))
    return ctx, inst, t2, t3


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [B.FP64, B.SPLIT_BF16X3], ids=["fp64-storage", "fp32-storage"])
@pytest.mark.parametrize("o,v,naux", [(1, 6, 8), (3, 7, 10), (4, 5, 9)])
def test_virtual_triangular_transposition_is_exact(prec, o, v, naux):
    ctx, _, _, t3 = _ctx(o, v, naux, prec)
    t3c = oc.pack(t3)
    if prec != B.FP64:  # the context stores T3 in FP32
        t3c = t3c.astype(np.float32).astype(np.float64)
    got = ctx.t3_virtual_triangular()
    assert np.array_equal(got, oq.pack_virtual_triangular(t3c, o))
    ctx.close()


@pytest.mark.gpu
@pytest.mark.parametrize("o,v,naux", SHAPES)
def test_q_energy_matches_oracle(o, v, naux):
    ctx, inst, t2, t3 = _ctx(o, v, naux)
    ref = oq.energy_q(inst.L, inst.fock_diag, t2, t3, o)
    e64, info = ctx.q_energy(B.Q_FP64)
    assert abs(e64 - ref) <= 1e-10 * abs(ref), (e64, ref)
    e32, _ = ctx.q_energy(B.Q_FP32)
    err32 = abs(e32 - ref) / abs(ref)
    print(f"o={o} v={v}: E(Q) = {ref:.12e}; FP64 rel. error {abs(e64 - ref) / abs(ref):.2e}, "
          f"FP32 rel. error {err32:.2e}; {int(info['quadruples'])} quadruples")
    assert err32 < 1e-5
    ctx.close()


@pytest.mark.gpu
def test_q_energy_vanishes_for_one_occupied_orbital():
    ctx, inst, t2, t3 = _ctx(1, 6, 8)
    e, _ = ctx.q_energy(B.Q_FP64)
    assert abs(e) < 1e-14
    ctx.close()


@pytest.mark.gpu
def test_q_energy_from_a_split_context_and_errors():
    """A 3xBF16 context (FP32 T3) feeds the same kernels; a context without
    amplitudes reports RCCSDT_ERR_STATE; an unknown arithmetic RCCSDT_ERR_ARG."""
    o, v, naux = 3, 9, 12
    ctx, inst, t2, t3 = _ctx(o, v, naux, B.SPLIT_BF16X3)
    t3_32 = oc.unpack_full(oc.pack(t3).astype(np.float32).astype(np.float64), o)
    ref = oq.energy_q(inst.L, inst.fock_diag, t2, t3_32, o)
    e, _ = ctx.q_energy(B.Q_FP64)
    assert abs(e - ref) <= 1e-10 * abs(ref)
    with pytest.raises(B.RccsdtError) as ei:
        ctx.q_energy(7)
    assert ei.value.status == B.ERR_ARG
    ctx.close()
    bare = B.Context(gpu_lib(), o, v, naux)
    with pytest.raises(B.RccsdtError) as ei:
        bare.q_energy(B.Q_FP64)
    assert ei.value.status == B.ERR_STATE
    bare.close()
