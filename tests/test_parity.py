"""Element-by-element parity of the library's iteration with the FP64 oracle.

Each check runs twice: on the CUDA library (marked gpu) and on the test-only
host simulation of the same plans (CPU).  Inputs are seeded; expected values
come from the oracle only.  FP64 bar: 1e-11 relative on every residual element
(the benchmark spec's bound is 1e-9 absolute), 1e-10 Eh on energies.
"""
import numpy as np
import pytest

from oracle import compact as oc
from oracle import rccsdt as ofull
from paper_2607_00981_gb300 import binding as B
from paper_2607_00981_gb300.synth import make_instance, random_amplitudes, workload

from ._helpers import gpu_lib, hostsim_lib, rel

BACKENDS = [pytest.param("hostsim", id="hostsim"), pytest.param("gpu", id="gpu", marks=pytest.mark.gpu)]


def _lib(kind):
    return gpu_lib() if kind == "gpu" else hostsim_lib()


def _ctx(kind, o, v, naux, **kw):
    return B.Context(_lib(kind), o, v, naux, **kw)


# sizes span several 64-wide tiles with ragged tails on the GPU, three 16-label pair tiles
# (v = 35, the last ragged) and hit o = 1 / v = 1
SHAPES = [(3, 4, 8), (2, 7, 10), (4, 5, 12), (1, 6, 6), (3, 1, 4), (3, 12, 40), (5, 9, 20), (2, 35, 16)]


@pytest.mark.parametrize("kind", BACKENDS)
@pytest.mark.parametrize("o,v,naux", SHAPES)
@pytest.mark.parametrize("zbatch", ["all", "one"])
def test_residual_matches_oracle(kind, o, v, naux, zbatch):
    """zbatch: step (iii) unpacks the blocks of every z at once, or of one z at a
    time (a 1-byte unpack budget)."""
    inst = make_instance(o, v, naux, seed=o * 31 + v)
    t1, t2, t3 = random_amplitudes(o, v, seed=v * 7 + o)
    t3c = oc.pack(t3)
    ctx = _ctx(kind, o, v, naux, unpack_bytes=(1 << 30) if zbatch == "all" else 1)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(t1, t2, t3c)
    ctx.build_intermediates()
    ctx.residual()
    norms = ctx.postprocess()
    r1, r2, r3 = ctx.residuals()
    R1, R2, R3 = oc.residuals_compact(inst.L, inst.fock_diag, t1, t2, t3c)
    P3 = oc.postprocess(R3, o)
    scale = max(1.0, np.abs(R3).max())
    assert np.abs(r1 - R1).max() / scale < 1e-11
    assert np.abs(r2 - R2).max() / scale < 1e-11
    # raw R3 equals the oracle's after symmetrisation except on i=j=k blocks,
    # which purification zeroes; compare the post-processed residual everywhere
    assert np.abs(oc.postprocess(r3, o) - P3).max() / scale < 1e-11
    sym_g, sym_o = oc.symmetrise(r3, o), oc.symmetrise(R3, o)
    for b, (i, j, k) in enumerate(oc.triples(o)):
        if not (i == j == k):
            assert np.abs(sym_g[b] - sym_o[b]).max() / scale < 1e-11
    ref_norm = oc.residual_norm(R1, R2, P3, o)
    assert abs(norms[3] - ref_norm) < 1e-11 * max(1.0, ref_norm)
    assert abs(ctx.energy() - ofull.energy(inst.L, inst.fock_diag, t1, t2)) < 1e-12
    ctx.close()


@pytest.mark.parametrize("kind", BACKENDS)
def test_intermediates_match_oracle(kind):
    o, v, naux = 3, 5, 12
    inst = make_instance(o, v, naux, seed=2)
    t1, t2, t3 = random_amplitudes(o, v, seed=3)
    t3c = oc.pack(t3)
    ctx = _ctx(kind, o, v, naux)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(t1, t2, t3c)
    ctx.build_intermediates()
    *_, I = oc.residuals_compact(inst.L, inst.fock_diag, t1, t2, t3c, return_intermediates=True)
    names = {"Fvv": ("Fvv", (v, v)), "Foo": ("Foo", (o, o)), "Woooo": ("Woooo", (o, o, o, o)),
             "Wovvo": ("Wovvo", (o, v, v, o)), "Wovov": ("Wovov", (o, v, o, v)),
             "Wvvvo": ("Wvvvo", (v, v, v, o)), "Wvooo": ("Wvooo", (v, o, o, o)),
             "Wb_ovvo": ("Wbar_ovvo", (o, v, v, o)), "Wb_ovov": ("Wbar_ovov", (o, v, o, v))}
    for name, (key, shape) in names.items():
        assert rel(ctx.debug_copy(name, shape), I[key]) < 1e-12, name
    # W^{ab}_{de} before the Fock fold of the residual step
    assert rel(ctx.debug_copy("Wvvvv", (v, v, v, v)), I["Wvvvv"]) < 1e-12
    ctx.close()


@pytest.mark.parametrize("kind", BACKENDS)
@pytest.mark.parametrize("o,v,naux", [(3, 12, 40), (4, 5, 12), (2, 21, 12), (5, 9, 20)])
def test_residual_f64_on_tensor_cores_matches_oracle(kind, o, v, naux):
    """FP64 contractions on the BF16 tensor cores (six digit planes per operand,
    exact chunk sums): every residual element within 1e-10 of the oracle's, relative
    to the largest, and the same intermediates."""
    inst = make_instance(o, v, naux, seed=o * 13 + v)
    t1, t2, t3 = random_amplitudes(o, v, seed=v * 3 + o)
    t3c = oc.pack(t3)
    ctx = _ctx(kind, o, v, naux, f64_tc=2)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(t1, t2, t3c)
    ctx.build_intermediates()
    ctx.residual()
    ctx.postprocess()
    r1, r2, r3 = ctx.residuals()
    R1, R2, R3 = oc.residuals_compact(inst.L, inst.fock_diag, t1, t2, t3c)
    scale = max(1.0, np.abs(R3).max())
    assert np.abs(r1 - R1).max() / scale < 1e-10
    assert np.abs(r2 - R2).max() / scale < 1e-10
    assert np.abs(oc.postprocess(r3, o) - oc.postprocess(R3, o)).max() / scale < 1e-10
    ctx.close()


@pytest.mark.parametrize("kind", BACKENDS)
def test_trajectory_matches_oracle_on_the_o3v12_workload(kind):
    """Six Jacobi+DIIS iterations of the o=3, v=12 workload from the MP2 guess:
    energies and residual norms agree iteration by iteration."""
    inst = workload("o3v12")
    hist = []
    try:
        oc.solve_compact(inst.L, inst.fock_diag, 3, tol=1e-30, max_iter=6,
                         callback=lambda it, E, n: hist.append((E, n)))
    except RuntimeError:
        pass
    ctx = _ctx(kind, 3, 12, 40)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.init_mp2()
    for k in range(6):
        e, norms = ctx.iterate()
        assert abs(e - hist[k][0]) < 1e-10, (k, e, hist[k][0])
        assert abs(norms[3] - hist[k][1]) < 1e-9 * max(1.0, hist[k][1]), (k, norms[3], hist[k][1])
    ctx.close()


@pytest.mark.parametrize("kind", BACKENDS)
def test_converged_energy_matches_oracle(kind):
    """Converged RCCSDT energy at a weakly coupled o=3, v=8 instance (|R| <= 1e-10)."""
    o, v, naux = 3, 8, 20
    inst = make_instance(o, v, naux, seed=11, scale=0.2)
    E0 = oc.solve_compact(inst.L, inst.fock_diag, o, tol=1e-10, max_iter=300)[0]
    ctx = _ctx(kind, o, v, naux, tol=1e-10, max_iter=300)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.init_mp2()
    E, it, nrm, conv = ctx.solve()
    assert conv and nrm <= 1e-10
    assert abs(E - E0) < 1e-10
    ctx.close()


@pytest.mark.parametrize("kind", BACKENDS)
def test_one_occupied_orbital_has_no_triples(kind):
    """o = 1: the only block is i=j=k, so the post-processed R3 vanishes."""
    inst = make_instance(1, 5, 8, seed=2)
    t1, t2, t3 = random_amplitudes(1, 5, seed=1)
    ctx = _ctx(kind, 1, 5, 8)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(t1, t2, oc.pack(t3))
    ctx.build_intermediates()
    ctx.residual()
    norms = ctx.postprocess()
    assert norms[2] == 0.0
    ctx.close()


@pytest.mark.parametrize("kind", BACKENDS)
def test_errors_are_reported_not_raised_on_device(kind):
    lib = _lib(kind)
    with pytest.raises(B.RccsdtError):
        B.Context(lib, 0, 4, 4)
    ctx = B.Context(lib, 2, 3, 4)
    with pytest.raises(B.RccsdtError) as ei:
        ctx.build_intermediates()  # no Hamiltonian yet
    assert ei.value.status == B.ERR_STATE
    ctx.close()


@pytest.mark.parametrize("prec,f64_tc", [(B.FP64, 0), (B.FP64, 2), (B.SPLIT_BF16X3, 0)],
                         ids=["fp64", "fp64-tensor-cores", "bf16x3"])
@pytest.mark.parametrize("o,v,naux", [(2, 16, 10), (2, 17, 10), (1, 33, 8)])
def test_pp_pair_tiles_edges_on_host(prec, f64_tc, o, v, naux):
    """Pair-tile edges of the pair-symmetric pp-ladder (one full 16-label tile; a tile
    plus one label, whose diagonal chunk has no difference pairs; two tiles plus one),
    per-plan engine on the host simulation of the same plans: the DFMA and digit-plane
    FP64 engines and 3xBF16, each with the row- and the column-mirror epilogue."""
    inst = make_instance(o, v, naux, seed=o + 5 * v)
    t1, t2, t3 = random_amplitudes(o, v, seed=v + 3 * o)
    t3c = oc.pack(t3)
    ctx = _ctx("hostsim", o, v, naux, precision=prec, grouped_bytes=0, f64_tc=f64_tc)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(t1, t2, t3c)
    ctx.build_intermediates()
    ctx.residual()
    ctx.postprocess()
    r1, r2, r3 = ctx.residuals()
    R1, R2, R3 = oc.residuals_compact(inst.L, inst.fock_diag, t1, t2, t3c)
    scale = max(1.0, np.abs(R3).max())
    tol = (1e-11 if f64_tc == 0 else 1e-10) if prec == B.FP64 else 5e-5
    assert np.abs(r1 - R1).max() / scale < tol
    assert np.abs(r2 - R2).max() / scale < tol
    assert np.abs(oc.postprocess(r3, o) - oc.postprocess(R3, o)).max() / scale < tol
    ctx.close()


@pytest.mark.parametrize("kind", BACKENDS)
@pytest.mark.parametrize("prec", [B.FP64, B.SPLIT_TF32X3], ids=["fp64", "tf32x3"])
def test_subspace_diis_trajectory_matches_oracle(kind, prec):
    """DIIS with T3 restricted to the 7 lowest of 12 virtual orbitals (the subspace
    DIIS of Sec. III.A.5): energies and residual norms of six iterations of the o=3,
    v=12 workload equal the oracle's iteration by iteration (FP32 T3 storage and
    3xTF32 products: 1e-5 relative)."""
    inst = workload("o3v12")
    hist = []
    try:
        oc.solve_compact(inst.L, inst.fock_diag, 3, tol=1e-30, max_iter=6, diis_t3_nvir=7,
                         callback=lambda it, E, n: hist.append((E, n)))
    except RuntimeError:
        pass
    ctx = _ctx(kind, 3, 12, 40, precision=prec, diis_t3_nvir=7)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.init_mp2()
    # 3xTF32 keeps about 21 bits per product; this strongly coupled workload (E ~ 1.4 Eh)
    # amplifies the first update's rounding to about 2e-6 of the next energy
    te, tn = (1e-10, 1e-9) if prec == B.FP64 else (1e-5, 1e-5)
    for k in range(6):
        e, norms = ctx.iterate()
        assert abs(e - hist[k][0]) < te * max(1.0, abs(hist[k][0])), (k, e, hist[k][0])
        assert abs(norms[3] - hist[k][1]) < tn * max(1.0, hist[k][1]), (k, norms[3], hist[k][1])
    ctx.close()


@pytest.mark.parametrize("kind", BACKENDS)
def test_subspace_diis_converges_to_the_oracle_energy(kind):
    """The converged energy does not depend on the DIIS subspace: a solve with T3 in
    DIIS over 4 of 8 virtual orbitals reaches the oracle's full-DIIS energy."""
    o, v, naux = 3, 8, 20
    inst = make_instance(o, v, naux, seed=11, scale=0.2)
    E0 = oc.solve_compact(inst.L, inst.fock_diag, o, tol=1e-10, max_iter=300)[0]
    ctx = _ctx(kind, o, v, naux, tol=1e-10, max_iter=300, diis_t3_nvir=4)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.init_mp2()
    E, it, nrm, conv = ctx.solve()
    assert conv and nrm <= 1e-10
    assert abs(E - E0) < 1e-10
    ctx.close()
