"""Checkpoint and resume (rccsdt_save / rccsdt_load): an iteration resumed in a new
context from a saved state repeats the one the saved context takes next (the DIIS
history, its device counters and B matrix travel with the amplitudes): bit for bit on
the host simulation of the library's plans and for FP64 on the GPU (every reduction
of the library runs in a fixed order, with no atomics), to 1e-6 relative for 3xBF16
on the GPU (a lost DIIS state moves the next step by orders of magnitude more)."""
import numpy as np
import pytest

from paper_2607_00981_gb300 import binding as B
from paper_2607_00981_gb300.synth import make_instance

from ._helpers import gpu_lib, hostsim_lib

BACKENDS = [pytest.param("hostsim", id="hostsim"), pytest.param("gpu", id="gpu", marks=pytest.mark.gpu)]


def _lib(kind):
    return gpu_lib() if kind == "gpu" else hostsim_lib()


def _state(ctx):
    t1, t2, t3 = ctx.amplitudes()
    return np.concatenate([t1.ravel(), t2.ravel(), t3.ravel()])


@pytest.mark.parametrize("kind", BACKENDS)
@pytest.mark.parametrize("prec", [B.FP64, B.SPLIT_BF16X3], ids=["fp64", "bf16x3"])
def test_resume_repeats_the_next_iteration(kind, prec, tmp_path):
    o, v, naux = 3, 8, 20
    inst = make_instance(o, v, naux, seed=4, scale=0.3)
    opt = dict(precision=prec, diis_space=4)
    a = B.Context(_lib(kind), o, v, naux, **opt)
    a.set_hamiltonian(inst.fock_diag, inst.L)
    a.init_mp2()
    for _ in range(3):  # past the DIIS start: the history is in use
        a.iterate()
    path = tmp_path / "state.ck"
    a.save(path)
    t_saved = a.amplitudes()
    e_a, n_a = a.iterate()
    e_a2, n_a2 = a.iterate()
    s_a = _state(a)
    a.close()

    b = B.Context(_lib(kind), o, v, naux, **opt)
    b.set_hamiltonian(inst.fock_diag, inst.L)
    b.load(path)
    e_b, n_b = b.iterate()
    e_b2, n_b2 = b.iterate()
    s_b = _state(b)
    b.close()
    # control: the same amplitudes without the DIIS history take a different step
    c = B.Context(_lib(kind), o, v, naux, **opt)
    c.set_hamiltonian(inst.fock_diag, inst.L)
    c.set_amplitudes(*t_saved)
    c.iterate()
    c.iterate()
    s_c = _state(c)
    c.close()
    assert np.abs(s_c - s_a).max() > 1e-4 * np.abs(s_a).max()
    if kind == "hostsim" or prec == B.FP64:
        assert e_a == e_b and e_a2 == e_b2
        assert np.array_equal(n_a, n_b) and np.array_equal(n_a2, n_b2)
        assert np.array_equal(s_a, s_b)
    else:
        tol = 1e-6
        assert abs(e_a - e_b) <= tol * abs(e_a) and abs(e_a2 - e_b2) <= tol * abs(e_a2)
        assert np.abs(n_a2 - n_b2).max() <= tol * np.abs(n_a2).max()
        assert np.abs(s_a - s_b).max() <= tol * np.abs(s_a).max()


@pytest.mark.parametrize("kind", BACKENDS)
def test_checkpoint_errors(kind, tmp_path):
    lib = _lib(kind)
    o, v, naux = 2, 5, 10
    inst = make_instance(o, v, naux, seed=1)
    a = B.Context(lib, o, v, naux, diis_space=4)
    with pytest.raises(B.RccsdtError):  # nothing to save yet
        a.save(tmp_path / "x.ck")
    a.set_hamiltonian(inst.fock_diag, inst.L)
    a.init_mp2()
    a.iterate()
    path = tmp_path / "a.ck"
    a.save(path)
    with pytest.raises(B.RccsdtError):  # a directory is not writable as a file
        a.save(tmp_path)
    a.close()
    for kw in (dict(o=3, v=5, naux=10), dict(o=2, v=5, naux=10, diis_space=3),
               dict(o=2, v=5, naux=10, precision=B.SPLIT_BF16X3)):
        kw = dict(kw)
        c = B.Context(lib, kw.pop("o"), kw.pop("v"), kw.pop("naux"), **kw)
        with pytest.raises(B.RccsdtError):  # other sizes, DIIS options or t3 storage
            c.load(path)
        c.close()
    c = B.Context(lib, o, v, naux, diis_space=4)
    with pytest.raises(B.RccsdtError):
        c.load(tmp_path / "missing.ck")
    bad = tmp_path / "bad.ck"
    bad.write_bytes(b"not a checkpoint at all, just bytes" * 4)
    with pytest.raises(B.RccsdtError):
        c.load(bad)
    short = tmp_path / "short.ck"
    short.write_bytes(path.read_bytes()[:200])
    with pytest.raises(B.RccsdtError):
        c.load(short)
    c.close()
