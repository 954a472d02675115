"""The allocation-free residual-norm entry point agrees with rccsdt_postprocess.

rccsdt_residual_norms_noalloc exists for callers that cannot allocate device
memory (a framework that owns all device memory through its pool allocator, or
a service that must not allocate after start-up).  This file is collected after the
parity suites so that a run stopping at the first failure has run those first.
"""
import ctypes

import numpy as np
import pytest

from oracle import compact as oc
from paper_2607_00981_gb300 import binding as B
from paper_2607_00981_gb300.synth import make_instance, random_amplitudes

from ._helpers import gpu_lib


def _noalloc(lib):
    fn = lib.rccsdt_residual_norms_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 5
    return fn


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2607_00981_gb300.build import build
    lib = ctypes.CDLL(build())
    fn = _noalloc(lib)
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    assert fn(29, 4, dummy, dummy, dummy, dummy, None) == B.ERR_ARG
    assert fn(0, 4, dummy, dummy, dummy, dummy, None) == B.ERR_ARG
    assert fn(3, 4, None, dummy, dummy, dummy, None) == B.ERR_ARG


@pytest.mark.gpu
def test_noalloc_norms_match_postprocess_on_two_calls():
    import torch
    lib = gpu_lib()
    fn = _noalloc(lib)
    o, v, naux = 4, 7, 12
    inst = make_instance(o, v, naux, seed=5)
    t1, t2, t3 = random_amplitudes(o, v, seed=6)
    ctx = B.Context(lib, o, v, naux)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.set_amplitudes(t1, t2, oc.pack(t3))
    ctx.build_intermediates()
    ctx.residual()
    ref = ctx.postprocess()
    r1, r2, _ = ctx.residuals()
    rp3 = ctx.debug_copy("rp3", (ctx.n3, v, v, v))
    ctx.close()
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (r1, r2, rp3)]
    for _ in range(2):
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        st = fn(o, v, dev[0].data_ptr(), dev[1].data_ptr(), dev[2].data_ptr(), out.data_ptr(),
                torch.cuda.current_stream().cuda_stream)
        assert st == B.OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-11 * np.maximum(1.0, np.abs(ref))), (got, ref)
