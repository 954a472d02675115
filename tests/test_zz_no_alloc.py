"""The allocation-free residual-norm entry point agrees with rccsdt_postprocess.

rccsdt_residual_norms_noalloc exists for callers that cannot allocate device
memory (a framework that owns all device memory through its pool allocator, or
a service that must not allocate after start-up).  Its norms are checked against
the library's own entry point and against the oracle's weighted compact norm
(itself pinned to the full-storage norm), the device's free memory is checked to
stay the same across calls, and the largest size its fixed scratch takes
(o = 28, n3 = 4060 blocks) is run.  This file is collected after the parity
suites so that a run stopping at the first failure has run those first.
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


def _oracle_norms(r1, r2, r3c, o):
    """{|R1|, |R2|, |R3|, |R|} with the oracle's block multiplicities."""
    w = oc.weights(o)
    s1, s2 = float(np.sum(r1 ** 2)), float(np.sum(r2 ** 2))
    s3 = float(np.sum(w * np.sum(r3c.reshape(len(w), -1) ** 2, axis=1)))
    full = oc.residual_norm(r1, r2, r3c, o)
    assert abs(full - np.sqrt(s1 + s2 + s3)) <= 1e-14 * max(1.0, full)
    return np.array([np.sqrt(s1), np.sqrt(s2), np.sqrt(s3), full])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2607_00981_gb300.build import build
    lib = ctypes.CDLL(build())
    fn = _noalloc(lib)
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    assert fn(29, 4, dummy, dummy, dummy, dummy, None) == B.ERR_ARG
    assert fn(0, 4, dummy, dummy, dummy, dummy, None) == B.ERR_ARG
    assert fn(3, 4, None, dummy, dummy, dummy, None) == B.ERR_ARG


def _run_twice(fn, o, v, dev_inputs, expected, tol):
    """Two calls in a row (after a first one that does the per-device set-up); each
    result within `tol` of every row of `expected`; device free memory unchanged."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    outs = [torch.full((4,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
    ptrs = [d.data_ptr() for d in dev_inputs]
    assert fn(o, v, *ptrs, outs[0].data_ptr(), stream) == B.OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for out in outs[1:]:
        assert fn(o, v, *ptrs, out.data_ptr(), stream) == B.OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for ref in expected:
            assert np.all(np.abs(got - ref) <= tol * np.maximum(1.0, np.abs(ref))), (got, ref)
    assert torch.cuda.mem_get_info()[0] == free0


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
    _run_twice(fn, o, v, dev, [ref, _oracle_norms(r1, r2, rp3, o)], 1e-11)


@pytest.mark.gpu
def test_noalloc_at_the_largest_occupied_count():
    """o = 28 fills 4060 of the 4096 block slots; the R1 and R2 slots follow them."""
    import torch
    lib = gpu_lib()
    fn = _noalloc(lib)
    o, v = 28, 2
    rng = np.random.default_rng(28)
    r1 = rng.standard_normal((o, v))
    r2 = rng.standard_normal((o, o, v, v))
    r3c = rng.standard_normal((oc.n3(o), v, v, v))
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (r1, r2, r3c)]
    _run_twice(fn, o, v, dev, [_oracle_norms(r1, r2, r3c, o)], 1e-12)
