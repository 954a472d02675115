"""Thin ctypes binding of the C ABI declared in ``include/rccsdt.h``.

Argument marshalling only: every step of the iteration runs in the CUDA
library.  Array arguments may be numpy arrays (host memory) or CUDA torch
tensors (device memory); both must be contiguous float64.  Functions keep the
C names without the ``rccsdt_`` prefix.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_NAME = "librccsdt.so"

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE, NOT_CONVERGED = 0, -1, -2, -3, -4, -5, -6, 1
FP64, SPLIT_BF16X3, SPLIT_TF32X3 = 0, 1, 2


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("diis_space", C.c_int),
                ("diis_start", C.c_int), ("diis_t3", C.c_int), ("max_iter", C.c_int),
                ("tol", C.c_double), ("watchdog_cycles", C.c_longlong), ("grouped_bytes", C.c_longlong),
                ("unpack_bytes", C.c_longlong), ("autotune", C.c_int), ("f64_tc", C.c_int),
                ("pp_unit_bytes", C.c_longlong), ("diis_t3_nvir", C.c_int)]


class RccsdtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rccsdt status {status}: {msg}")
        self.status = status


_P = C.c_void_p
_SIGS = {
    "rccsdt_options_default": (C.c_int, [C.POINTER(Options)]),
    "rccsdt_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(Options), _P, C.POINTER(_P)]),
    "rccsdt_device_bytes": (C.c_longlong, [_P]),
    "rccsdt_set_hamiltonian": (C.c_int, [_P, _P, _P]),
    "rccsdt_set_amplitudes": (C.c_int, [_P, _P, _P, _P]),
    "rccsdt_init_mp2": (C.c_int, [_P]),
    "rccsdt_set_precision": (C.c_int, [_P, C.c_int]),
    "rccsdt_build_intermediates": (C.c_int, [_P]),
    "rccsdt_residual": (C.c_int, [_P]),
    "rccsdt_postprocess": (C.c_int, [_P, _P]),
    "rccsdt_update": (C.c_int, [_P]),
    "rccsdt_energy": (C.c_int, [_P, _P]),
    "rccsdt_iterate": (C.c_int, [_P, _P, _P]),
    "rccsdt_solve": (C.c_int, [_P, _P, _P, _P]),
    "rccsdt_get_amplitudes": (C.c_int, [_P, _P, _P, _P]),
    "rccsdt_set_amplitudes_t3f32": (C.c_int, [_P, _P, _P, _P]),
    "rccsdt_get_amplitudes_t3f32": (C.c_int, [_P, _P, _P, _P]),
    "rccsdt_save": (C.c_int, [_P, C.c_char_p]),
    "rccsdt_load": (C.c_int, [_P, C.c_char_p]),
    "rccsdt_get_residuals": (C.c_int, [_P, _P, _P, _P]),
    "rccsdt_debug_copy": (C.c_int, [_P, C.c_char_p, _P, C.c_longlong]),
    "rccsdt_iteration_fma": (C.c_double, [C.c_int, C.c_int]),
    "rccsdt_step_times": (C.c_int, [_P, _P, C.c_int]),
    "rccsdt_enable_timing": (C.c_int, [_P, C.c_int]),
    "rccsdt_kernel_launches": (C.c_longlong, []),
    "rccsdt_engine_info": (C.c_int, [_P, _P, C.c_int]),
    "rccsdt_last_error": (C.c_char_p, [_P]),
    "rccsdt_destroy": (None, [_P]),
    "rccsdt_batch_create": (C.c_int, [C.c_int, _P, _P, _P, C.POINTER(Options), _P, C.POINTER(_P)]),
    "rccsdt_batch_instance": (_P, [_P, C.c_int]),
    "rccsdt_batch_solve": (C.c_int, [_P, _P, _P, _P, _P]),
    "rccsdt_batch_stats": (C.c_int, [_P, _P, C.c_int]),
    "rccsdt_batch_launch_times": (C.c_int, [_P, _P, C.c_int]),
    "rccsdt_batch_last_error": (C.c_char_p, [_P]),
    "rccsdt_batch_destroy": (None, [_P]),
    "rccsdt_q_energy": (C.c_int, [_P, C.c_int, _P, _P]),
    "rccsdt_t3_virtual_triangular": (C.c_int, [_P, _P]),
    "rccsdt_t4_create": (C.c_int, [C.c_int, C.c_int, C.c_int, _P, C.POINTER(_P)]),
    "rccsdt_t4_set": (C.c_int, [_P, _P, _P]),
    "rccsdt_t4_pp_ladder": (C.c_int, [_P]),
    "rccsdt_t4_postprocess": (C.c_int, [_P, _P]),
    "rccsdt_t4_get_r4": (C.c_int, [_P, _P]),
    "rccsdt_t4_last_error": (C.c_char_p, [_P]),
    "rccsdt_t4_destroy": (None, [_P]),
    "rccsdt_ijk_block_costs": (C.c_int, [C.c_int, C.c_int, _P]),
    "rccsdt_ijk_plan_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, _P, C.POINTER(_P)]),
    "rccsdt_ijk_plan_destroy": (None, [_P]),
    "rccsdt_ijk_plan_info": (C.c_int, [_P, _P]),
    "rccsdt_ijk_plan_owners": (C.c_int, [_P, _P]),
    "rccsdt_ijk_plan_local": (C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_int)]),
    "rccsdt_ijk_plan_batch": (C.c_int, [_P, C.c_int, _P, _P]),
    "rccsdt_ijk_plan_work": (C.c_int, [_P, _P, _P]),
}
Q_FP64, Q_FP32 = 0, 1


def load_library(path: str) -> C.CDLL:
    """Load a build of the library and declare the signatures it exports (the
    test-only host simulation has no (Q) kernels; the product library exports every
    declared entry point, which tests/test_abi.py checks)."""
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    return lib


def _ptr(x, f32=False):
    """Raw pointer of a contiguous float64 (float32 with ``f32``) numpy array or torch
    tensor (None -> NULL)."""
    if x is None:
        return None
    kind = "float32" if f32 else "float64"
    if isinstance(x, np.ndarray):
        if x.dtype != np.dtype(kind) or not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"arrays must be contiguous {kind}")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != getattr(torch, kind) or not x.is_contiguous():
            raise ValueError(f"tensors must be contiguous {kind}")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def default_options(lib, **kw) -> Options:
    opt = Options()
    lib.rccsdt_options_default(C.byref(opt))
    for k, val in kw.items():
        setattr(opt, k, val)
    return opt


class Context:
    """One RCCSDT problem (o occupied, v virtual spatial orbitals, naux factors)."""

    def __init__(self, lib, o: int, v: int, naux: int, stream: int = 0, _borrowed=None, **options):
        self.lib, self.o, self.v, self.naux = lib, o, v, naux
        self.n3 = o * (o + 1) * (o + 2) // 6
        self.options = default_options(lib, **options)
        self.owned = _borrowed is None
        if _borrowed is not None:  # a context owned by a Batch
            self.h = _borrowed
            return
        h = _P()
        st = lib.rccsdt_create(o, v, naux, C.byref(self.options), _P(stream) if stream else None, C.byref(h))
        if st != OK:
            raise RccsdtError(st, "rccsdt_create failed")
        self.h = h

    def _check(self, st, allow=(OK,)):
        if st not in allow:
            raise RccsdtError(st, self.lib.rccsdt_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "owned", True):
                self.lib.rccsdt_destroy(self.h)
            self.h = None

    __del__ = close

    def device_bytes(self) -> int:
        return self.lib.rccsdt_device_bytes(self.h)

    def set_hamiltonian(self, fock_diag, L):
        self._check(self.lib.rccsdt_set_hamiltonian(self.h, _ptr(fock_diag), _ptr(L)))

    def set_amplitudes(self, t1=None, t2=None, t3c=None):
        self._check(self.lib.rccsdt_set_amplitudes(self.h, _ptr(t1), _ptr(t2), _ptr(t3c)))

    def set_amplitudes_t3f32(self, t1=None, t2=None, t3c=None):
        """T3 in FP32, the split modes' storage type (t1, t2 float64)."""
        self._check(self.lib.rccsdt_set_amplitudes_t3f32(self.h, _ptr(t1), _ptr(t2), _ptr(t3c, f32=True)))

    def init_mp2(self):
        self._check(self.lib.rccsdt_init_mp2(self.h))

    def set_precision(self, precision: int):
        self._check(self.lib.rccsdt_set_precision(self.h, precision))

    def build_intermediates(self):
        self._check(self.lib.rccsdt_build_intermediates(self.h))

    def residual(self):
        self._check(self.lib.rccsdt_residual(self.h))

    def postprocess(self):
        norms = np.zeros(4)
        self._check(self.lib.rccsdt_postprocess(self.h, norms.ctypes.data))
        return norms

    def update(self):
        self._check(self.lib.rccsdt_update(self.h))

    def energy(self) -> float:
        e = np.zeros(1)
        self._check(self.lib.rccsdt_energy(self.h, e.ctypes.data))
        return float(e[0])

    def iterate(self):
        e = np.zeros(1)
        norms = np.zeros(4)
        self._check(self.lib.rccsdt_iterate(self.h, e.ctypes.data, norms.ctypes.data))
        return float(e[0]), norms

    def solve(self):
        e = np.zeros(1)
        it = C.c_int(0)
        nrm = np.zeros(1)
        st = self._check(self.lib.rccsdt_solve(self.h, e.ctypes.data, C.addressof(it), nrm.ctypes.data),
                         allow=(OK, NOT_CONVERGED))
        return float(e[0]), it.value, float(nrm[0]), st == OK

    def get_amplitudes(self, t1=None, t2=None, t3c=None):
        self._check(self.lib.rccsdt_get_amplitudes(self.h, _ptr(t1), _ptr(t2), _ptr(t3c)))

    def get_amplitudes_t3f32(self, t1=None, t2=None, t3c=None):
        self._check(self.lib.rccsdt_get_amplitudes_t3f32(self.h, _ptr(t1), _ptr(t2), _ptr(t3c, f32=True)))

    def save(self, path):
        """Write the iteration state (amplitudes, DIIS history, counters) to ``path``."""
        self._check(self.lib.rccsdt_save(self.h, str(path).encode()))

    def load(self, path):
        """Read a state written by ``save`` (same sizes and options; set the
        Hamiltonian before iterating)."""
        self._check(self.lib.rccsdt_load(self.h, str(path).encode()))

    def get_residuals(self, r1=None, r2=None, r3c=None):
        self._check(self.lib.rccsdt_get_residuals(self.h, _ptr(r1), _ptr(r2), _ptr(r3c)))

    def amplitudes(self):
        o, v = self.o, self.v
        t1, t2, t3 = np.empty((o, v)), np.empty((o, o, v, v)), np.empty((self.n3, v, v, v))
        self.get_amplitudes(t1, t2, t3)
        return t1, t2, t3

    def residuals(self):
        o, v = self.o, self.v
        r1, r2, r3 = np.empty((o, v)), np.empty((o, o, v, v)), np.empty((self.n3, v, v, v))
        self.get_residuals(r1, r2, r3)
        return r1, r2, r3

    def q_energy(self, arith: int = Q_FP64):
        """RCCSDT(Q) energy correction of the current amplitudes; returns (E_(Q), info)
        with info = {transpose_ms, intermediates_ms, main_ms, flop, quadruples, grid}."""
        e = np.zeros(1)
        info = np.zeros(6)
        self._check(self.lib.rccsdt_q_energy(self.h, arith, e.ctypes.data, info.ctypes.data))
        keys = ["transpose_ms", "intermediates_ms", "main_ms", "flop", "quadruples", "grid"]
        return float(e[0]), dict(zip(keys, info.tolist()))

    def t3_virtual_triangular(self):
        """Compact T3 transposed to the virtual-triangular layout [nv3][o][o][o]."""
        nv3 = self.v * (self.v + 1) * (self.v + 2) // 6
        out = np.empty((nv3, self.o, self.o, self.o))
        self._check(self.lib.rccsdt_t3_virtual_triangular(self.h, out.ctypes.data))
        return out

    def debug_copy(self, name: str, shape):
        out = np.empty(shape)
        self._check(self.lib.rccsdt_debug_copy(self.h, name.encode(), out.ctypes.data, out.size))
        return out

    def engine_info(self):
        out = np.zeros(13, dtype=np.int64)
        k = self.lib.rccsdt_engine_info(self.h, out.ctypes.data, 13)
        keys = ["grouped", "problems", "tiles", "gathers", "contributions", "bytes", "grid", "kind", "bn", "order",
                "tuned", "tuned_us", "fixed_us"]
        return dict(zip(keys[:k], out[:k].tolist()))

    def enable_timing(self, on=True):
        self._check(self.lib.rccsdt_enable_timing(self.h, 1 if on else 0))

    def step_times(self):
        ms = np.zeros(16)
        n = self.lib.rccsdt_step_times(self.h, ms.ctypes.data, 16)
        return ms[:n]


class Batch:
    """Independent instances iterated together (one CUDA graph launch per iteration).

    ``shapes`` is a list of (o, v, naux); ``instances[i]`` is a borrowed Context for
    setting the Hamiltonian and amplitudes of instance i.
    """

    def __init__(self, lib, shapes, stream: int = 0, **options):
        self.lib = lib
        self.shapes = [tuple(int(x) for x in s) for s in shapes]
        n = len(self.shapes)
        o = (C.c_int * n)(*[s[0] for s in self.shapes])
        v = (C.c_int * n)(*[s[1] for s in self.shapes])
        na = (C.c_int * n)(*[s[2] for s in self.shapes])
        self.options = default_options(lib, **options)
        h = _P()
        st = lib.rccsdt_batch_create(n, C.cast(o, _P), C.cast(v, _P), C.cast(na, _P), C.byref(self.options),
                                     _P(stream) if stream else None, C.byref(h))
        if st != OK:
            raise RccsdtError(st, "rccsdt_batch_create failed")
        self.h = h
        self.instances = [Context(lib, s[0], s[1], s[2], _borrowed=lib.rccsdt_batch_instance(h, i), **options)
                          for i, s in enumerate(self.shapes)]

    def close(self):
        if getattr(self, "h", None):
            for c in self.instances:
                c.h = None
            self.lib.rccsdt_batch_destroy(self.h)
            self.h = None

    __del__ = close

    def solve(self):
        """Returns (energies, iterations, final norms, statuses) as numpy arrays."""
        n = len(self.shapes)
        e, nrm = np.zeros(n), np.zeros(n)
        it, st = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.int32)
        rc = self.lib.rccsdt_batch_solve(self.h, e.ctypes.data, it.ctypes.data, nrm.ctypes.data, st.ctypes.data)
        if rc < 0:
            raise RccsdtError(rc, self.lib.rccsdt_batch_last_error(self.h).decode())
        return e, it, nrm, st

    def stats(self):
        out = np.zeros(14)
        k = self.lib.rccsdt_batch_stats(self.h, out.ctypes.data, 14)
        keys = ["launches", "device_ms", "flop", "kernels", "graph_nodes", "build_ms", "instantiate_ms",
                "first_launch_ms", "batch_gemm", "batch_gemm_problems", "batch_gemm_tiles", "batch_gemm_bn",
                "batch_gemm_tuned_ms", "batch_gemm_fixed_ms"]
        return dict(zip(keys[:k], out[:k].tolist()))

    def launch_times(self, cap: int = 100000):
        ms = np.zeros(cap)
        k = self.lib.rccsdt_batch_launch_times(self.h, ms.ctypes.data, cap)
        return ms[:k]


class T4Engine:
    """Compact T4 of RCCSDTQ: the six-term W^vv_vv * T4 ladder and the R4
    post-processing (rccsdt_t4_* in include/rccsdt.h)."""

    def __init__(self, lib, o: int, v: int, precision: int = FP64, stream: int = 0):
        self.lib, self.o, self.v = lib, o, v
        self.n4 = o * (o + 1) * (o + 2) * (o + 3) // 24
        h = _P()
        st = lib.rccsdt_t4_create(o, v, precision, _P(stream) if stream else None, C.byref(h))
        if st != OK:
            raise RccsdtError(st, "rccsdt_t4_create failed")
        self.h = h

    def _check(self, st):
        if st != OK:
            raise RccsdtError(st, self.lib.rccsdt_t4_last_error(self.h).decode())

    def set(self, W=None, t4c=None):
        self._check(self.lib.rccsdt_t4_set(self.h, _ptr(W), _ptr(t4c)))

    def pp_ladder(self):
        self._check(self.lib.rccsdt_t4_pp_ladder(self.h))

    def postprocess(self) -> float:
        nrm = np.zeros(1)
        self._check(self.lib.rccsdt_t4_postprocess(self.h, nrm.ctypes.data))
        return float(nrm[0])

    def r4(self):
        out = np.empty((self.n4, self.v, self.v, self.v, self.v))
        self._check(self.lib.rccsdt_t4_get_r4(self.h, out.ctypes.data))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.rccsdt_t4_destroy(self.h)
            self.h = None

    __del__ = close
