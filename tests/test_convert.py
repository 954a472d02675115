"""The integer-path binary64 -> binary32 conversion used by the FP64-source panel
gathers, against numpy's round-to-nearest-even cast (IEEE 754), bit for bit."""
import ctypes as C

import numpy as np

from ._helpers import hostsim_lib


def _convert(x):
    lib = hostsim_lib()
    f = lib.rcc_test_f64_to_f32
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_longlong]
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(x.shape, dtype=np.float32)
    f(x.ctypes.data, y.ctypes.data, x.size)
    return y


def test_f64_to_f32_matches_ieee_rounding():
    rng = np.random.default_rng(0)
    f32 = np.finfo(np.float32)
    parts = [
        rng.standard_normal(200000) * np.exp(rng.uniform(-40, 40, 200000)),
        # ties: a binary32 value plus exactly half an ulp (even and odd fractions)
        np.float32(rng.standard_normal(20000)).astype(np.float64) * (1 + 2.0 ** -24),
        np.nextafter(np.float32(rng.standard_normal(20000)).astype(np.float64), np.inf),
        # subnormal and overflow ranges, boundaries
        rng.uniform(-1, 1, 20000) * 2.0 ** -126, rng.uniform(-1, 1, 20000) * 2.0 ** -140,
        rng.uniform(-1, 1, 2000) * 2.0 ** -149, np.array([2.0 ** -150, 3 * 2.0 ** -151, 2.0 ** -151, 5e-324]),
        np.array([float(f32.max), float(f32.max) * (1 + 2.0 ** -25), float(f32.max) * (1 + 2.0 ** -23), 1e39, -1e300]),
        np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, float(f32.tiny), float(f32.smallest_subnormal)]),
    ]
    x = np.concatenate(parts)
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)
    got = _convert(x)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert np.isnan(_convert(np.array([np.nan]))).all()
