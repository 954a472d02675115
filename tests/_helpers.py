"""Shared test helpers: library loading and seeded inputs."""
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HOSTSIM_DIR = os.path.join(ROOT, "tests", "hostsim")


def gpu_lib():
    import paper_2607_00981_gb300 as pkg
    from paper_2607_00981_gb300.build import build
    build()
    return pkg.load()


def hostsim_lib():
    """Build (if stale) and load the test-only host simulation of the library's plans."""
    from paper_2607_00981_gb300 import binding
    from paper_2607_00981_gb300.build import CSRC, nvcc
    out = os.path.join(HOSTSIM_DIR, "_build", "librccsdt_hostsim.so")
    srcs = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HOSTSIM_DIR, "hostsim.cu"),
                                                                 os.path.join(ROOT, "include", "rccsdt.h")]
    if not os.path.exists(out) or any(os.path.getmtime(s) > os.path.getmtime(out) for s in srcs):
        os.makedirs(os.path.dirname(out), exist_ok=True)
        cmd = [nvcc(), "-std=c++17", "-O2", "-Xcompiler", "-fPIC", "-shared", "-DRCC_HOSTSIM", "-I", CSRC,
               os.path.join(CSRC, "runtime.cu"), os.path.join(CSRC, "batch.cu"), os.path.join(HOSTSIM_DIR, "hostsim.cu"),
               "-o", out]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode:
            sys.stderr.write(res.stdout + res.stderr)
            raise RuntimeError("hostsim build failed")
    return binding.load_library(out)


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(1.0, float(np.abs(b).max())))
