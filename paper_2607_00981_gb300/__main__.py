"""Command line: run RCCSDT iterations on one synthetic workload.

    python -m paper_2607_00981_gb300 --workload o8v80 --iters 2 --precision fp64

Prints the energy and residual norms of each iteration (the device work is
exactly one ``rccsdt_iterate`` per iteration after ``set_hamiltonian`` and the
MP2 guess), which makes it a small, fixed launch sequence for profilers.
"""
import argparse
import sys
import time

import paper_2607_00981_gb300 as pkg
from paper_2607_00981_gb300.synth import CONVERGENCE, WORKLOADS, make_instance


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2607_00981_gb300")
    ap.add_argument("--workload", default="o3v12", choices=sorted(WORKLOADS) + sorted(CONVERGENCE))
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "bf16x3", "tf32x3"])
    ap.add_argument("--scale", type=float, default=None, help="override the factor entry scale")
    ap.add_argument("--no-diis-t3", action="store_true", help="DIIS on T1 and T2 only")
    args = ap.parse_args(argv)
    spec = dict(WORKLOADS.get(args.workload) or CONVERGENCE[args.workload])
    if args.scale is not None:
        spec["scale"] = args.scale
    inst = make_instance(**spec)
    prec = {"fp64": 0, "bf16x3": 1, "tf32x3": 2}[args.precision]
    ctx = pkg.context(inst.o, inst.v, inst.naux, precision=prec, diis_t3=0 if args.no_diis_t3 else 1)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.init_mp2()
    for it in range(args.iters):
        t0 = time.perf_counter()
        e, n = ctx.iterate()
        print(f"iter {it + 1}  E = {e:.12f}  |R| = {n[3]:.3e}  ({time.perf_counter() - t0:.3f} s)", flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
