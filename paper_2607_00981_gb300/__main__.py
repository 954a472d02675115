"""Command line: run RCCSDT iterations on one synthetic workload.

    python -m paper_2607_00981_gb300 --workload o8v80 --iters 2 --precision fp64

Prints one JSON line per iteration: the energy and its change, the residual norms
(R1, R2, R3, total), the precision and the device ms of each step (the device work
is exactly one ``rccsdt_iterate`` per iteration after ``set_hamiltonian`` and the
MP2 guess, which makes it a small, fixed launch sequence for profilers).  With
``--resume PATH`` the iterations continue from a checkpoint instead of the MP2 guess;
``--checkpoint PATH`` saves the state after the last iteration.

    python -m paper_2607_00981_gb300 --workload o12v120w --solve --tol 1e-8 --precision bf16x3 --f64-tc 1

runs rccsdt_solve instead (split contexts switch to FP64 contractions at
|R| <= sqrt(tol)) and prints one JSON line: energy, iterations, norm, status, time.
With --refine-fp64 the converged amplitudes then seed an FP64 context (FP64
storage, FP64 DIIS of --refine-diis vectors, contractions per --f64-tc) iterated to
--tol again; its energy is the FP64 reference the split energy is compared with
(converged energies do not depend on the path).

    python -m paper_2607_00981_gb300 --t4 6,40 --precision bf16x3 --reps 2

runs the compact-T4 engine instead: seeded pair-symmetric W and T4 at o, v, then
--reps passes of the six-term ladder and the R4 post-processing, one JSON line per
pass with the device ms of each and the norm of the post-processed R4.

    python -m paper_2607_00981_gb300 --batch 6,40,64 --iters 4 --precision bf16x3

iterates a batch of n identical instances (o, v, naux = 4 (o + v), weak coupling) in
one CUDA graph launch per batch iteration for --iters batch iterations from the MP2
guess and prints the device ms of every launch.
"""
import argparse
import json
import sys
import time

import paper_2607_00981_gb300 as pkg
from paper_2607_00981_gb300.synth import CONVERGENCE, WORKLOADS, make_instance


def t4_passes(args):
    import numpy as np
    import torch

    from paper_2607_00981_gb300 import binding as B
    from paper_2607_00981_gb300.synth import random_pair_symmetric
    o, v = (int(x) for x in args.t4.split(","))
    n4 = o * (o + 1) * (o + 2) * (o + 3) // 24
    prec = {"fp64": B.FP64, "bf16x3": B.SPLIT_BF16X3, "tf32x3": B.SPLIT_TF32X3}[args.precision]
    W = random_pair_symmetric(v, seed=40)
    t4c = torch.from_numpy(0.05 * np.random.default_rng(6).standard_normal((n4, v, v, v, v))).cuda()
    eng = B.T4Engine(pkg.load(), o, v, precision=prec)
    eng.set(W, t4c)
    for rep in range(args.reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        ev[0].record()
        eng.pp_ladder()
        ev[1].record()
        norm = eng.postprocess()
        ev[2].record()
        torch.cuda.synchronize()
        print(json.dumps({"t4": [o, v], "precision": args.precision, "pass": rep, "n4": n4,
                          "ladder_ms": ev[0].elapsed_time(ev[1]), "post_ms": ev[1].elapsed_time(ev[2]),
                          "r4_norm": norm}), flush=True)
    eng.close()
    return 0


def batch_launches(args):
    from paper_2607_00981_gb300 import binding as B
    o, v, n = (int(x) for x in args.batch.split(","))
    naux = 4 * (o + v)
    inst = make_instance(o, v, naux, seed=7, scale=0.6 * 0.3 * (40 / naux) ** 0.5)
    prec = {"fp64": 0, "bf16x3": 1, "tf32x3": 2}[args.precision]
    b = B.Batch(pkg.load(), [(o, v, naux)] * n, precision=prec, tol=args.tol, max_iter=args.iters, autotune=0,
                f64_tc=args.f64_tc)
    for c in b.instances:
        c.set_hamiltonian(inst.fock_diag, inst.L)
        c.init_mp2()
    b.solve()
    print(json.dumps({"batch": [o, v, n], "precision": args.precision,
                      "launch_ms": [float(x) for x in b.launch_times()],
                      "kernels": float(b.stats()["kernels"])}), flush=True)
    b.close()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2607_00981_gb300")
    ap.add_argument("--workload", default="o3v12", choices=sorted(WORKLOADS) + sorted(CONVERGENCE))
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "bf16x3", "tf32x3"])
    ap.add_argument("--scale", type=float, default=None, help="override the factor entry scale")
    ap.add_argument("--no-diis-t3", action="store_true", help="DIIS on T1 and T2 only")
    ap.add_argument("--f64-tc", type=int, default=0, choices=[0, 1, 2],
                    help="FP64 contractions on the tensor cores (option f64_tc)")
    ap.add_argument("--solve", action="store_true", help="iterate to --tol with rccsdt_solve")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-iter", type=int, default=200)
    ap.add_argument("--diis-space", type=int, default=8)
    ap.add_argument("--refine-fp64", action="store_true", help="re-converge in an FP64 context afterwards")
    ap.add_argument("--refine-diis", type=int, default=2)
    ap.add_argument("--checkpoint", default=None, help="save the iteration state here at the end")
    ap.add_argument("--resume", default=None, help="continue from a saved iteration state")
    ap.add_argument("--grouped-bytes", type=int, default=None,
                    help="memory budget of the grouped residual of split contexts (0: per-plan engine)")
    ap.add_argument("--o", type=int, default=None, help="override the workload's occupied count (same v, naux)")
    ap.add_argument("--pp-unit-bytes", type=int, default=None,
                    help="bytes of one pp-ladder launch unit's T operand (option pp_unit_bytes)")
    ap.add_argument("--diis-t3-nvir", type=int, default=0,
                    help="DIIS on T3 over the lowest N virtual orbitals only (option diis_t3_nvir)")
    ap.add_argument("--contract-fp64", action="store_true",
                    help="split-storage context (FP32 T3) iterated with FP64 contractions throughout")
    ap.add_argument("--until-tol", action="store_true", help="with --iters: stop once |R| <= --tol")
    ap.add_argument("--q", default=None, choices=["fp64", "fp32"],
                    help="after the iterations (or the solve), the RCCSDT(Q) energy correction in this arithmetic")
    ap.add_argument("--t4", default=None, help="o,v: time the compact-T4 ladder and post-processing instead")
    ap.add_argument("--reps", type=int, default=2, help="with --t4: passes")
    ap.add_argument("--batch", default=None, help="o,v,n: n identical instances in one batch instead")
    args = ap.parse_args(argv)
    if args.t4:
        return t4_passes(args)
    if args.batch:
        return batch_launches(args)
    spec = dict(WORKLOADS.get(args.workload) or CONVERGENCE[args.workload])
    if args.scale is not None:
        spec["scale"] = args.scale
    if args.o is not None:
        spec["o"] = args.o
    inst = make_instance(**spec)
    prec = {"fp64": 0, "bf16x3": 1, "tf32x3": 2}[args.precision]
    extra = {} if args.grouped_bytes is None else {"grouped_bytes": args.grouped_bytes}
    if args.pp_unit_bytes is not None:
        extra["pp_unit_bytes"] = args.pp_unit_bytes
    ctx = pkg.context(inst.o, inst.v, inst.naux, precision=prec, diis_t3=0 if args.no_diis_t3 else 1,
                      f64_tc=args.f64_tc, tol=args.tol, max_iter=args.max_iter, diis_space=args.diis_space,
                      diis_t3_nvir=args.diis_t3_nvir, **extra)

    def q_correction():
        if args.q is None:
            return
        t0 = time.perf_counter()
        eq, info = ctx.q_energy(0 if args.q == "fp64" else 1)
        wall = time.perf_counter() - t0
        print(json.dumps({"workload": args.workload, "o": inst.o, "v": inst.v, "q_arith": args.q, "e_q": eq,
                          "seconds": wall, "main_tflops": info["flop"] / (info["main_ms"] / 1e3) / 1e12, **info}),
              flush=True)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    if args.contract_fp64:
        ctx.set_precision(0)
    if args.resume:
        ctx.load(args.resume)
    else:
        ctx.init_mp2()
    if args.solve:
        t0 = time.perf_counter()
        e, iters, norm, conv = ctx.solve()
        out = {"workload": args.workload, "precision": args.precision, "f64_tc": args.f64_tc, "tol": args.tol,
               "diis_space": args.diis_space, "energy": e, "iterations": iters, "norm": norm, "converged": conv,
               "seconds": time.perf_counter() - t0}
        print(json.dumps(out), flush=True)
        q_correction()
        if args.refine_fp64 and conv:
            t1, t2, t3 = ctx.amplitudes()
            ctx.close()
            ref = pkg.context(inst.o, inst.v, inst.naux, precision=0, diis_t3=1, diis_space=args.refine_diis,
                              f64_tc=args.f64_tc, tol=args.tol, max_iter=args.max_iter)
            ref.set_hamiltonian(inst.fock_diag, inst.L)
            ref.set_amplitudes(t1, t2, t3)
            del t1, t2, t3
            t0 = time.perf_counter()
            e64, it64, n64, c64 = ref.solve()
            print(json.dumps({"workload": args.workload, "reference": "fp64 storage", "f64_tc": args.f64_tc,
                              "energy": e64, "iterations": it64, "norm": n64, "converged": c64,
                              "seconds": time.perf_counter() - t0, "abs_energy_difference": abs(e64 - e)}),
                  flush=True)
            ref.close()
            return 0
        ctx.close()
        return 0
    steps = ["intermediates", "pp", "ring", "hh", "t2", "r12_setup", "post", "update", "energy"]
    e_prev = None
    for it in range(args.iters):
        ctx.enable_timing(True)  # a fresh window per iteration
        t0 = time.perf_counter()
        e, n = ctx.iterate()
        wall = time.perf_counter() - t0
        ms = ctx.step_times()
        print(json.dumps({"iter": it + 1, "energy": e, "delta_e": None if e_prev is None else e - e_prev,
                          "r1": n[0], "r2": n[1], "r3": n[2], "r": n[3], "precision": args.precision,
                          "seconds": wall, "step_ms": {k: float(x) for k, x in zip(steps, ms[:9])}}), flush=True)
        e_prev = e
        if args.until_tol and n[3] <= args.tol:
            break
    ctx.enable_timing(False)
    q_correction()
    if args.checkpoint:
        ctx.save(args.checkpoint)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
