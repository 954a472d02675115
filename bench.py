"""RCCSDT iteration benchmark on one GB300 (replicas under torchrun).

A step is one whole RCCSDT iteration through the C ABI (``rccsdt_iterate``):
energy, T1-dressing, intermediates, the T3 contributions to R1/R2/W, the
residuals R1, R2 and the compact R3 (pp-ladder, ring, hh-ladder, T2-driven
terms), post-processing of R3, the Jacobi update and DIIS.  Inputs are seeded
synthetic low-rank Hamiltonians; amplitudes start from the MP2 guess.

Prints one JSON line (rank 0).  ``value`` is seconds per iteration of the whole
job (the slowest rank's timed region divided by the iterations all ranks ran);
``tflops`` counts the algorithmic compact FMA n3 (3v^5 + 12ov^4 + 3o^2v^3) once.
``--impl reference`` times the FP64 CPU oracle instead, on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RCCSDT s/iteration and TFLOP/s at 1 GB300, FP64 vs split-precision at <=1e-6 Eh"
PRECISIONS = {"fp64": 0, "bf16x3": 1, "tf32x3": 2}
DTYPE = {"fp64": "f64", "bf16x3": "bf16x3 (fp32 accumulate, fp32 T3)", "tf32x3": "tf32x3 (fp32 accumulate, fp32 T3)"}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def measure_matmul_peaks(n=8192, reps=5):
    """FP64 and TF32 dense matmul rates of this GPU (cuBLAS through torch.matmul,
    2 n^3 flop, best of `reps`, CUDA events): the denominators of the FP64 (DFMA)
    and 3xTF32 rooflines, which MEASURED_PEAKS.json does not carry.  Takes a few
    seconds."""
    import torch
    out = {}
    for label, dt, tf32 in (("fp64_tflops", torch.float64, False), ("tf32_tflops", torch.float32, True)):
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = tf32
        m = n if dt == torch.float32 else n // 2   # the FP64 rate is ~1000x lower: a smaller cube
        a = torch.randn(m, m, dtype=dt, device="cuda")
        b = torch.randn(m, m, dtype=dt, device="cuda")
        c = a @ b
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c = a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[label] = 2.0 * m ** 3 / best / 1e12
        torch.backends.cuda.matmul.allow_tf32 = prev
        del a, b, c
    out["how"] = f"torch.matmul (cuBLAS) FP64 {n // 2}^3 and TF32 {n}^3, best of {reps}, CUDA events"
    return out


def cpu_model():
    """CPU model name of this host (lscpu, else /proc/cpuinfo)."""
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in txt.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample_one_core(workload, seconds_budget):
    """The oracle sample of ``oracle_sample`` in a child process limited to one thread
    (BLAS and OpenMP thread counts are fixed when numpy loads, hence the child)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1")
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "from paper_2607_00981_gb300.synth import workload; "
            "v, s = bench.oracle_sample(workload(%r), seconds_budget=%r); print(json.dumps([v, s]))"
            % (ROOT, workload, seconds_budget))
    try:
        res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                             timeout=30 * seconds_budget + 300)
        val, sample = json.loads(res.stdout.strip().splitlines()[-1])
        return {"value": val, "unit": "s/iteration", "cores": 1, "sample": sample}
    except (OSError, subprocess.SubprocessError, ValueError, IndexError) as exc:
        return {"value": None, "error": str(exc)[:200]}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu, self.rows, self.proc = gpu, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in self.rows for q in range(4) if len(r) > 5 + q and r[5 + q] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def oracle_sample(inst, seconds_budget=20.0):
    """Time one FP64 oracle iteration at this workload from bounded samples.

    Three parts, summed:
    * the T1-dressing and the RCCSD/RCCSDT intermediates (``oracle.rccsdt``), once;
    * the T3 contributions to R1, R2 and W (``oracle.compact.t3_contributions``, a loop
      of identical v-sized contractions over all o^3 occupied triples), timed on the
      same v and naux with two occupied orbitals (8 triples) and scaled by (o / 2)^3;
    * the compact R3 blocks (``oracle.compact.r3_block``: pp-ladder, ring, hh-ladder,
      F and T2 terms of one stored block) on blocks of a stride through the block list
      until `seconds_budget` is spent, scaled by block count.
    Returns (s/iteration, sample text)."""
    from oracle import compact as oc
    from oracle import rccsdt as of
    from paper_2607_00981_gb300.synth import make_instance
    o, v = inst.o, inst.v
    rng = np.random.default_rng(0)
    t1 = 1e-3 * rng.standard_normal((o, v))
    t2 = of.mp2_t2(inst.L, inst.fock_diag, o)
    t0 = time.perf_counter()
    Lt, ft = of.dress(inst.L, inst.fock_diag, t1)
    I = of.intermediates(Lt, ft, t2, None, triples=True)
    t_int = time.perf_counter() - t0
    small = make_instance(2, v, inst.naux, seed=inst.seed)
    Ls, fs = of.dress(small.L, small.fock_diag, 1e-3 * rng.standard_normal((2, v)))
    t3s = 1e-3 * rng.standard_normal((oc.n3(2), v, v, v))
    t0 = time.perf_counter()
    oc.t3_contributions(of.Eri(Ls, 2), fs, t3s, 2)
    t_a3 = (time.perf_counter() - t0) * (o / 2.0) ** 3
    tr = oc.triples(o)
    t3c = 1e-3 * rng.standard_normal((len(tr), v, v, v))
    stride = max(1, len(tr) // 16)
    picked, t_used = 0, 0.0
    t0 = time.perf_counter()
    for b in range(0, len(tr), stride):
        i, j, k = tr[b]
        oc.r3_block(I, t2, t3c, i, j, k)
        picked += 1
        t_used = time.perf_counter() - t0
        if t_used > seconds_budget:
            break
    t_r3 = t_used / picked * len(tr)
    total = t_int + t_a3 + t_r3
    return total, (f"oracle: intermediates {t_int:.1f} s (whole); T3 -> R1/R2/W {t_a3:.1f} s (8 occupied "
                   f"triples at v={v}, scaled by (o/2)^3); R3 {t_r3:.1f} s (r3_block on {picked} of {len(tr)} "
                   f"stored blocks, stride {stride}, {t_used:.1f} s, scaled by block count)")


def run_reference(args, rank, world):
    from paper_2607_00981_gb300.synth import workload
    if rank != 0:
        return
    inst = workload(args.workload)
    times = []
    sample = ""
    for s in range(args.warmup + args.steps):
        val, sample = oracle_sample(inst, seconds_budget=args.ref_seconds)
        if s >= args.warmup:
            times.append(val)
    value = statistics.mean(times)
    from oracle import opcount
    flop = opcount.flop_per_iteration(inst.o, inst.v)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/iteration", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(args, inst), "tflops": flop / value / 1e12,
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "sample": sample, "value": value,
                             "unit": "s/iteration"},
            "e2e": {"value": value, "unit": "s/iteration", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The slowest rank's value (all ranks get it); identity without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def per_iteration(seconds_max: float, steps: int, world: int) -> float:
    """Whole-job seconds per iteration: N replicas each ran `steps` iterations."""
    return seconds_max / (steps * world)


def config(args, inst):
    return {"workload": f"{args.workload}: RCCSDT iteration, o={inst.o} v={inst.v} naux={inst.naux}, "
                        f"compact T3 {inst.o * (inst.o + 1) * (inst.o + 2) // 6} x {inst.v}^3, seed {inst.seed}",
            "o": inst.o, "v": inst.v, "naux": inst.naux, "precision": args.precision,
            "l2": "inputs larger than L2 (compact T3/R3 and the operand panels exceed 129 MB)",
            "amplitudes": "MP2 guess, then the benchmark's own iterations",
            "coupling": ("weak: factor entries scaled by 0.6*0.3*sqrt(40/naux) (the literal 0.3 diverges and "
                         "overflows FP32 T3 within a few iterations; the work per iteration is the same)"
                         if args.workload.endswith("w") else "literal per-entry scale 0.3")}


def compare_fp64_split(pkg, stream, dev, name="o8v80w", warm=2, steps=2):
    """FP64 (contractions on the FP64 units, and on the tensor cores through digit
    planes), 3xBF16 and 3xTF32 s/iteration on the same o8v80 shapes (same MP2 start)."""
    import torch
    from paper_2607_00981_gb300.synth import workload
    inst = workload(name)
    out = {"workload": name}
    for label, prec, f64_tc in (("fp64", 0, 0), ("fp64_tc", 0, 1), ("bf16x3", 1, 0), ("tf32x3", 2, 0)):
        ctx = pkg.context(inst.o, inst.v, inst.naux, stream=stream.cuda_stream, precision=prec, f64_tc=f64_tc)
        ctx.set_hamiltonian(inst.fock_diag, inst.L)
        ctx.init_mp2()
        for _ in range(warm):
            ctx.iterate()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.iterate()
        e1.record(stream)
        torch.cuda.synchronize()
        out[label] = e0.elapsed_time(e1) / 1e3 / steps
        ctx.close()
    out["unit"] = "s/iteration"
    out["speedup_bf16x3"] = out["fp64"] / out["bf16x3"]
    out["speedup_tf32x3"] = out["fp64"] / out["tf32x3"]
    out["speedup_fp64_tc"] = out["fp64"] / out["fp64_tc"]
    out["speedup_bf16x3_vs_fp64_tc"] = out["fp64_tc"] / out["bf16x3"]
    return out


def fp64_tc_iteration(pkg, stream, inst, fp64_rate):
    """One FP64 iteration (FP64 storage, contractions on the tensor cores through
    digit planes, no DIIS history) at the benchmark workload, timed after one warm-up
    iteration; the DFMA path's time is estimated from its measured rate at o8v80w
    (one of its iterations here would take about ten minutes)."""
    import torch
    ctx = pkg.context(inst.o, inst.v, inst.naux, stream=stream.cuda_stream, precision=0, f64_tc=1, diis_space=0)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.init_mp2()
    ctx.iterate()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.iterate()
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    flop = 2.0 * ctx.lib.rccsdt_iteration_fma(inst.o, inst.v)
    ctx.close()
    out = {"fp64_tc_s_per_iteration": t, "fp64_tc_tflops": flop / t / 1e12}
    if fp64_rate:
        out["fp64_dfma_s_per_iteration_estimated"] = flop / fp64_rate
        out["note"] = "DFMA estimate = algorithmic flop / the DFMA path's measured flop rate at o8v80w"
    return out


def batch_solve(pkg, insts, prec, autotune, max_iter=100, tol=1e-8, host=False, f64_tc=1):
    """One rccsdt_batch_solve of the uneven-instance workload from the MP2 guess.

    host=True feeds every instance's Hamiltonian from pinned host memory inside the
    timed region (the end-to-end form); energies always come back to the host.
    """
    import torch
    from paper_2607_00981_gb300 import binding as B
    lib = pkg.load()
    b = B.Batch(lib, [(i.o, i.v, i.naux) for i in insts], precision=prec, tol=tol, max_iter=max_iter,
                autotune=autotune, f64_tc=f64_tc)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
    hL = [pin(i.L) for i in insts] if host else None
    hf = [pin(i.fock_diag) for i in insts] if host else None
    if not host:
        for c, inst in zip(b.instances, insts):
            c.set_hamiltonian(inst.fock_diag, inst.L)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d = 0
    if host:
        for c, L, f in zip(b.instances, hL, hf):
            c.set_hamiltonian(f, L)
            h2d += L.nbytes + f.nbytes
    for c in b.instances:
        c.init_mp2()
    e, it, nrm, st = b.solve()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    stats = b.stats()
    infos = [c.engine_info() for c in b.instances]
    b.close()
    return {"energies": e, "iterations": it, "norms": nrm, "status": st, "stats": stats, "wall_s": wall,
            "h2d_bytes": h2d, "d2h_bytes": int(8 * 8 * len(insts)), "infos": infos}


FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.07 / 1e3  # SMs x FP32 lanes x 2 flop x max SM clock (GHz), in TFLOP/s


def q_summary(pkg, stream, mm):
    """RCCSDT(Q) energy correction (ABC-based, Sec. II.E.2) on the o6v48w workload after
    two iterations from the MP2 guess, FP64 and FP32 arithmetic: device time of each
    phase, TFLOP/s of the main kernel (the flop it executes) and its fraction of the
    ALU peak (measured DGEMM for FP64; FP32 lanes x clock for FP32)."""
    from paper_2607_00981_gb300.synth import workload
    inst = workload("o6v48w")
    ctx = pkg.context(inst.o, inst.v, inst.naux, stream=stream.cuda_stream, precision=0)
    ctx.set_hamiltonian(inst.fock_diag, inst.L)
    ctx.init_mp2()
    for _ in range(2):
        ctx.iterate()
    out = {"workload": "o6v48w: (Q) on the amplitudes after two RCCSDT iterations, o=6 v=48"}
    for label, arith, peak in (("fp64", 0, mm["fp64_tflops"]), ("fp32", 1, FP32_SIMT_TFLOPS)):
        ctx.q_energy(arith)  # warm-up
        e, info = ctx.q_energy(arith)
        tf = info["flop"] / (info["main_ms"] / 1e3) / 1e12
        out[label] = {"e_q": e, "transpose_ms": info["transpose_ms"], "intermediates_ms": info["intermediates_ms"],
                      "main_ms": info["main_ms"], "quadruples": int(info["quadruples"]), "main_tflops": tf,
                      "roofline": {"bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                                   "frac": tf / peak, "peak_source": "measured DGEMM (this run)" if arith == 0 else
                                   "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"}}
    out["fp32_rel_error_vs_fp64"] = abs(out["fp32"]["e_q"] - out["fp64"]["e_q"]) / abs(out["fp64"]["e_q"])
    ctx.close()
    return out


def t4_summary(pkg, stream, pk):
    """Compact T4 ladder (six-term direct traversal, Sec. II.C.4) and R4 post-processing
    at o=6, v=40 (126 stored blocks of 40^4) in 3xBF16 and 3xTF32: device time,
    TFLOP/s of the ladder (2 x 6 n4 v^6 flop) against the split roof, and the GB/s of
    the post-processing pass (R4 read + written once) against the measured copy rate."""
    import torch
    from paper_2607_00981_gb300 import binding as B
    from paper_2607_00981_gb300.synth import random_pair_symmetric
    o, v = 6, 40
    n4 = o * (o + 1) * (o + 2) * (o + 3) // 24
    rng = np.random.default_rng(6)
    W = random_pair_symmetric(v, seed=40)
    # T4 values need no symmetry to time the kernels
    t4c = torch.from_numpy(0.05 * rng.standard_normal((n4, v, v, v, v))).cuda()
    flop = 2.0 * 6 * n4 * v ** 6
    out = {"workload": f"o={o} v={v}: {n4} stored blocks of v^4, seeded W (pair-symmetric) and T4"}
    for label, prec, peak in (("bf16x3", B.SPLIT_BF16X3, pk.get("bf16_tflops", 1893.2) / 3.0),
                              ("tf32x3", B.SPLIT_TF32X3, None)):
        eng = B.T4Engine(pkg.load(), o, v, precision=prec, stream=stream.cuda_stream)
        eng.set(W, t4c)
        eng.pp_ladder()
        eng.postprocess()
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        eng.pp_ladder()
        e1.record(stream)
        eng.postprocess()
        e2.record(stream)
        torch.cuda.synchronize()
        lad, post = e0.elapsed_time(e1), e1.elapsed_time(e2)
        tf = flop / (lad / 1e3) / 1e12
        gbs = 2 * n4 * v ** 4 * 4 / (post / 1e3) / 1e9
        out[label] = {"ladder_ms": lad, "ladder_tflops": tf, "post_ms": post, "post_gbs": gbs,
                      "post_frac_of_copy": gbs / pk.get("hbm_gbs", 6787.2)}
        if peak:
            out[label]["roofline"] = {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                                      "frac": tf / peak, "peak_source": "measured bf16 burst / 3"}
        eng.close()
    return out


def batch_summary(pkg, args):
    """The batched uneven-instance workload (64 RCCSDT problems, o in [3, 8], v in
    [20, 60]) iterated to |R| <= 1e-8 in one CUDA graph launch per batch iteration:
    split precision with the autotuned and the fixed grouped-GEMM shape (the final
    FP64 iterations with their large contractions on the tensor cores, f64_tc = 1),
    FP64 for a few batch iterations on the FP64 units and on the tensor cores
    (s/iteration), end to end from pinned host memory, and converged energies against
    the oracle's stored values where they exist."""
    import json as _json
    from paper_2607_00981_gb300.synth import batch_instances
    insts = batch_instances(64)
    prec = PRECISIONS[args.precision] if args.precision != "fp64" else 1
    out = {"workload": "batch64: 64 RCCSDT instances, o~U[3,8], v~U[20,60], naux=4(o+v), seeds 1000+i, "
                       "weak coupling 0.6*0.3*sqrt(40/naux)", "precision": args.precision, "tol": 1e-8,
           "flop_per_batch_iteration": float(sum(2 * pkg.load().rccsdt_iteration_fma(i.o, i.v) for i in insts))}
    runs = {}
    for label, tune in (("autotuned", 1), ("fixed", 0)):
        r = batch_solve(pkg, insts, prec, tune)
        s = r["stats"]
        runs[label] = {"s_per_batch_iteration": s["device_ms"] / 1e3 / max(1.0, s["launches"]),
                       "time_to_solution_s": s["device_ms"] / 1e3, "launches": int(s["launches"]),
                       "tflops": s["flop"] / (s["device_ms"] / 1e3) / 1e12, "kernels": int(s["kernels"]),
                       "graph_build_ms": s["build_ms"], "instantiate_ms": s["instantiate_ms"],
                       "converged": int((r["status"] == 0).sum()),
                       "iterations": [int(r["iterations"].min()), float(np.median(r["iterations"])),
                                      int(r["iterations"].max())]}
        runs[label]["batch_gemm"] = {
            "on": bool(s.get("batch_gemm", 0)), "problems": int(s.get("batch_gemm_problems", 0)),
            "tiles_all_active": int(s.get("batch_gemm_tiles", 0)), "tile_width": int(s.get("batch_gemm_bn", 0)),
            "ms_all_active": s.get("batch_gemm_tuned_ms"), "fixed_shape_ms_all_active": s.get("batch_gemm_fixed_ms"),
            "note": "one persistent grouped-GEMM launch per batch iteration over every instance's residual "
                    "products; shape tuned on the batch's table" if label == "autotuned" else "fixed shape"}
        if label == "autotuned":
            energies = r["energies"]
    out["split"] = runs
    out["split_final_phase"] = ("3xTF32 from |R| <= sqrt(tol), FP64 from tol^0.75 (or a 3xTF32 stall), "
                                "large FP64 contractions on the tensor cores")
    # FP64: per-iteration cost over three batch iterations (not to convergence)
    for label, f64_tc in (("fp64", 0), ("fp64_tc", 1)):
        r = batch_solve(pkg, insts, 0, 0, max_iter=3, f64_tc=f64_tc)
        s = r["stats"]
        out[label] = {"s_per_batch_iteration": s["device_ms"] / 1e3 / max(1.0, s["launches"]),
                      "tflops": s["flop"] / (s["device_ms"] / 1e3) / 1e12, "launches": int(s["launches"]),
                      "note": "three batch iterations from the MP2 guess"}
    out["speedup_split_vs_fp64_per_iteration"] = out["fp64"]["s_per_batch_iteration"] / \
        runs["autotuned"]["s_per_batch_iteration"]
    # end to end: Hamiltonians from pinned host memory, MP2 start, solve, energies to host
    r = batch_solve(pkg, insts, prec, 1, host=True)
    out["e2e"] = {"value": r["wall_s"] / max(1.0, r["stats"]["launches"]), "unit": "s/iteration",
                  "time_to_solution_s": r["wall_s"], "h2d_bytes_per_step": int(r["h2d_bytes"]),
                  "d2h_bytes_per_step": r["d2h_bytes"],
                  "note": "per batch iteration: wall time of set_hamiltonian (host buffers), init_mp2 and "
                          "rccsdt_batch_solve, divided by the batch iterations; h2d = the Hamiltonians once "
                          "per solve, d2h = the per-iteration norms and energies of all instances"}
    # converged energies against the oracle's stored values
    golden = os.path.join(ROOT, "tests", "golden", "energies.json")
    checks = {}
    if os.path.exists(golden):
        data = _json.load(open(golden))
        for k, vd in data.items():
            if k.startswith("batch64-"):
                i = int(k.split("-")[1])
                checks[k] = abs(float(energies[i]) - vd["energy"])
    out["abs_energy_error_vs_oracle"] = checks
    return out


def run_ours(args, rank, world):
    import torch
    import paper_2607_00981_gb300 as pkg
    from paper_2607_00981_gb300.synth import workload

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    inst = workload(args.workload)
    o, v, naux = inst.o, inst.v, inst.naux
    prec = PRECISIONS[args.precision]
    stream = torch.cuda.current_stream()
    n3 = o * (o + 1) * (o + 2) // 6
    # DIIS(8) over T1, T2 and T3; when the T3 history would exceed 64 GB it keeps the
    # T3 components with all virtual labels below ns (the largest multiple of 16 whose
    # history stays within 80 GB: ns = 112 at o16v160, 73 GB, with which that workload
    # converges)
    elem = 8 if prec == 0 else 4
    hist_t3 = 2 * 8 * n3 * v ** 3 * elem
    diis_t3 = 0 if args.no_diis_t3 else 1
    nvir = 0
    if diis_t3 and hist_t3 > 64e9:
        nvir = 16 * max(1, int((80e9 / (2 * 8 * n3 * elem)) ** (1 / 3) // 16))
        while nvir > 16 and 2 * 8 * n3 * nvir ** 3 * elem > 80e9:
            nvir -= 16
    ctx = pkg.context(o, v, naux, stream=stream.cuda_stream, precision=prec, diis_t3=diis_t3, diis_t3_nvir=nvir)
    lib = ctx.lib
    L = torch.from_numpy(inst.L).to(f"cuda:{dev}")
    f = torch.from_numpy(inst.fock_diag).to(f"cuda:{dev}")
    ctx.set_hamiltonian(f, L)
    ctx.init_mp2()
    for _ in range(args.warmup):
        ctx.iterate()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # --- device-timed region: K whole iterations, inputs resident in HBM
    barrier()
    launches0 = lib.rccsdt_kernel_launches()
    ctx.enable_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        e0.record(stream)
        energies = []
        for _ in range(args.steps):
            e, norms = ctx.iterate()
            energies.append(e)
        e1.record(stream)
        barrier()
    launches = lib.rccsdt_kernel_launches() - launches0
    ms_total = e0.elapsed_time(e1)
    st = ctx.step_times()
    ctx.enable_timing(False)
    ms_total = max_over_ranks(ms_total, dist, f"cuda:{dev}")
    s_per_iter = per_iteration(ms_total / 1e3, args.steps, world)
    fma = lib.rccsdt_iteration_fma(o, v)

    # --- end to end through the C ABI with pinned host buffers
    e2e = e2e64 = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        hL, hf = pin(inst.L), pin(inst.fock_diag)
        n3 = ctx.n3
        ht1, ht2, ht3 = ctx.amplitudes()
        ht1, ht2, ht3 = pin(ht1), pin(ht2), pin(ht3)
        split = prec != PRECISIONS["fp64"]
        ksteps = max(1, min(args.steps, 3 if n3 * v ** 3 < 1e9 else 1))

        def run_e2e(t3_f32):
            h3 = pin(ht3.astype(np.float32)) if t3_f32 else ht3
            setter = ctx.set_amplitudes_t3f32 if t3_f32 else ctx.set_amplitudes
            getter = ctx.get_amplitudes_t3f32 if t3_f32 else ctx.get_amplitudes
            bytes_in = hL.nbytes + hf.nbytes + ht1.nbytes + ht2.nbytes + h3.nbytes
            bytes_out = ht1.nbytes + ht2.nbytes + h3.nbytes + 8 * 5
            barrier()
            t0 = time.perf_counter()
            for _ in range(ksteps):
                ctx.set_hamiltonian(hf, hL)
                setter(ht1, ht2, h3)
                ctx.iterate()
                getter(ht1, ht2, h3)
            barrier()
            dt = max_over_ranks(time.perf_counter() - t0, dist, f"cuda:{dev}")
            return {"value": per_iteration(dt, ksteps, world), "unit": "s/iteration",
                    "h2d_bytes_per_step": int(bytes_in), "d2h_bytes_per_step": int(bytes_out), "steps": ksteps,
                    "note": "set_hamiltonian + " + ("set_amplitudes_t3f32 (T3 in its FP32 storage type)"
                                                    if t3_f32 else "set_amplitudes (float64 T3)")
                            + " from pinned host memory, rccsdt_iterate, "
                            + ("get_amplitudes_t3f32" if t3_f32 else "get_amplitudes")
                            + " to host; DIIS history restarts each step"}

        e2e = run_e2e(split)
        if split:
            e2e64 = run_e2e(False)

    # --- roofline of the dominant kernel (the pp-ladder GEMM)
    pk = peaks()
    mm = measure_matmul_peaks()
    gemm_ms, gemm_n, gemm_flop = float(st[9]), float(st[10]), float(st[11])
    roof = None
    if gemm_n > 0 and gemm_ms > 0:
        achieved = (gemm_flop / gemm_n) / (gemm_ms / gemm_n / 1e3) / 1e12
        if prec == 0:
            peak, bound, src = mm["fp64_tflops"], "alu", "measured FP64 DGEMM (cuBLAS, this run; DFMA path)"
        elif prec == 1:
            peak, bound, src = pk.get("bf16_tflops_sustained", 1700.0) / 3.0, "tensor", \
                "measured bf16 sustained / 3 (three BF16 products per FP32-accurate product)"
        else:
            peak, bound, src = mm["tf32_tflops"] / 3.0, "tensor", \
                "measured TF32 matmul (cuBLAS, this run) / 3"
        # DRAM bytes per pp-ladder launch: the mean over the six sum / difference GEMMs of
        # the three views of the first 65-block range (the launch shape of this workload)
        # captured at o=7, v=160 (dram__bytes_read.sum + dram__bytes_write.sum, one pass)
        traffic = 10.02e9 if (args.workload == "o16v160w" and prec == 1) else None
        roof = {"kernel": "pp-ladder GEMM (k_gemm_f64)" if prec == 0 else "pp-ladder GEMM (k_gemm_tc)",
                "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, "
                "mean of the six full-shape pp-ladder GEMMs (65-block units, three views) captured at o=7 v=160; "
                "algorithmic 3.33e9 B per launch" if traffic else None, "peak_source": src,
                "launches": int(gemm_n), "avg_launch_ms": gemm_ms / gemm_n}

    step_ms = {k: float(x) / args.steps for k, x in zip(
        ["intermediates", "pp", "ring", "hh", "t2", "r12_setup", "post", "update", "energy"], st[:9])}
    ctx.close()  # the comparisons below need the device memory

    compare = None
    if not args.no_compare and world == 1:
        compare = compare_fp64_split(pkg, stream, dev)
    fp64_here = None
    if not args.no_compare and world == 1 and prec != 0:
        rate = 2.0 * lib.rccsdt_iteration_fma(8, 80) / compare["fp64"] if compare else None
        fp64_here = fp64_tc_iteration(pkg, stream, inst, rate)
        fp64_here["speedup_split_vs_fp64_tc"] = fp64_here["fp64_tc_s_per_iteration"] / s_per_iter
        if rate:
            fp64_here["speedup_split_vs_fp64_dfma_estimated"] = \
                fp64_here["fp64_dfma_s_per_iteration_estimated"] / s_per_iter

    batch = None
    if rank == 0 and world == 1 and not args.no_batch:
        batch = batch_summary(pkg, args)

    extra_q = extra_t4 = None
    if rank == 0 and world == 1 and not args.no_next:
        extra_q = q_summary(pkg, stream, mm)
        extra_t4 = t4_summary(pkg, stream, pk)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, sample = oracle_sample(inst, seconds_budget=args.ref_seconds)
        cpu = {"value": val, "unit": "s/iteration", "cores": os.cpu_count(), "kind": "oracle", "sample": sample,
               "cpu_model": cpu_model(), "one_core": oracle_sample_one_core(args.workload, 5.0)}

    if rank == 0:
        line = {"metric": METRIC, "value": s_per_iter, "unit": "s/iteration", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
                "config": dict(config(args, inst), parallelism=f"replicas{world}"),
                "tflops": 2.0 * fma * world / (ms_total / 1e3 / args.steps) / 1e12,
                "energy_last": energies[-1], "e2e": e2e, "e2e_float64_t3": e2e64, "gpu_launches": int(launches), "roofline": roof,
                "cpu_baseline": cpu, "clocks": clk.summary(), "fp64_vs_split": compare, "fp64_here": fp64_here,
                "batch64": batch, "matmul_peaks": mm, "q_correction": extra_q, "t4_ladder": extra_t4,
                "diis": ("DIIS(8) over T1 and T2" if not diis_t3 else
                         "DIIS(8) over T1, T2 and T3" if not nvir else
                         f"DIIS(8) over T1, T2 and the T3 components with a, b, c < {nvir} "
                         f"({2 * 8 * n3 * nvir ** 3 * elem / 1e9:.0f} GB of history)"),
                "step_ms": step_ms}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="o16v160w")
    ap.add_argument("--precision", default="bf16x3", choices=list(PRECISIONS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-diis-t3", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 vs split comparison at o8v80w")
    ap.add_argument("--ref-seconds", type=float, default=20.0)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched uneven-instance workload")
    ap.add_argument("--no-next", action="store_true", help="skip the (Q) and compact-T4 measurements")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
