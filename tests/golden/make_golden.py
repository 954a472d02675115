"""Writes tests/golden/energies.json: converged RCCSDT energies from the FP64 oracle.

Run from the repository root:  python tests/golden/make_golden.py [name ...]
Calls only the oracle (compact storage, Jacobi + DIIS(8), |R| <= 1e-10) on the
seeded instances of paper_2607_00981_gb300.synth.CONVERGENCE, or on instance i of
the batched workload (synth.batch_instances) for a name "batch64-<i>".
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import compact as oc  # noqa: E402
from paper_2607_00981_gb300.synth import CONVERGENCE, batch_instances, workload  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "energies.json")


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        if name.startswith("batch64-"):
            inst = batch_instances(64)[int(name.split("-")[1])]
            spec = {"o": inst.o, "v": inst.v, "naux": inst.naux, "seed": inst.seed,
                    "scale": 0.6 * 0.3 * (40 / inst.naux) ** 0.5}
        else:
            inst = workload(name)
            spec = {k: CONVERGENCE[name][k] for k in ("o", "v", "naux", "seed", "scale")}
        t0 = time.time()
        E, t1, t2, t3c, it, hist = oc.solve_compact(inst.L, inst.fock_diag, inst.o, tol=1e-10, max_iter=400)
        data[name] = {"energy": E, "iterations": it, "residual_norm": hist[-1][2], "tol": 1e-10,
                      "spec": spec,
                      "solver": "oracle.compact.solve_compact, DIIS(8) from iteration 2",
                      "seconds": round(time.time() - t0, 1)}
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(name, E, it, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["o6v48w"])
