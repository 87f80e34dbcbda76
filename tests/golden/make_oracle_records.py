"""Run the FP64 oracle to the stopping tolerance on each named workload and record the outcome.

Writes tests/golden/oracle_records.json: per workload the outer iterations, bundles, final
objective, relative KKT and the oracle's wall time.  Calls only datagen (inputs) and oracle/.
The records give the benchmark's CPU-reference arm the number of bundles a full solve takes,
so that a bounded sample of oracle bundles can be projected to a whole solve.

    python tests/golden/make_oracle_records.py lr_2m_3m [more workloads]
"""
import json
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import datagen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_records.json")


def main(names):
    rec = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        wl = datagen.workload(name)
        t0 = time.time()
        p = datagen.generate(wl.spec, with_csr=False)
        tg = time.time() - t0
        o = oracle.Oracle.from_problem(p, wl.C, wl.loss)
        t0 = time.time()
        _, st = o.solve(wl.P, eps=wl.eps, seed=wl.solver_seed, max_epochs=1000)
        ts = time.time() - t0
        rec[name] = dict(workload=wl.describe(), nnz=p.nnz, epochs=int(st["epochs"]), bundles=int(st["bundles"]),
                         F_final=st["F_final"], kkt_rel=st["kkt_rel"], converged=bool(st["converged"]),
                         oracle_seconds=ts, generate_seconds=tg, machine=platform.machine(),
                         cpu=platform.processor() or platform.machine(), threads=1)
        print(name, rec[name], flush=True)
        with open(OUT, "w") as f:
            json.dump(rec, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["lr_2m_3m"])
