"""Write tests/golden/oracle_<config>.json: a full run of the FP64 oracle on a workload.

Calls only `oracle/` and the seeded input generators; stores the iteration count,
the wall time on this host, its core count and the eigenvalues.  Used to scale the
bounded oracle sample that the benchmark times into a time to solution.

    python tests/golden/make_oracle_runs.py q1_64
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle.gcg import gcg, Params  # noqa: E402


def main(name):
    p = W.make_config(name)
    nev, bs = W.CONFIGS[name]["nev"], W.CONFIGS[name]["bs"]
    X0 = W.initial_block(p.n, min(nev + 3 * bs, p.n), 0)
    t0 = time.perf_counter()
    r = gcg(p.A, p.B, nev, bs, 1e-8, X0, Params())
    dt = time.perf_counter() - t0
    out = {"config": name, "source": "oracle/gcg.py (FP64 CPU), seed 0, tol 1e-8",
           "iterations": int(r.iterations), "converged": bool(r.converged),
           "nconv": int(r.nconv), "seconds": round(dt, 2), "host_cores": os.cpu_count(),
           "evals": [float(x) for x in r.evals[:nev]]}
    with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, r.iterations, r.converged, f"{dt:.1f}s")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "q1_64")
