"""Write oracle/iteration_counts.json: the oracle's own Jacobi-PCG iteration
counts to a relative residual of 1e-10 on the benchmark workloads.

Test infrastructure: the timed CPU baseline runs the oracle's PCG for a
bounded number of iterations and scales its time per iteration by these
counts.  Only the oracle is called here.

Usage: python -m oracle.count_iterations [workload ...]
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import synth  # noqa: E402
from oracle import hybrid, krylov, pipeline  # noqa: E402

OUT = os.path.join(HERE, "iteration_counts.json")


def count(name, rtol=1e-10):
    p = synth.config_problem(name)
    topo, geom, A_K, D_K, R_K = pipeline.setup(p["coords"], p["elems"], p["nu"], p["mu"], p["fbar"][0], p["conv"])
    h = hybrid.hybridise(topo, A_K, D_K, R_K, p["mu"])
    t = time.perf_counter()
    _, it, hist = krylov.pcg(h["G"], h["S"], krylov.jacobi(h["G"]), rtol=rtol)
    return {"pcg_iterations": int(it), "rtol": rtol, "final_relres": float(hist[-1]),
            "seconds": time.perf_counter() - t}


if __name__ == "__main__":
    names = sys.argv[1:] or ["cfg1", "cfg2"]
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for n in names:
        data[n] = count(n)
        print(n, data[n], flush=True)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
