"""Writes tests/golden/cavity256_ra1e5.json from the FP64 CPU oracle only: the side-heated cavity
(256 x 256, Ra = 1e5, Pr = 0.71, u_c = 0.1, seed 0) stepped to E_R < 1e-8 (checked every 100
steps, cap 400k steps), with the Nusselt number (Eq. 29 along x) recorded at fixed step counts and at
convergence. Run: python tests/golden/make_cavity_golden.py  (tens of minutes on 8 cores)."""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1710_10569_gb300 import workloads as W  # noqa: E402

CHECKPOINTS = (2000, 5000, 10000, 20000, 50000)


def main():
    prob = W.cavity(256, Ra=1e5, Pr=0.71, u_c=0.1, seed=0)
    o = oracle.Oracle.from_problem(prob)
    p = prob.params
    prev = o.fields()[1:]
    out = {"problem": prob.name, "seed": 0, "interval": 100, "nusselt_at": {}, "threads": oracle.threads()}
    t0 = time.time()
    er = float("inf")
    while o.steps < 400000:
        o.step(100)
        cur = o.fields()[1:]
        er = oracle.residual(prev, cur, p["u_ref"], p["dT_ref"])
        prev = cur
        if o.steps in CHECKPOINTS:
            out["nusselt_at"][str(o.steps)] = oracle.nusselt(cur[0], cur[1], cur[2], p, 0)
            print(o.steps, out["nusselt_at"][str(o.steps)], er, f"{time.time() - t0:.0f}s", flush=True)
        if er < 1e-8:
            break
    out["steps"] = o.steps
    out["residual"] = er
    out["nusselt"] = oracle.nusselt(prev[0], prev[1], prev[2], p, 0)
    out["seconds"] = time.time() - t0
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "cavity256_ra1e5.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
