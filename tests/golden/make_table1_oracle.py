"""Writes tests/golden/table1_oracle.json from the FP64 CPU oracle only: for each Rayleigh number of
Table 1 (Sec. 3.3; 60 x 30, Pr = 0.71, Ma = 0.3, the workloads.rayleigh_benard_table1 set-up) the
Nusselt number of Eq. (29) after 10,000, 20,000 and 30,000 steps, and at steady state (Nu changing
by less than 1e-9 between two checks 1,000 steps apart, cap 200,000 steps).
Run: python tests/golden/make_table1_oracle.py  (about a minute on 8 cores)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1710_10569_gb300 import workloads as W  # noqa: E402

RA = (2000, 2500, 3000, 5000, 10000, 20000, 30000, 50000)


def main():
    out = {}
    for ra in RA:
        prob = W.rayleigh_benard_table1(float(ra))
        o = oracle.Oracle.from_problem(prob)
        rec = {"at": {}}
        prev = None
        while o.steps < 200000:
            o.step(1000)
            nu = o.nusselt(1)
            if o.steps in (10000, 20000, 30000):
                rec["at"][str(o.steps)] = nu
            if o.steps >= 30000 and prev is not None and abs(nu - prev) < 1e-9:
                break
            prev = nu
        rec["steady"] = nu
        rec["steady_steps"] = o.steps
        out[str(ra)] = rec
        print(ra, rec, flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "table1_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
