"""Write tests/golden/oracle_cases_64.json: the fp64 oracle's hot-wall Nusselt
history for the paper's four cases (Table 1: Ra, Pr) on a 64 x 64 cavity,
alpha = 0.1, walls +-0.5, rest start with seeded 1e-6 noise (seed 10 + case),
to Fourier number 4 (Eq. 20). Calls only the oracle.

    python tests/golden/make_oracle_cases.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_1601_04633_gb300 import inputs  # noqa: E402

CASES = [(1, 1e4, 0.01), (2, 5e4, 0.01), (3, 5e4, 0.005), (4, 1e5, 0.01)]
N, ALPHA, FO_END, EVERY, FO_KEEP = 64, 0.1, 4.0, 64, 1.5


def main():
    O.set_threads(0)
    steps = int(round(FO_END * N * N / ALPHA))
    out = {"_source": "fp64 oracle (oracle/dmrt_oracle.c) via tests/golden/make_oracle_cases.py",
           "n": N, "alpha": ALPHA, "steps": steps, "every": EVERY, "fo_first_kept": FO_KEEP, "cases": []}
    for case, Ra, Pr in CASES:
        cav = inputs.Cavity(N, N, Ra, Pr, ALPHA, seed=10 + case)
        m = O.derive(N, N, Ra, Pr, ALPHA)
        f, g = O.init(m, cav.theta0())
        r = O.run(m, steps, f, g)
        first = int(round(FO_KEEP * N * N / ALPHA))
        kept = r["nu_series"][first - 1::EVERY]
        out["cases"].append({"case": case, "Ra": Ra, "Pr": Pr, "first_step": first,
                             "nu": [float(x) for x in kept], "nu_local_last": [float(x) for x in r["nu_local"]]})
        print(case, Ra, Pr, float(r["nu_series"][-1]), flush=True)
    with open(os.path.join(HERE, "oracle_cases_64.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
