"""Write the fp64 oracle's Nusselt histories for two of the benchmark workloads,
so that GPU tests can compare full-length runs with it. Calls only the oracle.

* ``oracle_config2_256.json``: the oscillatory cavity 256 x 256, Ra = 1e5,
  Pr = 0.005, alpha = 0.1, seeded 1e-6 noise (seed 2), 1e6 steps; mean Nu every
  250 steps (about 1.8 h on 8 cores).
* ``oracle_config3_members.json``: three 128 x 128 members of the 64-cavity
  sweep (indices 0, 2, 60: Ra 2.5e5, 6.0e5, 1.3e5), 50,000 steps; mean Nu every
  100 steps.

    python tests/golden/make_baseline_goldens.py config3
    python tests/golden/make_baseline_goldens.py config2
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_1601_04633_gb300 import inputs  # noqa: E402

SOURCE = "fp64 oracle (oracle/dmrt_oracle.c) via tests/golden/make_baseline_goldens.py"


def _run(cav, steps):
    m = O.derive(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha)
    f, g = O.init(m, cav.theta0())
    return O.run(m, steps, f, g)["nu_series"]


def config2():
    cav = inputs.cavity_256_oscillatory()
    steps, every = 1_000_000, 250
    nu = _run(cav, steps)
    out = {"_source": SOURCE, "nx": cav.nx, "ny": cav.ny, "Ra": cav.Ra, "Pr": cav.Pr, "alpha": cav.alpha,
           "seed": cav.seed, "steps": steps, "every": every,
           "nu": [float(x) for x in nu[every - 1::every]]}
    with open(os.path.join(HERE, "oracle_config2_256.json"), "w") as fh:
        json.dump(out, fh)


def config3():
    cavs = inputs.batch_sweep()
    steps, every = 50_000, 100
    out = {"_source": SOURCE, "steps": steps, "every": every, "members": []}
    for i in (0, 2, 60):
        c = cavs[i]
        nu = _run(c, steps)
        out["members"].append({"index": i, "nx": c.nx, "ny": c.ny, "Ra": c.Ra, "Pr": c.Pr, "seed": c.seed,
                               "nu": [float(x) for x in nu[every - 1::every]]})
        print(i, c.nx, c.Ra, c.Pr, float(nu[-1]), flush=True)
    with open(os.path.join(HERE, "oracle_config3_members.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    O.set_threads(0)
    for name in sys.argv[1:] or ["config3", "config2"]:
        {"config2": config2, "config3": config3}[name]()
