"""Named runs of the library on the GPU, for profiling one kernel in isolation.

    python -m paper_1601_04633_gb300.workloads adjoint_128    # discrete adjoint, 128^2, 10k steps
    python -m paper_1601_04633_gb300.workloads cavity --n 64 --steps 20000 [--kernel 3] [--timed]
    python -m paper_1601_04633_gb300.workloads batch --steps 16 [--storage 3 --rounding 1]

Each prints one JSON line with its wall time; the runs are the benchmark's
workloads (``inputs``), so a profile of one of them covers the same launches.
``cavity --timed`` also times the steps on the device (CUDA events around the
``--steps`` steps, after 200 warm-up steps) and prints microseconds per step.
"""
from __future__ import annotations

import argparse
import json
import time


def main():
    from . import dmrt as D
    from . import inputs

    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("run", choices=("adjoint_128", "cavity", "batch"))
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--storage", type=int, default=0)
    ap.add_argument("--rounding", type=int, default=D.DMRT_ROUND_AUTO)
    ap.add_argument("--kernel", type=int, default=D.DMRT_KERNEL_AUTO, help="cavity: 0 auto, 1 direct, 2 TMA, 3 cluster")
    ap.add_argument("--timed", action="store_true", help="cavity: time the steps with CUDA events")
    args = ap.parse_args()
    import torch

    t0 = time.perf_counter()
    if args.run == "adjoint_128":
        cav = inputs.cavity_128_adjoint()
        sim = D.Cavity2D.from_inputs(cav, nu_capacity=2000)
        J, dth, dRa = sim.adjoint(args.steps, min(2000, args.steps))
        sim.close()
        out = {"J": J, "dJ_dRa": dRa}
    elif args.run == "cavity":
        cav = inputs.Cavity(args.n, args.n, 1e4, 0.01, seed=1)
        warm = 200 if args.timed else 0
        sim = D.Cavity2D.from_inputs(cav, nu_capacity=args.steps + warm, storage=args.storage,
                                     rounding=args.rounding, kernel=args.kernel)
        out = {}
        if warm:
            sim.step(warm)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(torch.cuda.current_stream())
        sim.step(args.steps)
        if warm:
            e1.record(torch.cuda.current_stream())
            torch.cuda.synchronize()
            out["us_per_step"] = 1e3 * e0.elapsed_time(e1) / args.steps
        sim.check()
        out.update({"nu": sim.nusselt()[0], "launch": sim.launch})
        sim.close()
    else:
        b = D.Batch.from_inputs(inputs.batch_sweep(), nu_capacity=args.steps, storage=args.storage,
                                rounding=args.rounding)
        b.step(args.steps)
        b.check()
        out = {"launch": b.launch}
        b.close()
    torch.cuda.synchronize()
    out.update({"run": args.run, "seconds": time.perf_counter() - t0})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
