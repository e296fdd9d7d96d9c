"""Autotuner for the step kernels' tile shape (nodes per thread, rows per work
item, pipeline stages) and CUDA-graph length.

Each candidate is timed on the actual workload with CUDA events after a short
warm-up, and the fastest is returned; results can be cached in a JSON file
keyed by the workload's shapes and the GPU name. Tuning never changes results:
every tile computes bit-identical steps.

    python -m paper_1601_04633_gb300.tune --batch      # the 64-cavity sweep
    python -m paper_1601_04633_gb300.tune --single 4096
    python -m paper_1601_04633_gb300.tune --batch --storage 3 --tile 4 4 2 --steps 16 --graph-steps 16
    python -m paper_1601_04633_gb300.tune --batch --group-mb 0 32 64    # with L2-sized cavity groups
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os

# Compiled tiles (see include/dmrt.h).
BATCH_TILES = [(1, 1, 2), (1, 2, 2), (1, 4, 2), (1, 4, 3), (2, 1, 2), (2, 1, 3), (2, 2, 2), (2, 2, 3), (2, 4, 2),
               (4, 1, 4), (4, 2, 2), (4, 4, 2)]
SINGLE_TILES_FP32 = ([(1, r, s) for r, s in [(1, 2), (1, 3), (1, 4), (1, 5), (2, 2), (2, 3), (3, 2), (4, 2), (4, 3)]]
                     + [(2, r, s) for r, s in [(1, 3), (1, 4), (1, 5), (2, 2), (2, 3), (4, 2)]]
                     + [(4, r, s) for r, s in [(1, 2), (1, 3), (1, 4), (1, 5), (1, 6), (2, 2), (2, 3), (2, 4),
                                              (4, 2), (4, 3)]])
SINGLE_TILES_16 = [(1, 1, 2), (1, 2, 2), (1, 4, 2), (1, 4, 3), (1, 4, 4), (2, 2, 2), (2, 4, 2), (2, 4, 3), (4, 2, 2),
                   (4, 4, 2)]
SINGLE_TILES_16_SR = [(1, 1, 2), (1, 4, 2), (2, 2, 2), (2, 4, 2), (4, 2, 2), (4, 4, 2)]
SINGLE_TILES_MIXED = [(1, 1, 2), (1, 1, 3), (1, 1, 4), (1, 2, 2), (1, 2, 3), (1, 4, 2), (2, 1, 2), (2, 1, 3),
                      (2, 1, 4), (2, 2, 2), (4, 1, 3), (4, 1, 4)]
SINGLE_TILES_MIXED_SR = [(1, 1, 2), (1, 2, 2), (1, 4, 2), (1, 4, 3), (2, 1, 2), (2, 1, 3), (2, 2, 2), (2, 4, 2),
                         (4, 1, 3)]
SINGLE_TILES_THETA = [(1, 1, 2), (2, 1, 2), (2, 1, 3), (2, 2, 2), (4, 1, 3)]
SINGLE_TILES_THETA_SR = [(1, 1, 2), (1, 2, 2), (2, 1, 2), (2, 1, 3), (2, 2, 2), (2, 4, 2), (4, 1, 3), (4, 2, 2)]


def _time_steps(step, steps, warmup):
    import torch

    step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    step(steps)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def _key(kind, shapes, extra=""):
    import torch

    h = hashlib.sha256(json.dumps([kind, shapes, extra]).encode()).hexdigest()[:16]
    return f"{torch.cuda.get_device_name()}|{kind}|{h}"


def _cache_get(path, key):
    if not path or not os.path.exists(path):
        return None
    with open(path) as fh:
        return json.load(fh).get(key)


def _cache_put(path, key, value):
    if not path:
        return
    d = {}
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
    d[key] = value
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1)
    os.replace(tmp, path)


# Cavity-group sizes tried for the batched sweep (bytes of both population
# buffers per group; 0: one group, every cavity in every launch). The GB300's
# L2 holds about 126 MB.
GROUP_BYTES = [0, 24 << 20, 40 << 20, 64 << 20, 96 << 20]
# Tiles compiled for the multi-step batched kernel (several steps per launch).
BATCH_MSTEP_TILES = {0: [(1, 2, 2), (2, 1, 2), (2, 2, 2), (2, 2, 3), (4, 2, 2), (4, 4, 2)],
                     3: [(2, 2, 2), (4, 2, 2), (4, 4, 2)]}
STEPS_PER_LAUNCH = [1, 8, 32]
# Tiles compiled with the tensor-store epilogue (one launch per step).
BATCH_TS_TILES = {0: [(2, 1, 2), (2, 2, 2)], 3: [(2, 2, 2), (4, 2, 2), (4, 4, 2)]}


def tune_batch(cavities, steps=200, warmup=20, tiles=None, graph_steps=(64,), cache=None, storage=0, rounding=0,
               group_bytes=(0,), steps_per_launch=(1,), tensor_store=False, finalists=3, strip_fill=(0, 1)):
    """Pick the batched kernel's tile, strip policy, cavity-group size and steps
    per launch for these cavities (storage 0: float32, 3: mixed). Every tile is
    timed with each strip policy, the first group size and one step per launch;
    the `finalists` fastest are then timed with each other combination (steps
    per launch > 1 only for the tiles the multi-step kernel is compiled for).
    Returns {"opts": {...}, "mlups": best, "trials": [...]}."""
    from . import dmrt as D

    key = _key("batch", [(c.nx, c.ny) for c in cavities],
               f"{steps}-{storage}-{rounding}-{list(group_bytes)}-{list(steps_per_launch)}-{tensor_store}-"
               f"{list(strip_fill)}")
    hit = _cache_get(cache, key)
    if hit:
        return hit
    nodes = sum(c.nx * c.ny for c in cavities)
    trials = []

    def trial(npt, R, S, g, gb, K, ts=0, fill=0):
        opts = dict(tma_npt=npt, tma_rows=R, tma_stages=S, graph_steps=g, group_bytes=gb, steps_per_launch=K,
                    tensor_store=ts, strip_fill=fill)
        glen = 2 * K if K > 1 else g
        # The warm-up covers one whole graph, so its instantiation is not timed.
        b = D.Batch.from_inputs(cavities, opts=opts, nu_capacity=steps + warmup + glen + 8, storage=storage,
                                rounding=rounding)
        sec = _time_steps(b.step, steps, max(warmup, glen))
        b.check()
        trials.append({"opts": opts, "mlups": nodes * steps / sec / 1e6, "groups": b.groups})
        b.close()

    for npt, R, S in (tiles or BATCH_TILES):
        for g in graph_steps:
            for fill in strip_fill:
                trial(npt, R, S, g, group_bytes[0], 1, fill=fill)
    if len(group_bytes) > 1 or len(steps_per_launch) > 1 or tensor_store:
        top = sorted(trials, key=lambda r: -r["mlups"])[:finalists]
        for t in top:
            o = t["opts"]
            tile = (o["tma_npt"], o["tma_rows"], o["tma_stages"])
            for K in steps_per_launch:
                if K > 1 and tile not in BATCH_MSTEP_TILES.get(storage, []):
                    continue
                for gb in group_bytes:
                    if (gb, K) == (group_bytes[0], 1):
                        continue
                    trial(*tile, o["graph_steps"], gb, K, fill=o["strip_fill"])
            if tensor_store and tile in BATCH_TS_TILES.get(storage, []):
                for gb in group_bytes:
                    trial(*tile, o["graph_steps"], gb, 1, 1, fill=o["strip_fill"])
    best = max(trials, key=lambda r: r["mlups"])
    out = {"opts": best["opts"], "mlups": best["mlups"], "trials": trials}
    _cache_put(cache, key, out)
    return out


def tune_single(cav, storage=0, rounding=0, steps=200, warmup=20, tiles=None, cache=None):
    """Pick the single-cavity TMA tile. Returns {"kw": {...}, "mlups": best, "trials": [...]}."""
    from . import dmrt as D

    if tiles is None:
        if storage == 3:
            tiles = SINGLE_TILES_MIXED_SR if rounding else SINGLE_TILES_MIXED
        elif storage == 4:
            tiles = SINGLE_TILES_THETA_SR if rounding else SINGLE_TILES_THETA
        else:
            tiles = SINGLE_TILES_FP32 if storage == 0 else (SINGLE_TILES_16_SR if rounding else SINGLE_TILES_16)
    key = _key("single", [(cav.nx, cav.ny)], f"{storage}-{rounding}-{steps}")
    hit = _cache_get(cache, key)
    if hit:
        return hit
    trials = []
    for npt, R, S in tiles:
        kw = dict(kernel=D.DMRT_KERNEL_TMA, tma_npt=npt, tma_rows=R, tma_stages=S, storage=storage,
                  rounding=rounding)
        sim = D.Cavity2D.from_inputs(cav, nu_capacity=steps + warmup + 72, **kw)
        sec = _time_steps(sim.step, steps, max(warmup, 64))  # one whole graph before timing
        sim.check()
        sim.close()
        trials.append({"kw": kw, "mlups": cav.nx * cav.ny * steps / sec / 1e6})
    best = max(trials, key=lambda r: r["mlups"])
    out = {"kw": best["kw"], "mlups": best["mlups"], "trials": trials}
    _cache_put(cache, key, out)
    return out


def main():
    from . import inputs

    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--batch", action="store_true")
    ap.add_argument("--single", type=int, default=0, help="side of a square cavity")
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--storage", type=int, default=0, help="0 float32, 1 float16, 2 bfloat16, 3 mixed")
    ap.add_argument("--rounding", type=int, default=0, help="0 nearest, 1 stochastic")
    ap.add_argument("--tile", type=int, nargs=3, metavar=("NPT", "R", "S"), help="time this tile only")
    ap.add_argument("--graph-steps", type=int, default=64, help="steps per CUDA graph (batched sweep)")
    ap.add_argument("--group-mb", type=int, nargs="*", default=[0],
                    help="cavity-group sizes to try, MB of both buffers (batched sweep; 0: one group)")
    ap.add_argument("--steps-per-launch", type=int, nargs="*", default=[1],
                    help="steps per launch to try (batched sweep; 1: one launch per step)")
    ap.add_argument("--tensor-store", action="store_true", help="also try the tensor-store epilogue (batched sweep)")
    ap.add_argument("--strip-fill", type=int, nargs="*", default=[0, 1],
                    help="strip policies to try (batched sweep; 0 widest strips, 1 fullest blocks)")
    ap.add_argument("--cache", default=None)
    args = ap.parse_args()
    tiles = [tuple(args.tile)] if args.tile else None
    if args.batch:
        print(json.dumps(tune_batch(inputs.batch_sweep(), steps=args.steps, tiles=tiles,
                                    graph_steps=(args.graph_steps,), cache=args.cache, storage=args.storage,
                                    rounding=args.rounding, group_bytes=[m << 20 for m in args.group_mb],
                                    steps_per_launch=args.steps_per_launch, tensor_store=args.tensor_store,
                                    strip_fill=args.strip_fill),
                         indent=1))
    if args.single:
        cav = inputs.Cavity(args.single, args.single, 1e7, 0.001, seed=5)
        print(json.dumps(tune_single(cav, storage=args.storage, rounding=args.rounding, steps=args.steps,
                                     tiles=tiles, cache=args.cache), indent=1))


if __name__ == "__main__":
    main()
