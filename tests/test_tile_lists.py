"""The tile lists the autotuner and the tests walk agree with the variant tables
compiled into the library (host logic; no GPU).

Each `csrc/tma_*.cu` holds a table of (storage, rounding, nodes per thread,
rows, stages, epilogue, kernel) entries; a tile the tuner times must be in
the table (or creating the context fails), every table entry must be reachable
through the tuner, each entry's template arguments must repeat its (npt, R, S),
and the default tiles the library picks must be compiled.
"""
import glob
import os
import re

from paper_1601_04633_gb300 import tune

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1601_04633_gb300", "csrc")
STORAGE = {"DMRT_FP32": 0, "DMRT_FP16": 1, "DMRT_BF16": 2, "DMRT_MIXED": 3, "DMRT_THETA32": 4}
ROUNDING = {"DMRT_ROUND_NEAREST": 0, "DMRT_ROUND_STOCHASTIC": 1}
ENTRY = re.compile(r"\{(DMRT_\w+), (DMRT_ROUND_\w+), (\d+), (\d+), (\d+), ([01]), \(const void\*\)(\w+)<(.*)>\}")


def _tables(with_mstep=False):
    single, batch, mstep = set(), set(), set()
    for path in sorted(glob.glob(os.path.join(CSRC, "tma_*.cu"))):
        with open(path) as fh:
            for line in fh:
                m = ENTRY.search(line)
                if not m:
                    continue
                st, rd, npt, R, S, ts, kernel, targs = m.groups()
                key = (STORAGE[st], ROUNDING[rd], int(npt), int(R), int(S))
                # The template arguments after the layout repeat (npt, R, S).
                rest = re.sub(r"^\w+(<[^>]*>)?,\s*", "", targs).split(",")
                assert [int(x) for x in rest[:3]] == [int(npt), int(R), int(S)], line
                if kernel == "step_tma_batch_kernel":
                    batch.add(key)
                elif kernel == "step_tma_batch_mstep_kernel":
                    mstep.add(key)
                else:
                    single.add(key)
    return (single, batch, mstep) if with_mstep else (single, batch)


def test_tables_parse():
    single, batch = _tables()
    assert len(single) > 50 and len(batch) > 20


def test_single_tuner_tiles_are_compiled_and_complete():
    single, _ = _tables()
    lists = {(0, 0): tune.SINGLE_TILES_FP32, (1, 0): tune.SINGLE_TILES_16, (1, 1): tune.SINGLE_TILES_16_SR,
             (2, 0): tune.SINGLE_TILES_16, (2, 1): tune.SINGLE_TILES_16_SR, (3, 0): tune.SINGLE_TILES_MIXED,
             (3, 1): tune.SINGLE_TILES_MIXED_SR, (4, 0): tune.SINGLE_TILES_THETA, (4, 1): tune.SINGLE_TILES_THETA_SR}
    for (st, rd), tiles in lists.items():
        listed = {(st, rd) + tuple(t) for t in tiles}
        compiled = {k for k in single if k[:2] == (st, rd)}
        assert listed == compiled, (st, rd, sorted(listed ^ compiled))


def test_batch_tuner_tiles_are_compiled_for_every_batch_storage():
    _, batch = _tables()
    for st, rd in ((0, 0), (3, 0), (3, 1)):
        compiled = {k[2:] for k in batch if k[:2] == (st, rd)}
        assert compiled == set(map(tuple, tune.BATCH_TILES)), (st, rd)
    assert {k[:2] for k in batch} == {(0, 0), (3, 0), (3, 1)}


def test_multistep_batch_tiles_match_the_tuner_and_have_single_step_twins():
    # Every multi-step tile the tuner may pick is compiled, and also compiled as
    # a one-step-per-launch tile (a batch call runs its remainder steps that way).
    _, batch, mstep = _tables(with_mstep=True)
    for st, rd in ((0, 0), (3, 0), (3, 1)):
        compiled = {k[2:] for k in mstep if k[:2] == (st, rd)}
        assert compiled == set(map(tuple, tune.BATCH_MSTEP_TILES[st])), (st, rd)
        assert {(st, rd) + t for t in compiled} <= batch
    assert {k[:2] for k in mstep} == {(0, 0), (3, 0), (3, 1)}


def test_tensor_store_batch_tiles_match_the_tuner():
    import re as _re

    ts = set()
    with open(os.path.join(CSRC, "tma_batch.cu")) as fh:
        for line in fh:
            m = ENTRY.search(line)
            if m and m.group(6) == "1":
                ts.add((STORAGE[m.group(1)], ROUNDING[m.group(2)], int(m.group(3)), int(m.group(4)), int(m.group(5))))
                assert _re.search(r", true>\}", line), line  # the TS template argument
    for st, rd in ((0, 0), (3, 0), (3, 1)):
        assert {k[2:] for k in ts if k[:2] == (st, rd)} == set(tune.BATCH_TS_TILES[st]), (st, rd)


def test_default_tiles_are_compiled():
    # The library's defaults (storage, rounding -> tile) and the small-grid
    # tiles it switches to: float32 (1,4,2), one-row (1,1,2) and (2,1,3);
    # 16-bit nearest (2,4,2) and stochastic (4,4,2), 2-row (2,2,2) / (4,2,2),
    # one-row (1,1,2); mixed (2,1,2); THETA32 nearest (2,1,2), stochastic (4,2,2).
    single, batch = _tables()
    want = [(0, 0, 1, 4, 2), (0, 0, 1, 1, 2), (0, 0, 2, 1, 3)]
    for st in (1, 2):
        want += [(st, 0, 2, 4, 2), (st, 0, 2, 2, 2), (st, 0, 1, 1, 2),
                 (st, 1, 4, 4, 2), (st, 1, 4, 2, 2), (st, 1, 1, 1, 2)]
    want += [(3, 0, 2, 1, 2), (3, 1, 2, 1, 2)]
    want += [(4, 0, 2, 1, 2), (4, 1, 4, 2, 2), (4, 0, 1, 1, 2), (4, 1, 1, 1, 2)]
    for k in want:
        assert k in single, k
    for k in [(0, 0, 2, 2, 2), (3, 0, 4, 2, 2), (3, 1, 4, 2, 2)]:
        assert k in batch, k
