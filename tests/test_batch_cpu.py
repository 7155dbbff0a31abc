"""Host-side checks of the batched runner's task lists (sft_batch_plan; no
GPU): the persistent kernel relies on each list being a topological order of
the passes of Algorithm 2, with every pass cut into tasks that cover it
exactly once."""
import collections

import pytest

SHAPES = [((300, 200, 100), 8, 20_000), ((50, 60, 70, 80, 90, 40), 4, 3_001),
          ((1000, 1000), 32, 70_000), ((7, 9, 11), 16, 257)]
FACTOR, REFRESH, CORE, APPLY, LOSS, LOSSFIN = range(6)


@pytest.fixture(scope="module")
def sft():
    from paper_2210_06014_gb300 import build, sft as mod
    build.build()
    mod.load()
    return mod


def plan(sft, which, chunk, workers, shapes=SHAPES):
    recs = sft.batch_problem_records(shapes)
    return sft.sft_batch_plan(recs, which, chunk, workers)


@pytest.mark.parametrize("workers", [1, 7, 304])
@pytest.mark.parametrize("chunk", [256, 4096])
def test_epoch_plan_is_a_topological_order_of_algorithm_2(sft, workers, chunk):
    tasks = plan(sft, 0, chunk, workers)
    first = {}   # counter -> position of its first task
    count = collections.Counter(t["done"] for t in tasks)
    seen = collections.Counter()
    for pos, t in enumerate(tasks):
        if t["wait"] >= 0:
            # every task of the pass it waits for was handed out earlier
            assert seen[t["wait"]] == count[t["wait"]], (pos, t)
        seen[t["done"]] += 1
        first.setdefault(t["done"], pos)
    for p, (dims, R, nnz) in enumerate(SHAPES):
        mine = [t for t in tasks if t["prob"] == p]
        phases = []
        for t in sorted(mine, key=lambda t: first[t["done"]]):
            key = (t["kind"], t["mode"], t["done"])
            if not phases or phases[-1] != key:
                phases.append(key)
        N = len(dims)
        want = [(FACTOR, n) for n in range(N) for _ in (0,)]
        want = []
        for n in range(N):
            want += [(FACTOR, n), (REFRESH, n)]
        for n in range(N):
            want += [(CORE, n), (APPLY, n), (REFRESH, n)]
        assert [(k, m) for k, m, _ in phases] == want
        # each pass waits for the one before it
        for (k0, m0, c0), (k1, m1, c1) in zip(phases, phases[1:]):
            assert all(t["wait"] == c0 for t in mine if t["done"] == c1)
        # tasks of a pass cover it exactly
        for k, m, c in phases:
            ts = sorted((t for t in mine if t["done"] == c), key=lambda t: t["begin"])
            total = {FACTOR: nnz, CORE: nnz, REFRESH: dims[m], APPLY: 1}[k]
            assert ts[0]["begin"] == 0 and ts[-1]["end"] == total
            assert all(a["end"] == b["begin"] for a, b in zip(ts, ts[1:]))
            if k in (FACTOR, CORE):
                assert all(t["end"] - t["begin"] <= chunk for t in ts)
            if k == CORE:
                assert sorted(t["slot"] for t in ts) == list(range(len(ts)))
                ncore = len(ts)
            if k == APPLY:
                assert ts[0]["nslots"] == ncore


def test_refresh_and_loss_plans(sft):
    ref = plan(sft, 1, 1024, 16)
    assert all(t["wait"] == -1 and t["kind"] == REFRESH for t in ref)
    for p, (dims, R, nnz) in enumerate(SHAPES):
        for n, I in enumerate(dims):
            ts = sorted((t for t in ref if t["prob"] == p and t["mode"] == n), key=lambda t: t["begin"])
            assert ts[0]["begin"] == 0 and ts[-1]["end"] == I
    loss = plan(sft, 2, 1024, 16)
    for p, (dims, R, nnz) in enumerate(SHAPES):
        parts = [t for t in loss if t["prob"] == p and t["kind"] == LOSS]
        fin = [t for t in loss if t["prob"] == p and t["kind"] == LOSSFIN]
        assert len(fin) == 1 and fin[0]["nslots"] == len(parts) == -(-nnz // 1024)
        assert fin[0]["wait"] == parts[0]["done"]
        assert loss.index(fin[0]) > max(loss.index(t) for t in parts)


def test_big_problems_start_first(sft):
    """The list is the problems with R <= 16, then those with R = 32 (one
    persistent kernel each); within each part the list scheduler hands out
    the problem with the most work first."""
    tasks = plan(sft, 0, 256, 4)
    small = [p for p, (_, R, _) in enumerate(SHAPES) if R <= 16]
    cls = [0 if t["prob"] in small else 1 for t in tasks]
    assert cls == sorted(cls)  # the R <= 16 part, then the R = 32 part
    assert tasks[0]["prob"] == 0  # 20k nonzeros at R = 8: most work of the small ranks
    assert tasks[cls.index(1)]["prob"] == 2  # the only R = 32 problem


@pytest.mark.parametrize("shape", [((10, 10), 12, 100), ((10,) * 9, 8, 100), ((10, 10), 8, 0)])
def test_invalid_problems_are_rejected(sft, shape):
    recs = sft.batch_problem_records([shape])
    lib = sft.load()
    assert lib.sft_batch_plan(1, recs, 0, 1024, 8, None, 0) == -1
    assert lib.sft_batch_workspace_bytes(1, recs, 1024) == 0


def test_chunk_below_minimum_is_rejected(sft):
    recs = sft.batch_problem_records(SHAPES)
    lib = sft.load()
    assert lib.sft_batch_plan(len(SHAPES), recs, 0, 128, 8, None, 0) == -1
    assert lib.sft_batch_workspace_bytes(len(SHAPES), recs, 128) == 0
    assert lib.sft_batch_workspace_bytes(len(SHAPES), recs, 256) > 0
