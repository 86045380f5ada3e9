"""Host model of the backward rasterizer's record pipeline (no GPU): one
producer fills a ring of NS stages, each consumer warp queues the indices of
its live records, processes them 32 at a time (carrying items across tiles),
and releases a stage once all of the stage's items are processed, at the latest
before the wait that reuses the stage's slot; at a tile's first stage it first
processes the items of the tile before the previous one (the pixel factors
are kept for two tiles), and at the end the queue's last items. The model
follows the kernel's rules step by step on random per-stage item counts
(dense, sparse and empty footprints, tiles of one or many stages) and checks
what the kernel relies on: every warp always makes progress (no wait for a slot
that a consumer still holds), every stage is released exactly once by every
consumer, every item is processed exactly once, only while its stage is held
and while its tile's pixel factors are kept, and the queue never holds more
than a round's remainder plus one stage."""
import numpy as np
import pytest

BATCHES = (64, 128, 256)  # records per stage of the compiled backward variants


def _simulate(ns, tiles, warps, rng, BATCH=128):
    """tiles: list of per-tile stage counts; returns the largest queue fill."""
    # the stream of stages: (tile index, first stage of its tile?, per-warp live item counts)
    stages = []
    for t, n_st in enumerate(tiles):
        for j in range(n_st):
            cnt = [int(rng.choice([0, rng.integers(0, 8), rng.integers(0, BATCH + 1)]))
                   for _ in range(warps)]
            stages.append((t, j == 0, cnt))
    total = len(stages)
    released = [[False] * total for _ in range(warps)]  # by warp, by stage
    filled = [False] * total
    # producer: stage k may be filled once every warp released stage k - ns
    produced = 0

    def produce():
        nonlocal produced
        while produced < total and (produced < ns or
                                    all(released[w][produced - ns] for w in range(warps))):
            filled[produced] = True
            produced += 1

    state = []
    for w in range(warps):
        state.append(dict(k=0, qhead=0, qtail=0, qend={}, krel=0, items=[], done=False,
                          tile=-1, qmark={0: 0, 1: 0}))
    max_fill = 0
    processed = [set() for _ in range(warps)]

    def round_(w):
        st = state[w]
        n = min(st["qtail"] - st["qhead"], 32)
        for i in range(st["qhead"], st["qhead"] + n):
            stage, item = st["items"][i]
            assert not released[w][stage], "item read after its stage was released"
            assert (stage, item) not in processed[w]
            assert st["tile"] - stages[stage][0] <= 1, "item read after its factors were replaced"
            processed[w].add((stage, item))
        st["qhead"] += n

    def release(w, last):
        st = state[w]
        while st["krel"] <= last and st["qend"][st["krel"]] <= st["qhead"]:
            assert not released[w][st["krel"]]
            released[w][st["krel"]] = True
            st["krel"] += 1

    produce()
    steps = 0
    while not all(s["done"] for s in state):
        progressed = False
        for w in range(warps):
            st = state[w]
            if st["done"]:
                continue
            k = st["k"]
            if k == total:
                while st["qtail"] > st["qhead"]:  # the queue's last items
                    round_(w)
                release(w, total - 1)  # (the kernel leaves these unreleased: the producer is done)
                st["done"] = True
                progressed = True
                continue
            if k >= ns and st["krel"] + ns <= k:
                # the wait reuses the slot of stage k - ns: process its items first
                while st["qhead"] < st["qend"][k - ns]:
                    round_(w)
                release(w, k - 1)
                progressed = True
            if not filled[k]:
                continue  # waits for the producer
            tile, first, cnt = stages[k]
            if first:
                if st["tile"] >= 0:
                    st["qmark"][st["tile"] & 1] = st["qtail"]
                while st["qhead"] < st["qmark"][tile & 1]:  # the tile before the previous one
                    round_(w)
                st["tile"] = tile  # its pixel factors replace those of tile - 2
            for i in range(cnt[w]):
                st["items"].append((k, i))
            st["qtail"] += cnt[w]
            st["qend"][k] = st["qtail"]
            max_fill = max(max_fill, st["qtail"] - st["qhead"])
            while st["qtail"] - st["qhead"] >= 32:
                round_(w)
            release(w, k)
            st["k"] = k + 1
            progressed = True
        produce()
        steps += 1
        assert progressed or all(s["done"] for s in state), "no warp can make progress"
        assert steps < 100000
    for w in range(warps):
        assert all(released[w]), "a stage was never released"
        assert len(processed[w]) == sum(c[w] for _, _, c in stages)
    return max_fill


@pytest.mark.parametrize("ns", [2, 3, 4])
@pytest.mark.parametrize("batch", BATCHES)
def test_release_protocol_progresses_and_releases_every_stage(ns, batch):
    rng = np.random.default_rng(ns * 1000 + batch)
    worst = 0
    for _ in range(60):
        tiles = [int(rng.integers(1, 6)) for _ in range(int(rng.integers(1, 12)))]
        worst = max(worst, _simulate(ns, tiles, warps=4, rng=rng, BATCH=batch))
    assert worst <= 31 + batch


def test_queue_capacity_in_the_kernel_covers_the_bound():
    """The kernel's queue (a ring of BwdQueue<BATCH>::kLen entries) holds the
    model's bound for every records-per-stage count, and the kernel asserts it
    at compile time; the stage count fits the queue entries' two bits."""
    import re
    from pathlib import Path
    src = (Path(__file__).resolve().parents[1] / "paper_2505_05643_gb300" / "csrc" /
           "ug_render.cu").read_text()
    m = re.search(r"kLen = BATCH <= (\d+) \? (\d+) : (\d+);", src)
    cut, small, large = (int(x) for x in m.groups())
    for batch in BATCHES:
        assert (small if batch <= cut else large) >= 31 + batch
    assert "static_assert(kLen >= 31 + BATCH" in src
    ns = int(re.search(r"constexpr int kBwdStages = (\d+);", src).group(1))
    assert 2 <= ns <= 4
    for v_ns, v_batch in re.findall(r"bwd_launch<TILE, \d, CUT, (\d), (\d+),", src):
        assert 2 <= int(v_ns) <= 4 and int(v_batch) in BATCHES
