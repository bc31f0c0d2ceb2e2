"""The serving loop's scheduler on the host (pg_serve_simulate: the same
scheduler code as pg_serve_start, with simulated work and no GPU).

Checked from the event log: an insertion runs on a worker beside the
query groups dispatched before it (they search the version they started
on) and ends before every later request starts; query groups hold
consecutive requests of one shape, never more than max_batch queries; with
several workers groups overlap, with one they never do; the scratch of the
groups in flight never exceeds the budget, and a group that can never fit
is refused while the rest still run."""
import numpy as np
import pytest

import paper_2410_01231_gb300 as pg


def plan(seed, count=120, p_insert=0.08, shapes=3, max_rows=40):
    rs = np.random.default_rng(seed)
    kind = (rs.random(count) < p_insert).astype(np.int32)
    rows = rs.integers(1, max_rows + 1, size=count).astype(np.int32)
    shape = rs.integers(0, shapes, size=count).astype(np.int32)
    return kind, rows, shape


def overlaps(a0, a1, b0, b1):
    return a0 < b1 and b0 < a1


@pytest.mark.parametrize("seed,slots", [(0, 4), (1, 2), (2, 1), (3, 8)])
def test_insertions_publish_before_later_requests(seed, slots):
    kind, rows, shape = plan(seed)
    r = pg.serve_simulate(kind, rows, shape, slots=slots, max_batch=64, work_us=300)
    start, end = r["start"], r["end"]
    assert (start >= 0).all() and (end > start).all()
    for t in np.flatnonzero(kind == 1):
        assert 0 <= r["slot"][t] < slots
        # nothing submitted later starts before it has published
        assert (start[t + 1:] > end[t]).all(), t
        if slots == 1:
            assert (end[:t] < start[t]).all(), t
    # each query group searched the version left by the insertions submitted
    # before it, wherever its worker started
    before = np.cumsum(kind) - kind
    q = kind == 0
    assert (r["version"][q] == before[q]).all()
    assert (r["version"][kind == 1] == before[kind == 1] + 1).all()
    st = r["stats"]
    assert st["requests"] == len(kind)
    assert st["queries"] == rows[kind == 0].sum() and st["inserted"] == rows[kind == 1].sum()
    assert st["max_in_flight"] <= slots


@pytest.mark.parametrize("seed", [4, 5])
def test_groups_merge_consecutive_requests_of_one_shape(seed):
    kind, rows, shape = plan(seed, shapes=2, max_rows=20)
    r = pg.serve_simulate(kind, rows, shape, slots=3, max_batch=50, work_us=200)
    group = r["group"]
    for g in np.unique(group):
        members = np.flatnonzero(group == g)
        assert (np.diff(members) == 1).all(), members
        if kind[members[0]] == 1:
            assert len(members) == 1
            continue
        assert (kind[members] == 0).all()
        assert len(set(shape[members])) == 1
        assert rows[members].sum() <= 50
        # merging is greedy: the request after the group did not fit or differs
        nxt = members[-1] + 1
        if nxt < len(kind) and kind[nxt] == 0 and shape[nxt] == shape[members[0]]:
            assert rows[members].sum() + rows[nxt] > 50
    assert r["stats"]["batches"] == len(np.unique(group))


def test_workers_overlap_and_one_worker_serialises():
    count = 16
    kind = np.zeros(count, np.int32)
    rows = np.full(count, 4, np.int32)
    shape = np.arange(count, dtype=np.int32)  # nothing merges
    r4 = pg.serve_simulate(kind, rows, shape, slots=4, work_us=3000)
    pairs = [(i, j) for i in range(count) for j in range(i + 1, count)
             if overlaps(r4["start"][i], r4["end"][i], r4["start"][j], r4["end"][j])]
    assert pairs and r4["stats"]["max_in_flight"] >= 2
    assert len(set(r4["slot"])) > 1
    r1 = pg.serve_simulate(kind, rows, shape, slots=1, work_us=500)
    order = np.argsort(r1["start"])
    assert (r1["end"][order][:-1] < r1["start"][order][1:]).all()
    assert r1["stats"]["max_in_flight"] == 1 and set(r1["slot"]) == {0}


def test_budget_bounds_the_scratch_in_flight():
    count = 40
    rs = np.random.default_rng(9)
    kind = np.zeros(count, np.int32)
    rows = rs.integers(1, 9, size=count).astype(np.int32)
    shape = np.arange(count, dtype=np.int32)
    rows[7] = 30  # 30 x 100 bytes can never fit in 1,000
    r = pg.serve_simulate(kind, rows, shape, slots=8, budget_bytes=1000, work_us=1500,
                          bytes_per_row=100)
    start, end = r["start"], r["end"]
    assert start[7] == -1 and end[7] == -1  # refused, nothing ran
    ran = np.flatnonzero(start >= 0)
    assert len(ran) == count - 1
    for i in ran:
        live = [j for j in ran if start[j] <= start[i] < end[j]]
        assert rows[live].sum() * 100 <= 1000, (i, live)
    assert r["stats"]["requests"] == count
    assert r["stats"]["admission_waits"] > 0


def test_simulation_rejects_bad_arguments():
    with pytest.raises(pg.PGError):
        pg.serve_simulate([0], [1], [0], slots=0)
    with pytest.raises(pg.PGError):
        pg.serve_simulate([2], [1], [0])
    with pytest.raises(pg.PGError):
        pg.serve_simulate([0], [0], [0])


def test_insertion_overlaps_the_groups_before_it():
    # three long query groups of distinct shapes, then an insertion: with
    # four workers it starts while they still run, and the query after it
    # waits for its end
    kind = np.array([0, 0, 0, 1, 0], np.int32)
    rows = np.array([64, 64, 64, 4, 4], np.int32)
    shape = np.array([0, 1, 2, 0, 0], np.int32)
    r = pg.serve_simulate(kind, rows, shape, slots=4, max_batch=64, work_us=4000)
    start, end = r["start"], r["end"]
    assert any(overlaps(start[i], end[i], start[3], end[3]) for i in range(3))
    assert start[4] > end[3]
    assert r["stats"]["max_in_flight"] >= 2
