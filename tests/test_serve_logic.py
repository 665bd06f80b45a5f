"""Serving loop logic on the CPU (fake executor): admission by HBM footprint,
LRU eviction of unpinned histograms, continuous batching, query pinning."""
import numpy as np

from paper_1711_01919_gb300 import serve


class Clock:
    def __init__(self, step=1e-4):
        self.t, self.step = 0.0, step

    def __call__(self):
        self.t += self.step
        return self.t


def frames(n, h=10, w=10, b=4, dt=0.0):
    return [serve.FrameRequest(i, i * dt, h, w, b) for i in range(n)]


def test_continuous_batching_groups_arrivals():
    ex = serve.FakeExecutor(frame_latency=1e-3)
    srv = serve.Server(ex, budget_bytes=1 << 30)
    done = srv.run(frames(10), Clock())
    assert len(done) == 10 and all(d.status == "ok" for d in done)
    kinds = [l for l in ex.launches if l[0] == "frames"]
    assert kinds[0][1] == list(range(10))  # all arrived together -> one launch


def test_plain_mode_launches_one_frame_each():
    ex = serve.FakeExecutor()
    srv = serve.Server(ex, budget_bytes=1 << 30, mode="plain")
    srv.run(frames(5), Clock())
    assert [l[1] for l in ex.launches] == [[0], [1], [2], [3], [4]]


def test_admission_waits_for_budget_and_evicts_lru():
    nb = serve.hist_bytes(10, 10, 4)
    ex = serve.FakeExecutor(frame_latency=1e-3)
    srv = serve.Server(ex, budget_bytes=3 * nb, max_batch=2)
    done = srv.run(frames(8, dt=1e-3), Clock(2e-4))
    assert sum(d.status == "ok" for d in done) == 8
    assert srv.store.used <= 3 * nb
    assert srv.store.evicted == 5
    assert srv.store.resident() == [5, 6, 7]


def test_oversized_frame_rejected():
    ex = serve.FakeExecutor()
    srv = serve.Server(ex, budget_bytes=100)
    done = srv.run(frames(2), Clock())
    assert all(d.status == "rejected" for d in done)


def test_unsupported_shapes_are_rejected_not_launched():
    reqs = [serve.FrameRequest(0, 0.0, 10, 10, 4), serve.FrameRequest(1, 0.0, 10, 70000, 4),
            serve.FrameRequest(2, 0.0, 10, 10, 300), serve.FrameRequest(3, 0.0, 0, 10, 4),
            serve.FrameRequest(4, 0.0, 10, 10, 0), serve.FrameRequest(5, 0.0, 10, 8192, 4),
            serve.FrameRequest(6, 0.0, 3, 20000, 4), serve.FrameRequest(7, 0.0, 70000, 10, 4)]
    ex = serve.FakeExecutor()
    srv = serve.Server(ex, budget_bytes=1 << 30)
    done = {d.rid: d.status for d in srv.run(reqs, Clock())}
    assert done == {0: "ok", 1: "rejected", 2: "rejected", 3: "rejected", 4: "rejected", 5: "ok", 6: "ok",
                    7: "rejected"}
    launched = [rid for l in ex.launches if l[0] == "frames" for rid in l[1]]
    assert sorted(launched) == [0, 5, 6]


def test_query_pins_its_target_until_answered():
    nb = serve.hist_bytes(10, 10, 4)
    ex = serve.FakeExecutor(frame_latency=1e-4, query_latency=5e-3)
    srv = serve.Server(ex, budget_bytes=2 * nb, max_batch=1, seed=0)
    reqs = frames(1) + [serve.QueryRequest(100, 1e-3, np.zeros((3, 4), np.int32))] + \
        [serve.FrameRequest(1 + i, 2e-3 + i * 1e-4, 10, 10, 4) for i in range(3)]
    evicted = []
    ex.release = lambda rid, payload: evicted.append(rid)
    done = srv.run(reqs, Clock(1e-4))
    q = [d for d in done if d.kind == "query"][0]
    assert q.status == "ok" and q.target == 0
    # frame 0 is held by the slow query, so the later frames evict each other instead
    assert evicted == [1, 2]
    assert 0 in srv.store.resident() and 3 in srv.store.resident()


def test_query_without_resident_histogram_is_rejected():
    ex = serve.FakeExecutor()
    srv = serve.Server(ex, budget_bytes=1 << 20)
    done = srv.run([serve.QueryRequest(0, 0.0, np.zeros((1, 4), np.int32))], Clock())
    assert done[0].status == "rejected"


def test_workload_mix():
    reqs = serve.serving_workload(7, 0.2, rects_per_query=10)
    nf = sum(isinstance(r, serve.FrameRequest) for r in reqs)
    nq = len(reqs) - nf
    assert 320 < nf < 480 and 20 < nq < 60
    assert all(a.t_arrival <= b.t_arrival for a, b in zip(reqs, reqs[1:]))


def test_report_percentiles():
    ex = serve.FakeExecutor(frame_latency=2e-3)
    srv = serve.Server(ex, budget_bytes=1 << 30)
    srv.run(frames(20, dt=1e-4), Clock(1e-4))
    rep = srv.report(1.0)
    assert rep["frame"]["completed"] == 20
    assert rep["frame"]["p50_ms"] <= rep["frame"]["p99_ms"] <= rep["frame"]["max_ms"]


def test_short_queues_launch_frames_one_by_one():
    ex = serve.FakeExecutor(frame_latency=1e-3)
    srv = serve.Server(ex, budget_bytes=1 << 30, min_batch=4)
    srv.run(frames(3), Clock())
    assert [l[1] for l in ex.launches] == [[0], [1], [2]]
    ex = serve.FakeExecutor(frame_latency=1e-3)
    srv = serve.Server(ex, budget_bytes=1 << 30, min_batch=4)
    srv.run(frames(4), Clock())
    assert [l[1] for l in ex.launches] == [[0, 1, 2, 3]]
    assert srv.report(1.0)["launch_sizes"] == {"4": 1}


def test_query_targets_only_finished_histograms():
    # frame 0 is still computing when the query arrives: no target yet -> rejected;
    # frame 1 finished before the second query -> that one is served on it
    ex = serve.FakeExecutor(frame_latency=5e-3)
    srv = serve.Server(ex, budget_bytes=1 << 30, seed=1)
    reqs = [serve.FrameRequest(0, 0.0, 10, 10, 4), serve.QueryRequest(10, 1e-3, np.zeros((1, 4), np.int32)),
            serve.QueryRequest(11, 2e-2, np.zeros((1, 4), np.int32))]
    done = {d.rid: d for d in srv.run(reqs, Clock(1e-4))}
    assert done[10].status == "rejected"
    assert done[11].status == "ok" and done[11].target == 0


def test_search_requests_are_held_and_answered_like_queries():
    nb = serve.hist_bytes(10, 10, 4)
    ex = serve.FakeExecutor(frame_latency=1e-4, query_latency=2e-3)
    srv = serve.Server(ex, budget_bytes=10 * nb, seed=0)
    reqs = frames(2) + [serve.SearchRequest(50, 1e-3, 0, 0, 4, 4, 2)]
    done = {d.rid: d for d in srv.run(reqs, Clock(1e-4))}
    assert done[50].kind == "search" and done[50].status == "ok" and done[50].target in (0, 1)
    assert ("search", 50, done[50].target) in ex.launches
    assert srv.report(1.0)["search"]["completed"] == 1


def test_search_workload_patches_sit_on_the_grid_inside_the_smallest_frame():
    reqs = serve.serving_workload(3, 0.5, rects_per_query=4, search_rate=100.0, search_win=(64, 64), search_stride=8)
    ss = [r for r in reqs if isinstance(r, serve.SearchRequest)]
    assert 20 < len(ss) < 90
    for r in ss:
        assert r.y % 8 == 0 and r.x % 8 == 0 and r.y + 64 <= 240 and r.x + 64 <= 320


def test_decode_best():
    assert serve.decode_best(0, 10) is None
    v = (4096 << 32) | (0xffffffff - 23)
    assert serve.decode_best(v, 10) == (4096, 2, 3)


class _Ev:
    def synchronize(self):
        pass


class _Rows:
    """A result that views a slot's host buffer (clone copies it)."""

    def __init__(self, buf):
        self.buf = buf

    def clone(self):
        return _Rows(list(self.buf))


def test_query_slot_reuse_keeps_results_the_server_has_not_taken():
    ex = object.__new__(serve.GpuExecutor)  # only the slot bookkeeping, no GPU
    ex.keep_results = True
    ex.qslots = [{"free": None, "owner": None, "buf": [0]}, {"free": None, "owner": None, "buf": [0]}]
    ex.next_qslot = 0
    handles = []
    for value in (11, 22, 33):  # the third request reuses the first one's slot
        slot = ex._take_qslot()
        slot["buf"][0] = value  # the request's rows land in the slot's host buffer
        h = {"result": _Rows(slot["buf"]), "slot": slot}
        slot["owner"] = h
        slot["free"] = _Ev()
        handles.append(h)
    assert [h["result"].buf[0] for h in handles] == [11, 22, 33]  # the first result was copied out
    ex.finish(handles[1])
    slot = ex._take_qslot()  # the second slot: its result was taken, nothing to copy
    assert slot["owner"] is None and handles[1]["result"].buf is slot["buf"]


def test_store_evictable_bytes_track_every_change():
    # the running count of evictable bytes (ready, unpinned) and the set of
    # evictable entries equal a full recount after any sequence of reserve /
    # ready / pin / unpin / eviction
    rng = np.random.default_rng(5)
    store = serve.HistStore(budget_bytes := 10_000)
    evicted = []
    live = []
    for step in range(3000):
        op = rng.integers(4)
        if op == 0:
            rid = step
            if store.reserve(rid, int(rng.integers(100, 900)), lambda k, p: evicted.append(k)):
                live.append(rid)
        elif op == 1 and live:
            store.set_ready(live[int(rng.integers(len(live)))], payload=("h",))
        elif op == 2 and store.ready_ids():
            store.pin(store.ready_ids()[int(rng.integers(len(store.ready_ids())))])
        elif op == 3:
            pinned = [k for k, e in store.entries.items() if e[1] > 0]
            if pinned:
                store.unpin(pinned[int(rng.integers(len(pinned)))])
        live = [k for k in live if k in store.entries]
        want = sum(e[0] for e in store.entries.values() if e[1] == 0 and e[2])
        assert store.evictable == want, step
        assert set(store.lru) == {k for k, e in store.entries.items() if e[1] == 0 and e[2]}, step
        assert store.used == sum(e[0] for e in store.entries.values()) <= budget_bytes
    assert evicted


def test_busy_gpu_holds_partial_batches_until_launches_drain():
    # a burst of 100 frames, 16 per shared launch: while two launches are in
    # flight the rest wait to fill whole launches, so only the last is partial
    ex = serve.FakeExecutor(frame_latency=2e-3)
    srv = serve.Server(ex, budget_bytes=1 << 30, max_batch=16, min_batch=4)
    done = srv.run(frames(100), Clock())
    assert len(done) == 100 and all(d.status == "ok" for d in done)
    sizes = [len(l[1]) for l in ex.launches if l[0] == "frames"]
    assert sizes == [16] * 6 + [4]
    # spaced arrivals (5 ms apart, each frame done in 2 ms) go out alone at once
    ex = serve.FakeExecutor(frame_latency=2e-3)
    srv = serve.Server(ex, budget_bytes=1 << 30, max_batch=16, min_batch=4)
    done = srv.run(frames(10, dt=5e-3), Clock())
    assert [len(l[1]) for l in ex.launches if l[0] == "frames"] == [1] * 10
    assert max(d.t_launch - d.t_arrival for d in done) < 1e-3
