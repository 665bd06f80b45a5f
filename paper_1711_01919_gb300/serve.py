"""Continuous-batching server for integral histograms.

Requests arrive over time (Sec. 4.4's image sequences, served):

* ``FrameRequest``  a uint8 frame and a bin count.  Its integral histogram
  (Eq. 1) is computed on the GPU and then stays resident in device memory
  for follow-up queries.  A frame is admitted only when its histogram
  (h * w * nbins * 4 bytes) fits the HBM budget, after evicting the least
  recently used resident histograms that no pending query holds.
* ``QueryRequest``  rectangles whose region histograms (Eq. 2) are wanted
  from a resident histogram.  The server picks the target among the
  resident frames whose histogram is complete when the query is admitted
  (seeded, uniform) and holds it until the query is answered; the rows are
  copied back to the host.
* ``SearchRequest``  a patch of a resident frame to find again: its region
  histogram becomes the target of a sliding-window search over the frame,
  and the best window (score, i, j) comes back (tracking, Sec. 1).  Targets
  are chosen and held like a query's.

The loop is continuous batching, not a queue: every iteration it admits
what has arrived and fits, puts all admitted frames that are not yet
running into ONE batched launch (``ihist_batch_upload_compute``: uploads on
a copy stream, compute as soon as they land), so frames that arrive while
a batch runs join the next one and their uploads overlap the running
compute.  Queries whose histogram is ready are launched as they come.
Latency is taken from GPU event timestamps against a reference event
recorded at the start, so it does not depend on how often the host polls.

When fewer than ``min_batch`` (8) frames are waiting, the batched server
launches them one by one (``ihist_compute`` with a per-shape plan): a short
queue gains nothing from a shared launch, whose first frame would wait for
the others (at 2000 frames/s a threshold of 4 still sent 4-6 bursts per 10 s
through shared launches, and their frames set the p99).  Queries run on a stream of their own, so they do not
queue behind frames that do not concern them.

``mode="plain"`` serves every frame with its own ``ihist_compute`` launch
(no batching) -- the baseline the batched form is compared with.

The GPU work sits behind ``GpuExecutor``; the admission, eviction and
batching logic runs unchanged on a ``FakeExecutor`` in the CPU tests.
"""
from __future__ import annotations

import collections
import dataclasses
import gc
import heapq
import time

import numpy as np

from . import synth


@dataclasses.dataclass
class FrameRequest:
    rid: int
    t_arrival: float          # seconds from the start of the run
    h: int
    w: int
    nbins: int
    frame: object = None      # host uint8 [h][w] (page-locked torch tensor on the GPU path)


@dataclasses.dataclass
class QueryRequest:
    rid: int
    t_arrival: float
    rects: object             # int32 [n][4] host array
    target: int = -1          # frame rid, chosen at admission


@dataclasses.dataclass
class SearchRequest:
    """Where in a resident frame does this patch's histogram fit best?  The
    target is the histogram of the win_h x win_w patch at (y, x) of the
    chosen frame (a region query); the answer is the best window of the
    sliding-window search over that frame (score, i, j) -- the tracking use
    of the integral histogram (Sec. 1)."""
    rid: int
    t_arrival: float
    y: int
    x: int
    win_h: int
    win_w: int
    stride: int
    target: int = -1          # frame rid, chosen at admission


@dataclasses.dataclass
class Done:
    rid: int
    kind: str                 # "frame", "query" or "search"
    t_arrival: float
    t_done: float
    status: str = "ok"        # ok | rejected
    target: int = -1
    t_launch: float = -1.0    # host time of the launch that served it
    launch_n: int = 0         # frames: how many frames shared that launch (1 = a per-frame launch)


def hist_bytes(h: int, w: int, nbins: int) -> int:
    return h * w * nbins * 4


def frame_supported(h: int, w: int, nbins: int) -> bool:
    """Shapes both executors take: the library's frame limits (1 <= h, w <=
    65535, h * w < 2^32, 1 <= nbins <= 256)."""
    return 1 <= h <= 65535 and 1 <= w <= 65535 and h * w < (1 << 32) and 1 <= nbins <= 256


class HistStore:
    """Resident histograms under a byte budget; LRU over entries not pinned.
    The entries that may be evicted (ready, not pinned) are also kept in an
    LRU-ordered dict of their own, with their total bytes, so admission and
    eviction cost O(1) however many histograms are resident or waiting (a
    full store at saturation holds hundreds of admitted frames not yet
    computed)."""

    def __init__(self, budget: int):
        self.budget = budget
        self.used = 0
        self.evictable = 0
        self.entries = collections.OrderedDict()  # rid -> [bytes, pins, ready, payload], LRU order
        self.lru = collections.OrderedDict()      # the evictable rids, LRU order
        self.evicted = 0

    def can_fit(self, nbytes: int) -> bool:
        return self.used - self.evictable + nbytes <= self.budget

    def _add_evictable(self, rid, e):
        self.lru[rid] = None
        self.evictable += e[0]

    def _drop_evictable(self, rid, e):
        if self.lru.pop(rid, 0) is None:
            self.evictable -= e[0]

    def reserve(self, rid: int, nbytes: int, evict_cb=None) -> bool:
        """Make room (evicting the least recently used ready, unpinned
        entries) and reserve nbytes."""
        if not self.can_fit(nbytes):
            return False
        while self.used + nbytes > self.budget and self.lru:
            k, _ = self.lru.popitem(last=False)
            e = self.entries.pop(k)
            self.used -= e[0]
            self.evictable -= e[0]
            self.evicted += 1
            if evict_cb:
                evict_cb(k, e[3])
        if self.used + nbytes > self.budget:
            return False
        self.entries[rid] = [nbytes, 0, False, None]
        self.used += nbytes
        return True

    def set_ready(self, rid: int, payload=None):
        e = self.entries.get(rid)
        if e is not None:
            if not e[2] and e[1] == 0:
                self._add_evictable(rid, e)
            e[2] = True
            if payload is not None:
                e[3] = payload

    def touch(self, rid: int):
        if rid in self.entries:
            self.entries.move_to_end(rid)
            if rid in self.lru:
                self.lru.move_to_end(rid)

    def pin(self, rid: int):
        e = self.entries[rid]
        if e[1] == 0 and e[2]:
            self._drop_evictable(rid, e)
        e[1] += 1
        self.touch(rid)

    def unpin(self, rid: int):
        e = self.entries.get(rid)
        if e is not None:
            e[1] -= 1
            if e[1] == 0 and e[2]:
                self._add_evictable(rid, e)

    def resident(self):
        return list(self.entries.keys())

    def ready_ids(self):
        """Resident histograms whose computation has finished."""
        return [rid for rid, e in self.entries.items() if e[2]]

    def payload(self, rid: int):
        return self.entries[rid][3]

    def ready(self, rid: int) -> bool:
        return rid in self.entries and self.entries[rid][2]


class FakeExecutor:
    """CPU stand-in for the GPU: work finishes `latency` seconds after launch."""

    def __init__(self, frame_latency=1e-4, query_latency=5e-5):
        self.frame_latency, self.query_latency = frame_latency, query_latency
        self.launches = []

    def now(self):
        return self._now

    def launch_frames(self, reqs, t):
        self.launches.append(("frames", [r.rid for r in reqs]))
        return {"t": t + self.frame_latency, "payloads": {r.rid: ("hist", r.rid) for r in reqs}}

    def launch_query(self, q, payload, t):
        self.launches.append(("query", q.rid, q.target))
        return {"t": t + self.query_latency, "result": ("rows", q.rid, payload)}

    def launch_search(self, q, payload, t):
        self.launches.append(("search", q.rid, q.target))
        return {"t": t + self.query_latency, "result": ("best", q.rid, payload)}

    def poll(self, handle, t):
        return t >= handle["t"]

    def done_time(self, handle):
        return handle["t"]

    def release(self, rid, payload):
        pass

    def finish(self, handle):
        pass


class Server:
    """Continuous-batching request loop over an executor (see module doc)."""

    def __init__(self, executor, budget_bytes: int, max_batch: int = 64, mode: str = "batched",
                 seed: int = 4, min_batch: int = 8, keep_results: bool = True, hold: int = 2):
        self.ex = executor
        self.store = HistStore(budget_bytes)
        self.max_batch = max_batch if mode == "batched" else 1
        # fewer waiting frames than this go out one launch each: a short
        # queue gains nothing from a shared launch, and the first frame of a
        # batch would wait for the others
        self.min_batch = min_batch if mode == "batched" else 1
        # frame launches in flight from which waiting frames are held back to
        # fill a whole shared launch (batched mode only)
        self.hold = hold if mode == "batched" else 1 << 30
        self.mode = mode
        self.rng = np.random.default_rng(seed)
        self.done = []
        self.results = {}
        self.keep_results = keep_results  # copy each query's rows out of the executor's reusable buffers
        self.batch_sizes = collections.Counter()
        self.host_ms = {"frames": [], "query": [], "search": []}  # host time spent issuing each launch

    def run(self, requests, clock, max_wall: float = 600.0):
        """Serve `requests` (sorted by t_arrival).  clock() returns seconds since
        the start; the loop ends when every request has completed.  Python's
        cyclic garbage collector is paused meanwhile: its full passes over the
        request objects take milliseconds and would show as latency."""
        was_enabled = gc.isenabled()
        gc.disable()
        try:
            return self._run(requests, clock, max_wall)
        finally:
            if was_enabled:
                gc.enable()

    def _run(self, requests, clock, max_wall):
        pending = collections.deque(requests)
        admit_frames = collections.deque()   # arrived, waiting for budget
        ready_frames = []                    # admitted, not launched
        waiting_queries = collections.deque()
        inflight = []                        # (handle, kind, payload)
        arrived_frames = {}
        t_start_wall = time.perf_counter()
        while pending or admit_frames or ready_frames or waiting_queries or inflight:
            if time.perf_counter() - t_start_wall > max_wall:
                raise RuntimeError("serving loop exceeded %.0f s" % max_wall)
            t = clock()
            # 1. arrivals
            while pending and pending[0].t_arrival <= t:
                r = pending.popleft()
                if isinstance(r, FrameRequest):
                    admit_frames.append(r)
                    arrived_frames[r.rid] = r
                else:
                    live = self.store.ready_ids()
                    if not live:
                        self.done.append(Done(r.rid, _kind(r), r.t_arrival, t, "rejected"))
                        continue
                    r.target = int(live[int(self.rng.integers(len(live)))])
                    self.store.pin(r.target)
                    waiting_queries.append(r)
            # 2. admission by HBM footprint (FIFO)
            while admit_frames:
                r = admit_frames[0]
                nb = hist_bytes(r.h, r.w, r.nbins)
                if nb > self.store.budget or not frame_supported(r.h, r.w, r.nbins):
                    admit_frames.popleft()
                    self.done.append(Done(r.rid, "frame", r.t_arrival, t, "rejected"))
                    continue
                if not self.store.reserve(r.rid, nb, self.ex.release):
                    break
                admit_frames.popleft()
                ready_frames.append(r)
            # 3. queries whose histogram is ready (first: they are short and wait on nothing)
            for _ in range(len(waiting_queries)):
                q = waiting_queries.popleft()
                if self.store.ready(q.target):
                    t_call = clock()
                    launch = self.ex.launch_search if isinstance(q, SearchRequest) else self.ex.launch_query
                    h = launch(q, self.store.payload(q.target), t)
                    h["t_launch"] = clock()
                    self.host_ms[_kind(q)].append(1e3 * (h["t_launch"] - t_call))
                    inflight.append((h, _kind(q), q))
                else:
                    waiting_queries.append(q)
            # 4. frame launches (continuous batching).  While `hold` or more
            # frame launches are in flight the GPU has work queued, so admitted
            # frames wait to fill a whole shared launch; otherwise they go out
            # at once: one by one if fewer than min_batch wait, else together
            frame_launches = sum(1 for _, kind, _ in inflight if kind == "frames")
            while ready_frames:
                if frame_launches >= self.hold and len(ready_frames) < self.max_batch:
                    break
                take = self.max_batch if len(ready_frames) >= self.min_batch else 1
                batch, ready_frames = ready_frames[:take], ready_frames[take:]
                t_call = clock()
                h = self.ex.launch_frames(batch, t)
                h["t_launch"] = clock()
                self.host_ms["frames"].append(1e3 * (h["t_launch"] - t_call))
                self.batch_sizes[len(batch)] += 1
                inflight.append((h, "frames", batch))
                frame_launches += 1
                if len(batch) > 1:
                    break  # one shared launch per iteration; later arrivals join the next
            # 5. completions
            still = []
            for h, kind, obj in inflight:
                if self.ex.poll(h, clock()):
                    td = self.ex.done_time(h)
                    if kind == "frames":
                        for r in obj:
                            self.store.set_ready(r.rid, h["payloads"][r.rid])
                            self.store.touch(r.rid)
                            self.done.append(Done(r.rid, "frame", r.t_arrival, td, t_launch=h["t_launch"],
                                                  launch_n=len(obj)))
                    else:
                        self.store.unpin(obj.target)
                        self.store.touch(obj.target)
                        if self.keep_results:
                            r = h.get("result")
                            self.results[obj.rid] = r.clone() if hasattr(r, "clone") else r
                        self.ex.finish(h)  # the executor may now reuse the result's buffers
                        self.done.append(Done(obj.rid, kind, obj.t_arrival, td, target=obj.target,
                                              t_launch=h["t_launch"]))
                else:
                    still.append((h, kind, obj))
            inflight = still
        return self.done

    def report(self, wall_s: float):
        out = {"mode": self.mode, "evicted": self.store.evicted,
               "launch_sizes": {str(k): v for k, v in sorted(self.batch_sizes.items())},
               "host_issue_p50_ms": {k: float(np.percentile(v, 50)) if v else None for k, v in self.host_ms.items()}}
        for kind in ("frame", "query", "search"):
            ok = [d for d in self.done if d.kind == kind and d.status == "ok"]
            lat = np.array([d.t_done - d.t_arrival for d in ok]) * 1e3
            wait = np.array([d.t_launch - d.t_arrival for d in ok]) * 1e3  # host: arrival -> launched
            out[kind] = {
                "latencies_ms": lat,  # every completed request's latency (for pooling runs)
                "completed": len(ok),
                "rejected": sum(1 for d in self.done if d.kind == kind and d.status != "ok"),
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                "max_ms": float(lat.max()) if len(lat) else None,
                "launch_wait_p50_ms": float(np.percentile(wait, 50)) if len(wait) else None,
                "launch_wait_p99_ms": float(np.percentile(wait, 99)) if len(wait) else None,
                "per_s": len(ok) / wall_s if wall_s > 0 else None,
            }
        # frame latency by the path that served it: per-frame launches and
        # shared (batched) launches
        frames = [d for d in self.done if d.kind == "frame" and d.status == "ok"]
        by_path = {}
        for name, sel in (("solo", [d for d in frames if d.launch_n == 1]),
                          ("shared", [d for d in frames if d.launch_n > 1])):
            lat = np.array([d.t_done - d.t_arrival for d in sel]) * 1e3
            wait = np.array([d.t_launch - d.t_arrival for d in sel]) * 1e3
            by_path[name] = {"frames": len(sel),
                             "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                             "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                             "launch_wait_p99_ms": float(np.percentile(wait, 99)) if len(wait) else None}
        out["frame"]["by_path"] = by_path
        return out


def _kind(r) -> str:
    return "search" if isinstance(r, SearchRequest) else "query"


def decode_best(v: int, nx: int):
    """(score, i, j) of a packed best window (see ihist_window_search), or None."""
    v &= 0xffffffffffffffff
    if v == 0:
        return None
    idx = 0xffffffff - (v & 0xffffffff)
    return v >> 32, idx // nx, idx % nx


# ----------------------------------------------------------------- workload

def serving_workload(seed: int, duration_s: float, frame_rate: float = 2000.0, query_rate: float = 200.0,
                     rects_per_query: int = 10000, frame_pool=None, search_rate: float = 0.0,
                     search_win=(64, 64), search_stride: int = 8):
    """Poisson frame arrivals (mix of the uneven batch), Poisson query
    arrivals with `rects_per_query` random rectangles each, and Poisson
    search arrivals (a search_win patch of the chosen frame, searched for on
    a search_stride grid).  frame_pool: optional {(h, w): [frames]} of host
    frames to cycle through."""
    ft = synth.poisson_arrivals(seed, frame_rate, duration_s)
    qt = synth.poisson_arrivals(seed + 1, query_rate, duration_s)
    specs = synth.uneven_batch_specs(seed + 2, len(ft))
    reqs = []
    use = collections.Counter()
    for i, (t, (h, w, b, s)) in enumerate(zip(ft, specs)):
        fr = None
        if frame_pool is not None:
            pool = frame_pool[(h, w)]
            fr = pool[use[(h, w)] % len(pool)]
            use[(h, w)] += 1
        reqs.append(FrameRequest(i, float(t), h, w, b, fr))
    n0 = len(reqs)
    for j, t in enumerate(qt):
        # rectangles in the smallest resolution of the mix, valid in every frame
        reqs.append(QueryRequest(n0 + j, float(t), synth.rects(seed + 10 + j, rects_per_query, 240, 320)))
    if search_rate > 0:
        st = synth.poisson_arrivals(seed + 3, search_rate, duration_s)
        wh, ww = search_win
        # patch corners on the stride grid inside the smallest resolution of the mix
        corners = synth.splitmix64(seed + 4, 2 * len(st)).reshape(-1, 2)
        n1 = len(reqs)
        for k, t in enumerate(st):
            y = int(corners[k, 0] % np.uint64((240 - wh) // search_stride + 1)) * search_stride
            x = int(corners[k, 1] % np.uint64((320 - ww) // search_stride + 1)) * search_stride
            reqs.append(SearchRequest(n1 + k, float(t), y, x, wh, ww, search_stride))
    reqs.sort(key=lambda r: r.t_arrival)
    return reqs


# ----------------------------------------------------------------- the GPU

class GpuExecutor:
    """Runs the server's launches with libihist on one GPU.

    batched: a ring of four `nslots`-frame batch plans whose slots are
    sized for the largest frame of the mix; every launch of two or more
    frames rebinds the slots to the admitted frames (ihist_batch_set_io) and
    uploads them on the copy stream; a single frame takes the plain path.
    plain: one ihist_compute per frame with a plan per shape, its upload on
    the copy stream into one of two staging buffers.  Queries: rectangles
    up, Eq. 2 launch and rows back, all on a high-priority query stream.
    Output histograms come from torch's allocator on the compute stream the
    first time a shape is seen; evicted ones are kept per shape and reused.
    """

    def __init__(self, mode="batched", nslots=64, max_shape=(1080, 1920, 64), query_slots=8, max_rects=10000,
                 trace=False, keep_results=True):
        """trace: mark every launch with an NVTX range (frames / query, with
        sizes) so a profiler's timeline shows the serving loop's issue."""
        import torch

        from . import ihist
        self.torch, self.ih = torch, ihist
        self.mode = mode
        self.keep_results = keep_results  # the server reads query results (copy them before a slot is reused)
        self.free_outputs = {}  # (h, w, b) -> evicted output buffers for reuse
        self.trace = trace
        self.stream = torch.cuda.current_stream()
        self.copy = torch.cuda.Stream()
        self.qstream = torch.cuda.Stream(priority=-1)
        self.s = self.stream.cuda_stream
        h, w, b = max_shape
        self.plans = {}
        self.batches = []
        self.inputs = []
        self.inputs.append([torch.empty((h, w), dtype=torch.uint8, device="cuda") for _ in range(2)])
        if mode == "batched":
            # a ring of 4 batches: binding a batch waits (on the host) for its
            # previous descriptor copy, so with 4 the host can run that many
            # launches ahead of the GPU before it waits (2 measured host-bound
            # at saturation)
            for _ in range(4):
                ins = [torch.empty((h, w), dtype=torch.uint8, device="cuda") for _ in range(nslots)]
                outs = [torch.empty((b, h, w), dtype=torch.int32, device="cuda") for _ in range(1)] * nslots
                self.batches.append(ihist.Batch(ins, b, outs=outs))
                self.inputs.append(ins)
            del outs
        self.next_batch = 0
        self.next_input = 0
        self.read_done = [torch.cuda.Event() for _ in range(2)]
        self.upload_done = [torch.cuda.Event() for _ in range(2)]
        for e in self.read_done:
            e.record(self.stream)
        self.t0_event = torch.cuda.Event(enable_timing=True)
        self.t0_wall = 0.0
        # query slots, reused round robin: pinned and device buffers for the
        # rectangles and the rows, so that issuing a query allocates nothing
        self.max_rects = max_rects
        self.qslots = [self._new_qslot() for _ in range(query_slots)]
        self.next_qslot = 0

    def _new_qslot(self):
        torch = self.torch
        m = self.max_rects
        return {
            "h_rects": torch.empty((m, 4), dtype=torch.int32, pin_memory=True),
            "d_rects": torch.empty((m, 4), dtype=torch.int32, device="cuda"),
            "d_out": torch.empty((m * 256,), dtype=torch.int32, device="cuda"),
            "h_out": torch.empty((m * 256,), dtype=torch.int32, pin_memory=True),
            "d_best": torch.zeros((1,), dtype=torch.int64, device="cuda"),
            "h_best": torch.zeros((1,), dtype=torch.int64, pin_memory=True),
            "free": None,   # event: the slot's last rows have reached the host
            "owner": None,  # handle whose result the slot holds until the server takes it
        }

    def _take_qslot(self):
        """The next query slot, round robin over a fixed pool.  Its previous
        request's rows must be on the host (wait for its event, rarely
        needed) and, if the server has not taken that result yet, they are
        copied into the request's handle first, so reuse never changes a
        result the server will read."""
        slot = self.qslots[self.next_qslot]
        self.next_qslot = (self.next_qslot + 1) % len(self.qslots)
        if slot["free"] is not None:
            slot["free"].synchronize()
        owner = slot["owner"]
        if owner is not None and self.keep_results:
            owner["result"] = owner["result"].clone()
        slot["owner"] = None
        return slot

    def finish(self, handle):
        """The server has taken the handle's result: its query slot no longer
        holds a result anyone will read."""
        slot = handle.get("slot")
        if slot is not None and slot["owner"] is handle:
            slot["owner"] = None

    def warm(self, shapes):
        """Create the per-shape plans and run every kernel once before
        serving: plan creation allocates and synchronises the device, and a
        kernel's first launch loads its code, neither of which may happen
        inside the timed loop."""
        torch = self.torch
        shapes = list(shapes)
        for (h, w, b) in shapes:
            p = self._plan(h, w, b)
            out = torch.empty((b, h, w), dtype=torch.int32, device="cuda")
            p.compute(torch.zeros((h, w), dtype=torch.uint8, device="cuda"), out, stream=self.s)
            p.query(out, torch.zeros((1, 4), dtype=torch.int32, device="cuda"), stream=self.s)
        if self.mode == "batched" and shapes:
            for batch, ins in zip(self.batches, self.inputs[1:]):
                sel = shapes[:min(len(shapes), len(ins))]
                views = [ins[i].view(-1)[:h * w].view(h, w) for i, (h, w, b) in enumerate(sel)]
                outs = [torch.empty((b, h, w), dtype=torch.int32, device="cuda") for (h, w, b) in sel]
                batch.set_io(views, outs, nbins=[b for (h, w, b) in sel], layouts=[0] * len(sel), stream=self.s)
                batch.compute(stream=self.s)
        torch.cuda.synchronize()
        for p in self.plans.values():
            if p.status() != self.ih.IHIST_OK:
                raise RuntimeError("device status error while warming up")
        for batch in self.batches:
            if batch.status() != self.ih.IHIST_OK:
                raise RuntimeError("device status error while warming up a batch")

    def start(self):
        self.torch.cuda.synchronize()
        self.t0_event.record(self.stream)
        self.torch.cuda.synchronize()
        self.t0_wall = time.perf_counter()

    def clock(self):
        return time.perf_counter() - self.t0_wall

    def _plan(self, h, w, b):
        p = self.plans.get((h, w, b))
        if p is None:
            p = self.plans[(h, w, b)] = self.ih.Plan(h, w, b)
        return p

    def launch_frames(self, reqs, t):
        if self.trace:
            self.torch.cuda.nvtx.range_push("ihist frames n=%d" % len(reqs))
        try:
            return self._launch_frames(reqs, t)
        finally:
            if self.trace:
                self.torch.cuda.nvtx.range_pop()

    def _launch_frames(self, reqs, t):
        torch, ih = self.torch, self.ih
        outs = {r.rid: self._output(r.h, r.w, r.nbins) for r in reqs}
        ev = torch.cuda.Event(enable_timing=True)
        if self.mode == "batched" and len(reqs) > 1:
            b = self.batches[self.next_batch]
            ins = self.inputs[1 + self.next_batch]
            self.next_batch = (self.next_batch + 1) % len(self.batches)
            # bind the slots with raw pointers (rows packed at the frame's
            # width in each slot buffer): no tensor views on the issue path
            ih.ihist_batch_set_io(b.handle, [(r.h, r.w, r.nbins, 0, ins[i].data_ptr(), r.w, outs[r.rid].data_ptr())
                                             for i, r in enumerate(reqs)], self.s)
            ih.ihist_batch_upload_compute(b.handle, [r.frame.data_ptr() for r in reqs], self.s,
                                          self.copy.cuda_stream)
        else:
            (r,) = reqs
            k = self.next_input
            self.next_input ^= 1
            view = self.inputs[0][k].view(-1)[:r.h * r.w].view(r.h, r.w)
            # the upload into buffer k waits only for the compute that last read it
            self.copy.wait_event(self.read_done[k])
            with torch.cuda.stream(self.copy):
                view.copy_(r.frame, non_blocking=True)
                self.upload_done[k].record(self.copy)
            self.stream.wait_event(self.upload_done[k])
            # the plan's entry point with raw pointers (the shapes were checked at admission)
            ih.ihist_compute(self._plan(r.h, r.w, r.nbins).handle, view.data_ptr(), r.w, outs[r.rid].data_ptr(), self.s)
            self.read_done[k].record(self.stream)
        ev.record(self.stream)
        return {"ev": ev, "payloads": {r.rid: (outs[r.rid], r.h, r.w, r.nbins) for r in reqs}}

    def launch_query(self, q, payload, t):
        if self.trace:
            self.torch.cuda.nvtx.range_push("ihist query rects=%d" % len(q.rects))
        try:
            return self._launch_query(q, payload, t)
        finally:
            if self.trace:
                self.torch.cuda.nvtx.range_pop()

    def launch_search(self, q, payload, t):
        if self.trace:
            self.torch.cuda.nvtx.range_push("ihist search %dx%d/%d" % (q.win_h, q.win_w, q.stride))
        try:
            return self._launch_search(q, payload, t)
        finally:
            if self.trace:
                self.torch.cuda.nvtx.range_pop()

    def _launch_search(self, q, payload, t):
        # the target is the patch's own region histogram (Eq. 2), then the
        # search keeps only the best window; 8 bytes come back
        torch, ih = self.torch, self.ih
        hist, h, w, b = payload
        slot = self._take_qslot()
        slot["h_rects"].numpy()[0] = (q.x, q.y, q.x + q.win_w - 1, q.y + q.win_h - 1)
        qs = self.qstream.cuda_stream
        plan = self._plan(h, w, b)
        with torch.cuda.stream(self.qstream):
            slot["d_rects"][:1].copy_(slot["h_rects"][:1], non_blocking=True)
            ih.ihist_query(plan.handle, hist.data_ptr(), slot["d_rects"].data_ptr(), 1, slot["d_out"].data_ptr(), qs)
            ih.ihist_window_search(plan.handle, hist.data_ptr(), slot["d_out"].data_ptr(), q.win_h, q.win_w, q.stride,
                                   0, slot["d_best"].data_ptr(), qs)
            slot["h_best"].copy_(slot["d_best"], non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(self.qstream)
        slot["free"] = ev
        hist.record_stream(self.qstream)
        handle = {"ev": ev, "result": slot["h_best"], "slot": slot,
                  "nx": ih.window_grid(h, w, q.win_h, q.win_w, q.stride)[1]}
        slot["owner"] = handle
        return handle

    def _launch_query(self, q, payload, t):
        # the server launches a query only once its histogram is complete,
        # and keeps the histogram resident until the query is done
        torch, ih = self.torch, self.ih
        hist, h, w, b = payload
        n = len(q.rects)
        if n > self.max_rects:
            raise ValueError("query of %d rectangles exceeds the executor's %d" % (n, self.max_rects))
        slot = self._take_qslot()
        slot["h_rects"].numpy()[:n] = q.rects
        qs = self.qstream.cuda_stream
        d_rects, d_out, h_out = slot["d_rects"], slot["d_out"], slot["h_out"]
        with torch.cuda.stream(self.qstream):
            d_rects[:n].copy_(slot["h_rects"][:n], non_blocking=True)
            ih.ihist_query(self._plan(h, w, b).handle, hist.data_ptr(), d_rects.data_ptr(), n, d_out.data_ptr(), qs)
            h_out[:n * b].copy_(d_out[:n * b], non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(self.qstream)
        slot["free"] = ev
        hist.record_stream(self.qstream)
        handle = {"ev": ev, "result": h_out[:n * b].view(n, b), "slot": slot}
        slot["owner"] = handle
        return handle

    def poll(self, handle, t):
        return handle["ev"].query()

    def done_time(self, handle):
        return self.t0_event.elapsed_time(handle["ev"]) / 1e3

    def _output(self, h, w, b):
        """An output buffer for a (h, w, b) histogram: an evicted one of the
        same shape if there is one, else a new allocation.  Reusing evicted
        buffers keeps torch's allocator (whose cudaMalloc / cudaFree can
        stall the host) out of the serving loop once the shapes have been
        seen."""
        free = self.free_outputs.get((h, w, b))
        if free:
            return free.pop()
        return self.torch.empty((b, h, w), dtype=self.torch.int32, device="cuda")

    def release(self, rid, payload):
        # an evicted histogram has no pending query (queries pin their
        # targets) and its compute has completed, so its buffer can take the
        # next histogram of the same shape on the compute stream
        hist, h, w, b = payload
        self.free_outputs.setdefault((h, w, b), []).append(hist)

    def close(self):
        for b in self.batches:
            b.close()
        for p in self.plans.values():
            p.close()


def serve(mode="batched", duration_s=2.0, budget_gb=40.0, seed=None, frame_rate=2000.0, query_rate=200.0,
          rects_per_query=10000, pool_per_shape=8, saturate=False, trace=False, search_rate=50.0):
    """Run the serving workload on the GPU; returns the server's report."""
    import torch
    seed = synth.workload_seed(4) if seed is None else seed
    pool = {}
    for (w, h) in synth.BATCH_RESOLUTIONS:
        pool[(h, w)] = [torch.from_numpy(synth.uniform_frame(seed + 100 * k + w, h, w)).pin_memory()
                        for k in range(pool_per_shape)]
    reqs = serving_workload(seed, duration_s, frame_rate, query_rate, rects_per_query, pool, search_rate)
    if saturate:
        # the same requests, arriving 1000 times faster than the server can take them
        for r in reqs:
            r.t_arrival *= 1e-3
    ex = GpuExecutor(mode, nslots=128, max_rects=max(1, rects_per_query), trace=trace, keep_results=False)
    ex.warm(sorted({(r.h, r.w, r.nbins) for r in reqs if isinstance(r, FrameRequest)}))
    srv = Server(ex, int(budget_gb * (1 << 30)), max_batch=128, mode=mode, keep_results=False)
    ex.start()
    t0 = time.perf_counter()
    srv.run(reqs, ex.clock)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    rep = srv.report(wall)
    rep["wall_s"] = wall
    rep["requests"] = len(reqs)
    ex.close()
    return rep
