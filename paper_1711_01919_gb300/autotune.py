"""Autotuner: pick the scan kernel's tiling (and, if allowed, the layout) by
measurement, cached per device and frame shape.

Search space (ihist_tune_t fields): rows per band R, bins per CTA G (4 or
8), 128-column chunks per warp m, bin groups per CTA (and, for batches,
warps per CTA).  Each candidate is
timed with CUDA events on a seeded uniform frame (median of a few launches
after warm-up); candidates the library rejects (shared memory, registers)
are skipped.  For a batch the search covers R and G of the batched launch.
``choose_layout`` (one frame) and ``tune_batch_layout`` (a batch) time
compute plus a query load for bin-major, pixel-major and (bin counts that
are multiples of 4) quad-major output and keep the fastest, for callers
that accept any.

Results are cached in a JSON file (``IHIST_TUNE_CACHE`` or
``~/.cache/ihist_tune.json``) keyed by device name and shape.  The timing
function is injectable, so the search and cache logic run on the CPU in the
tests.
"""
from __future__ import annotations

import json
import os
import statistics
import threading

from . import ihist, synth

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("IHIST_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "ihist_tune.json")


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(path, cache):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def plan_candidates(h: int, w: int, nbins: int):
    """Tilings worth timing for one frame shape (the default first)."""
    nchunks = -(-w // 128)
    out = [{}]
    for G in (4, 8):
        for m in (1, 2, 4, 8):
            wpg = -(-nchunks // m)
            if wpg > 16 or (m > 1 and wpg < 2):
                continue  # needs more than 16 warps, or leaves a single warp per group
            ngroups = -(-nbins // G)
            for gpc in sorted({1, min(ngroups, max(1, 16 // wpg))}):
                for R in (0, 16, 24, 32, 48, 64):
                    if R and R > h:
                        continue
                    t = {"bins_per_cta": G, "chunks_per_warp": m, "groups_per_cta": gpc}
                    if R:
                        t["rows_per_band"] = R
                    out.append(t)
    return out


def batch_candidates(shapes=(), tables=False):
    """Batch launch shapes to time (the default first); 16-bin groups too
    when some frame is pixel-major (their longer pieces of pixel records)."""
    gs = (4, 8, 16) if any(s[3] == ihist.IHIST_PIXEL_MAJOR for s in shapes) and not tables else (4, 8)
    return [{}] + [{"warps_per_cta": nw, "bins_per_cta": G, "rows_per_band": R}
                   for nw in (8, 16) for G in gs for R in (24, 32, 40, 48, 56)]


def _device_key():
    import torch
    return torch.cuda.get_device_name()


def time_plan(h, w, nbins, layout, tune, reps=5):
    """Median ms of ihist_compute with this tiling (raises IhistError if rejected)."""
    import torch
    frame = torch.from_numpy(synth.uniform_frame(12345, h, w)).cuda()
    with ihist.Plan(h, w, nbins, layout, tune=tune or None) as plan:
        out = plan.empty_output()
        for _ in range(2):
            plan.compute(frame, out)
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan.compute(frame, out)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        if plan.status() != ihist.IHIST_OK:
            raise RuntimeError("device status error while tuning")
    return statistics.median(ms)


def time_batch(shapes, tune, reps=3, tables=False, queries=0):
    """Median ms of one batched launch over frames of these (h, w, nbins,
    layout), plus one batched query launch of `queries` rectangles per frame;
    tables: every frame bins through a value -> bin table."""
    import torch
    frames = [torch.from_numpy(synth.uniform_frame(100 + i, h, w)).cuda() for i, (h, w, b, l) in enumerate(shapes)]
    tb = [[(v * s[2]) >> 8 for v in range(256)] for s in shapes] if tables else None
    rects = None
    if queries:
        import numpy as np
        rects = torch.from_numpy(np.stack([synth.rects(200 + i, queries, h, w)
                                           for i, (h, w, b, l) in enumerate(shapes)])).cuda()  # [frames][n][4]
    with ihist.Batch(frames, [s[2] for s in shapes], [s[3] for s in shapes], tune=tune or None, tables=tb) as batch:
        qout = (torch.empty((queries * sum(s[2] for s in shapes),), dtype=torch.int32, device="cuda")
                if queries else None)

        def step():
            batch.compute()
            if queries:
                batch.query_all(rects, out=qout)

        for _ in range(2):
            step()
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            step()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        if batch.status() != ihist.IHIST_OK:
            raise RuntimeError("device status error while tuning")
    return statistics.median(ms)


def _search(cands, timer):
    best, best_ms, tried = None, float("inf"), []
    for t in cands:
        try:
            ms = timer(t)
        except ihist.IhistError:
            continue
        tried.append((ms, t))
        if ms < best_ms:
            best, best_ms = t, ms
    if best is None:
        raise RuntimeError("no tiling candidate ran")
    return best, best_ms, tried


def tune_plan(h, w, nbins, layout=ihist.IHIST_BIN_MAJOR, timer=None, device=None, use_cache=True):
    """Best tiling for ihist_plan_tuned on this device and shape."""
    device = device or _device_key()
    key = "plan|%s|%dx%dx%d|%d" % (device, h, w, nbins, layout)
    path = cache_path()
    with _lock:
        cache = _load_cache(path) if use_cache else {}
        if key in cache:
            return cache[key]["tune"]
    timer = timer or (lambda t: time_plan(h, w, nbins, layout, t))
    best, ms, _ = _search(plan_candidates(h, w, nbins), timer)
    if use_cache:
        with _lock:
            cache = _load_cache(path)
            cache[key] = {"tune": best, "ms": ms}
            _store_cache(path, cache)
    return best


def tune_batch(shapes, timer=None, device=None, use_cache=True, tables=False):
    """Best (warps_per_cta, bins_per_cta, rows_per_band) for a batch of (h, w,
    nbins, layout) frames; tables: a table batch (other bin structures)."""
    device = device or _device_key()
    sig = ",".join("%dx%dx%dx%d" % tuple(s) for s in sorted(set(tuple(s) for s in shapes)))
    key = "batch|%s|%d|%s%s" % (device, len(shapes), sig, "|tables" if tables else "")
    path = cache_path()
    with _lock:
        cache = _load_cache(path) if use_cache else {}
        if key in cache:
            return cache[key]["tune"]
    timer = timer or (lambda t: time_batch(shapes, t, tables=tables))
    best, ms, _ = _search(batch_candidates(shapes, tables), timer)
    if use_cache:
        with _lock:
            cache = _load_cache(path)
            cache[key] = {"tune": best, "ms": ms}
            _store_cache(path, cache)
    return best


def layouts_for(nbins_list):
    """Layouts every frame can take: bin-major, pixel-major, and quad-major
    when every bin count is a multiple of 4."""
    out = [ihist.IHIST_BIN_MAJOR, ihist.IHIST_PIXEL_MAJOR]
    if all(b % 4 == 0 for b in nbins_list):
        out.append(ihist.IHIST_QUAD_MAJOR)
    return out


def tune_batch_layout(shapes, queries_per_frame=0, timer=None, device=None, use_cache=True):
    """Layout and launch shape of a batch of (h, w, nbins) frames that are
    computed once and then queried `queries_per_frame` times each.  For each
    layout (the same for every frame) the launch shape comes from
    tune_batch; the layout whose batched launch plus batched queries take
    less time wins.  timer(shapes, tune, queries) -> ms replaces the
    measurement (tests).  Returns (layout, tune, {layout: ms})."""
    device = device or _device_key()
    times, tunes = {}, {}
    for layout in layouts_for([b for (h, w, b) in shapes]):
        sh = [(h, w, b, layout) for (h, w, b) in shapes]
        shape_timer = None if timer is None else (lambda t, sh=sh: timer(sh, t, 0))
        try:
            tunes[layout] = tune_batch(sh, timer=shape_timer, device=device, use_cache=use_cache)
        except RuntimeError:
            continue  # no launch shape runs this layout
        times[layout] = (timer(sh, tunes[layout], queries_per_frame) if timer is not None
                         else time_batch(sh, tunes[layout], queries=queries_per_frame))
    if not times:
        raise RuntimeError("no layout ran")
    layout = min(times, key=times.get)
    return layout, tunes[layout], times


def choose_layout(h, w, nbins, queries_per_frame=1000, timer=None):
    """The layout (bin-major, pixel-major or, when nbins % 4 == 0,
    quad-major) for a frame that is computed once and then queried
    `queries_per_frame` times: whichever takes less time in total."""
    if timer is None:
        import torch

        def timer(layout):
            frame = torch.from_numpy(synth.uniform_frame(77, h, w)).cuda()
            rects = torch.from_numpy(synth.rects(78, max(1, queries_per_frame), h, w)).cuda()
            with ihist.Plan(h, w, nbins, layout) as plan:
                out = plan.empty_output()
                for _ in range(2):
                    plan.compute(frame, out)
                    if queries_per_frame:
                        plan.query(out, rects)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                for _ in range(3):
                    plan.compute(frame, out)
                    if queries_per_frame:
                        plan.query(out, rects)
                b.record()
                torch.cuda.synchronize()
                return a.elapsed_time(b) / 3
    times = {layout: timer(layout) for layout in layouts_for([nbins])}
    return min(times, key=times.get)
