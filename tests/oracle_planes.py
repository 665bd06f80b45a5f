"""Worker side of the full-size plane comparison in test_gpu_large.py: each
worker process computes oracle bin planes of the 8192 x 8192 frame (one
independent run of Algorithm 1 per plane) and the oracle's Eq. 2 region
counts of that bin for every query rectangle, and returns SHA-256 digests of
both; also the per-frame digests of the bench's 1080p sequence for
test_gpu_bench_workload.py.  Imports nothing but numpy and the oracle at
module level (bench only inside that function), so spawned workers start
quickly."""
import hashlib

import numpy as np

import oracle

_IMG = None
_RECTS = None


def init(img, rects=None):
    global _IMG, _RECTS
    _IMG = img
    _RECTS = rects


def plane_digest(args):
    """(k, digest of oracle plane k, digest of its query column or None)."""
    nbins, k = args
    ref = oracle.integral_histogram_plane(_IMG, nbins, k)
    d_plane = hashlib.sha256(np.ascontiguousarray(ref)).hexdigest()
    d_query = None
    if _RECTS is not None:
        col = np.ascontiguousarray(oracle.query(ref[None], _RECTS)[:, 0], dtype=np.uint32)
        d_query = hashlib.sha256(col).hexdigest()
    return k, d_plane, d_query


def bench_frame_digests(f):
    """(f, digest of the oracle's H of frame f of the bench's 64-frame 1080p
    sequence, digest of its Eq. 2 rows for the bench's 1000 rectangles).
    The worker makes the frame and the rectangles itself from their seeds."""
    import bench
    img = bench.make_frame(0, f)
    ref = oracle.integral_histogram(img, bench.NBINS)
    rows = np.ascontiguousarray(oracle.query(ref, bench.make_rects()), dtype=np.uint32)
    return f, hashlib.sha256(np.ascontiguousarray(ref)).hexdigest(), hashlib.sha256(rows).hexdigest()
