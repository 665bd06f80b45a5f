"""The bench's own workload at full size, in its launch configuration: the
64 frames of 1920x1080 (gradient + N(0, 20^2) noise) with 64 bins, one
batched scan launch over the 64 resident frames with the default batch
tiling, one query launch for the 64 x 1000 rectangles, the launch pair run
twice as in the bench's steps.

Checks: every frame's H and every frame's 1000 query rows against the
oracle's Algorithm 1 (Eq. 1) and Eq. 2 by SHA-256 digest (the oracle runs
in spawned worker processes on the host cores, each making its frame from
the seed), and frames 0 and 63 word for word."""
import concurrent.futures as cf
import hashlib
import multiprocessing
import os

import numpy as np
import pytest

import bench
import oracle
import oracle_planes
from paper_1711_01919_gb300 import ihist

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def oracle_digests():
    # the pool starts before this module's first GPU call
    nproc = max(1, min(16, (os.cpu_count() or 2) - 1))
    with cf.ProcessPoolExecutor(nproc, mp_context=multiprocessing.get_context("spawn")) as ex:
        return {f: (dh, dq) for f, dh, dq in ex.map(oracle_planes.bench_frame_digests, range(bench.NFRAMES))}


@pytest.fixture(scope="module")
def bench_run(oracle_digests):
    from paper_1711_01919_gb300 import build as cuda_build
    cuda_build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    frames = bench.make_frames(0)
    rects = bench.make_rects()
    d_frames = torch.from_numpy(frames).cuda()
    d_rects = torch.from_numpy(np.ascontiguousarray(
        np.broadcast_to(rects, (bench.NFRAMES,) + rects.shape))).cuda()
    outs = [torch.empty((bench.NBINS, bench.H, bench.W), dtype=torch.int32, device="cuda")
            for _ in range(bench.NFRAMES)]
    for o in outs:
        o.fill_(-1)
    q = torch.full((bench.NFRAMES * bench.NRECTS * bench.NBINS,), -1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    with ihist.Batch([d_frames[f] for f in range(bench.NFRAMES)], bench.NBINS, [0] * bench.NFRAMES,
                     outs=outs) as batch:
        for _ in range(2):
            ihist.ihist_batch_compute(batch.handle, s)
            ihist.ihist_batch_query_all(batch.handle, d_rects.data_ptr(), bench.NRECTS, q.data_ptr(), s)
        torch.cuda.synchronize()
        st = batch.status()
    yield frames, rects, outs, q, st
    del outs, q, d_frames
    torch.cuda.empty_cache()


def test_status_ok(bench_run):
    assert bench_run[4] == ihist.IHIST_OK


def test_every_frame_and_query_row_by_digest(bench_run, oracle_digests):
    _, _, outs, q, _ = bench_run
    rows = q.view(bench.NFRAMES, bench.NRECTS * bench.NBINS)

    def digests(f):
        h = outs[f].cpu().numpy().view(np.uint32)
        r = rows[f].cpu().numpy().view(np.uint32)
        return f, hashlib.sha256(np.ascontiguousarray(h)).hexdigest(), hashlib.sha256(np.ascontiguousarray(r)).hexdigest()

    with cf.ThreadPoolExecutor(8) as ex:
        got = {f: (dh, dq) for f, dh, dq in ex.map(digests, range(bench.NFRAMES))}
    bad_h = [f for f in range(bench.NFRAMES) if got[f][0] != oracle_digests[f][0]]
    bad_q = [f for f in range(bench.NFRAMES) if got[f][1] != oracle_digests[f][1]]
    assert not bad_h, "frames whose H differs from the oracle: %s" % bad_h
    assert not bad_q, "frames whose query rows differ from the oracle: %s" % bad_q


@pytest.mark.parametrize("f", [0, 63])
def test_frames_word_for_word(bench_run, f):
    frames, rects, outs, q, _ = bench_run
    ref = oracle.integral_histogram(frames[f], bench.NBINS)
    got = outs[f].cpu().numpy().view(np.uint32)
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        raise AssertionError("frame %d: %d words differ, first at %s" % (f, len(bad), tuple(bad[0])))
    rows = q.view(bench.NFRAMES, bench.NRECTS, bench.NBINS)[f].cpu().numpy().view(np.uint32)
    assert np.array_equal(rows, oracle.query(ref, rects))
