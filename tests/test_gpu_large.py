"""The 8192 x 8192, 128-bin workload (32 GiB of output) at full size, in the
launch configuration the bench uses.

Checks: sampled bin planes word for word against the oracle (each plane is
an independent run of Algorithm 1), and every one of the 128 planes against
the oracle's by SHA-256 digest (the planes computed in parallel on the host
cores); every word through the second-difference
property (Algorithm 1 solved for Q: the 2-D second difference of H is the
one-hot of the pixel's bin); the 2^20 region queries against the oracle's
Eq. 2 word for word on the sampled bins and by digest of each bin's column on
all 128 bins (bins from 64 up sit past element offset 2^32 of H), and
per-rectangle totals equal to the rectangle's area.
"""
import concurrent.futures as cf
import hashlib
import multiprocessing
import os

import numpy as np
import pytest

import oracle
import oracle_planes
from paper_1711_01919_gb300 import ihist, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

H = W = 8192
NBINS = 128
SAMPLE_PLANES = (0, 1, 37, 64, 101, 127)


@pytest.fixture(scope="module")
def big():
    from paper_1711_01919_gb300 import build as cuda_build
    cuda_build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 40 * (1 << 30):
        pytest.skip("needs 40 GiB of free device memory")
    seed = synth.workload_seed(5)
    img = synth.sinusoid_frame(seed, H, W)
    rects = synth.rects(seed + 1, 1 << 20, H, W)
    plan = ihist.Plan(H, W, NBINS, ihist.IHIST_BIN_MAJOR)
    d_img = torch.from_numpy(img).cuda()
    out = plan.compute(d_img)
    d_rects = torch.from_numpy(rects).cuda()
    q = plan.query(out, d_rects)
    st = plan.status()
    yield img, rects, d_img, out, d_rects, q, st, plan
    del out, q
    plan.close()
    torch.cuda.empty_cache()


def test_status_ok(big):
    assert big[6] == ihist.IHIST_OK


@pytest.mark.parametrize("k", SAMPLE_PLANES)
def test_sampled_plane_vs_oracle(big, k):
    img, _, _, out, _, _, _, _ = big
    ref = oracle.integral_histogram_plane(img, NBINS, k)
    got = out[k].cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ref), "plane %d: %d words differ" % (k, int((got != ref).sum()))


@pytest.fixture(scope="module")
def oracle_digests(big):
    """{bin: (plane digest, query-column digest)} of the oracle, all 128 bins.

    The oracle computes every plane (and Eq. 2 on it for every rectangle) in
    spawned host processes; a worker that dies breaks the pool with an error
    (no silent wait)."""
    img, rects = big[0], big[1]
    oracle.default()  # the oracle library exists before any worker loads it
    nproc = max(1, min(16, os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(nproc, mp_context=multiprocessing.get_context("spawn"),
                                initializer=oracle_planes.init, initargs=(img, rects)) as pool:
        pending = [pool.submit(oracle_planes.plane_digest, (NBINS, k)) for k in range(NBINS)]
        ref = {}
        for f in pending:
            k, dp, dq = f.result(timeout=1800)
            ref[k] = (dp, dq)
    return ref


def test_every_plane_vs_oracle_by_digest(big, oracle_digests):
    # all 128 planes (32 GiB): the GPU planes are copied back and hashed in
    # threads; equal SHA-256 digests per plane mean equal words.
    img, _, _, out, _, _, _, _ = big

    def gpu_digest(k):
        return k, hashlib.sha256(out[k].cpu().numpy()).hexdigest()

    with cf.ThreadPoolExecutor(8) as ex:
        got = dict(ex.map(gpu_digest, range(NBINS)))
    bad = [k for k in range(NBINS) if got[k] != oracle_digests[k][0]]
    if bad:
        k = bad[0]
        plane = out[k].cpu().numpy().view(np.uint32)
        want = oracle.integral_histogram_plane(img, NBINS, k)
        raise AssertionError("%d planes differ; plane %d: %d words" % (len(bad), k, int((plane != want).sum())))


def test_every_word_by_second_difference(big):
    _, _, d_img, out, _, _, _, _ = big
    binned = (d_img.to(torch.int32) * NBINS) >> 8
    for b0 in range(0, NBINS, 8):
        P = out[b0:b0 + 8]
        d2 = P.clone()
        d2[:, 1:, :] -= P[:, :-1, :]
        d2[:, :, 1:] -= P[:, :, :-1]
        d2[:, 1:, 1:] += P[:, :-1, :-1]
        onehot = (binned.unsqueeze(0) == torch.arange(b0, b0 + 8, device="cuda").view(8, 1, 1)).to(torch.int32)
        assert torch.equal(d2, onehot), "bins %d..%d" % (b0, b0 + 7)
        del d2, onehot


def test_bottom_row_and_right_column_sums(big):
    img, _, _, out, _, _, _, _ = big
    bottom = out[:, H - 1, :].to(torch.int64).sum(0).cpu().numpy()
    right = out[:, :, W - 1].to(torch.int64).sum(0).cpu().numpy()
    assert np.array_equal(bottom, H * np.arange(1, W + 1))
    assert np.array_equal(right, W * np.arange(1, H + 1))
    counts = np.bincount(((img.astype(np.int64) * NBINS) >> 8).ravel(), minlength=NBINS)
    assert np.array_equal(out[:, H - 1, W - 1].cpu().numpy().view(np.uint32), counts)


def test_queries(big):
    img, rects, _, out, d_rects, q, _, _ = big
    area = ((d_rects[:, 2] - d_rects[:, 0] + 1).to(torch.int64) * (d_rects[:, 3] - d_rects[:, 1] + 1))
    assert torch.equal(q.to(torch.int64).sum(1), area)
    for k in SAMPLE_PLANES:  # 64, 101 and 127 read H past element offset 2^32
        ref_plane = oracle.integral_histogram_plane(img, NBINS, k)
        ref_q = oracle.query(ref_plane[None], rects)[:, 0]
        got = q[:, k].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, ref_q), "bin %d" % k


def test_queries_every_bin_vs_oracle_by_digest(big, oracle_digests):
    q = big[5]
    bad = []
    for k in range(NBINS):
        col = np.ascontiguousarray(q[:, k].cpu().numpy().view(np.uint32))
        if hashlib.sha256(col).hexdigest() != oracle_digests[k][1]:
            bad.append(k)
    assert not bad, "query columns of %d bins differ from the oracle's Eq. 2, first bin %d" % (len(bad), bad[0])


@pytest.mark.parametrize("bpp", [0, 16])
def test_sorted_queries_equal_the_checked_queries(big, bpp):
    # the row-bucketed query on the same 2^20 rectangles equals the plain
    # query word for word (the plain one is checked against the oracle above)
    _, _, _, out, d_rects, q, _, plan = big
    got = plan.query_sorted(out, d_rects, bins_per_pass=bpp)
    assert plan.status() == ihist.IHIST_OK
    assert torch.equal(got, q)
    del got
