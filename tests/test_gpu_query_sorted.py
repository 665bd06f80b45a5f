"""Region histograms (Eq. 2) with the corners bucketed by row first
(ihist_query_sorted): word for word against the oracle's Eq. 2 and against
ihist_query, for every group width, bin counts that leave a partial last
group, rectangles touching the frame's top and left edges (absent corners),
out-of-range rectangles (zero rows, status latched) and reused scratch."""
import numpy as np
import pytest

import oracle
from paper_1711_01919_gb300 import ihist, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1711_01919_gb300 import build as cuda_build
    cuda_build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def edge_rects(h, w):
    """Rectangles on the frame's edges (corners at row or column -1 are
    absent from Eq. 2); only those inside the frame are kept."""
    r = np.array([[0, 0, w - 1, h - 1], [0, 0, 0, 0], [w - 1, h - 1, w - 1, h - 1], [0, 3, 5, h - 1],
                  [2, 0, w - 1, 1], [0, h - 1, w - 1, h - 1], [w - 1, 0, w - 1, h - 1]], dtype=np.int32)
    ok = (r[:, 0] <= r[:, 2]) & (r[:, 2] < w) & (r[:, 1] <= r[:, 3]) & (r[:, 3] < h)
    return r[ok]


@pytest.mark.parametrize("h,w,nbins,n,bpp", [(37, 131, 37, 777, 0), (37, 131, 37, 777, 4), (37, 131, 37, 777, 16),
                                             (480, 640, 32, 1000, 8), (64, 300, 3, 5000, 4), (1, 1, 1, 10, 0),
                                             (300, 20000, 12, 3000, 16)])
def test_sorted_query_matches_oracle_and_plain_query(h, w, nbins, n, bpp):
    img = synth.uniform_frame(h * 3 + w + nbins, h, w)
    rects = np.concatenate([edge_rects(h, w), synth.rects(h + w + n, n, h, w)])
    ref = oracle.query(oracle.integral_histogram(img, nbins), rects)
    with ihist.Plan(h, w, nbins) as plan:
        out = plan.compute(torch.from_numpy(img).cuda())
        d_rects = torch.from_numpy(rects).cuda()
        work = torch.empty((plan.query_work_bytes(len(rects), bpp),), dtype=torch.uint8, device="cuda")
        for _ in range(2):  # the scratch is reused as the previous call left it
            got = plan.query_sorted(out, d_rects, work=work, bins_per_pass=bpp)
            assert plan.status() == ihist.IHIST_OK
            g = got.cpu().numpy().view(np.uint32)
            assert np.array_equal(g, ref), "%d words differ" % int((g != ref).sum())
        assert torch.equal(got, plan.query(out, d_rects))


def test_sorted_query_bad_rects_give_zero_rows_and_status():
    h, w, nbins = 50, 70, 8
    img = synth.uniform_frame(9, h, w)
    rects = np.array([[0, 0, 10, 10], [5, 5, 4, 9], [-1, 0, 3, 3], [0, 0, w, 3], [0, 0, 3, h], [3, 3, 3, 3]],
                     dtype=np.int32)
    ref = oracle.query(oracle.integral_histogram(img, nbins), rects)
    ref[1:5] = 0
    with ihist.Plan(h, w, nbins) as plan:
        out = plan.compute(torch.from_numpy(img).cuda())
        got = plan.query_sorted(out, torch.from_numpy(rects).cuda())
        assert plan.status() == ihist.IHIST_ERR_BAD_RECT
        assert np.array_equal(got.cpu().numpy().view(np.uint32), ref)
        assert plan.status() == ihist.IHIST_OK


def test_sorted_query_argument_checks():
    with ihist.Plan(16, 16, 4, ihist.IHIST_PIXEL_MAJOR) as plan:
        out = plan.compute(torch.zeros((16, 16), dtype=torch.uint8, device="cuda"))
        with pytest.raises(ihist.IhistError) as e:
            plan.query_sorted(out, torch.zeros((3, 4), dtype=torch.int32, device="cuda"))
        assert e.value.code == ihist.IHIST_ERR_UNSUPPORTED
    with ihist.Plan(16, 16, 4) as plan:
        out = plan.compute(torch.zeros((16, 16), dtype=torch.uint8, device="cuda"))
        rects = torch.zeros((100, 4), dtype=torch.int32, device="cuda")
        res = torch.empty((100, 4), dtype=torch.int32, device="cuda")
        need = plan.query_work_bytes(100)
        work = torch.empty((need,), dtype=torch.uint8, device="cuda")
        for args in ((res.data_ptr(), 0, work.data_ptr(), need - 1), (res.data_ptr(), 5, work.data_ptr(), need),
                     (res.data_ptr(), 0, work.data_ptr() + 16, need)):
            with pytest.raises(ihist.IhistError) as e:
                ihist.ihist_query_sorted(plan.handle, out.data_ptr(), rects.data_ptr(), 100, *args)
            assert e.value.code == ihist.IHIST_ERR_INVALID_ARG
        ihist.ihist_query_sorted(plan.handle, out.data_ptr(), rects.data_ptr(), 0, res.data_ptr(), 0, 0, 0)
        assert plan.query_work_bytes(100, 5) == 0
