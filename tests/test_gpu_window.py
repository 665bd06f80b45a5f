"""Sliding-window histogram search on the GPU (Eq. 2 per window, histogram
intersection with a target) against the oracle, which counts every window's
pixels directly: exact uint32 equality, both layouts."""
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
    ihist.load()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [(1, 1, 4, 1, 1, 1), (20, 31, 8, 5, 7, 1), (33, 40, 16, 8, 8, 3), (16, 16, 4, 16, 16, 5),
         (9, 50, 32, 1, 1, 2), (30, 30, 3, 7, 4, 4), (64, 300, 64, 17, 33, 5), (100, 129, 256, 10, 10, 7),
         (240, 320, 100, 32, 48, 8)]


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("h,w,nbins,wh,ww,st", CASES)
def test_window_search_matches_oracle(layout, h, w, nbins, wh, ww, st):
    img = synth.uniform_frame(h * 131 + w + nbins, h, w)
    rng = np.random.default_rng(h + w)
    target = rng.integers(0, wh * ww // max(1, nbins // 4) + 2, size=nbins).astype(np.int32)
    exp = oracle.window_intersection(img, nbins, target.astype(np.uint32), wh, ww, st)
    with ihist.Plan(h, w, nbins, layout) as plan:
        hist = plan.compute(torch.from_numpy(img).cuda())
        got = plan.window_search(hist, torch.from_numpy(target).cuda(), wh, ww, st)
        best = plan.window_best(hist, torch.from_numpy(target).cuda(), wh, ww, st)
        assert plan.status() == ihist.IHIST_OK
    assert np.array_equal(got.cpu().numpy().view(np.uint32), exp)
    # numpy's argmax takes the first of equal maxima in row-major order, as the kernel must
    k = int(np.argmax(exp))
    assert best == (int(exp.max()), k // exp.shape[1], k % exp.shape[1])


def test_window_search_1080p_tracks_the_planted_patch():
    # the target is the histogram of one 64x64 patch; on a smooth frame with
    # noise that window scores its full area and the map agrees with the oracle
    h, w, nbins = 1080, 1920, 64
    img = synth.gradient_frame(9, h, w)
    y, x = 520, 1200
    target = np.bincount(((img[y:y + 64, x:x + 64].astype(np.int64) * nbins) >> 8).ravel(),
                         minlength=nbins).astype(np.int32)
    exp = oracle.window_intersection(img, nbins, target.astype(np.uint32), 64, 64, 8)
    for layout in (0, 1):
        with ihist.Plan(h, w, nbins, layout) as plan:
            hist = plan.compute(torch.from_numpy(img).cuda())
            got = plan.window_search(hist, torch.from_numpy(target).cuda(), 64, 64, 8).cpu().numpy().view(np.uint32)
            assert plan.status() == ihist.IHIST_OK
        assert np.array_equal(got, exp), layout
        assert got[y // 8, x // 8] == 64 * 64
        with ihist.Plan(h, w, nbins, layout) as plan:
            hist = plan.compute(torch.from_numpy(img).cuda())
            best = plan.window_best(hist, torch.from_numpy(target).cuda(), 64, 64, 8)
        k = int(np.argmax(exp))
        assert best == (64 * 64, k // exp.shape[1], k % exp.shape[1])


def test_window_search_rejects_bad_windows():
    with ihist.Plan(32, 32, 4) as plan:
        hist = plan.compute(torch.zeros((32, 32), dtype=torch.uint8, device="cuda"))
        t = torch.zeros(4, dtype=torch.int32, device="cuda")
        for (wh, ww, st) in [(33, 1, 1), (1, 33, 1), (0, 4, 1), (4, 4, 0)]:
            with pytest.raises(ihist.IhistError) as e:
                plan.window_search(hist, t, wh, ww, st)
            assert e.value.code == ihist.IHIST_ERR_INVALID_ARG
