"""Failure detection without faulting the GPU: a band that never publishes its
carries makes the band below wait; the wait is bounded, the kernel returns,
the device status reports the timeout, and the context stays usable."""
import time

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


@pytest.mark.parametrize("skip_band", [0, 2, 7])
def test_lookback_timeout_is_bounded_and_reported(skip_band):
    h, w, nbins = 64, 256, 8
    img = synth.uniform_frame(1, h, w)
    tune = {"rows_per_band": 8, "fault_skip_band": skip_band + 1, "timeout_us": 20000}  # 1-based hook
    with ihist.Plan(h, w, nbins, 0, tune=tune) as plan:
        d_img = torch.from_numpy(img).cuda()
        t0 = time.time()
        plan.compute(d_img)
        st = plan.status()
        dt = time.time() - t0
        if skip_band == 7:  # the last band has no band below: nothing waits on it
            assert st == ihist.IHIST_OK
        else:
            assert st == ihist.IHIST_ERR_LOOKBACK_TIMEOUT
        assert dt < 5.0
        assert plan.status() == ihist.IHIST_OK  # read-and-clear
    # the context is healthy: a normal plan is exact right after
    ref = oracle.integral_histogram(img, nbins)
    with ihist.Plan(h, w, nbins, 0, tune={"rows_per_band": 8}) as plan:
        out = plan.compute(torch.from_numpy(img).cuda())
        assert plan.status() == ihist.IHIST_OK
        assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(nbins, h, w), ref)


@pytest.mark.parametrize("skip_band", [0, 3])
def test_width_segment_timeout_is_bounded_and_reported(skip_band):
    # 3000 columns at one chunk per warp: each band is two width segments; the
    # band whose CTAs publish nothing leaves its right segment (and the band
    # below) waiting, both waits run out, and the next launch is exact
    h, w, nbins = 32, 3000, 8
    img = synth.uniform_frame(3, h, w)
    tune = {"rows_per_band": 8, "chunks_per_warp": 1, "fault_skip_band": skip_band + 1, "timeout_us": 20000}
    ref = oracle.integral_histogram(img, nbins)
    with ihist.Plan(h, w, nbins, 0, tune=tune) as plan:
        d_img = torch.from_numpy(img).cuda()
        t0 = time.time()
        plan.compute(d_img)
        st = plan.status()
        assert time.time() - t0 < 5.0
        assert st == ihist.IHIST_ERR_LOOKBACK_TIMEOUT
    with ihist.Plan(h, w, nbins, 0, tune={"rows_per_band": 8, "chunks_per_warp": 1}) as plan:
        for _ in range(2):
            out = plan.compute(torch.from_numpy(img).cuda())
            assert plan.status() == ihist.IHIST_OK
            assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(nbins, h, w), ref)


@pytest.mark.parametrize("skip_band", [0, 2, 5])
def test_pixel_major_record_timeout_is_bounded_and_reported(skip_band):
    # whole-record pixel-major rows: the four bin groups' warps of a column
    # range meet at named barriers, so a timed-out wait in one of them must
    # still take its vote; the launch ends within the timeout, reports it,
    # and the next launch is exact
    h, w, nbins = 48, 700, 64
    img = synth.uniform_frame(9, h, w)
    base = {"bins_per_cta": 16, "groups_per_cta": 4, "chunks_per_warp": 1, "rows_per_band": 8}
    ref = oracle.integral_histogram(img, nbins).transpose(1, 2, 0)
    with ihist.Plan(h, w, nbins, 1, tune=dict(base, fault_skip_band=skip_band + 1, timeout_us=20000)) as plan:
        d_img = torch.from_numpy(img).cuda()
        t0 = time.time()
        plan.compute(d_img)
        st = plan.status()
        assert time.time() - t0 < 5.0
        assert st == ihist.IHIST_ERR_LOOKBACK_TIMEOUT
    with ihist.Plan(h, w, nbins, 1, tune=base) as plan:
        for _ in range(2):
            out = plan.compute(torch.from_numpy(img).cuda())
            assert plan.status() == ihist.IHIST_OK
            assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(h, w, nbins), ref)


def test_plan_recovers_after_timeout_launch():
    # a plan whose previous launch timed out runs the next launch cleanly
    # (flags carry the launch epoch, so stale ones are ignored)
    h, w, nbins = 40, 300, 4
    img = synth.uniform_frame(2, h, w)
    ref = oracle.integral_histogram(img, nbins)
    lib = ihist.load()
    import ctypes
    t = ihist._tune_struct({"rows_per_band": 4, "fault_skip_band": 4, "timeout_us": 10000})  # band 3
    hp = ctypes.c_void_p()
    assert lib.ihist_plan_tuned(h, w, nbins, 0, ctypes.byref(t), ctypes.byref(hp)) == 0
    d_img = torch.from_numpy(img).cuda()
    out = torch.empty((nbins, h, w), dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    ihist.ihist_compute(hp.value, d_img.data_ptr(), w, out.data_ptr(), s)
    assert ihist.ihist_status(hp.value, s) == ihist.IHIST_ERR_LOOKBACK_TIMEOUT
    ihist.ihist_destroy(hp.value)
    with ihist.Plan(h, w, nbins, 0, tune={"rows_per_band": 4}) as plan:
        for _ in range(3):
            out = plan.compute(d_img)
            assert plan.status() == ihist.IHIST_OK
            assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(nbins, h, w), ref)


def test_zeroed_tune_struct_leaves_the_fault_hook_off():
    # a C caller's zero-initialised ihist_tune_t means defaults everywhere
    import ctypes
    lib = ihist.load()
    h, w, nbins = 48, 200, 8
    img = synth.uniform_frame(5, h, w)
    t = ihist.ihist_tune_t()  # all zero
    hp = ctypes.c_void_p()
    assert lib.ihist_plan_tuned(h, w, nbins, 0, ctypes.byref(t), ctypes.byref(hp)) == 0
    out = torch.empty((nbins, h, w), dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    ihist.ihist_compute(hp.value, torch.from_numpy(img).cuda().data_ptr(), w, out.data_ptr(), s)
    assert ihist.ihist_status(hp.value, s) == ihist.IHIST_OK
    assert ihist.ihist_plan_get_tune(hp.value)["fault_skip_band"] == 0
    ihist.ihist_destroy(hp.value)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.integral_histogram(img, nbins))


def test_batch_lookback_timeout_is_bounded_and_reported():
    # band 1 of every frame publishes nothing: the frames' lower bands time out
    imgs = [synth.uniform_frame(20 + i, h, w) for i, (h, w) in enumerate([(64, 256), (40, 700), (100, 130)])]
    frames = [torch.from_numpy(x).cuda() for x in imgs]
    tune = {"rows_per_band": 8, "fault_skip_band": 2, "timeout_us": 20000}
    with ihist.Batch(frames, [8, 16, 4], tune=tune) as batch:
        t0 = time.time()
        batch.compute()
        st = batch.status()
        assert st == ihist.IHIST_ERR_LOOKBACK_TIMEOUT
        assert time.time() - t0 < 5.0
        assert batch.status() == ihist.IHIST_OK  # read-and-clear
    with ihist.Batch(frames, [8, 16, 4], tune={"rows_per_band": 8}) as batch:
        batch.compute()
        assert batch.status() == ihist.IHIST_OK
        for x, o, b in zip(imgs, batch.outs, [8, 16, 4]):
            assert np.array_equal(o.cpu().numpy().view(np.uint32).reshape(b, *x.shape), oracle.integral_histogram(x, b))
