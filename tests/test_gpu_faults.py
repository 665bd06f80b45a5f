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
    tune = {"rows_per_band": 8, "fault_skip_band": skip_band, "timeout_us": 20000}
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


def test_plan_recovers_after_timeout_launch():
    # a plan whose previous launch timed out runs the next launch cleanly
    # (flags carry the launch epoch, so stale ones are ignored)
    h, w, nbins = 40, 300, 4
    img = synth.uniform_frame(2, h, w)
    ref = oracle.integral_histogram(img, nbins)
    lib = ihist.load()
    import ctypes
    t = ihist._tune_struct({"rows_per_band": 4, "fault_skip_band": 3, "timeout_us": 10000})
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
