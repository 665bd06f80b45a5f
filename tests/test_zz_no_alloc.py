"""The allocation-free entry point gives the same words as the plan path.

ihist_compute_noalloc serves callers that cannot allocate device memory
(callbacks, allocator hooks, pools that must not grow): it runs the same
kernel with its carry scratch in a fixed array inside the library.  Each case
calls it twice in a row on different frames (the scratch keeps the previous
call's contents, so the second call checks that reuse is clean) and compares
every word with ihist_plan + ihist_compute.  This file is collected last.
"""
import numpy as np
import pytest

from paper_1711_01919_gb300 import ihist, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1711_01919_gb300 import build as cuda_build
    cuda_build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("h,w,nbins,layout", [(480, 640, 32, 0), (300, 1000, 24, 1), (1080, 1920, 64, 0),
                                              (61, 333, 9, 0), (1, 1, 1, 0), (270, 480, 16, 2), (61, 333, 12, 2)])
def test_noalloc_matches_plan_twice(h, w, nbins, layout):
    s = torch.cuda.current_stream().cuda_stream
    with ihist.Plan(h, w, nbins, layout) as plan:
        for call in range(2):
            img = synth.uniform_frame(7000 + 13 * call + h + w, h, w) if call == 0 else \
                synth.gradient_frame(7100 + h + w, h, w)
            d_in = torch.from_numpy(img).cuda()
            ref = plan.compute(d_in)
            assert plan.status() == ihist.IHIST_OK
            got = plan.empty_output()
            got.fill_(-1)
            st = ihist.ihist_compute_noalloc(h, w, nbins, layout, d_in.data_ptr(), d_in.stride(0),
                                             got.data_ptr(), s)
            assert st == ihist.IHIST_OK
            assert torch.equal(got, ref), "call %d differs" % call


def test_noalloc_async_then_status():
    h, w, nbins = 200, 512, 16
    img = synth.uniform_frame(11, h, w)
    d_in = torch.from_numpy(img).cuda()
    with ihist.Plan(h, w, nbins) as plan:
        ref = plan.compute(d_in)
        got = plan.empty_output()
        s = torch.cuda.current_stream().cuda_stream
        assert ihist.ihist_compute_noalloc(h, w, nbins, 0, d_in.data_ptr(), w, got.data_ptr(), s,
                                           wait=False) is None
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def test_noalloc_rejects_frames_beyond_the_scratch():
    d = torch.zeros((16,), dtype=torch.uint8, device="cuda")
    o = torch.zeros((16,), dtype=torch.int32, device="cuda")
    with pytest.raises(ihist.IhistError) as e:
        ihist.ihist_compute_noalloc(8192, 8192, 128, 0, d.data_ptr(), 8192, o.data_ptr())
    assert e.value.code == ihist.IHIST_ERR_UNSUPPORTED
    with pytest.raises(ihist.IhistError) as e:
        ihist.ihist_compute_noalloc(0, 8, 4, 0, d.data_ptr(), 8, o.data_ptr())
    assert e.value.code == ihist.IHIST_ERR_INVALID_ARG
