"""The allocation-free entry point against the oracle and the plan path.

ihist_compute_noalloc serves callers that cannot allocate device memory
(callbacks, allocator hooks, pools that must not grow): it runs the same
kernel with its carry scratch in a fixed array inside the library.  Each case
calls it twice in a row on different frames (the scratch keeps the previous
call's contents, so the second call checks that reuse is clean) and compares
every word with the oracle's Algorithm 1 (Eq. 1) and with ihist_plan +
ihist_compute.  The cases cover the entry point's own tiling choices: one,
two, four and eight 128-column chunks per warp (frames up to 16384 columns),
bands pushed past 64 rows by the scratch bound, and inputs whose row pitch
is larger than the width (aligned for the TMA path, odd for plain loads).
This file is collected last.
"""
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


def to_layout(ref, layout):
    """Bin-major oracle result in the requested layout (a transpose only)."""
    if layout == ihist.IHIST_QUAD_MAJOR:
        b, h, w = ref.shape
        return np.ascontiguousarray(ref.reshape(b // 4, 4, h, w).transpose(0, 2, 3, 1))
    return ref if layout == ihist.IHIST_BIN_MAJOR else np.ascontiguousarray(ref.transpose(1, 2, 0))


def device_frame(img, pitch_pad):
    h, w = img.shape
    if not pitch_pad:
        return torch.from_numpy(img).cuda()
    buf = torch.zeros(h * (w + pitch_pad), dtype=torch.uint8, device="cuda")
    view = buf.view(h, w + pitch_pad)[:, :w]
    view.copy_(torch.from_numpy(img))
    return view


def assert_same(got, ref, what):
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        i = tuple(bad[0])
        raise AssertionError("%s: %d words differ, first at %s: got %d want %d"
                             % (what, len(bad), i, got[i], ref[i]))


CASES = [
    (480, 640, 32, 0, 0), (300, 1000, 24, 1, 0), (1080, 1920, 64, 0, 0), (61, 333, 9, 0, 0), (1, 1, 1, 0, 0),
    (270, 480, 16, 2, 0), (61, 333, 12, 2, 0),
    # two, four and eight chunks per warp (16 warps at most)
    (120, 4096, 16, 0, 0), (64, 8192, 8, 0, 0), (32, 16384, 4, 0, 0), (40, 8192, 8, 2, 0),
    # 1024 columns, 256 bins: the 8 MiB bound raises the band height to 150 rows
    (900, 1024, 256, 0, 0),
    # row pitch larger than the width: 16-byte aligned (TMA) and odd (plain loads)
    (200, 640, 32, 0, 64), (77, 300, 16, 1, 37),
]


@pytest.mark.parametrize("h,w,nbins,layout,pitch_pad", CASES)
def test_noalloc_matches_oracle_and_plan_twice(h, w, nbins, layout, pitch_pad):
    s = torch.cuda.current_stream().cuda_stream
    with ihist.Plan(h, w, nbins, layout) as plan:
        for call in range(2):
            img = synth.uniform_frame(7000 + 13 * call + h + w, h, w) if call == 0 else \
                synth.gradient_frame(7100 + h + w, h, w)
            d_in = device_frame(img, pitch_pad)
            got = plan.empty_output()
            got.fill_(-1)
            st = ihist.ihist_compute_noalloc(h, w, nbins, layout, d_in.data_ptr(), d_in.stride(0),
                                             got.data_ptr(), s)
            assert st == ihist.IHIST_OK
            want = to_layout(oracle.integral_histogram(img, nbins), layout)
            assert_same(got.cpu().numpy().view(np.uint32).reshape(want.shape), want,
                        "call %d vs the oracle" % call)
            ref = plan.compute(d_in)
            assert plan.status() == ihist.IHIST_OK
            assert torch.equal(got, ref), "call %d differs from the plan path" % call


def test_noalloc_async_then_status():
    h, w, nbins = 200, 512, 16
    img = synth.uniform_frame(11, h, w)
    d_in = torch.from_numpy(img).cuda()
    with ihist.Plan(h, w, nbins) as plan:
        got = plan.empty_output()
        s = torch.cuda.current_stream().cuda_stream
        assert ihist.ihist_compute_noalloc(h, w, nbins, 0, d_in.data_ptr(), w, got.data_ptr(), s,
                                           wait=False) is None
        torch.cuda.synchronize()
        assert_same(got.cpu().numpy().view(np.uint32).reshape(nbins, h, w),
                    oracle.integral_histogram(img, nbins), "asynchronous call vs the oracle")
        assert torch.equal(got, plan.compute(d_in))


def test_noalloc_rejects_frames_beyond_the_scratch():
    d = torch.zeros((16,), dtype=torch.uint8, device="cuda")
    o = torch.zeros((16,), dtype=torch.int32, device="cuda")
    with pytest.raises(ihist.IhistError) as e:
        ihist.ihist_compute_noalloc(8192, 8192, 128, 0, d.data_ptr(), 8192, o.data_ptr())
    assert e.value.code == ihist.IHIST_ERR_UNSUPPORTED
    with pytest.raises(ihist.IhistError) as e:
        ihist.ihist_compute_noalloc(0, 8, 4, 0, d.data_ptr(), 8, o.data_ptr())
    assert e.value.code == ihist.IHIST_ERR_INVALID_ARG
