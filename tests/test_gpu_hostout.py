"""Stand-alone mode: integral histograms written by the scan kernel straight
into page-locked host memory (the results-to-host half of the sequence
pipeline), bit-exact against the oracle, per frame and through the host
sequence pipeline."""
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


@pytest.mark.parametrize("h,w,nbins", [(37, 131, 16), (240, 320, 32), (1080, 1920, 8)])
def test_compute_into_pinned_host_memory(h, w, nbins):
    img = synth.uniform_frame(h * 3 + w, h, w)
    host = torch.zeros((nbins, h, w), dtype=torch.int32).pin_memory()
    with ihist.Plan(h, w, nbins) as plan:
        d = torch.from_numpy(img).cuda()
        s = torch.cuda.current_stream()
        ihist.ihist_compute(plan.handle, d.data_ptr(), w, host.data_ptr(), s.cuda_stream)
        s.synchronize()
        assert plan.status() == ihist.IHIST_OK
    assert np.array_equal(host.numpy().view(np.uint32), oracle.integral_histogram(img, nbins))


def test_sequence_with_outputs_in_host_memory():
    h, w, nbins, n = 120, 700, 16, 5
    frames = np.stack([synth.gradient_frame(50 + i, h, w) for i in range(n)])
    hf = torch.from_numpy(frames).pin_memory()
    outs = torch.zeros((n, nbins, h, w), dtype=torch.int32).pin_memory()  # every frame's H lands on the host
    slots = torch.empty((2, h, w), dtype=torch.uint8, device="cuda")
    copy = torch.cuda.Stream()
    s = torch.cuda.current_stream()
    with ihist.Plan(h, w, nbins) as plan:
        ihist.ihist_sequence_host(plan.handle, hf.data_ptr(), h * w, n, slots.data_ptr(), outs.data_ptr(), n,
                                  0, 0, 0, 0, s.cuda_stream, copy.cuda_stream)
        s.synchronize()
        assert plan.status() == ihist.IHIST_OK
    for i in range(n):
        assert np.array_equal(outs[i].numpy().view(np.uint32), oracle.integral_histogram(frames[i], nbins)), i
