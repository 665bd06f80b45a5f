"""The paper's three GPU mappings (CW-STS, CW-TiS, WF-TiS), rebuilt as
comparison kernels, give exactly the oracle's integral histogram."""
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


def run_mapping(name, img, nbins, pitch_pad=0):
    h, w = img.shape
    m = ihist.MAPPINGS[name]
    buf = torch.zeros((h, w + pitch_pad), dtype=torch.uint8, device="cuda")
    buf[:, :w].copy_(torch.from_numpy(img))
    out = torch.full((nbins, h, w), -1, dtype=torch.int32, device="cuda")
    nb = ihist.ihist_mapping_workspace_bytes(m, h, w, nbins)
    work = torch.empty((max(nb, 1),), dtype=torch.uint8, device="cuda")
    ihist.ihist_mapping_compute(m, h, w, nbins, buf.data_ptr(), w + pitch_pad, out.data_ptr(),
                                work.data_ptr() if nb else 0, torch.cuda.current_stream().cuda_stream)
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("name", ["cw_sts", "cw_tis", "wf_tis"])
@pytest.mark.parametrize("h,w", [(1, 1), (1, 40), (45, 1), (33, 65), (64, 64), (100, 130), (480, 640)])
@pytest.mark.parametrize("nbins", [1, 5, 32])
def test_mapping_matches_oracle(name, h, w, nbins):
    img = synth.uniform_frame(h * 7 + w + nbins, h, w)
    assert np.array_equal(run_mapping(name, img, nbins, pitch_pad=(h + w) % 5), oracle.integral_histogram(img, nbins))


@pytest.mark.parametrize("name", ["cw_sts", "cw_tis", "wf_tis"])
def test_mapping_1080p_equals_fused_kernel(name):
    img = synth.gradient_frame(3, 1080, 1920)
    with ihist.Plan(1080, 1920, 16) as plan:
        ref = plan.compute(torch.from_numpy(img).cuda()).cpu().numpy().view(np.uint32)
    assert np.array_equal(run_mapping(name, img, 16), ref)
    assert np.array_equal(ref[:, -1, -1], np.bincount((img.astype(np.int64) * 16 >> 8).ravel(), minlength=16))
