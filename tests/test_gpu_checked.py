"""The checked build (every carry index and output store guarded on the
device; a failed guard latches IHIST_ERR_CHECK_FAILED and skips the access,
in place of a memory sanitizer) runs the main paths clean: status OK and
results equal to the oracle.  It runs in a child process that loads
libihist_checked.so through IHIST_LIB."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys, os
sys.path.insert(0, os.environ["ROOT"])
import numpy as np, torch
import oracle
from paper_1711_01919_gb300 import ihist, synth
assert ihist.LIB_PATH.endswith("libihist_checked.so"), ihist.LIB_PATH
def u32(t): return t.cpu().numpy().view(np.uint32)
def ref_layout(img, b, l):
    r = oracle.integral_histogram(img, b)
    if l == 2:
        return np.ascontiguousarray(r.reshape(b // 4, 4, r.shape[1], r.shape[2]).transpose(0, 2, 3, 1))
    return r if l == 0 else np.ascontiguousarray(r.transpose(1, 2, 0))
n = 0
for (h, w, b, l, tune) in [(1, 1, 3, 0, None), (37, 131, 16, 0, None), (64, 257, 7, 1, None), (100, 1000, 64, 1, None),
                           (33, 2049, 100, 0, {"bins_per_cta": 8}), (130, 640, 64, 1, {"bins_per_cta": 8}),
                           (300, 4096, 8, 0, None), (17, 128, 256, 1, None), (37, 131, 16, 2, None),
                           (130, 643, 64, 2, {"bins_per_cta": 16}),
                           (130, 700, 64, 1, {"bins_per_cta": 16, "groups_per_cta": 4, "chunks_per_warp": 1}),
                           (40, 500, 128, 1, {"bins_per_cta": 16, "groups_per_cta": 8, "chunks_per_warp": 1})]:
    img = synth.uniform_frame(h + w + b, h, w)
    with ihist.Plan(h, w, b, l, tune=tune) as p:
        got = u32(p.compute(torch.from_numpy(img).cuda())).reshape(p.out_shape)
        assert p.status() == ihist.IHIST_OK, (h, w, b, l)
    assert np.array_equal(got, ref_layout(img, b, l)), (h, w, b, l)
    n += 1
img = synth.uniform_frame(5, 90, 500)
with ihist.Plan(90, 500, edges=[0, 10, 11, 100, 255]) as p:
    got = u32(p.compute(torch.from_numpy(img).cuda()))
    assert p.status() == ihist.IHIST_OK
assert np.array_equal(got.reshape(4, 90, 500), oracle.integral_histogram_edges(img, [0, 10, 11, 100, 255]))
rgb = np.random.default_rng(3).integers(0, 256, size=(60, 300, 3), dtype=np.uint8)
with ihist.Plan(60, 300, bins_per_channel=[4, 4, 4]) as p:
    got = u32(p.compute(torch.from_numpy(rgb).cuda()))
    assert p.status() == ihist.IHIST_OK
assert np.array_equal(got.reshape(64, 60, 300), oracle.integral_histogram_joint(rgb, [4, 4, 4]))
shapes = [(37, 131, 16, 0), (240, 320, 16, 1), (100, 1000, 64, 0), (720, 1280, 32, 1), (5, 3, 3, 1), (90, 250, 12, 2)]
imgs = [synth.uniform_frame(40 + i, h, w) for i, (h, w, b, l) in enumerate(shapes)]
with ihist.Batch([torch.from_numpy(x).cuda() for x in imgs], [s[2] for s in shapes], [s[3] for s in shapes]) as bt:
    bt.compute()
    assert bt.status() == ihist.IHIST_OK
    for x, o, (h, w, b, l) in zip(imgs, bt.outs, shapes):
        assert np.array_equal(u32(o).reshape(ihist.out_shape(h, w, b, l)), ref_layout(x, b, l)), (h, w, b, l)
# a table batch: frames with value -> bin tables next to a uniform frame
edges = [0, 16, 64, 128, 129, 256]
tabs = [ihist.edges_table(edges), None, [(v * 7) % 9 - 1 for v in range(256)]]
tshapes = [(270, 480, 5, 0), (64, 257, 7, 1), (100, 1000, 8, 1)]
timgs = [synth.gradient_frame(60 + i, h, w) for i, (h, w, b, l) in enumerate(tshapes)]
with ihist.Batch([torch.from_numpy(x).cuda() for x in timgs], [s[2] for s in tshapes], [s[3] for s in tshapes],
                 tables=tabs) as bt:
    bt.compute()
    assert bt.status() == ihist.IHIST_OK
    for x, o, t, (h, w, b, l) in zip(timgs, bt.outs, tabs, tshapes):
        r = ref_layout(x, b, 0) if t is None else oracle.integral_histogram_mapped(x, np.asarray(t, np.int32), b)
        r = r if l == 0 else np.ascontiguousarray(r.transpose(1, 2, 0))
        assert np.array_equal(u32(o).reshape(ihist.out_shape(h, w, b, l)), r), (h, w, b, l)
print("checked ok", n)
'''


def test_checked_build_runs_clean():
    from paper_1711_01919_gb300 import build as cuda_build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = cuda_build.build(checked=True)
    env = dict(os.environ, IHIST_LIB=lib, ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked ok" in r.stdout
