"""The quad-major layout H[b/4][y][x][b%4]: the same counts as the oracle's
bin-major planes, regrouped four bins per 16-byte word, word for word --
per frame over tails, tilings, bin-group sizes, pitched and unaligned
buffers, overlapped launches and host-memory outputs; in batches next to the
other layouts; and through the region queries (Eq. 2)."""
import numpy as np
import pytest

import oracle
from paper_1711_01919_gb300 import ihist, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

Q = ihist.IHIST_QUAD_MAJOR


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1711_01919_gb300 import build as cuda_build
    cuda_build.build()
    ihist.load()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def quad(ref):
    b, h, w = ref.shape
    return np.ascontiguousarray(ref.reshape(b // 4, 4, h, w).transpose(0, 2, 3, 1))


def assert_same(got, ref, what):
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        i = tuple(bad[0])
        raise AssertionError("%s: %d words differ, first at %s: got %d want %d"
                             % (what, len(bad), i, got[i], ref[i]))


@pytest.mark.parametrize("h,w,nbins,tune", [
    (1, 1, 4, None), (5, 3, 8, None), (37, 131, 16, None), (64, 256, 12, {"rows_per_band": 7}),
    (97, 130, 4, {"rows_per_band": 3, "ctas_per_sm": 1}), (130, 643, 64, {"bins_per_cta": 8}),
    (130, 643, 64, {"bins_per_cta": 16}), (300, 1000, 32, {"chunks_per_warp": 2}),
    (200, 640, 24, {"groups_per_cta": 3, "rows_per_band": 11}), (17, 128, 256, None),
    (480, 640, 32, None), (1080, 1920, 64, None), (9, 16384, 4, None), (65535, 3, 4, None)])
def test_plan_equals_the_oracle(h, w, nbins, tune):
    img = synth.uniform_frame(h * 7 + w + nbins, h, w)
    with ihist.Plan(h, w, nbins, Q, tune=tune) as plan:
        out = plan.compute(torch.from_numpy(img).cuda())
        assert plan.status() == ihist.IHIST_OK
        assert plan.out_shape == (nbins // 4, h, w, 4)
        assert_same(u32(out).reshape(plan.out_shape), quad(oracle.integral_histogram(img, nbins)),
                    "%dx%d B=%d %s" % (h, w, nbins, tune))


def test_pitched_input_and_unaligned_output():
    h, w, nbins = 61, 333, 12
    img = synth.gradient_frame(77, h, w)
    ref = quad(oracle.integral_histogram(img, nbins))
    buf = torch.zeros(3 + h * (w + 5) + 16, dtype=torch.uint8, device="cuda")
    view = buf[3:3 + h * (w + 5)].view(h, w + 5)[:, :w]
    view.copy_(torch.from_numpy(img))
    n = h * w * nbins
    with ihist.Plan(h, w, nbins, Q) as plan:
        # output 4 bytes past a 16-byte boundary: the element-wise store path
        store = torch.full((n + 64,), -1, dtype=torch.int32, device="cuda")
        ihist.ihist_compute(plan.handle, view.data_ptr(), view.stride(0), store[1:].data_ptr(), 0)
        torch.cuda.synchronize()
        assert plan.status() == ihist.IHIST_OK
        host = u32(store)
        assert_same(host[1:1 + n].reshape(plan.out_shape), ref, "unaligned output")
        assert host[0] == 0xffffffff and (host[1 + n:] == 0xffffffff).all()  # nothing written outside


def test_queries_and_overlapped_launches():
    h, w, nbins = 270, 480, 16
    imgs = [synth.uniform_frame(900 + k, h, w) for k in range(4)]
    rects = synth.rects(901, 500, h, w)
    rects[7] = (0, 0, w, 3)  # out of range: a zero row and BAD_RECT
    d_rects = torch.from_numpy(rects).cuda()
    with ihist.Plan(h, w, nbins, Q, tune={"overlap": 1}) as plan:
        outs = [plan.empty_output() for _ in range(2)]
        rows = []
        for k, img in enumerate(imgs):
            plan.compute(torch.from_numpy(img).cuda(), outs[k % 2])
            rows.append(plan.query(outs[k % 2], d_rects))
        torch.cuda.synchronize()
        assert plan.status() == ihist.IHIST_ERR_BAD_RECT
        valid = rects.copy()
        valid[7] = (0, 0, 0, 0)  # the oracle is only asked about rectangles inside the frame
        for img, r in zip(imgs, rows):
            ref = oracle.query(oracle.integral_histogram(img, nbins), valid)
            ref[7] = 0
            assert np.array_equal(u32(r), ref)
        # window search works on bin-major and pixel-major outputs only
        target = torch.zeros(nbins, dtype=torch.int32, device="cuda")
        with pytest.raises(ihist.IhistError) as e:
            plan.window_search(outs[0], target, 32, 32, 8)
        assert e.value.code == ihist.IHIST_ERR_UNSUPPORTED


def test_batch_with_all_three_layouts_and_query_all():
    shapes = [(37, 131, 16, 2), (240, 320, 8, 0), (100, 1000, 64, 2), (64, 257, 7, 1), (480, 640, 32, 2)]
    imgs = [synth.uniform_frame(950 + i, h, w) for i, (h, w, b, l) in enumerate(shapes)]
    nb = [b for (h, w, b, l) in shapes]
    ly = [l for (h, w, b, l) in shapes]
    n = 40
    rects = np.stack([synth.rects(960 + i, n, h, w) for i, (h, w, b, l) in enumerate(shapes)])
    for tune in (None, {"bins_per_cta": 8, "rows_per_band": 13}):
        with ihist.Batch([torch.from_numpy(x).cuda() for x in imgs], nb, ly, tune=tune) as batch:
            batch.compute()
            assert batch.status() == ihist.IHIST_OK
            q = u32(batch.query_all(torch.from_numpy(rects).cuda()))
            off = 0
            for i, (img, (h, w, b, l)) in enumerate(zip(imgs, shapes)):
                ref = oracle.integral_histogram(img, b)
                want = quad(ref) if l == 2 else ref if l == 0 else np.ascontiguousarray(ref.transpose(1, 2, 0))
                assert_same(u32(batch.outs[i]).reshape(ihist.out_shape(h, w, b, l)), want, "frame %d %s" % (i, tune))
                assert np.array_equal(q[off:off + n * b].reshape(n, b), oracle.query(ref, rects[i])), i
                off += n * b


def test_host_memory_output():
    h, w, nbins = 120, 400, 8
    img = synth.gradient_frame(990, h, w)
    with ihist.Plan(h, w, nbins, Q) as plan:
        host = torch.empty(plan.out_shape, dtype=torch.int32).pin_memory()
        d_img = torch.from_numpy(img).cuda()
        ihist.ihist_compute(plan.handle, d_img.data_ptr(), w, host.data_ptr(), 0)
        torch.cuda.synchronize()
        assert plan.status() == ihist.IHIST_OK
        assert_same(host.numpy().view(np.uint32), quad(oracle.integral_histogram(img, nbins)), "host output")


def test_other_bin_structures_in_quad_major():
    h, w = 150, 300
    edges = [0, 10, 50, 51, 200, 210, 220, 240, 256]  # 8 bins
    img = synth.gradient_frame(1500, h, w)
    rgb = np.ascontiguousarray(np.stack([synth.uniform_frame(1501 + c, h, w) for c in range(3)], axis=2))
    with ihist.Plan(h, w, layout=Q, edges=edges) as ep, ihist.Plan(h, w, layout=Q, bins_per_channel=[4, 2, 2]) as jp:
        he = ep.compute(torch.from_numpy(img).cuda())
        hj = jp.compute(torch.from_numpy(rgb).cuda())
        assert ep.status() == ihist.IHIST_OK and jp.status() == ihist.IHIST_OK
        assert_same(u32(he).reshape(ep.out_shape), quad(oracle.integral_histogram_edges(img, edges)), "edges")
        assert_same(u32(hj).reshape(jp.out_shape), quad(oracle.integral_histogram_joint(rgb, [4, 2, 2])), "joint")
