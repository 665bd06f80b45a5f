"""Batched persistent launch over frames of uneven size: every frame's result
equals the oracle (and the single-frame path) word for word."""
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


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def ref_layout(img, nbins, layout):
    ref = oracle.integral_histogram(img, nbins)
    if layout == ihist.IHIST_QUAD_MAJOR:
        b, h, w = ref.shape
        return np.ascontiguousarray(ref.reshape(b // 4, 4, h, w).transpose(0, 2, 3, 1))
    return ref if layout == 0 else np.ascontiguousarray(ref.transpose(1, 2, 0))


def check_batch(batch, imgs, nbins, layouts):
    for i, (img, b, l) in enumerate(zip(imgs, nbins, layouts)):
        got = u32(batch.outs[i]).reshape(ihist.out_shape(img.shape[0], img.shape[1], b, l))
        ref = ref_layout(img, b, l)
        assert np.array_equal(got, ref), "frame %d (%dx%d B=%d layout %d): %d words differ" % (
            i, img.shape[0], img.shape[1], b, l, int((got != ref).sum()))


MIXED = [(1, 1, 1, 0), (5, 3, 3, 1), (37, 131, 16, 0), (240, 320, 16, 0), (64, 257, 7, 1),
         (480, 640, 32, 0), (100, 1000, 64, 1), (720, 1280, 64, 0), (33, 2049, 100, 0),
         (300, 4096, 8, 0), (17, 128, 256, 1)]


@pytest.mark.parametrize("tune", [None, {"rows_per_band": 8}, {"rows_per_band": 64, "bins_per_cta": 8},
                                  {"rows_per_band": 3, "ctas_per_sm": 1}, {"warps_per_cta": 8},
                                  {"warps_per_cta": 8, "bins_per_cta": 8, "rows_per_band": 40},
                                  {"bins_per_cta": 16}, {"bins_per_cta": 16, "rows_per_band": 9},
                                  {"bins_per_cta": 8, "warps_per_cta": 16}, {"bins_per_cta": 8, "warps_per_cta": 8,
                                                                             "rows_per_band": 20}])
def test_mixed_batch(tune):
    imgs = [synth.uniform_frame(1000 + i, h, w) for i, (h, w, b, l) in enumerate(MIXED)]
    nbins = [b for (h, w, b, l) in MIXED]
    layouts = [l for (h, w, b, l) in MIXED]
    with ihist.Batch([torch.from_numpy(x).cuda() for x in imgs], nbins, layouts, tune=tune) as batch:
        batch.compute()
        assert batch.status() == ihist.IHIST_OK
        check_batch(batch, imgs, nbins, layouts)


def test_unaligned_frames_take_the_plain_path():
    imgs = [synth.uniform_frame(7 + i, 90, 300) for i in range(3)]
    dev = []
    for i, img in enumerate(imgs):
        buf = torch.zeros(1 + 90 * 311 + 16, dtype=torch.uint8, device="cuda")
        v = buf[1:1 + 90 * 311].view(90, 311)[:, :300]
        v.copy_(torch.from_numpy(img))
        dev.append(v)
    with ihist.Batch(dev, [12, 5, 64], [0, 1, 0]) as batch:
        batch.compute()
        assert batch.status() == ihist.IHIST_OK
        check_batch(batch, imgs, [12, 5, 64], [0, 1, 0])


def test_uneven_batch_workload_256_frames():
    # 256 frames, resolutions {320x240, 640x480, 1280x720, 1920x1080}, B in {16, 32, 64}
    specs = synth.uneven_batch_specs(synth.workload_seed(3), 256)
    imgs = [synth.uniform_frame(s, h, w) for (h, w, b, s) in specs]
    nbins = [b for (h, w, b, s) in specs]
    with ihist.Batch([torch.from_numpy(x).cuda() for x in imgs], nbins) as batch:
        batch.compute()
        assert batch.status() == ihist.IHIST_OK
        for i in range(len(imgs)):
            got = u32(batch.outs[i]).reshape(nbins[i], imgs[i].shape[0], imgs[i].shape[1])
            assert np.array_equal(got, oracle.integral_histogram(imgs[i], nbins[i])), "frame %d" % i
        # the same frames through single-frame plans give the same words
        for i in (0, 1, 2):
            with ihist.Plan(imgs[i].shape[0], imgs[i].shape[1], nbins[i]) as p:
                assert torch.equal(p.compute(batch.frames[i]), batch.outs[i])


def test_graph_replay_and_set_io():
    shapes = [(200, 700, 24), (64, 128, 8), (480, 640, 32)]
    a = [synth.uniform_frame(50 + i, h, w) for i, (h, w, b) in enumerate(shapes)]
    b_ = [synth.gradient_frame(60 + i, h, w) for i, (h, w, b) in enumerate(shapes)]
    nb = [b for (h, w, b) in shapes]
    da = [torch.from_numpy(x).cuda() for x in a]
    db = [torch.from_numpy(x).cuda() for x in b_]
    with ihist.Batch(da, nb) as batch:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            batch.compute(stream=s)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            batch.compute(stream=s)
        for _ in range(2):
            for o in batch.outs:
                o.fill_(-1)
            g.replay()
            torch.cuda.synchronize()
            check_batch(batch, a, nb, [0, 0, 0])
        outs2 = [torch.empty_like(o) for o in batch.outs]
        batch.set_io(db, outs2)
        batch.compute()
        assert batch.status() == ihist.IHIST_OK
        check_batch(batch, b_, nb, [0, 0, 0])
        q = batch.query(2, torch.from_numpy(synth.rects(3, 50, 480, 640)).cuda())
        ref = oracle.query(oracle.integral_histogram(b_[2], 32), synth.rects(3, 50, 480, 640))
        assert np.array_equal(u32(q), ref)


def test_batch_rejects_bad_frames():
    d = torch.zeros((10, 10), dtype=torch.uint8, device="cuda")
    o = torch.zeros((4, 10, 10), dtype=torch.int32, device="cuda")
    with pytest.raises(ihist.IhistError):
        ihist.ihist_batch_plan([(10, 10, 0, 0, d.data_ptr(), 10, o.data_ptr())])
    with pytest.raises(ihist.IhistError):
        ihist.ihist_batch_plan([(10, 10, 4, 0, d.data_ptr(), 5, o.data_ptr())])
    with pytest.raises(ihist.IhistError):
        ihist.ihist_batch_plan([])


def test_query_all_over_a_mixed_batch():
    shapes = [(37, 131, 16, 0), (240, 320, 7, 1), (5, 3, 3, 0), (100, 1000, 64, 1)]
    imgs = [synth.uniform_frame(300 + i, h, w) for i, (h, w, b, l) in enumerate(shapes)]
    nb = [b for (h, w, b, l) in shapes]
    ly = [l for (h, w, b, l) in shapes]
    n = 40
    rects = np.stack([synth.rects(400 + i, n, h, w) for i, (h, w, b, l) in enumerate(shapes)])
    rects[1, 5] = (0, 0, 320, 3)   # out of range: zero row and BAD_RECT
    with ihist.Batch([torch.from_numpy(x).cuda() for x in imgs], nb, ly) as batch:
        batch.compute()
        q = u32(batch.query_all(torch.from_numpy(rects).cuda()))
        assert batch.status() == ihist.IHIST_ERR_BAD_RECT
        off = 0
        for i, (img, b) in enumerate(zip(imgs, nb)):
            got = q[off:off + n * b].reshape(n, b)
            ref = oracle.query(oracle.integral_histogram(img, b), rects[i])
            assert np.array_equal(got, ref), "frame %d" % i
            off += n * b
        assert not q[n * nb[0] + 5 * nb[1]: n * nb[0] + 6 * nb[1]].any()


def test_upload_compute_from_pinned_host_frames():
    shapes = [(120, 500, 24), (64, 256, 8), (90, 640, 32)]
    nb = [b for (h, w, b) in shapes]
    d_in = [torch.empty((h, w), dtype=torch.uint8, device="cuda") for (h, w, b) in shapes]
    with ihist.Batch(d_in, nb) as batch:
        copy = torch.cuda.Stream()
        for rep in range(3):
            imgs = [synth.gradient_frame(500 + 10 * rep + i, h, w) for i, (h, w, b) in enumerate(shapes)]
            host = [torch.from_numpy(x).pin_memory() for x in imgs]
            batch.upload_compute(host, copy_stream=copy)
            torch.cuda.synchronize()
            assert batch.status() == ihist.IHIST_OK
            check_batch(batch, imgs, nb, [0, 0, 0])


def test_set_io_rebinds_different_shapes_within_slot_capacity():
    # plan 4 slots at 480x640x32, then bind smaller and mixed frames
    cap = [(480, 640, 32)] * 4
    d0 = [torch.empty((h, w), dtype=torch.uint8, device="cuda") for (h, w, b) in cap]
    with ihist.Batch(d0, [b for (h, w, b) in cap]) as batch:
        for shapes in ([(100, 300, 16), (480, 640, 32), (7, 5, 3)],
                       [(240, 320, 32), (480, 640, 8), (480, 640, 32), (33, 129, 24)],
                       [(1, 1, 1)]):
            imgs = [synth.uniform_frame(900 + h + w + b, h, w) for (h, w, b) in shapes]
            frames = [torch.from_numpy(x).cuda() for x in imgs]
            outs = [torch.empty((b, h, w), dtype=torch.int32, device="cuda") for (h, w, b) in shapes]
            batch.nbins = [b for (h, w, b) in shapes]
            batch.layouts = [0] * len(shapes)
            batch.set_io(frames, outs)
            batch.compute()
            assert batch.status() == ihist.IHIST_OK
            check_batch(batch, imgs, batch.nbins, batch.layouts)
        # a frame larger than its slot is refused and the binding stays usable
        big = torch.empty((960, 640), dtype=torch.uint8, device="cuda")
        bo = torch.empty((32, 960, 640), dtype=torch.int32, device="cuda")
        with pytest.raises(ihist.IhistError) as e:
            ihist.ihist_batch_set_io(batch.handle, [(960, 640, 32, 0, big.data_ptr(), 640, bo.data_ptr())])
        assert e.value.code == ihist.IHIST_ERR_UNSUPPORTED
        batch.compute()
        assert batch.status() == ihist.IHIST_OK


def test_set_io_narrower_frames_keep_the_planned_launch_shape():
    # slots planned at 1920 wide: 1280- and 640-wide frames bound later must
    # fit the planned chunks per warp and per-CTA carry width
    d0 = [torch.empty((1080, 1920), dtype=torch.uint8, device="cuda") for _ in range(2)]
    shapes = [(720, 1280, 32), (480, 640, 16)]
    imgs = [synth.uniform_frame(40 + h, h, w) for (h, w, b) in shapes]
    for tune in (None, {"bins_per_cta": 8}):
        with ihist.Batch(d0, [64, 64], tune=tune) as batch:
            frames = [torch.from_numpy(x).cuda() for x in imgs]
            outs = [torch.empty((b, h, w), dtype=torch.int32, device="cuda") for (h, w, b) in shapes]
            batch.set_io(frames, outs, nbins=[b for (h, w, b) in shapes], layouts=[0, 0])
            batch.compute()
            assert batch.status() == ihist.IHIST_OK
            check_batch(batch, imgs, [b for (h, w, b) in shapes], [0, 0])


def test_warps_per_cta_4_and_wide_frames_in_width_segments():
    small = [(37, 131, 16, 0), (240, 320, 16, 0), (64, 257, 7, 1), (100, 1000, 64, 1)]
    imgs = [synth.uniform_frame(2000 + i, h, w) for i, (h, w, b, l) in enumerate(small)]
    nbins = [b for (h, w, b, l) in small]
    layouts = [l for (h, w, b, l) in small]
    with ihist.Batch([torch.from_numpy(x).cuda() for x in imgs], nbins, layouts,
                     tune={"warps_per_cta": 4}) as batch:
        batch.compute()
        assert batch.status() == ihist.IHIST_OK
        check_batch(batch, imgs, nbins, layouts)
    # frames wider than a CTA's warps x 4 chunks: each band splits into width
    # segments (4-warp CTAs: 300x4096 needs 32 chunks = 2 segments; 16-warp
    # CTAs: 9000 columns = 2 segments, 20000 = 3, 65535 = 8), mixed with
    # ordinary frames in one launch
    for shapes, tune in (([(300, 4096, 8, 0), (50, 700, 16, 1)], {"warps_per_cta": 4}),
                         ([(16, 9000, 8, 0), (240, 320, 16, 0)], None),
                         ([(70, 20000, 12, 0), (33, 20000, 32, 2), (480, 640, 32, 0), (5, 20000, 16, 1)], None),
                         ([(9, 65535, 5, 0), (61, 333, 9, 0)], {"rows_per_band": 4})):
        imgs = [synth.uniform_frame(2100 + i + w, h, w) for i, (h, w, b, l) in enumerate(shapes)]
        nbins = [b for (h, w, b, l) in shapes]
        layouts = [l for (h, w, b, l) in shapes]
        with ihist.Batch([torch.from_numpy(x).cuda() for x in imgs], nbins, layouts, tune=tune) as batch:
            batch.compute()
            assert batch.status() == ihist.IHIST_OK
            check_batch(batch, imgs, nbins, layouts)
            batch.compute()  # the next launch (other epoch) is exact too
            assert batch.status() == ihist.IHIST_OK
            check_batch(batch, imgs, nbins, layouts)


def test_pixel_major_batch_defaults_to_16_bin_groups():
    shapes = [(240, 320, 16), (480, 640, 32), (720, 1280, 64), (37, 131, 100), (1, 1, 16)]
    imgs = [synth.uniform_frame(3000 + i, h, w) for i, (h, w, b) in enumerate(shapes)]
    nbins = [b for (h, w, b) in shapes]
    with ihist.Batch([torch.from_numpy(x).cuda() for x in imgs], nbins, [1] * len(shapes)) as batch:
        assert batch.tune["bins_per_cta"] == 16
        batch.compute()
        assert batch.status() == ihist.IHIST_OK
        check_batch(batch, imgs, nbins, [1] * len(shapes))


@pytest.mark.parametrize("tune", [None, {"warps_per_cta": 16}, {"warps_per_cta": 8, "rows_per_band": 5}])
def test_pixel_major_batch_stores_whole_records(tune):
    # pixel-major frames whose bin groups all fit one CTA (B = 32, 64, 128
    # with 16-bin groups) take the whole-record rows, with width segments
    # where the CTA's warps cannot span the frame; a bin-major frame and a
    # pixel-major one outside that path (16 bins: one group; 100 bins:
    # records of 25 units) share the launch
    shapes = [(200, 1920, 64, 1), (150, 700, 32, 1), (61, 1000, 128, 1), (90, 333, 16, 1), (45, 640, 64, 0),
              (37, 131, 100, 1)]
    imgs = [synth.uniform_frame(5000 + i, h, w) for i, (h, w, b, l) in enumerate(shapes)]
    nbins = [b for (h, w, b, l) in shapes]
    layouts = [l for (h, w, b, l) in shapes]
    with ihist.Batch([torch.from_numpy(x).cuda() for x in imgs], nbins, layouts, tune=tune) as batch:
        assert batch.tune["bins_per_cta"] == 16
        for _ in range(2):
            batch.compute()
            assert batch.status() == ihist.IHIST_OK
            check_batch(batch, imgs, nbins, layouts)


def test_autotuned_layout_and_launch_shape_give_exact_batches(tmp_path, monkeypatch):
    # the autotuner times both layouts (each with its own tuned launch shape)
    # with and without a query load; whatever it picks computes exactly
    from paper_1711_01919_gb300 import autotune
    monkeypatch.setenv("IHIST_TUNE_CACHE", str(tmp_path / "tune.json"))
    shapes = [(240, 320, 16), (480, 640, 32), (100, 1000, 8)]
    imgs = [synth.uniform_frame(70 + i, h, w) for i, (h, w, b) in enumerate(shapes)]
    nbins = [b for (h, w, b) in shapes]
    for queries in (0, 4000):
        layout, tune, times = autotune.tune_batch_layout(shapes, queries, use_cache=False)
        assert set(times) == {ihist.IHIST_BIN_MAJOR, ihist.IHIST_PIXEL_MAJOR, ihist.IHIST_QUAD_MAJOR}
        assert times[layout] == min(times.values())
        with ihist.Batch([torch.from_numpy(x).cuda() for x in imgs], nbins, [layout] * 3, tune=tune or None) as batch:
            batch.compute()
            assert batch.status() == ihist.IHIST_OK
            check_batch(batch, imgs, nbins, [layout] * 3)
