"""CUDA path vs the CPU oracle, through the C ABI: bit-exact uint32 equality.

The counts are integers, so every comparison is exact (no tolerance).  Small
and odd shapes are compared word for word over the whole tensor; the
full-size 64-MP workload is compared on sampled bin planes plus invariants
over every plane (test_gpu_large.py).
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
    ihist.load()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def to_layout(ref, layout):
    """Bin-major oracle result in the requested layout (a transpose only)."""
    if layout == ihist.IHIST_QUAD_MAJOR:
        b, h, w = ref.shape
        return np.ascontiguousarray(ref.reshape(b // 4, 4, h, w).transpose(0, 2, 3, 1))
    return ref if layout == ihist.IHIST_BIN_MAJOR else np.ascontiguousarray(ref.transpose(1, 2, 0))


def run_gpu(img, nbins, layout=0, tune=None, pitch_pad=0, offset=0):
    h, w = img.shape
    dev = torch.device("cuda")
    if pitch_pad or offset:
        buf = torch.zeros(offset + h * (w + pitch_pad) + 16, dtype=torch.uint8, device=dev)
        view = buf[offset:offset + h * (w + pitch_pad)].view(h, w + pitch_pad)[:, :w]
        view.copy_(torch.from_numpy(img))
        d_img = view
    else:
        d_img = torch.from_numpy(img).to(dev)
    with ihist.Plan(h, w, nbins, layout, tune=tune) as plan:
        out = plan.compute(d_img)
        st = plan.status()
    assert st == ihist.IHIST_OK, ihist.ihist_error_string(st)
    return u32(out).reshape(plan.out_shape)


def assert_same(got, ref, what):
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        i = tuple(bad[0])
        raise AssertionError("%s: %d words differ, first at %s: got %d want %d"
                             % (what, len(bad), i, got[i], ref[i]))


SHAPES = [(1, 1), (1, 5), (7, 1), (2, 3), (3, 129), (17, 128), (33, 130), (64, 255), (65, 257),
          (100, 384), (31, 1000), (480, 640)]


@pytest.mark.parametrize("h,w", SHAPES)
@pytest.mark.parametrize("nbins", [1, 3, 8, 32, 100, 256])
def test_small_shapes_bin_major(h, w, nbins):
    img = synth.uniform_frame(synth.workload_seed(1) + h * 7919 + w, h, w)
    ref = oracle.integral_histogram(img, nbins)
    assert_same(run_gpu(img, nbins), ref, "%dx%d B=%d" % (h, w, nbins))


@pytest.mark.parametrize("h,w", [(1, 1), (5, 3), (37, 131), (64, 256), (130, 640)])
@pytest.mark.parametrize("nbins", [2, 5, 16, 64])
def test_small_shapes_pixel_major(h, w, nbins):
    img = synth.gradient_frame(h * 31 + w, h, w)
    ref = oracle.integral_histogram(img, nbins)
    got = run_gpu(img, nbins, layout=ihist.IHIST_PIXEL_MAJOR)
    assert_same(got, to_layout(ref, 1), "pixel-major %dx%d B=%d" % (h, w, nbins))


TUNINGS = [
    {"rows_per_band": 1},
    {"rows_per_band": 3, "bins_per_cta": 4},
    {"rows_per_band": 7, "bins_per_cta": 16},
    {"rows_per_band": 255, "bins_per_cta": 8, "chunks_per_warp": 4},
    {"rows_per_band": 16, "chunks_per_warp": 2},
    {"rows_per_band": 5, "chunks_per_warp": 4, "bins_per_cta": 4},
    {"rows_per_band": 9, "chunks_per_warp": 8, "bins_per_cta": 8},
    {"rows_per_band": 20, "chunks_per_warp": 2, "bins_per_cta": 16},
    {"rows_per_band": 12, "ctas_per_sm": 1},
    # at most 8 (4) warps per CTA: frames wider than 8 (4) chunks per warp slot
    # split into width segments
    {"warps_per_cta": 8, "chunks_per_warp": 1, "rows_per_band": 10},
    {"warps_per_cta": 4, "chunks_per_warp": 2, "bins_per_cta": 8},
]


@pytest.mark.parametrize("tune", TUNINGS, ids=lambda t: "-".join("%s%d" % (k[:4], v) for k, v in t.items()))
def test_tilings(tune):
    # deep look-back chains (R=1 gives one band per row) and multi-chunk warps
    for (h, w, nbins) in [(300, 1000, 24), (77, 2049, 8), (260, 130, 64)]:
        img = synth.uniform_frame(h + w + nbins, h, w)
        ref = oracle.integral_histogram(img, nbins)
        assert_same(run_gpu(img, nbins, tune=tune), ref, "%s %dx%d B=%d" % (tune, h, w, nbins))


@pytest.mark.parametrize("h,w,nbins,tune", [
    (300, 640, 24, {"groups_per_cta": 3, "rows_per_band": 11}),
    (300, 384, 40, {"groups_per_cta": 5, "rows_per_band": 7}),
    (100, 130, 44, {"groups_per_cta": 7, "rows_per_band": 9}),      # last group set partial
    (61, 1000, 30, {"groups_per_cta": 2, "chunks_per_warp": 2, "rows_per_band": 5}),
    (40, 256, 64, {"groups_per_cta": 4, "bins_per_cta": 8, "rows_per_band": 3}),
])
@pytest.mark.parametrize("layout", [0, 1])
def test_multi_group_ctas(h, w, nbins, tune, layout):
    img = synth.uniform_frame(h * w + nbins, h, w)
    ref = oracle.integral_histogram(img, nbins)
    got = run_gpu(img, nbins, layout=layout, tune=tune)
    assert_same(got, to_layout(ref, layout), "%s %dx%d B=%d" % (tune, h, w, nbins))


# Pixel-major frames whose CTA owns every bin group (groups_per_cta =
# number of groups, B / 4 a power of two) store whole pixel records: the
# warps of one column range meet at a named barrier per row.  Records of
# 4..64 16-byte units, 8 and 16 bins per group, ragged and unaligned widths
# (scalar stores), width segments, one-row bands and pitched input.
RECORD_CASES = [
    (300, 640, 64, {"bins_per_cta": 16, "groups_per_cta": 4, "chunks_per_warp": 1}, 0),
    (130, 1920, 64, {"bins_per_cta": 16, "groups_per_cta": 4, "chunks_per_warp": 2, "rows_per_band": 29}, 0),
    (77, 333, 32, {"bins_per_cta": 16, "groups_per_cta": 2}, 0),
    (50, 200, 16, {"bins_per_cta": 8, "groups_per_cta": 2, "rows_per_band": 7}, 0),
    (40, 500, 128, {"bins_per_cta": 16, "groups_per_cta": 8, "chunks_per_warp": 1}, 0),
    (20, 300, 256, {"bins_per_cta": 16, "groups_per_cta": 16, "rows_per_band": 6}, 0),
    (64, 256, 32, {"bins_per_cta": 16, "groups_per_cta": 2, "rows_per_band": 1}, 0),
    (90, 1000, 64, {"bins_per_cta": 8, "groups_per_cta": 8, "chunks_per_warp": 1, "rows_per_band": 11}, 0),
    (60, 700, 64, {"bins_per_cta": 16, "groups_per_cta": 4}, 7),
]


@pytest.mark.parametrize("h,w,nbins,tune,pitch_pad", RECORD_CASES)
def test_pixel_major_whole_records(h, w, nbins, tune, pitch_pad):
    img = synth.uniform_frame(h * 13 + w * 7 + nbins, h, w)
    ref = to_layout(oracle.integral_histogram(img, nbins), 1)
    got = run_gpu(img, nbins, layout=1, tune=tune, pitch_pad=pitch_pad, offset=3 if pitch_pad else 0)
    assert_same(got, ref, "%s %dx%d B=%d pad %d" % (tune, h, w, nbins, pitch_pad))
    img = synth.gradient_frame(h + w + nbins, h, w)
    assert_same(run_gpu(img, nbins, layout=1, tune=tune), to_layout(oracle.integral_histogram(img, nbins), 1),
                "gradient %s" % tune)


def test_warps_per_cta_caps_the_plan_and_round_trips():
    with ihist.Plan(64, 3000, 16, 0, tune={"warps_per_cta": 8, "chunks_per_warp": 1}) as plan:
        assert plan.tune["warps_per_cta"] <= 8
        tune = plan.tune
    with ihist.Plan(64, 3000, 16, 0, tune=tune) as again:
        assert again.tune == tune  # the reported tiling recreates itself
    with pytest.raises(ihist.IhistError) as e:
        ihist.Plan(64, 256, 8, 0, tune={"warps_per_cta": 17})
    assert e.value.code == ihist.IHIST_ERR_INVALID_ARG


def test_infeasible_tiling_is_rejected():
    # 8 warps x 255 rows x 128 bytes of staged input exceed shared memory
    with pytest.raises(ihist.IhistError) as e:
        ihist.Plan(300, 1000, 24, 0, tune={"rows_per_band": 255, "bins_per_cta": 8, "chunks_per_warp": 1})
    assert e.value.code == ihist.IHIST_ERR_UNSUPPORTED


def test_pitch_and_unaligned_input():
    img = synth.uniform_frame(5, 90, 300)
    ref = oracle.integral_histogram(img, 12)
    assert_same(run_gpu(img, 12, pitch_pad=13), ref, "pitch+13")
    assert_same(run_gpu(img, 12, pitch_pad=4, offset=1), ref, "unaligned base")
    assert_same(run_gpu(img, 12, layout=1, pitch_pad=7, offset=3), to_layout(ref, 1), "pixel-major unaligned")


def test_closed_form_frames():
    h, w = 200, 300
    area = (np.arange(1, h + 1)[:, None] * np.arange(1, w + 1)[None, :]).astype(np.uint32)
    for v, nbins in [(0, 16), (255, 16), (131, 7), (255, 256)]:
        got = run_gpu(np.full((h, w), v, dtype=np.uint8), nbins)
        b = oracle.bin_of(v, nbins)
        assert np.array_equal(got[b], area)
        assert not np.delete(got, b, axis=0).any()


def test_workload_640x480_b32_and_1000_queries():
    seed = synth.workload_seed(1)
    img = synth.uniform_frame(seed, 480, 640)
    rects = synth.rects(seed + 1, 1000, 480, 640)
    ref = oracle.integral_histogram(img, 32)
    ref_q = oracle.query(ref, rects)
    for layout in (0, 1):
        with ihist.Plan(480, 640, 32, layout) as plan:
            out = plan.compute(torch.from_numpy(img).cuda())
            q = plan.query(out, torch.from_numpy(rects).cuda())
            assert plan.status() == ihist.IHIST_OK
        assert_same(u32(out).reshape(plan.out_shape), to_layout(ref, layout), "640x480 layout %d" % layout)
        assert_same(u32(q), ref_q, "1000 queries layout %d" % layout)


def test_workload_1080p_b64_gradient_frames():
    seed = synth.workload_seed(2)
    with ihist.Plan(1080, 1920, 64, 0) as plan:
        for f in range(2):
            img = synth.gradient_frame(synth.substream_seed(seed, f), 1080, 1920)
            ref = oracle.integral_histogram(img, 64)
            out = plan.compute(torch.from_numpy(img).cuda())
            assert plan.status() == ihist.IHIST_OK
            assert_same(u32(out).reshape(64, 1080, 1920), ref, "1080p frame %d" % f)


def test_repeated_launches_and_graph_replay():
    # the epoch in device memory lets launches (and graph replays) run back to
    # back with no host-side reset of the carry flags
    img1 = synth.uniform_frame(21, 150, 520)
    img2 = synth.uniform_frame(22, 150, 520)
    ref1, ref2 = oracle.integral_histogram(img1, 20), oracle.integral_histogram(img2, 20)
    with ihist.Plan(150, 520, 20, 0, tune={"rows_per_band": 8}) as plan:
        d_in = torch.from_numpy(img1).cuda()
        out = plan.empty_output()
        for _ in range(5):
            out.fill_(-1)
            plan.compute(d_in, out)
            assert_same(u32(out).reshape(plan.out_shape), ref1, "repeat")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            plan.compute(d_in, out, stream=s)  # warm-up on the capture stream
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            plan.compute(d_in, out, stream=s)
        for img, ref in ((img2, ref2), (img1, ref1), (img2, ref2)):
            d_in.copy_(torch.from_numpy(img))
            out.fill_(-1)
            g.replay()
            torch.cuda.synchronize()
            assert_same(u32(out).reshape(plan.out_shape), ref, "graph replay")
        assert plan.status() == ihist.IHIST_OK


def test_output_guard_words_untouched():
    img = synth.uniform_frame(3, 61, 333)
    ref = oracle.integral_histogram(img, 9)
    n = ref.size
    for layout in (0, 1):
        buf = torch.full((64 + n + 64,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        with ihist.Plan(61, 333, 9, layout) as plan:
            ihist.ihist_compute(plan.handle, torch.from_numpy(img).cuda().data_ptr(), 333,
                                buf[64:].data_ptr(), torch.cuda.current_stream().cuda_stream)
            assert plan.status() == ihist.IHIST_OK
        host = u32(buf)
        assert (host[:64] == 0x5A5A5A5A).all() and (host[64 + n:] == 0x5A5A5A5A).all()
        assert_same(host[64:64 + n].reshape(plan.out_shape), to_layout(ref, layout), "guarded")


def test_query_edge_rectangles_and_bad_rect_status():
    h, w, nbins = 50, 70, 6
    img = synth.uniform_frame(8, h, w)
    ref = oracle.integral_histogram(img, nbins)
    good = [(0, 0, w - 1, h - 1), (0, 0, 0, 0), (w - 1, h - 1, w - 1, h - 1), (0, 5, 0, 9),
            (3, 0, 9, 0), (10, 10, 10, 49), (69, 0, 69, 49)]
    bad = [(-1, 0, 3, 3), (0, 0, w, 3), (5, 5, 4, 6), (0, 9, 2, 8), (0, 0, 3, h)]
    rects = np.array(good + bad, dtype=np.int32)
    for layout in (0, 1):
        with ihist.Plan(h, w, nbins, layout) as plan:
            out = plan.compute(torch.from_numpy(img).cuda())
            q = u32(plan.query(out, torch.from_numpy(rects[:len(good)]).cuda()))
            assert plan.status() == ihist.IHIST_OK
            assert_same(q, oracle.query(ref, rects[:len(good)]), "good rects")
            for r, row in zip(good, q):
                assert np.array_equal(row, oracle.region_brute(img, nbins, r))
            qa = u32(plan.query(out, torch.from_numpy(rects).cuda()))
            assert plan.status() == ihist.IHIST_ERR_BAD_RECT
            assert not qa[len(good):].any()
            assert_same(qa[:len(good)], q, "good rows beside bad ones")
            assert plan.status() == ihist.IHIST_OK  # read-and-clear
            z = plan.query(out, torch.zeros((0, 4), dtype=torch.int32, device="cuda"))
            assert z.shape == (0, nbins)


@pytest.mark.parametrize("h,w,nbins,layout", [(9, 16384, 5, 0), (9, 16384, 5, 1), (65535, 3, 2, 0), (65535, 3, 2, 1),
                                              (40, 300, 256, 1), (3, 8192, 256, 0), (1, 16384, 1, 0),
                                              (9, 65535, 5, 0), (9, 65535, 5, 1), (9, 65535, 8, 2),
                                              (3, 40000, 256, 0), (3, 40000, 256, 1), (3, 40000, 256, 2),
                                              (1, 65535, 1, 0)])
def test_extreme_shapes(h, w, nbins, layout):
    # the widest frames (65535 columns: width segments), the tallest (65535
    # rows) and 256 bins in every layout
    img = synth.uniform_frame(h + 3 * w + nbins, h, w)
    got = run_gpu(img, nbins, layout=layout)
    assert_same(got, to_layout(oracle.integral_histogram(img, nbins), layout),
                "%dx%d B=%d layout %d" % (h, w, nbins, layout))


@pytest.mark.parametrize("h,w,nbins,layout,tune", [
    # one chunk per warp: 24-chunk frames split into 2 segments of 12 warps
    (100, 3000, 16, 0, {"chunks_per_warp": 1}), (100, 3000, 16, 1, {"chunks_per_warp": 1}),
    (100, 3000, 16, 2, {"chunks_per_warp": 1}),
    (97, 5000, 37, 0, {"chunks_per_warp": 1, "rows_per_band": 5}),           # 3 segments, ragged tail
    (64, 4100, 64, 1, {"chunks_per_warp": 2, "bins_per_cta": 16}),           # 17 warps -> 2 segments
    (130, 20000, 24, 0, {"bins_per_cta": 8, "rows_per_band": 17}), (130, 20000, 24, 1, None),
    (300, 17000, 4, 0, {"chunks_per_warp": 8, "ctas_per_sm": 1}),            # 133 chunks -> 2 segments
    (2, 65535, 64, 0, None), (255, 33000, 16, 2, {"rows_per_band": 64}),
])
def test_width_segments(h, w, nbins, layout, tune):
    # frames wider than one CTA's warps cover: each band's segments add the
    # per-row bin totals of the segments to their left (Eq. 1's row sums
    # split at the segment edges); exact against Algorithm 1 word for word
    img = synth.uniform_frame(h * 7 + w + nbins, h, w)
    got = run_gpu(img, nbins, layout=layout, tune=tune)
    assert_same(got, to_layout(oracle.integral_histogram(img, nbins), layout),
                "%dx%d B=%d layout %d %s" % (h, w, nbins, layout, tune))


def test_width_segments_pitched_and_gradient():
    # a pitched, unaligned wide input (plain loads, no TMA) and a smooth frame
    # whose bins change slowly across the segment edges
    h, w, nbins = 40, 30000, 32
    img = synth.gradient_frame(77, h, w)
    ref = oracle.integral_histogram(img, nbins)
    assert_same(run_gpu(img, nbins, pitch_pad=13, offset=1), ref, "pitched wide frame")
    assert_same(run_gpu(img, nbins, tune={"chunks_per_warp": 1, "rows_per_band": 3}), ref, "1 chunk per warp")


@pytest.mark.parametrize("h,w,nbins,tune", [
    (30, 9000, 24, {"bins_per_cta": 8, "groups_per_cta": 2, "chunks_per_warp": 8}),  # 2 groups in 2 segments
    (45, 5000, 36, {"groups_per_cta": 4, "chunks_per_warp": 2, "rows_per_band": 9}),  # 4 groups in 5 segments
])
@pytest.mark.parametrize("layout", [0, 1])
def test_width_segments_with_several_groups_per_cta(h, w, nbins, tune, layout):
    # groups_per_cta > 1 leaves 16 / groups_per_cta warps to a group, so
    # narrower frames already split into segments
    img = synth.uniform_frame(h + 5 * w + nbins, h, w)
    ref = to_layout(oracle.integral_histogram(img, nbins), layout)
    assert_same(run_gpu(img, nbins, layout=layout, tune=tune), ref, "%s %dx%d B=%d" % (tune, h, w, nbins))
