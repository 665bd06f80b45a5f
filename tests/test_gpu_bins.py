"""Other bin structures and joint multi-channel bins on the GPU, through the
C ABI, against the oracle: bit-exact uint32 equality over whole tensors.

Bins by edges and by a value -> bin map (values in no bin count nowhere) run
the scan kernel with its shared-memory table; joint bins of [h][w][C]
frames run the joint-index pass and then the scan on its plane."""
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
    return ref if layout == 0 else np.ascontiguousarray(ref.transpose(1, 2, 0))


def assert_same(got, ref, what):
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        i = tuple(bad[0])
        raise AssertionError("%s: %d words differ, first at %s: got %d want %d"
                             % (what, len(bad), i, got[i], ref[i]))


def compute(plan, frame, pitch_pad=0):
    if pitch_pad:
        h = frame.shape[0]
        row = int(np.prod(frame.shape[1:]))
        buf = torch.zeros((h, row + pitch_pad), dtype=torch.uint8, device="cuda")
        buf[:, :row].copy_(torch.from_numpy(frame.reshape(h, row)))
        d = buf[:, :row].view(frame.shape) if frame.ndim == 2 else buf[:, :row].view(*frame.shape)
    else:
        d = torch.from_numpy(np.ascontiguousarray(frame)).cuda()
    out = plan.compute(d)
    assert plan.status() == ihist.IHIST_OK
    return u32(out).reshape(plan.out_shape)


EDGE_SETS = [[0, 256], [10, 50, 51, 200], [0, 1, 2, 255, 256], [0, 16, 48, 96, 160, 255],
             [3, 17, 90, 91, 92, 200, 255], list(range(0, 257, 4)), sorted(set(np.linspace(5, 250, 40).astype(int)))]
SHAPES = [(1, 1), (3, 129), (37, 131), (64, 256), (100, 384), (33, 1000), (240, 320), (17, 2300)]


@pytest.mark.parametrize("h,w", SHAPES)
@pytest.mark.parametrize("ei", range(len(EDGE_SETS)))
def test_edges_bin_major(h, w, ei):
    edges = EDGE_SETS[ei]
    img = synth.uniform_frame(900 + h * 7 + w, h, w)
    ref = oracle.integral_histogram_edges(img, edges)
    with ihist.Plan(h, w, edges=edges) as plan:
        assert_same(compute(plan, img), ref, "edges %s %dx%d" % (edges[:4], h, w))


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("tune", [None, {"bins_per_cta": 8}, {"bins_per_cta": 8, "rows_per_band": 7},
                                  {"chunks_per_warp": 2, "groups_per_cta": 2}])
def test_value_map_layouts_and_tilings(layout, tune):
    rng = np.random.default_rng(12)
    nbins = 21
    bin_map = rng.integers(-1, nbins, size=256)
    h, w = 130, 700
    img = synth.gradient_frame(44, h, w)
    ref = oracle.integral_histogram_mapped(img, bin_map, nbins)
    with ihist.Plan(h, w, nbins, layout, tune=tune, bin_of_value=bin_map.tolist()) as plan:
        assert_same(compute(plan, img), to_layout(ref, layout), "map layout %d tune %s" % (layout, tune))


def test_value_map_unaligned_pitch_and_wide_frames():
    rng = np.random.default_rng(3)
    bin_map = rng.integers(-1, 40, size=256)
    for (h, w) in [(50, 300), (9, 5000), (70, 8200)]:
        img = synth.uniform_frame(h + w, h, w)
        ref = oracle.integral_histogram_mapped(img, bin_map, 40)
        with ihist.Plan(h, w, 40, bin_of_value=bin_map.tolist()) as plan:
            assert_same(compute(plan, img, pitch_pad=3), ref, "map %dx%d pitch+3" % (h, w))
            assert_same(compute(plan, img), ref, "map %dx%d" % (h, w))


def test_value_map_all_in_no_bin_and_uniform_table():
    img = synth.uniform_frame(5, 64, 200)
    with ihist.Plan(64, 200, 3, bin_of_value=[-1] * 256) as plan:
        assert not compute(plan, img).any()
    # the table of the uniform bins gives the uniform plan's result
    table = [v * 64 // 256 for v in range(256)]
    with ihist.Plan(64, 200, 64, bin_of_value=table) as a, ihist.Plan(64, 200, 64) as b:
        assert_same(compute(a, img), compute(b, img), "uniform table vs uniform plan")


def test_edges_queries_match_oracle():
    h, w = 480, 640
    edges = [0, 30, 31, 100, 180, 181, 250]
    img = synth.uniform_frame(77, h, w)
    ref = oracle.integral_histogram_edges(img, edges)
    rects = synth.rects(78, 500, h, w)
    with ihist.Plan(h, w, edges=edges) as plan:
        d = torch.from_numpy(img).cuda()
        hist = plan.compute(d)
        q = plan.query(hist, torch.from_numpy(rects).cuda())
        assert plan.status() == ihist.IHIST_OK
    assert_same(u32(q), oracle.query(ref, rects), "edges queries")


JOINT = [([2, 3, 2], (2, 2)), ([4, 4, 4], (37, 131)), ([8, 8, 4], (64, 256)), ([6, 6, 6], (100, 384)),
         ([5, 7], (33, 1000)), ([4, 4, 4, 4], (48, 300)), ([16], (29, 130)), ([3, 3, 3], (1, 1)),
         ([4, 4, 4], (240, 320))]


@pytest.mark.parametrize("cbins,shape", JOINT)
def test_joint_bin_major(cbins, shape):
    h, w = shape
    C = len(cbins)
    rng = np.random.default_rng(h * 131 + w + C)
    img = rng.integers(0, 256, size=(h, w, C), dtype=np.uint8)
    ref = oracle.integral_histogram_joint(img, cbins)
    with ihist.Plan(h, w, layout=0, bins_per_channel=cbins) as plan:
        assert ihist.ihist_plan_channels(plan.handle) == C
        assert_same(compute(plan, img), ref, "joint %s %dx%d" % (cbins, h, w))


@pytest.mark.parametrize("tune", [None, {"bins_per_cta": 8}])
def test_joint_pixel_major_and_padded_pitch(tune):
    h, w, cbins = 90, 500, [4, 4, 4]
    rng = np.random.default_rng(8)
    img = rng.integers(0, 256, size=(h, w, 3), dtype=np.uint8)
    ref = oracle.integral_histogram_joint(img, cbins)
    with ihist.Plan(h, w, layout=1, tune=tune, bins_per_channel=cbins) as plan:
        assert_same(compute(plan, img), to_layout(ref, 1), "joint pixel-major")
    with ihist.Plan(h, w, layout=0, tune=tune, bins_per_channel=cbins) as plan:
        buf = torch.zeros((h, w * 3 + 5), dtype=torch.uint8, device="cuda")
        buf[:, :w * 3].copy_(torch.from_numpy(img.reshape(h, w * 3)))
        out = torch.empty(plan.out_shape, dtype=torch.int32, device="cuda")
        ihist.ihist_compute(plan.handle, buf.data_ptr(), buf.stride(0), out.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
        assert plan.status() == ihist.IHIST_OK
        assert_same(u32(out).reshape(plan.out_shape), ref, "joint padded pitch")


def test_joint_1080p_rgb_with_queries_and_sequence():
    h, w, cbins = 1080, 1920, [4, 4, 4]
    frames = [np.stack([synth.gradient_frame(300 + 3 * i + c, h, w) for c in range(3)], axis=2) for i in range(3)]
    rects = synth.rects(21, 200, h, w)
    with ihist.Plan(h, w, layout=0, bins_per_channel=cbins) as plan:
        ref0 = oracle.integral_histogram_joint(frames[0], cbins)
        d = torch.from_numpy(frames[0]).cuda()
        hist = plan.compute(d)
        q = plan.query(hist, torch.from_numpy(rects).cuda())
        assert plan.status() == ihist.IHIST_OK
        assert_same(u32(hist).reshape(plan.out_shape), ref0, "joint 1080p")
        assert_same(u32(q), oracle.query(ref0, rects), "joint 1080p queries")
        # host sequence pipeline over three RGB frames
        hf = torch.from_numpy(np.stack(frames)).pin_memory()
        slots = torch.empty((2, h, w, 3), dtype=torch.uint8, device="cuda")
        outs = torch.empty((3,) + plan.out_shape, dtype=torch.int32, device="cuda")
        dq = torch.empty((200, 64), dtype=torch.int32, device="cuda")
        hq = torch.empty((3, 200, 64), dtype=torch.int32).pin_memory()
        d_rects = torch.from_numpy(rects).cuda()
        copy = torch.cuda.Stream()
        s = torch.cuda.current_stream()
        ihist.ihist_sequence_host(plan.handle, hf.data_ptr(), h * w * 3, 3, slots.data_ptr(), outs.data_ptr(), 3,
                                  d_rects.data_ptr(), 200, dq.data_ptr(), hq.data_ptr(), s.cuda_stream,
                                  copy.cuda_stream)
        torch.cuda.synchronize()
        assert plan.status() == ihist.IHIST_OK
        for i in range(3):
            ref = ref0 if i == 0 else oracle.integral_histogram_joint(frames[i], cbins)
            assert_same(u32(outs[i]).reshape(plan.out_shape), ref, "sequence frame %d" % i)
            assert_same(hq[i].numpy().view(np.uint32), oracle.query(ref, rects), "sequence queries %d" % i)
