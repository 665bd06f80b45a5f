"""Overlapped launches (programmatic dependent launch): every scan and
query may start while the kernel before it finishes; by default a scan
waits for it before reading its frame, with tune "overlap": 1 only before
its first store, so back-to-back computes of one plan run at the same time.  Results must still equal
the oracle word for word: across many launches (both control-block
parities), interleaved with queries and other kernels on the stream, in a
captured graph, after a launch that timed out, and in the host-frame
sequence (which always overlaps)."""
import ctypes

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


def assert_same(got, ref, what):
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        i = tuple(bad[0])
        raise AssertionError("%s: %d words differ, first at %s: got %d want %d"
                             % (what, len(bad), i, got[i], ref[i]))


def to_layout(ref, layout):
    return ref if layout == ihist.IHIST_BIN_MAJOR else np.ascontiguousarray(ref.transpose(1, 2, 0))


def test_tune_reports_overlap_and_rejects_bad_values():
    with ihist.Plan(64, 256, 8, tune={"overlap": 1}) as plan:
        assert ihist.ihist_plan_get_tune(plan.handle)["overlap"] == 1
    with ihist.Plan(64, 256, 8) as plan:
        assert ihist.ihist_plan_get_tune(plan.handle)["overlap"] == 0
    lib = ihist.load()
    t = ihist._tune_struct({"overlap": 2})
    hp = ctypes.c_void_p()
    assert lib.ihist_plan_tuned(64, 256, 8, 0, ctypes.byref(t), ctypes.byref(hp)) == ihist.IHIST_ERR_INVALID_ARG


@pytest.mark.parametrize("h,w,nbins,layout,tune", [
    (1080, 1920, 64, 0, {}),
    (333, 517, 20, 0, {"rows_per_band": 8}),
    (480, 640, 32, 1, {}),
    (97, 130, 5, 0, {"rows_per_band": 3, "ctas_per_sm": 1}),
    (130, 3000, 16, 0, {"chunks_per_warp": 1}),  # two width segments per band
    (300, 1920, 64, 1, {"bins_per_cta": 16, "groups_per_cta": 4, "chunks_per_warp": 1}),  # whole records
])
def test_back_to_back_launches_equal_the_oracle(h, w, nbins, layout, tune):
    # 9 launches: both control blocks several times, distinct frames, a ring
    # of three outputs (so launch i+3 overwrites what launch i wrote)
    n = 9
    imgs = [synth.uniform_frame(300 + k, h, w) if k % 2 else synth.gradient_frame(300 + k, h, w)
            for k in range(3)]
    refs = [to_layout(oracle.integral_histogram(img, nbins), layout) for img in imgs]
    d_imgs = [torch.from_numpy(img).cuda() for img in imgs]
    with ihist.Plan(h, w, nbins, layout, tune=dict(tune, overlap=1)) as plan:
        outs = [plan.empty_output() for _ in range(3)]
        for o in outs:
            o.fill_(-1)
        for k in range(n):
            plan.compute(d_imgs[k % 3], outs[k % 3])
        torch.cuda.synchronize()
        assert plan.status() == ihist.IHIST_OK
        for k in range(3):
            assert_same(u32(outs[k]).reshape(plan.out_shape), refs[k], "output %d" % k)
        # the same output buffer every launch, a fill kernel in between
        for k in range(5):
            outs[0].fill_(-1)
            plan.compute(d_imgs[k % 3], outs[0])
        torch.cuda.synchronize()
        assert_same(u32(outs[0]).reshape(plan.out_shape), refs[4 % 3], "reused output")


def test_interleaved_queries_and_sequence():
    h, w, nbins = 270, 480, 16
    imgs = [synth.uniform_frame(400 + k, h, w) for k in range(4)]
    rects = synth.rects(401, 300, h, w)
    d_rects = torch.from_numpy(rects).cuda()
    with ihist.Plan(h, w, nbins, tune={"overlap": 1}) as plan:
        out = plan.empty_output()
        rows = []
        for img in imgs:
            plan.compute(torch.from_numpy(img).cuda(), out)
            rows.append(plan.query(out, d_rects))
        torch.cuda.synchronize()
        assert plan.status() == ihist.IHIST_OK
        for img, r in zip(imgs, rows):
            assert np.array_equal(u32(r), oracle.query(oracle.integral_histogram(img, nbins), rects))


def test_graph_capture_of_overlapped_launches():
    h, w, nbins = 200, 700, 24
    imgs = [synth.uniform_frame(500 + k, h, w) for k in range(3)]
    refs = [oracle.integral_histogram(img, nbins) for img in imgs]
    d_imgs = [torch.from_numpy(img).cuda() for img in imgs]
    with ihist.Plan(h, w, nbins, tune={"overlap": 1, "rows_per_band": 12}) as plan:
        outs = [plan.empty_output() for _ in range(3)]
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            for k in range(3):
                plan.compute(d_imgs[k], outs[k], stream=s)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for k in range(3):
                plan.compute(d_imgs[k], outs[k], stream=s)
        for _ in range(3):
            for o in outs:
                o.fill_(-1)
            g.replay()
            torch.cuda.synchronize()
            for k in range(3):
                assert_same(u32(outs[k]).reshape(plan.out_shape), refs[k], "replay %d" % k)
        assert plan.status() == ihist.IHIST_OK


def test_timeout_is_reported_from_either_launch_parity_and_plan_recovers():
    h, w, nbins = 64, 256, 8
    img = synth.uniform_frame(600, h, w)
    ref = oracle.integral_histogram(img, nbins)
    d_img = torch.from_numpy(img).cuda()
    tune = {"rows_per_band": 8, "fault_skip_band": 3, "timeout_us": 20000, "overlap": 1}
    with ihist.Plan(h, w, nbins, tune=tune) as plan:
        for launches in (1, 2):  # the second launch uses the other control block
            for _ in range(launches):
                plan.compute(d_img)
            torch.cuda.synchronize()
            assert plan.status() == ihist.IHIST_ERR_LOOKBACK_TIMEOUT
            assert plan.status() == ihist.IHIST_OK  # reading clears it
    with ihist.Plan(h, w, nbins, tune={"rows_per_band": 8, "overlap": 1}) as plan:
        out = plan.empty_output()
        for _ in range(4):
            out.fill_(-1)
            plan.compute(d_img, out)
        torch.cuda.synchronize()
        assert plan.status() == ihist.IHIST_OK
        assert_same(u32(out).reshape(plan.out_shape), ref, "after recovery")


def test_joint_and_table_plans_with_overlap():
    h, w = 150, 300
    rgb = np.stack([synth.uniform_frame(700 + c, h, w) for c in range(3)], axis=2)
    ref = oracle.integral_histogram_joint(rgb, [4, 2, 3])
    edges = [0, 10, 50, 51, 200, 256]
    img = synth.gradient_frame(710, h, w)
    ref_e = oracle.integral_histogram_edges(img, edges)
    with ihist.Plan(h, w, bins_per_channel=[4, 2, 3], tune={"overlap": 1}) as jp, \
            ihist.Plan(h, w, edges=edges, tune={"overlap": 1}) as ep:
        d_rgb = torch.from_numpy(np.ascontiguousarray(rgb)).cuda()
        d_img = torch.from_numpy(img).cuda()
        for _ in range(3):
            hj = jp.compute(d_rgb)
            he = ep.compute(d_img)
        torch.cuda.synchronize()
        assert jp.status() == ihist.IHIST_OK and ep.status() == ihist.IHIST_OK
        assert_same(u32(hj).reshape(jp.out_shape), ref, "joint")
        assert_same(u32(he).reshape(ep.out_shape), ref_e, "edges")


def test_default_launch_is_safe_when_the_kernel_before_writes_the_frame():
    # without overlap=1 a scan reads nothing of its frame before the kernel
    # launched just before it completed, so a kernel that writes the frame
    # right before ihist_compute is fine (and so is one that writes the
    # rectangles right before ihist_query)
    h, w, nbins = 1080, 1920, 16
    base = synth.gradient_frame(800, h, w)
    rects = synth.rects(801, 500, h, w)
    d = torch.from_numpy(base).cuda()
    d_r = torch.from_numpy(rects).cuda()
    d_r2 = torch.empty_like(d_r)
    with ihist.Plan(h, w, nbins) as plan:
        out = plan.empty_output()
        for key in (0x5a, 0x33, 0xff, 0x01):
            frame = torch.bitwise_xor(d, key)  # an elementwise kernel writes the frame ...
            plan.compute(frame, out)           # ... and the scan is launched right after it
            d_r2.copy_(d_r.flip(0))            # a kernel writes the rectangles right before the query
            rows = plan.query(out, d_r2)
            torch.cuda.synchronize()
            img = base ^ key
            ref = oracle.integral_histogram(img, nbins)
            assert_same(u32(out).reshape(plan.out_shape), ref, "frame xor %#x" % key)
            assert np.array_equal(u32(rows), oracle.query(ref, np.ascontiguousarray(rects[::-1])))
        assert plan.status() == ihist.IHIST_OK


def test_sequence_pipeline_rows_and_histograms_after_syncing_the_compute_stream():
    # 9 host frames through the 2-slot ring, 3 outputs in rotation, 200 rects
    # per frame; only the compute stream is synchronised before reading
    h, w, nbins, n, nrects = 180, 300, 16, 9, 200
    frames = np.stack([synth.uniform_frame(1600 + i, h, w) for i in range(n)])
    rects = synth.rects(1601, nrects, h, w)
    hf = torch.from_numpy(frames).pin_memory()
    slots = torch.empty((2, h, w), dtype=torch.uint8, device="cuda")
    d_rects = torch.from_numpy(rects).cuda()
    dq = torch.empty((nrects, nbins), dtype=torch.int32, device="cuda")
    hq = torch.zeros((n, nrects, nbins), dtype=torch.int32).pin_memory()
    s, copy = torch.cuda.Stream(), torch.cuda.Stream()
    with ihist.Plan(h, w, nbins) as plan:
        outs = torch.empty((3,) + plan.out_shape, dtype=torch.int32, device="cuda")
        for _ in range(2):  # the plan's events and control blocks are reused by a second call
            hq.zero_()
            ihist.ihist_sequence_host(plan.handle, hf.data_ptr(), h * w, n, slots.data_ptr(), outs.data_ptr(), 3,
                                      d_rects.data_ptr(), nrects, dq.data_ptr(), hq.data_ptr(), s.cuda_stream,
                                      copy.cuda_stream)
            s.synchronize()
            for i in range(n):
                ref = oracle.integral_histogram(frames[i], nbins)
                assert np.array_equal(hq[i].numpy().view(np.uint32), oracle.query(ref, rects)), i
            for i in range(n - 3, n):  # the last frame written to each output
                assert_same(u32(outs[i % 3]), oracle.integral_histogram(frames[i], nbins), "output of frame %d" % i)
        assert plan.status() == ihist.IHIST_OK
