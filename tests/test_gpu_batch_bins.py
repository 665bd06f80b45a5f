"""Batches with other bin structures: frames that bin through their own
value -> bin table (bins by edges, arbitrary maps, values in no bin) next to
uniform-bin frames in one persistent launch.  Every frame equals the
oracle's mapped integral histogram word for word."""
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


def random_table(seed, nbins):
    """Any value -> bin map; about a tenth of the values in no bin."""
    rng = np.random.default_rng(seed)
    t = rng.integers(0, nbins, 256)
    t[rng.random(256) < 0.1] = -1
    return [int(v) for v in t]


def reference(img, nbins, table, layout):
    if table is None:
        ref = oracle.integral_histogram(img, nbins)
    else:
        ref = oracle.integral_histogram_mapped(img, np.asarray(table, dtype=np.int32), nbins)
    if layout == 2:
        b, h, w = ref.shape
        return np.ascontiguousarray(ref.reshape(b // 4, 4, h, w).transpose(0, 2, 3, 1))
    return ref if layout == 0 else np.ascontiguousarray(ref.transpose(1, 2, 0))


def check(batch, imgs, nbins, tables, layouts):
    for i, (img, b, t, l) in enumerate(zip(imgs, nbins, tables, layouts)):
        got = u32(batch.outs[i]).reshape(ihist.out_shape(img.shape[0], img.shape[1], b, l))
        ref = reference(img, b, t, l)
        assert np.array_equal(got, ref), "frame %d (%dx%d B=%d layout %d table %s): %d words differ" % (
            i, img.shape[0], img.shape[1], b, l, t is not None, int((got != ref).sum()))


CASES = [(1, 1, 3, 0), (37, 131, 16, 0), (240, 320, 16, 1), (480, 640, 32, 0), (64, 257, 7, 1),
         (720, 1280, 64, 0), (33, 2049, 100, 0), (17, 128, 256, 1), (200, 700, 5, 0), (90, 333, 12, 2),
         (240, 320, 64, 2)]


def frames_and_tables(seed, cases):
    imgs = [synth.uniform_frame(seed + i, h, w) if i % 2 else synth.gradient_frame(seed + i, h, w)
            for i, (h, w, b, l) in enumerate(cases)]
    nbins = [b for (h, w, b, l) in cases]
    layouts = [l for (h, w, b, l) in cases]
    tables = []
    for i, b in enumerate(nbins):
        if i % 3 == 1:
            tables.append(None)  # uniform bins
        elif i % 3 == 2:
            edges = sorted(set([0, 256] + [int(e) for e in np.linspace(7, 250, b - 1)]))
            tables.append(ihist.edges_table(edges) if len(edges) == b + 1 else random_table(seed + i, b))
        else:
            tables.append(random_table(seed + i, b))
    return imgs, nbins, layouts, tables


@pytest.mark.parametrize("tune", [None, {"rows_per_band": 8}, {"bins_per_cta": 8},
                                  {"warps_per_cta": 16, "rows_per_band": 5}, {"rows_per_band": 3, "ctas_per_sm": 1}])
def test_tables_and_uniform_frames_in_one_batch(tune):
    imgs, nbins, layouts, tables = frames_and_tables(900, CASES)
    with ihist.Batch([torch.from_numpy(x).cuda() for x in imgs], nbins, layouts, tune=tune,
                     tables=tables) as batch:
        batch.compute()
        assert batch.status() == ihist.IHIST_OK
        check(batch, imgs, nbins, tables, layouts)


def test_edges_batch_equals_edges_plans():
    edges = [0, 16, 64, 128, 129, 256]
    imgs = [synth.gradient_frame(950 + i, 270, 480) for i in range(4)]
    d = [torch.from_numpy(x).cuda() for x in imgs]
    with ihist.Batch(d, 5, tables=[ihist.edges_table(edges)] * 4) as batch:
        batch.compute()
        assert batch.status() == ihist.IHIST_OK
        with ihist.Plan(270, 480, edges=edges) as plan:
            for i in range(4):
                assert torch.equal(plan.compute(d[i]), batch.outs[i])
        for i in range(4):
            got = u32(batch.outs[i]).reshape(5, 270, 480)
            assert np.array_equal(got, oracle.integral_histogram_edges(imgs[i], edges))


def test_set_io_rebinds_tables_and_graph_replay():
    imgs, nbins, layouts, tables = frames_and_tables(970, CASES[:6])
    imgs2, _, _, tables2 = frames_and_tables(980, CASES[:6])
    tables2 = [random_table(990 + i, b) for i, b in enumerate(nbins)]
    with ihist.Batch([torch.from_numpy(x).cuda() for x in imgs], nbins, layouts, tables=tables) as batch:
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
            check(batch, imgs, nbins, tables, layouts)
        outs2 = [torch.empty_like(o) for o in batch.outs]
        batch.set_io([torch.from_numpy(x).cuda() for x in imgs2], outs2, tables=tables2)
        batch.compute()
        torch.cuda.synchronize()
        assert batch.status() == ihist.IHIST_OK
        check(batch, imgs2, nbins, tables2, layouts)
        # the same slots back to uniform bins
        batch.set_io([torch.from_numpy(x).cuda() for x in imgs2], outs2)
        batch.compute()
        torch.cuda.synchronize()
        check(batch, imgs2, nbins, [None] * len(nbins), layouts)


def test_tables_need_a_table_batch_and_small_bin_groups():
    imgs = [synth.uniform_frame(5 + i, 64, 256) for i in range(2)]
    d = [torch.from_numpy(x).cuda() for x in imgs]
    t = random_table(3, 16)
    with ihist.Batch(d, 16) as batch:  # planned without tables
        with pytest.raises(ihist.IhistError) as e:
            batch.set_io(d, batch.outs, tables=[t, None])
        assert e.value.code == ihist.IHIST_ERR_UNSUPPORTED
    with pytest.raises(ihist.IhistError) as e:
        ihist.Batch(d, 16, tune={"bins_per_cta": 16}, tables=[t, t])
    assert e.value.code == ihist.IHIST_ERR_UNSUPPORTED
    with ihist.Batch(d, 16, [1, 1], tables=[t, t]) as batch:  # pixel-major tables: 8 bins per CTA
        assert batch.tune["bins_per_cta"] == 8
        batch.compute()
        assert batch.status() == ihist.IHIST_OK
        check(batch, imgs, [16, 16], [t, t], [1, 1])


def test_upload_compute_with_tables():
    imgs, nbins, layouts, tables = frames_and_tables(1100, CASES[1:5])
    h = [torch.from_numpy(x).pin_memory() for x in imgs]
    d = [torch.empty_like(x, device="cuda") for x in h]
    with ihist.Batch(d, nbins, layouts, tables=tables) as batch:
        s, cs = torch.cuda.Stream(), torch.cuda.Stream()
        batch.upload_compute(h, stream=s, copy_stream=cs)
        torch.cuda.synchronize()
        assert batch.status() == ihist.IHIST_OK
        check(batch, imgs, nbins, tables, layouts)


def joint_frame(seed, h, w, c):
    return np.ascontiguousarray(np.stack([synth.uniform_frame(seed + k, h, w) for k in range(c)], axis=2))


JOINT_CASES = [  # (h, w, bins per channel, layout)
    (150, 300, [4, 4, 4], 0), (64, 257, [8, 2], 1), (37, 131, [2, 2, 2, 2], 0), (240, 320, [16, 16], 0),
    (1, 5, [3, 5], 1), (200, 700, [5], None), (120, 250, [4, 2, 2], 2)]


@pytest.mark.parametrize("with_tables", [False, True])
def test_joint_frames_next_to_uniform_and_table_frames(with_tables):
    frames, nbins, layouts, tables, joint, refs = [], [], [], [], [], []
    for i, (h, w, bins, l) in enumerate(JOINT_CASES):
        if l is None:  # a one-channel frame between the joint ones
            img = synth.gradient_frame(1200 + i, h, w)
            t = random_table(1200 + i, bins[0]) if with_tables else None
            frames.append(img), nbins.append(bins[0]), layouts.append(0), tables.append(t), joint.append(None)
            refs.append(reference(img, bins[0], t, 0))
            continue
        img = joint_frame(1200 + 10 * i, h, w, len(bins))
        nb = int(np.prod(bins))
        frames.append(img), nbins.append(nb), layouts.append(l), tables.append(None), joint.append(bins)
        ref = oracle.integral_histogram_joint(img, bins)
        if l == 2:
            refs.append(np.ascontiguousarray(ref.reshape(nb // 4, 4, h, w).transpose(0, 2, 3, 1)))
        else:
            refs.append(ref if l == 0 else np.ascontiguousarray(ref.transpose(1, 2, 0)))
    with ihist.Batch([torch.from_numpy(x).cuda() for x in frames], nbins, layouts, tables=tables,
                     joint=joint) as batch:
        for _ in range(2):  # the joint-bin planes are recomputed each launch
            batch.compute()
        assert batch.status() == ihist.IHIST_OK
        for i, (img, b, l) in enumerate(zip(frames, nbins, layouts)):
            got = u32(batch.outs[i]).reshape(ihist.out_shape(img.shape[0], img.shape[1], b, l))
            assert np.array_equal(got, refs[i]), "frame %d" % i
        # joint frames computed alone through joint plans give the same words
        h, w, bins, l = JOINT_CASES[0]
        with ihist.Plan(h, w, bins_per_channel=bins) as plan:
            assert torch.equal(plan.compute(torch.from_numpy(frames[0]).cuda()), batch.outs[0])


def test_joint_frames_rebind_and_upload():
    shapes = [(120, 400, [4, 4, 4]), (90, 640, [8, 4])]
    imgs = [joint_frame(1300 + 10 * i, h, w, len(b)) for i, (h, w, b) in enumerate(shapes)]
    nbins = [int(np.prod(b)) for (h, w, b) in shapes]
    joint = [b for (h, w, b) in shapes]
    d = [torch.from_numpy(x).cuda() for x in imgs]
    with ihist.Batch(d, nbins, joint=joint) as batch:
        # new joint frames of the same shapes, uploaded from pinned host memory
        imgs2 = [joint_frame(1400 + 10 * i, h, w, len(b)) for i, (h, w, b) in enumerate(shapes)]
        batch.set_io(d, batch.outs, nbins=nbins, joint=joint)
        s, cs = torch.cuda.Stream(), torch.cuda.Stream()
        batch.upload_compute([torch.from_numpy(x).pin_memory() for x in imgs2], stream=s, copy_stream=cs)
        torch.cuda.synchronize()
        assert batch.status() == ihist.IHIST_OK
        for i, (h, w, b) in enumerate(shapes):
            got = u32(batch.outs[i]).reshape(nbins[i], h, w)
            assert np.array_equal(got, oracle.integral_histogram_joint(imgs2[i], b)), "frame %d" % i
        # a slot planned for a one-channel frame has no joint-bin plane
    with ihist.Batch([torch.from_numpy(synth.uniform_frame(5, 64, 256)).cuda()], [16]) as batch:
        with pytest.raises(ihist.IhistError) as e:
            batch.set_io([torch.from_numpy(joint_frame(6, 64, 256, 2)).cuda()], batch.outs, nbins=[16],
                         joint=[[4, 4]])
        assert e.value.code == ihist.IHIST_ERR_UNSUPPORTED
