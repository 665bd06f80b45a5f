"""Served results against the oracle and against results computed alone,
word for word: each frame's resident histogram (Eq. 1, Algorithm 1), each
query's rows (Eq. 2) and each search's best window, in the batched
(continuous batching) and the plain server, with small pools of distinct
frames."""
import numpy as np
import pytest

import oracle
from paper_1711_01919_gb300 import ihist, serve, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1711_01919_gb300 import build as cuda_build
    cuda_build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run_server(mode, duration=0.04, budget_gb=40.0, saturate=False, nslots=16, max_batch=16):
    seed = synth.workload_seed(4)
    pool = {}
    for (w, h) in synth.BATCH_RESOLUTIONS:
        pool[(h, w)] = [torch.from_numpy(synth.uniform_frame(seed + 7 * k + w, h, w)).pin_memory() for k in range(3)]
    reqs = serve.serving_workload(seed, duration, 2000.0, 200.0, 500, pool, search_rate=300.0)
    if saturate:
        for r in reqs:
            r.t_arrival = 0.0
    ex = serve.GpuExecutor(mode, nslots=nslots, trace=True)  # NVTX ranges must not disturb anything
    ex.warm(sorted({(r.h, r.w, r.nbins) for r in reqs if isinstance(r, serve.FrameRequest)}))
    srv = serve.Server(ex, int(budget_gb * (1 << 30)), max_batch=max_batch, mode=mode)
    ex.start()
    srv.run(reqs, ex.clock)
    torch.cuda.synchronize()
    return srv, ex, reqs


def check_alone(srv, reqs):
    frames = {r.rid: r for r in reqs if isinstance(r, serve.FrameRequest)}
    alone = {}
    plans = {}
    for rid in srv.store.resident():
        r = frames[rid]
        key = (r.h, r.w, r.nbins)
        if key not in plans:
            plans[key] = ihist.Plan(*key)
        ref = plans[key].compute(r.frame.cuda())
        hist = srv.store.payload(rid)[0]
        assert torch.equal(hist, ref), "frame %d differs from its histogram computed alone" % rid
        alone[rid] = ref
    nq = 0
    for q in reqs:
        if isinstance(q, serve.QueryRequest) and q.rid in srv.results and q.target in alone:
            r = frames[q.target]
            d_rects = torch.from_numpy(np.ascontiguousarray(q.rects)).cuda()
            ref = plans[(r.h, r.w, r.nbins)].query(alone[q.target], d_rects)
            assert torch.equal(srv.results[q.rid], ref.cpu()), "query %d differs" % q.rid
            nq += 1
        if isinstance(q, serve.SearchRequest) and q.rid in srv.results and q.target in alone:
            r = frames[q.target]
            plan = plans[(r.h, r.w, r.nbins)]
            rect = torch.tensor([[q.x, q.y, q.x + q.win_w - 1, q.y + q.win_h - 1]], dtype=torch.int32, device="cuda")
            target = plan.query(alone[q.target], rect)[0].contiguous()
            ref = plan.window_best(alone[q.target], target, q.win_h, q.win_w, q.stride)
            nx = ihist.window_grid(r.h, r.w, q.win_h, q.win_w, q.stride)[1]
            assert serve.decode_best(int(srv.results[q.rid].item()), nx) == ref, "search %d differs" % q.rid
            assert ref[0] == q.win_h * q.win_w  # the patch itself matches fully
            nq += 1
    for p in plans.values():
        p.close()
    return nq


def check_oracle(srv, reqs):
    """Every resident histogram, query row and search answer against the
    oracle computed from the request's own host frame.  Frames of the pool
    repeat, so the oracle runs once per (frame, bin count)."""
    frames = {r.rid: r for r in reqs if isinstance(r, serve.FrameRequest)}
    groups = {}
    for rid in srv.store.resident():
        r = frames[rid]
        groups.setdefault((id(r.frame), r.nbins), []).append(rid)
    nq = 0
    for (_, nbins), rids in groups.items():
        img = frames[rids[0]].frame.numpy()
        ref = oracle.integral_histogram(img, nbins)
        for rid in rids:
            got = srv.store.payload(rid)[0].cpu().numpy().view(np.uint32).reshape(ref.shape)
            assert np.array_equal(got, ref), "frame %d differs from the oracle" % rid
        for q in reqs:
            if q.rid not in srv.results or getattr(q, "target", None) not in rids:
                continue
            if isinstance(q, serve.QueryRequest):
                want = oracle.query(ref, np.ascontiguousarray(q.rects))
                got = srv.results[q.rid].numpy().view(np.uint32).reshape(want.shape)
                assert np.array_equal(got, want), "query %d differs from the oracle" % q.rid
                nq += 1
            elif isinstance(q, serve.SearchRequest):
                rect = np.array([[q.x, q.y, q.x + q.win_w - 1, q.y + q.win_h - 1]], dtype=np.int32)
                target = oracle.query(ref, rect)[0]
                scores = oracle.window_intersection(img, nbins, target, q.win_h, q.win_w, q.stride)
                i = int(np.argmax(scores))
                nx = scores.shape[1]
                assert serve.decode_best(int(srv.results[q.rid].item()), nx) == (int(scores.flat[i]), i // nx, i % nx), \
                    "search %d differs from the oracle" % q.rid
                nq += 1
    return nq


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_served_results_equal_alone(mode):
    srv, ex, reqs = run_server(mode)
    done = srv.done
    assert len(done) == len(reqs)
    assert all(d.status == "ok" for d in done if d.kind == "frame")
    # a query is refused only if it came before any histogram was complete
    first_ready = min(d.t_done for d in done if d.kind == "frame")
    assert all(d.status == "ok" or d.t_arrival < first_ready for d in done if d.kind == "query")
    nq = check_alone(srv, reqs)
    assert nq >= 3
    assert check_oracle(srv, reqs) == nq
    ex.close()


def test_batched_server_under_a_small_budget_evicts_and_stays_exact():
    srv, ex, reqs = run_server("batched", duration=0.04, budget_gb=1.0, saturate=True)
    assert srv.store.evicted > 0
    assert srv.store.used <= 1 << 30
    assert all(d.status == "ok" for d in srv.done if d.kind == "frame")
    assert check_alone(srv, reqs) == check_oracle(srv, reqs)
    ex.close()


def test_serving_configuration_saturated_stays_exact():
    # the bench's server shape (128-frame slots, launches of up to 128
    # frames from a ring of batches, the hold rule) with 0.2 s of requests
    # all arriving at once: several large shared launches, evictions under
    # the 40 GB budget, every resident histogram and query row exact
    srv, ex, reqs = run_server("batched", duration=0.2, saturate=True, nslots=128, max_batch=128)
    assert all(d.status == "ok" for d in srv.done if d.kind == "frame")
    sizes = {int(k): v for k, v in srv.report(1.0)["launch_sizes"].items()}
    assert max(sizes) >= 64 and sum(v for k, v in sizes.items() if k >= 8) >= 2
    assert check_alone(srv, reqs) == check_oracle(srv, reqs)
    ex.close()
