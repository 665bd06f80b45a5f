"""Autotuner search and cache logic on the CPU (injected timer)."""
import json

from paper_1711_01919_gb300 import autotune, ihist


def test_candidates_respect_warp_limit():
    for (h, w, b) in [(1080, 1920, 64), (8192, 8192, 128), (240, 320, 16), (5, 3, 2)]:
        cands = autotune.plan_candidates(h, w, b)
        assert cands[0] == {}
        nchunks = -(-w // 128)
        for t in cands[1:]:
            wpg = -(-nchunks // t["chunks_per_warp"])
            assert wpg * t["groups_per_cta"] <= 16 or t["groups_per_cta"] == 1
            assert wpg <= 16
            assert t.get("rows_per_band", 0) <= h


def test_search_picks_fastest_and_skips_rejected(tmp_path, monkeypatch):
    monkeypatch.setenv("IHIST_TUNE_CACHE", str(tmp_path / "c.json"))
    calls = []

    def timer(t):
        calls.append(t)
        if t.get("bins_per_cta") == 8:
            raise ihist.IhistError(ihist.IHIST_ERR_UNSUPPORTED, "plan")
        return 1.0 / (1 + t.get("rows_per_band", 0)) + 0.01 * t.get("chunks_per_warp", 1)

    best = autotune.tune_plan(1080, 1920, 64, timer=timer, device="fake")
    assert best["rows_per_band"] == 64 and best["bins_per_cta"] == 4 and best["chunks_per_warp"] == 1
    cache = json.load(open(tmp_path / "c.json"))
    assert "plan|fake|1080x1920x64|0" in cache
    # second call is served from the cache: the timer is not called again
    n = len(calls)
    assert autotune.tune_plan(1080, 1920, 64, timer=timer, device="fake") == best
    assert len(calls) == n


def test_batch_tuning_key_and_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("IHIST_TUNE_CACHE", str(tmp_path / "c.json"))
    shapes = [(240, 320, 16, 0), (1080, 1920, 64, 0), (240, 320, 16, 0)]
    def timer(t):
        if t.get("warps_per_cta") == 8 and t.get("rows_per_band") == 56:
            raise ihist.IhistError(ihist.IHIST_ERR_UNSUPPORTED, "batch")
        return (abs(t.get("rows_per_band", 0) - 40) + 0.5 * (t.get("bins_per_cta", 4) == 8)
                + 0.25 * (t.get("warps_per_cta", 16) == 16))

    best = autotune.tune_batch(shapes, timer=timer, device="fake")
    assert best == {"warps_per_cta": 8, "bins_per_cta": 4, "rows_per_band": 40}
    cache = json.load(open(tmp_path / "c.json"))
    assert any(k.startswith("batch|fake|3|") for k in cache)


def test_choose_layout():
    assert autotune.choose_layout(10, 10, 4, timer=lambda l: 2.0 if l == 0 else 1.0) == ihist.IHIST_PIXEL_MAJOR
    assert autotune.choose_layout(10, 10, 4, timer=lambda l: 1.0 if l == 0 else 2.0) == ihist.IHIST_BIN_MAJOR


def test_batch_candidates_add_16_bin_groups_for_pixel_major():
    bm = autotune.batch_candidates([(240, 320, 16, 0)])
    pm = autotune.batch_candidates([(240, 320, 16, 0), (480, 640, 32, 1)])
    assert bm[0] == {} and pm[0] == {}
    assert not any(t.get("bins_per_cta") == 16 for t in bm)
    assert any(t.get("bins_per_cta") == 16 for t in pm)
    assert len(pm) > len(bm)


def test_table_batches_never_try_16_bin_groups():
    pm = autotune.batch_candidates([(240, 320, 16, 0), (480, 640, 32, 1)], tables=True)
    assert pm[0] == {}
    assert not any(t.get("bins_per_cta") == 16 for t in pm)


def test_batch_layout_takes_the_faster_layout_with_its_own_launch_shape(tmp_path, monkeypatch):
    monkeypatch.setenv("IHIST_TUNE_CACHE", str(tmp_path / "cache.json"))
    shapes = [(240, 320, 16), (1080, 1920, 64)]
    seen = []

    def timer(sh, tune, queries):
        layout = sh[0][3]
        assert all(s[3] == layout for s in sh)
        seen.append((layout, queries))
        # pixel-major: slower to compute, faster to query
        base = 5.0 if layout == ihist.IHIST_BIN_MAJOR else 8.0
        per_query = 0.004 if layout == ihist.IHIST_BIN_MAJOR else 0.001
        return base + per_query * queries + (0.0 if tune == {} else 0.5)

    layout, tune, times = autotune.tune_batch_layout(shapes, 0, timer=timer, device="fake")
    assert layout == ihist.IHIST_BIN_MAJOR and tune == {}
    assert times[ihist.IHIST_BIN_MAJOR] == 5.0 and times[ihist.IHIST_PIXEL_MAJOR] == 8.0
    layout, tune, times = autotune.tune_batch_layout(shapes, 2000, timer=timer, device="fake")
    assert layout == ihist.IHIST_PIXEL_MAJOR  # 8 + 2 < 5 + 8
    assert (ihist.IHIST_PIXEL_MAJOR, 2000) in seen
