"""Pins for the CPU oracle: checks against what the paper and mathematics fix.

Every check takes an ``oracle.Oracle`` so the same suite runs on the oracle as
committed (test_oracle_pins.py) and on deliberately mutated builds of it
(test_oracle_mutations.py), where at least one check must fail.

The checks never re-call the oracle's own formula to produce an expected
value.  Expected values come from:
  * hand-worked fixtures in tests/golden/ (Eq. 1 and Eq. 2 worked by hand);
  * brute-force counting in pure Python on tiny frames (Eq. 1 as a count);
  * invariants that hold for any image: sum over bins = (x+1)(y+1),
    bottom-right = numpy.bincount of the binned image, monotonicity;
  * closed forms: constant frame, column ramp, row ramp, single bright pixel;
  * special cases of the binning: power-of-two B is a right shift, every
    bin is a contiguous run of width floor(256/B) or ceil(256/B).

Other bin structures (edges, any value -> bin map) and joint multi-channel
bins are pinned the same way: hand-worked fixtures, numpy's binary search
(``searchsorted``) as an independent bin lookup, brute-force counting,
reduction to the pinned uniform case, and marginals of the joint histogram
that must equal the single-channel integral histograms.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def in_bin(v: int, b: int, nbins: int) -> bool:
    """v in the b-th of nbins equal sub-intervals of [0, 256): b/B <= v/256 < (b+1)/B."""
    return 256 * b <= v * nbins < 256 * (b + 1)


def brute_bin(v: int, nbins: int) -> int:
    for b in range(nbins):
        if in_bin(v, b, nbins):
            return b
    raise AssertionError("no bin for %d" % v)


def binned(img: np.ndarray, nbins: int) -> np.ndarray:
    table = np.array([brute_bin(v, nbins) for v in range(256)], dtype=np.int64)
    return table[img]


def brute_integral_histogram(img: np.ndarray, nbins: int) -> np.ndarray:
    """Eq. 1 as a literal count over the rectangle [0..y] x [0..x] (tiny frames)."""
    h, w = img.shape
    bins = [[brute_bin(int(img[r, c]), nbins) for c in range(w)] for r in range(h)]
    out = np.zeros((nbins, h, w), dtype=np.uint32)
    for y in range(h):
        for x in range(w):
            counts = [0] * nbins
            for r in range(y + 1):
                for c in range(x + 1):
                    counts[bins[r][c]] += 1
            for b in range(nbins):
                out[b, y, x] = counts[b]
    return out


def brute_from_bins(bins: np.ndarray, nbins: int) -> np.ndarray:
    """Eq. 1 as a literal count, given each pixel's bin (-1 = no bin)."""
    h, w = bins.shape
    out = np.zeros((nbins, h, w), dtype=np.uint32)
    for y in range(h):
        for x in range(w):
            counts = [0] * nbins
            for r in range(y + 1):
                for c in range(x + 1):
                    if bins[r, c] >= 0:
                        counts[bins[r, c]] += 1
            out[:, y, x] = counts
    return out


def edges_bin(v: int, edges) -> int:
    """Bin of v for bins [e_k, e_k+1), by numpy's binary search; -1 outside."""
    k = int(np.searchsorted(np.asarray(edges), v, side="right")) - 1
    return k if 0 <= k < len(edges) - 1 else -1


def brute_region(img: np.ndarray, nbins: int, rect) -> np.ndarray:
    x0, y0, x1, y1 = rect
    out = np.zeros(nbins, dtype=np.uint32)
    for r in range(y0, y1 + 1):
        for c in range(x0, x1 + 1):
            out[brute_bin(int(img[r, c]), nbins)] += 1
    return out


def load_golden(name: str) -> dict:
    """Parse a hand-worked fixture (see the files for the format)."""
    lines = [ln.strip() for ln in open(os.path.join(GOLDEN, name)) if ln.strip() and not ln.startswith("#")]
    d = {"planes": {}, "queries": [], "rest_zero": False}
    i = 0

    def rows(n):
        nonlocal i
        m = [list(map(int, lines[i + k].split())) for k in range(n)]
        i += n
        return np.array(m, dtype=np.int64)

    while i < len(lines):
        tok = lines[i].split()
        i += 1
        if tok[0] in ("h", "w", "bins", "channels"):
            d[tok[0]] = int(tok[1])
        elif tok[0] in ("edges", "cbins"):
            d[tok[0]] = [int(v) for v in tok[1:]]
        elif tok[0] == "image":
            d["image"] = rows(d["h"]).astype(np.uint8)
            if "channels" in d:
                d["image"] = d["image"].reshape(d["h"], d["w"], d["channels"])
        elif tok[0] == "H":
            d["planes"][int(tok[1])] = rows(d["h"])
        elif tok[0] == "rest":
            d["rest_zero"] = True
        elif tok[0] == "query":
            rect = tuple(int(v) for v in tok[1:5])
            ans = lines[i].split()
            i += 1
            exp = np.zeros(d["bins"], dtype=np.int64)
            if ans[0] == "sparse":
                for k in range(1, len(ans), 2):
                    exp[int(ans[k])] = int(ans[k + 1])
            else:
                exp[:] = list(map(int, ans))
            d["queries"].append((rect, exp))
        else:
            raise ValueError("bad fixture line: %r" % (tok,))
    return d


GOLDEN_FILES = ("ih_3x4_b2.txt", "ih_2x4_b3_edges.txt", "ih_2x2_b256.txt")
GOLDEN_EDGES = "ih_2x4_b3_edges_gap.txt"
GOLDEN_JOINT = "ih_2x2_joint_2x3x2.txt"
TINY_BINS = (1, 2, 3, 5, 8, 32, 256)


# ---------------------------------------------------------------- checks

def check_bins(o) -> None:
    """Q: uniform bins, power-of-two shift, contiguous runs, full range."""
    for nbins in range(1, 257):
        got = [o.bin_of(v, nbins) for v in range(256)]
        assert got[0] == 0 and got[255] == nbins - 1, nbins
        assert all(got[v] <= got[v + 1] <= got[v] + 1 for v in range(255)), nbins
        widths = np.bincount(np.array(got), minlength=nbins)
        assert set(widths.tolist()) <= {256 // nbins, -(-256 // nbins)}, nbins
        for v in range(256):
            assert in_bin(v, got[v], nbins), (v, nbins)
    for k in range(9):
        nbins = 1 << k
        for v in range(256):
            assert o.bin_of(v, nbins) == (v >> (8 - k)), (v, nbins)


def check_golden(o) -> None:
    for name in GOLDEN_FILES:
        d = load_golden(name)
        H = o.integral_histogram(d["image"], d["bins"]).astype(np.int64)
        for b, plane in d["planes"].items():
            assert np.array_equal(H[b], plane), (name, b)
        if d["rest_zero"]:
            others = [b for b in range(d["bins"]) if b not in d["planes"]]
            assert not H[others].any(), name
        else:
            assert sorted(d["planes"]) == list(range(d["bins"])), name
        for rect, exp in d["queries"]:
            q = o.query(H.astype(np.uint32), [rect])[0].astype(np.int64)
            assert np.array_equal(q, exp), (name, rect)
            r = o.region_brute(d["image"], d["bins"], rect).astype(np.int64)
            assert np.array_equal(r, exp), (name, rect)


def tiny_images():
    rng = np.random.default_rng(1711)
    shapes = [(1, 1), (1, 7), (6, 1), (2, 3), (5, 4), (7, 9), (12, 12), (3, 13)]
    imgs = [rng.integers(0, 256, size=s, dtype=np.uint8) for s in shapes]
    edge = np.array([[0, 255, 127, 128], [85, 86, 170, 171], [63, 64, 191, 192]], dtype=np.uint8)
    return imgs + [edge]


def check_brute_force(o) -> None:
    for img in tiny_images():
        for nbins in TINY_BINS:
            exp = brute_integral_histogram(img, nbins)
            got = o.integral_histogram(img, nbins)
            assert np.array_equal(got, exp), (img.shape, nbins)
            for k in (0, nbins - 1):
                assert np.array_equal(o.integral_histogram_plane(img, nbins, k), exp[k])


def invariant_errors(img: np.ndarray, nbins: int, H: np.ndarray) -> list:
    """Properties any correct integral histogram of img satisfies."""
    errs = []
    h, w = img.shape
    Hi = H.astype(np.int64)
    area = (np.arange(1, h + 1)[:, None] * np.arange(1, w + 1)[None, :])
    if not np.array_equal(Hi.sum(axis=0), area):
        errs.append("sum over bins != (x+1)(y+1)")
    counts = np.bincount(binned(img, nbins).ravel(), minlength=nbins)
    if not np.array_equal(Hi[:, -1, -1], counts):
        errs.append("bottom-right != bin counts")
    if (np.diff(Hi, axis=1) < 0).any() or (np.diff(Hi, axis=2) < 0).any():
        errs.append("not monotone")
    first = np.zeros(nbins, dtype=np.int64)
    first[brute_bin(int(img[0, 0]), nbins)] = 1
    if not np.array_equal(Hi[:, 0, 0], first):
        errs.append("H[:,0,0] != one-hot of first pixel")
    # 2-D second difference recovers the one-hot of each pixel (Alg. 1 solved for Q)
    P = np.pad(Hi, ((0, 0), (1, 0), (1, 0)))
    d2 = P[:, 1:, 1:] - P[:, :-1, 1:] - P[:, 1:, :-1] + P[:, :-1, :-1]
    onehot = (binned(img, nbins)[None, :, :] == np.arange(nbins)[:, None, None]).astype(np.int64)
    if not np.array_equal(d2, onehot):
        errs.append("second difference != one-hot")
    return errs


def check_invariants(o) -> None:
    rng = np.random.default_rng(20171106)
    for (h, w, nbins) in [(37, 53, 16), (64, 64, 3), (31, 130, 64), (5, 257, 256), (100, 1, 7)]:
        img = rng.integers(0, 256, size=(h, w), dtype=np.uint8)
        errs = invariant_errors(img, nbins, o.integral_histogram(img, nbins))
        assert not errs, (h, w, nbins, errs)


def check_closed_forms(o) -> None:
    h, w = 9, 13
    area = np.arange(1, h + 1)[:, None] * np.arange(1, w + 1)[None, :]
    for v, nbins in [(0, 4), (255, 4), (200, 7), (128, 2), (127, 2)]:
        H = o.integral_histogram(np.full((h, w), v, dtype=np.uint8), nbins).astype(np.int64)
        b = brute_bin(v, nbins)
        assert np.array_equal(H[b], area), (v, nbins)
        assert not np.delete(H, b, axis=0).any(), (v, nbins)
    # column ramp I(y, x) = x on W = 256: H[b][y][x] = (y+1) * #{x' <= x in bin b}
    ramp = np.tile(np.arange(256, dtype=np.uint8), (5, 1))
    for nbins in (1, 3, 8, 100):
        H = o.integral_histogram(ramp, nbins).astype(np.int64)
        for b in range(nbins):
            run = np.cumsum([1 if in_bin(x, b, nbins) else 0 for x in range(256)])
            assert np.array_equal(H[b], np.arange(1, 6)[:, None] * run[None, :]), (nbins, b)
    # row ramp (the transposed case): I(y, x) = y on H = 256, width 3
    H = o.integral_histogram(np.tile(np.arange(256, dtype=np.uint8)[:, None], (1, 3)), 5).astype(np.int64)
    for b in range(5):
        run = np.cumsum([1 if in_bin(y, b, 5) else 0 for y in range(256)])
        assert np.array_equal(H[b], run[:, None] * np.arange(1, 4)[None, :]), b
    # single bright pixel on a dark frame: H[q][y][x] = [x >= x*][y >= y*]
    img = np.zeros((11, 17), dtype=np.uint8)
    img[4, 9] = 250
    H = o.integral_histogram(img, 8).astype(np.int64)
    yy, xx = np.mgrid[0:11, 0:17]
    assert np.array_equal(H[7], ((yy >= 4) & (xx >= 9)).astype(np.int64))
    assert np.array_equal(H[0], (yy + 1) * (xx + 1) - H[7])
    # checkerboard of two bins: bin 1 holds floor/ceil halves of every prefix
    cb = ((np.add.outer(np.arange(8), np.arange(10)) % 2) * 255).astype(np.uint8)
    H = o.integral_histogram(cb, 2).astype(np.int64)
    n = (yy[:8, :10] + 1) * (xx[:8, :10] + 1)
    assert np.array_equal(H[1], n // 2) and np.array_equal(H[0], n - n // 2)


def check_query(o) -> None:
    rng = np.random.default_rng(4)
    for (h, w, nbins) in [(13, 17, 5), (8, 8, 32), (1, 9, 2), (9, 1, 3), (20, 31, 256)]:
        img = rng.integers(0, 256, size=(h, w), dtype=np.uint8)
        H = o.integral_histogram(img, nbins)
        rects = [(0, 0, w - 1, h - 1), (0, 0, 0, 0), (w - 1, h - 1, w - 1, h - 1)]
        for _ in range(25):
            xa, xb = sorted(rng.integers(0, w, size=2).tolist())
            ya, yb = sorted(rng.integers(0, h, size=2).tolist())
            rects.append((xa, ya, xb, yb))
        got = o.query(H, rects)
        for i, r in enumerate(rects):
            exp = brute_region(img, nbins, r)
            assert np.array_equal(got[i], exp), (h, w, nbins, r)
            assert np.array_equal(o.region_brute(img, nbins, r), exp), (h, w, nbins, r)
        full = np.bincount(binned(img, nbins).ravel(), minlength=nbins)
        assert np.array_equal(got[0].astype(np.int64), full)
    # out-of-range rectangles give zeros and are counted
    img = rng.integers(0, 256, size=(6, 7), dtype=np.uint8)
    H = o.integral_histogram(img, 4)
    bad = [(-1, 0, 2, 2), (0, 0, 7, 1), (3, 2, 2, 2), (0, 4, 1, 3), (0, 0, 0, 6)]
    assert not o.query(H, bad).any()


def check_threads(o) -> None:
    rng = np.random.default_rng(9)
    img = rng.integers(0, 256, size=(45, 67), dtype=np.uint8)
    ref = o.integral_histogram(img, 11)
    for t in (1, 2, 3, 16):
        got, used = o.integral_histogram_threads(img, 11, t)
        assert 1 <= used <= min(t, 11)
        assert np.array_equal(got, ref), t


def check_fixture(d, H, name) -> None:
    H = H.astype(np.int64)
    for b, plane in d["planes"].items():
        assert np.array_equal(H[b], plane), (name, b)
    if d["rest_zero"]:
        others = [b for b in range(d["bins"]) if b not in d["planes"]]
        assert not H[others].any(), name
    else:
        assert sorted(d["planes"]) == list(range(d["bins"])), name


EDGE_SETS = ([0, 256], [10, 50, 51, 200], [0, 1, 2, 255, 256], [100, 101], [0, 64, 65, 128, 250],
             [3, 17, 90, 91, 92, 200, 255])


def check_edges(o) -> None:
    """Bins given by edges: fixture, numpy lookup, uniform reduction, brute force."""
    d = load_golden(GOLDEN_EDGES)
    H = o.integral_histogram_edges(d["image"], d["edges"])
    check_fixture(d, H, GOLDEN_EDGES)
    for rect, exp in d["queries"]:
        assert np.array_equal(o.query(H, [rect])[0].astype(np.int64), exp), rect
    for edges in EDGE_SETS:
        for v in range(256):
            assert o.bin_of_edges(v, edges) == edges_bin(v, edges), (edges, v)
    # uniform edges e_k = ceil(256 k / B) give the uniform bins of Eq. 1's Q
    rng = np.random.default_rng(31)
    img = rng.integers(0, 256, size=(9, 14), dtype=np.uint8)
    for nbins in (1, 3, 7, 64, 256):
        edges = [-(-256 * k // nbins) for k in range(nbins + 1)]
        assert np.array_equal(o.integral_histogram_edges(img, edges), o.integral_histogram(img, nbins)), nbins
    for img in tiny_images()[:6]:
        for edges in EDGE_SETS[1:4]:
            bins = np.vectorize(lambda v: edges_bin(int(v), edges))(img)
            exp = brute_from_bins(bins, len(edges) - 1)
            assert np.array_equal(o.integral_histogram_edges(img, edges), exp), (img.shape, edges)


def check_mapped(o) -> None:
    """Any value -> bin map: brute force, plane permutation, values in no bin."""
    rng = np.random.default_rng(77)
    img = rng.integers(0, 256, size=(11, 19), dtype=np.uint8)
    nbins = 6
    bin_map = rng.integers(-1, nbins, size=256)
    H = o.integral_histogram_mapped(img, bin_map, nbins)
    assert np.array_equal(H, brute_from_bins(bin_map[img], nbins))
    # renaming the bins renames the planes
    perm = rng.permutation(nbins)
    renamed = np.where(bin_map >= 0, perm[np.maximum(bin_map, 0)], -1)
    H2 = o.integral_histogram_mapped(img, renamed, nbins)
    for k in range(nbins):
        assert np.array_equal(H2[perm[k]], H[k]), k
    # the sum over bins counts exactly the pixels that have a bin
    inbin = (bin_map[img] >= 0).astype(np.int64)
    assert np.array_equal(H.astype(np.int64).sum(axis=0), inbin.cumsum(axis=0).cumsum(axis=1))
    assert not o.integral_histogram_mapped(img, np.full(256, -1), 3).any()


def joint_digits(k: int, cbins) -> list:
    """Channel bins of joint bin k (channel 0 most significant)."""
    out = []
    for b in reversed(cbins):
        out.append(k % b)
        k //= b
    return out[::-1]


def check_joint(o) -> None:
    """Joint multi-channel bins: fixture, one channel, marginals, brute force."""
    d = load_golden(GOLDEN_JOINT)
    H = o.integral_histogram_joint(d["image"], d["cbins"])
    assert H.shape[0] == d["bins"]
    check_fixture(d, H, GOLDEN_JOINT)
    for rect, exp in d["queries"]:
        assert np.array_equal(o.query(H, [rect])[0].astype(np.int64), exp), rect
    rng = np.random.default_rng(5)
    img1 = rng.integers(0, 256, size=(8, 13, 1), dtype=np.uint8)
    for b in (1, 5, 16):
        assert np.array_equal(o.integral_histogram_joint(img1, [b]), o.integral_histogram(img1[:, :, 0], b)), b
    # summing the joint planes over the other channels' bins leaves channel
    # c's own integral histogram (pins the digit order and each channel's Q)
    for cbins in ([2, 3, 4], [5, 2], [4, 1, 3, 2]):
        C = len(cbins)
        img = rng.integers(0, 256, size=(7, 10, C), dtype=np.uint8)
        H = o.integral_histogram_joint(img, cbins).astype(np.int64)
        assert H.shape[0] == int(np.prod(cbins))
        digits = np.array([joint_digits(k, cbins) for k in range(H.shape[0])])
        for c in range(C):
            ref = o.integral_histogram(np.ascontiguousarray(img[:, :, c]), cbins[c]).astype(np.int64)
            for j in range(cbins[c]):
                assert np.array_equal(H[digits[:, c] == j].sum(axis=0), ref[j]), (cbins, c, j)
    img = rng.integers(0, 256, size=(5, 6, 3), dtype=np.uint8)
    cbins = [3, 2, 4]
    bins = np.zeros((5, 6), dtype=np.int64)
    for y in range(5):
        for x in range(6):
            q = [brute_bin(int(img[y, x, c]), cbins[c]) for c in range(3)]
            bins[y, x] = (q[0] * cbins[1] + q[1]) * cbins[2] + q[2]
    assert np.array_equal(o.integral_histogram_joint(img, cbins), brute_from_bins(bins, 24))


def numpy_window_intersection(img, nbins, target, win_h, win_w, stride):
    """Window counts by numpy's sliding_window_view over the one-hot planes."""
    onehot = (binned(img, nbins)[None, :, :] == np.arange(nbins)[:, None, None]).astype(np.int64)
    win = np.lib.stride_tricks.sliding_window_view(onehot, (win_h, win_w), axis=(1, 2))[:, ::stride, ::stride]
    counts = win.sum(axis=(-1, -2))
    return np.minimum(counts, np.asarray(target, dtype=np.int64)[:, None, None]).sum(axis=0)


def check_window_search(o) -> None:
    """Sliding-window histogram intersection: numpy windows, closed forms, self-match."""
    rng = np.random.default_rng(99)
    for (h, w, nbins, wh, ww, st) in [(20, 31, 8, 5, 7, 1), (33, 40, 16, 8, 8, 3), (16, 16, 4, 16, 16, 5),
                                      (9, 50, 32, 1, 1, 2), (30, 30, 3, 7, 4, 4)]:
        img = rng.integers(0, 256, size=(h, w), dtype=np.uint8)
        target = rng.integers(0, wh * ww + 1, size=nbins)
        got = o.window_intersection(img, nbins, target, wh, ww, st)
        exp = numpy_window_intersection(img, nbins, target, wh, ww, st)
        assert got.shape == ((h - wh) // st + 1, (w - ww) // st + 1), (h, w, wh, ww, st)
        assert np.array_equal(got.astype(np.int64), exp), (h, w, nbins, wh, ww, st)
    # constant frame: every window holds area pixels of one bin
    img = np.full((12, 17), 200, dtype=np.uint8)
    target = np.arange(8) * 3
    got = o.window_intersection(img, 8, target, 4, 5, 2)
    assert (got == min(20, int(target[brute_bin(200, 8)]))).all()
    # the target taken from one window scores that window's full area there and no more anywhere
    img = rng.integers(0, 256, size=(24, 24), dtype=np.uint8)
    target = brute_region(img, 6, (8, 4, 15, 11)).astype(np.int64)  # window at row 4, col 8
    got = o.window_intersection(img, 6, target, 8, 8, 4)
    assert got[1, 2] == 64 and got.max() == 64


ALL_CHECKS = (check_bins, check_golden, check_brute_force, check_invariants,
              check_closed_forms, check_query, check_threads, check_edges, check_mapped, check_joint,
              check_window_search)
