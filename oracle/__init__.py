"""CPU oracle for the integral histogram -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
legs may import this package.  The product library (``paper_1711_01919_gb300``)
never imports it, and the two share no code.

The arithmetic lives in ``ihist_oracle.c`` (plain single-threaded C following
Eq. 1 / Algorithm 1 and Eq. 2 of arXiv 1711.01919, Sec. 2.1).  This module only
compiles that file with gcc (on first use, or from ``build()``) and marshals
numpy arrays through ctypes.

Functions (module level, on the default build)
---------------------------------------------
bin_of(v, nbins)                  Q of Eq. 1: the uniform bin of intensity v.
integral_histogram(img, nbins)    Algorithm 1 over all bins -> [nbins][h][w] uint32.
integral_histogram_plane(img, nbins, k)   one bin plane of Algorithm 1.
integral_histogram_threads(img, nbins, nthreads)  same result, bins split over
                                  threads (timing only; Sec. 4.7 methodology).
query(hist, rects)                Eq. 2 on an inclusive rect list -> [n][nbins].
region_brute(img, nbins, rect)    direct count over a rectangle (no Eq. 2).
bin_of_edges(v, edges)            the bin of v for bins given by edges, or -1.
integral_histogram_mapped(img, bin_map, nbins)   Algorithm 1 for any value -> bin map.
integral_histogram_edges(img, edges)             Algorithm 1 for bins given by edges.
integral_histogram_joint(img, bins)              Algorithm 1 over the joint bins of a
                                  [h][w][C] frame (channel 0 most significant).
window_intersection(img, nbins, target, win_h, win_w, stride)
                                  histogram-intersection score of every window on a
                                  stride grid, each window counted directly.

``Oracle(path)`` wraps any shared object built from ``ihist_oracle.c``; the
tests use it to load deliberately mutated copies and check that the pins
reject them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(HERE, "ihist_oracle.c")
_LIB = os.path.join(HERE, "libihist_oracle.so")
_lock = threading.Lock()
_default = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)


def compile_c(src: str, out: str) -> str:
    """gcc -O2 shared object from one C file (atomic replace)."""
    tmp = out + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-pthread", src, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ihist_oracle.c into libihist_oracle.so next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(SOURCE):
        compile_c(SOURCE, _LIB)
    return _LIB


def _img(img) -> np.ndarray:
    a = np.asarray(img)
    if a.dtype != np.uint8 or a.ndim != 2:
        raise ValueError("image must be a 2-D uint8 array")
    if a.strides[1] != 1 or a.strides[0] < a.shape[1]:
        a = np.ascontiguousarray(a)
    return a


def _p8(a):
    return a.ctypes.data_as(_u8p)


def _p32(a):
    return a.ctypes.data_as(_u32p)


class Oracle:
    """ctypes view of one build of ihist_oracle.c."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        lib.oracle_bin_of.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.oracle_bin_of.restype = ctypes.c_int
        lib.oracle_ih_plane.argtypes = [_u8p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, _u32p]
        lib.oracle_ih_plane.restype = None
        lib.oracle_ih.argtypes = [_u8p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, _u32p]
        lib.oracle_ih.restype = None
        lib.oracle_ih_threads.argtypes = [_u8p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _u32p, ctypes.c_int]
        lib.oracle_ih_threads.restype = ctypes.c_int
        lib.oracle_query.argtypes = [_u32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     _i32p, ctypes.c_int, _u32p]
        lib.oracle_query.restype = ctypes.c_int
        lib.oracle_region_brute.argtypes = [_u8p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, _u32p]
        lib.oracle_region_brute.restype = ctypes.c_int
        lib.oracle_bin_of_edges.argtypes = [ctypes.c_int, _i32p, ctypes.c_int]
        lib.oracle_bin_of_edges.restype = ctypes.c_int
        lib.oracle_ih_mapped.argtypes = [_u8p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, _i32p,
                                         ctypes.c_int, _u32p]
        lib.oracle_ih_mapped.restype = None
        lib.oracle_ih_joint.argtypes = [_u8p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        _i32p, _u32p]
        lib.oracle_ih_joint.restype = None
        lib.oracle_window_intersection.argtypes = [_u8p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, _u32p, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, _u32p]
        lib.oracle_window_intersection.restype = None
        self.lib = lib
        self.path = path

    def bin_of(self, v: int, nbins: int) -> int:
        """Q of Eq. 1 for one intensity value."""
        return int(self.lib.oracle_bin_of(int(v), int(nbins)))

    def integral_histogram(self, img, nbins: int, out=None) -> np.ndarray:
        """Algorithm 1: the [nbins][h][w] uint32 integral histogram of img."""
        a = _img(img)
        h, w = a.shape
        if out is None:
            out = np.empty((nbins, h, w), dtype=np.uint32)
        if out.shape != (nbins, h, w) or out.dtype != np.uint32 or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous uint32 [nbins][h][w] array")
        if h and w and nbins:
            self.lib.oracle_ih(_p8(a), a.strides[0], h, w, nbins, _p32(out))
        return out

    def integral_histogram_plane(self, img, nbins: int, k: int, out=None) -> np.ndarray:
        """Bin plane k of Algorithm 1, [h][w] uint32."""
        a = _img(img)
        h, w = a.shape
        if out is None:
            out = np.empty((h, w), dtype=np.uint32)
        if out.shape != (h, w) or out.dtype != np.uint32 or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous uint32 [h][w] array")
        if h and w:
            self.lib.oracle_ih_plane(_p8(a), a.strides[0], h, w, nbins, k, _p32(out))
        return out

    def integral_histogram_threads(self, img, nbins: int, nthreads: int, out=None):
        """Bins-parallel run of Algorithm 1; returns (hist, threads_used)."""
        a = _img(img)
        h, w = a.shape
        if out is None:
            out = np.empty((nbins, h, w), dtype=np.uint32)
        used = self.lib.oracle_ih_threads(_p8(a), a.strides[0], h, w, nbins, _p32(out), int(nthreads))
        return out, int(used)

    def query(self, hist: np.ndarray, rects) -> np.ndarray:
        """Eq. 2 for each inclusive rect (x0, y0, x1, y1); out-of-range rects give zeros."""
        hist = np.ascontiguousarray(hist, dtype=np.uint32)
        nbins, h, w = hist.shape
        r = np.ascontiguousarray(np.asarray(rects, dtype=np.int32).reshape(-1, 4))
        out = np.zeros((r.shape[0], nbins), dtype=np.uint32)
        if r.shape[0]:
            self.lib.oracle_query(_p32(hist), h, w, nbins, r.ctypes.data_as(_i32p), r.shape[0], _p32(out))
        return out

    def region_brute(self, img, nbins: int, rect) -> np.ndarray:
        """Histogram of the pixels inside an inclusive rect, counted directly."""
        a = _img(img)
        h, w = a.shape
        x0, y0, x1, y1 = (int(v) for v in rect)
        out = np.zeros(nbins, dtype=np.uint32)
        self.lib.oracle_region_brute(_p8(a), a.strides[0], h, w, nbins, x0, y0, x1, y1, _p32(out))
        return out


    def bin_of_edges(self, v: int, edges) -> int:
        """The bin of intensity v for bins given by edges (nbins + 1 ints), or -1."""
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32))
        return int(self.lib.oracle_bin_of_edges(int(v), e.ctypes.data_as(_i32p), e.size - 1))

    def integral_histogram_mapped(self, img, bin_map, nbins: int, out=None) -> np.ndarray:
        """Algorithm 1 with bin_map[v] (256 ints in [-1, nbins)) as Q."""
        a = _img(img)
        h, w = a.shape
        m = np.ascontiguousarray(np.asarray(bin_map, dtype=np.int32))
        if m.shape != (256,) or m.min() < -1 or m.max() >= nbins:
            raise ValueError("bin_map must be 256 ints in [-1, nbins)")
        if out is None:
            out = np.empty((nbins, h, w), dtype=np.uint32)
        if h and w and nbins:
            self.lib.oracle_ih_mapped(_p8(a), a.strides[0], h, w, m.ctypes.data_as(_i32p), nbins, _p32(out))
        return out

    def integral_histogram_edges(self, img, edges, out=None) -> np.ndarray:
        """Algorithm 1 for bins [edges[k], edges[k+1]); values outside count nowhere."""
        nbins = len(edges) - 1
        bin_map = [self.bin_of_edges(v, edges) for v in range(256)]
        return self.integral_histogram_mapped(img, bin_map, nbins, out)

    def integral_histogram_joint(self, img, bins, out=None) -> np.ndarray:
        """Algorithm 1 over the joint bins of a uint8 [h][w][C] frame."""
        a = np.asarray(img)
        if a.dtype != np.uint8 or a.ndim != 3:
            raise ValueError("image must be a 3-D uint8 [h][w][C] array")
        a = np.ascontiguousarray(a)
        h, w, c = a.shape
        b = np.ascontiguousarray(np.asarray(bins, dtype=np.int32))
        if b.shape != (c,):
            raise ValueError("one bin count per channel")
        nbins = int(np.prod(b))
        if out is None:
            out = np.empty((nbins, h, w), dtype=np.uint32)
        if h and w:
            self.lib.oracle_ih_joint(_p8(a), a.strides[0], h, w, c, b.ctypes.data_as(_i32p), _p32(out))
        return out

    def window_intersection(self, img, nbins: int, target, win_h: int, win_w: int, stride: int) -> np.ndarray:
        """[ny][nx] uint32 scores sum_b min(window count_b, target_b)."""
        a = _img(img)
        h, w = a.shape
        if not (1 <= win_h <= h and 1 <= win_w <= w and stride >= 1):
            raise ValueError("window must fit the frame and stride must be >= 1")
        t = np.ascontiguousarray(np.asarray(target, dtype=np.uint32))
        if t.shape != (nbins,):
            raise ValueError("target must hold nbins counts")
        ny, nx = (h - win_h) // stride + 1, (w - win_w) // stride + 1
        out = np.zeros((ny, nx), dtype=np.uint32)
        self.lib.oracle_window_intersection(_p8(a), a.strides[0], h, w, nbins, _p32(t), win_h, win_w, stride,
                                            _p32(out))
        return out


def default() -> Oracle:
    """The oracle built from ihist_oracle.c as committed."""
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def bin_of(v, nbins):
    return default().bin_of(v, nbins)


def integral_histogram(img, nbins, out=None):
    return default().integral_histogram(img, nbins, out)


def integral_histogram_plane(img, nbins, k, out=None):
    return default().integral_histogram_plane(img, nbins, k, out)


def integral_histogram_threads(img, nbins, nthreads, out=None):
    return default().integral_histogram_threads(img, nbins, nthreads, out)


def query(hist, rects):
    return default().query(hist, rects)


def region_brute(img, nbins, rect):
    return default().region_brute(img, nbins, rect)


def bin_of_edges(v, edges):
    return default().bin_of_edges(v, edges)


def integral_histogram_mapped(img, bin_map, nbins, out=None):
    return default().integral_histogram_mapped(img, bin_map, nbins, out)


def integral_histogram_edges(img, edges, out=None):
    return default().integral_histogram_edges(img, edges, out)


def integral_histogram_joint(img, bins, out=None):
    return default().integral_histogram_joint(img, bins, out)


def window_intersection(img, nbins, target, win_h, win_w, stride):
    return default().window_intersection(img, nbins, target, win_h, win_w, stride)
