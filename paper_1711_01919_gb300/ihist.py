"""Thin ctypes binding of libihist.so (declared in include/ihist.h).

The functions named ``ihist_*`` mirror the C entry points one to one and only
marshal arguments: device pointers and streams are plain integers (for torch
tensors, ``t.data_ptr()`` and ``torch.cuda.current_stream().cuda_stream``).
Non-zero return codes raise :class:`IhistError`.  ``Plan`` adds the torch
plumbing (output allocation, stream lookup) around the same calls.

There is no fallback: if libihist.so is missing the import of this module
succeeds but the first call raises, naming the build step.  The environment
variable IHIST_LIB selects another build of the same library (for example
libihist_checked.so, whose kernels guard every carry index and output store).
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("IHIST_LIB") or os.path.join(PKG, "libihist.so")

IHIST_OK = 0
IHIST_ERR_INVALID_ARG = 1
IHIST_ERR_UNSUPPORTED = 2
IHIST_ERR_OOM = 3
IHIST_ERR_CUDA = 4
IHIST_ERR_LOOKBACK_TIMEOUT = 5
IHIST_ERR_BAD_RECT = 6
IHIST_ERR_CHECK_FAILED = 7
IHIST_BIN_MAJOR = 0
IHIST_PIXEL_MAJOR = 1
IHIST_QUAD_MAJOR = 2  # H[b/4][y][x][b%4]

EXPORTED = (
    "ihist_plan", "ihist_plan_tuned", "ihist_plan_get_tune", "ihist_workspace_bytes",
    "ihist_output_bytes", "ihist_compute", "ihist_query", "ihist_sequence_host", "ihist_status",
    "ihist_destroy", "ihist_error_string", "ihist_batch_plan", "ihist_batch_set_io",
    "ihist_batch_compute", "ihist_batch_query", "ihist_batch_status", "ihist_batch_workspace_bytes",
    "ihist_batch_items", "ihist_batch_destroy", "ihist_batch_query_all", "ihist_batch_upload_compute",
    "ihist_compute_noalloc", "ihist_plan_lut", "ihist_plan_edges", "ihist_plan_joint",
    "ihist_plan_channels", "ihist_window_search", "ihist_mapping_workspace_bytes", "ihist_mapping_compute",
    "ihist_batch_get_tune", "ihist_edges_table", "ihist_query_work_bytes", "ihist_query_sorted",
)


class IhistError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s failed: %s (code %d)" % (what, ihist_error_string(code), code))
        self.code = code


class ihist_tune_t(ctypes.Structure):
    _fields_ = [
        ("rows_per_band", ctypes.c_int),
        ("bins_per_cta", ctypes.c_int),
        ("chunks_per_warp", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int),
        ("timeout_us", ctypes.c_uint),
        ("fault_skip_band", ctypes.c_int),
        ("groups_per_cta", ctypes.c_int),
        ("warps_per_cta", ctypes.c_int),
        ("overlap", ctypes.c_int),
        ("reserved", ctypes.c_int),
    ]


class ihist_frame_t(ctypes.Structure):
    _fields_ = [
        ("h", ctypes.c_int),
        ("w", ctypes.c_int),
        ("nbins", ctypes.c_int),
        ("layout", ctypes.c_int),
        ("d_in", ctypes.c_void_p),
        ("in_pitch", ctypes.c_size_t),
        ("d_out", ctypes.c_void_p),
        ("bin_of_value", ctypes.POINTER(ctypes.c_int)),
        ("channels", ctypes.c_int),
        ("bins_per_channel", ctypes.c_int * 4),
    ]


TUNE_FIELDS = ("rows_per_band", "bins_per_cta", "chunks_per_warp", "ctas_per_sm", "timeout_us",
               "fault_skip_band", "groups_per_cta", "warps_per_cta", "overlap")

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libihist.so and declare its signatures (once)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("libihist.so is not built (%s); run __graft_entry__.build() or "
                               "python -m paper_1711_01919_gb300.build" % path)
        L = ctypes.CDLL(path)
        vp, sz, ci, cu = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint
        L.ihist_plan.argtypes = [ci, ci, ci, ci, ctypes.POINTER(vp)]
        L.ihist_plan.restype = ci
        L.ihist_plan_tuned.argtypes = [ci, ci, ci, ci, ctypes.POINTER(ihist_tune_t), ctypes.POINTER(vp)]
        L.ihist_plan_tuned.restype = ci
        L.ihist_plan_get_tune.argtypes = [vp, ctypes.POINTER(ihist_tune_t)]
        L.ihist_plan_get_tune.restype = ci
        L.ihist_workspace_bytes.argtypes = [vp]
        L.ihist_workspace_bytes.restype = sz
        L.ihist_output_bytes.argtypes = [ci, ci, ci]
        L.ihist_output_bytes.restype = sz
        L.ihist_compute.argtypes = [vp, vp, sz, vp, vp]
        L.ihist_compute.restype = ci
        L.ihist_query.argtypes = [vp, vp, vp, ci, vp, vp]
        L.ihist_query.restype = ci
        L.ihist_query_work_bytes.argtypes = [vp, ci, ci]
        L.ihist_query_work_bytes.restype = sz
        L.ihist_query_sorted.argtypes = [vp, vp, vp, ci, vp, ci, vp, sz, vp]
        L.ihist_query_sorted.restype = ci
        L.ihist_sequence_host.argtypes = [vp, vp, sz, ci, vp, vp, ci, vp, ci, vp, vp, vp, vp]
        L.ihist_sequence_host.restype = ci
        L.ihist_status.argtypes = [vp, vp, ctypes.POINTER(ci)]
        L.ihist_status.restype = ci
        L.ihist_destroy.argtypes = [vp]
        L.ihist_destroy.restype = None
        fp = ctypes.POINTER(ihist_frame_t)
        L.ihist_batch_plan.argtypes = [fp, ci, ctypes.POINTER(ihist_tune_t), ctypes.POINTER(vp)]
        L.ihist_batch_plan.restype = ci
        L.ihist_batch_get_tune.argtypes = [vp, ctypes.POINTER(ihist_tune_t)]
        L.ihist_batch_get_tune.restype = ci
        L.ihist_batch_set_io.argtypes = [vp, fp, ci, vp]
        L.ihist_batch_set_io.restype = ci
        L.ihist_batch_compute.argtypes = [vp, vp]
        L.ihist_batch_compute.restype = ci
        L.ihist_batch_query.argtypes = [vp, ci, vp, vp, ci, vp, vp]
        L.ihist_batch_query.restype = ci
        L.ihist_batch_query_all.argtypes = [vp, vp, ci, vp, vp]
        L.ihist_batch_query_all.restype = ci
        L.ihist_batch_upload_compute.argtypes = [vp, ctypes.POINTER(vp), vp, vp]
        L.ihist_batch_upload_compute.restype = ci
        L.ihist_batch_status.argtypes = [vp, vp, ctypes.POINTER(ci)]
        L.ihist_batch_status.restype = ci
        L.ihist_batch_workspace_bytes.argtypes = [vp]
        L.ihist_batch_workspace_bytes.restype = sz
        L.ihist_batch_items.argtypes = [vp]
        L.ihist_batch_items.restype = cu
        L.ihist_batch_destroy.argtypes = [vp]
        L.ihist_batch_destroy.restype = None
        L.ihist_compute_noalloc.argtypes = [ci, ci, ci, ci, vp, sz, vp, vp, ctypes.POINTER(ci)]
        L.ihist_compute_noalloc.restype = ci
        ip = ctypes.POINTER(ci)
        tp = ctypes.POINTER(ihist_tune_t)
        L.ihist_plan_lut.argtypes = [ci, ci, ci, ci, ip, tp, ctypes.POINTER(vp)]
        L.ihist_plan_lut.restype = ci
        L.ihist_plan_edges.argtypes = [ci, ci, ci, ci, ip, tp, ctypes.POINTER(vp)]
        L.ihist_plan_edges.restype = ci
        L.ihist_edges_table.argtypes = [ci, ip, ip]
        L.ihist_edges_table.restype = ci
        L.ihist_plan_joint.argtypes = [ci, ci, ci, ip, ci, tp, ctypes.POINTER(vp)]
        L.ihist_plan_joint.restype = ci
        L.ihist_mapping_workspace_bytes.argtypes = [ci, ci, ci, ci]
        L.ihist_mapping_workspace_bytes.restype = sz
        L.ihist_mapping_compute.argtypes = [ci, ci, ci, ci, vp, sz, vp, vp, vp]
        L.ihist_mapping_compute.restype = ci
        L.ihist_window_search.argtypes = [vp, vp, vp, ci, ci, ci, vp, vp, vp]
        L.ihist_window_search.restype = ci
        L.ihist_plan_channels.argtypes = [vp]
        L.ihist_plan_channels.restype = ci
        L.ihist_error_string.argtypes = [ci]
        L.ihist_error_string.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(code: int, what: str) -> None:
    if code != IHIST_OK:
        raise IhistError(code, what)


def ihist_error_string(code: int) -> str:
    return load().ihist_error_string(int(code)).decode()


def ihist_output_bytes(h: int, w: int, nbins: int) -> int:
    return int(load().ihist_output_bytes(h, w, nbins))


def _tune_struct(tune) -> ihist_tune_t:
    t = ihist_tune_t()
    t.fault_skip_band = -1
    for k, v in (tune or {}).items():
        if k not in TUNE_FIELDS:
            raise KeyError("unknown tuning field %r" % k)
        setattr(t, k, int(v))
    return t


def ihist_plan(h: int, w: int, nbins: int, layout: int = IHIST_BIN_MAJOR) -> int:
    out = ctypes.c_void_p()
    _check(load().ihist_plan(h, w, nbins, layout, ctypes.byref(out)), "ihist_plan")
    return out.value


def ihist_plan_tuned(h: int, w: int, nbins: int, layout: int = IHIST_BIN_MAJOR, tune=None) -> int:
    out = ctypes.c_void_p()
    t = _tune_struct(tune)
    _check(load().ihist_plan_tuned(h, w, nbins, layout, ctypes.byref(t), ctypes.byref(out)),
           "ihist_plan_tuned")
    return out.value


def _ints(vals):
    vals = [int(v) for v in vals]
    return (ctypes.c_int * max(1, len(vals)))(*vals)


def ihist_plan_lut(h: int, w: int, nbins: int, layout: int, bin_of_value, tune=None) -> int:
    """Plan whose bins come from a 256-entry value -> bin map (-1 = no bin)."""
    vals = list(bin_of_value)
    if len(vals) != 256:
        raise ValueError("bin_of_value must have 256 entries")
    out = ctypes.c_void_p()
    t = _tune_struct(tune) if tune else None
    _check(load().ihist_plan_lut(h, w, nbins, layout, _ints(vals), ctypes.byref(t) if t else None,
                                 ctypes.byref(out)), "ihist_plan_lut")
    return out.value


def ihist_plan_edges(h: int, w: int, layout: int, edges, tune=None) -> int:
    """Plan with bins [edges[k], edges[k+1]); values outside count nowhere."""
    e = list(edges)
    out = ctypes.c_void_p()
    t = _tune_struct(tune) if tune else None
    _check(load().ihist_plan_edges(h, w, len(e) - 1, layout, _ints(e), ctypes.byref(t) if t else None,
                                   ctypes.byref(out)), "ihist_plan_edges")
    return out.value


def ihist_plan_joint(h: int, w: int, bins_per_channel, layout: int = IHIST_BIN_MAJOR, tune=None) -> int:
    """Plan for the joint bins of frames with len(bins_per_channel) interleaved channels."""
    b = list(bins_per_channel)
    out = ctypes.c_void_p()
    t = _tune_struct(tune) if tune else None
    _check(load().ihist_plan_joint(h, w, len(b), _ints(b), layout, ctypes.byref(t) if t else None,
                                   ctypes.byref(out)), "ihist_plan_joint")
    return out.value


def ihist_plan_channels(plan: int) -> int:
    return int(load().ihist_plan_channels(plan))


def ihist_plan_get_tune(plan: int) -> dict:
    t = ihist_tune_t()
    _check(load().ihist_plan_get_tune(plan, ctypes.byref(t)), "ihist_plan_get_tune")
    return {k: getattr(t, k) for k in TUNE_FIELDS}


def ihist_workspace_bytes(plan: int) -> int:
    return int(load().ihist_workspace_bytes(plan))


def ihist_compute(plan: int, d_in: int, in_pitch: int, d_out: int, stream: int = 0) -> None:
    _check(load().ihist_compute(plan, d_in, in_pitch, d_out, stream), "ihist_compute")


def ihist_query(plan: int, d_hist: int, d_rects: int, n: int, d_hist_out: int, stream: int = 0) -> None:
    _check(load().ihist_query(plan, d_hist, d_rects, n, d_hist_out, stream), "ihist_query")


def ihist_query_work_bytes(plan: int, n: int, bins_per_pass: int = 0) -> int:
    return int(load().ihist_query_work_bytes(plan, n, bins_per_pass))


def ihist_query_sorted(plan: int, d_hist: int, d_rects: int, n: int, d_hist_out: int, bins_per_pass: int,
                       d_work: int, work_bytes: int, stream: int = 0) -> None:
    _check(load().ihist_query_sorted(plan, d_hist, d_rects, n, d_hist_out, bins_per_pass, d_work, work_bytes,
                                     stream), "ihist_query_sorted")


def ihist_window_search(plan: int, d_hist: int, d_target: int, win_h: int, win_w: int, stride: int,
                        d_scores: int, d_best: int = 0, stream: int = 0) -> None:
    _check(load().ihist_window_search(plan, d_hist, d_target, win_h, win_w, stride, d_scores or None,
                                      d_best or None, stream), "ihist_window_search")


IHIST_MAPPING_CW_STS, IHIST_MAPPING_CW_TIS, IHIST_MAPPING_WF_TIS = 1, 2, 3
MAPPINGS = {"cw_sts": IHIST_MAPPING_CW_STS, "cw_tis": IHIST_MAPPING_CW_TIS, "wf_tis": IHIST_MAPPING_WF_TIS}


def ihist_mapping_workspace_bytes(mapping: int, h: int, w: int, nbins: int) -> int:
    return int(load().ihist_mapping_workspace_bytes(mapping, h, w, nbins))


def ihist_mapping_compute(mapping: int, h: int, w: int, nbins: int, d_in: int, in_pitch: int, d_out: int,
                          d_work: int = 0, stream: int = 0) -> None:
    """One of the paper's mappings (comparison kernels; see include/ihist.h)."""
    _check(load().ihist_mapping_compute(mapping, h, w, nbins, d_in, in_pitch, d_out, d_work or None, stream),
           "ihist_mapping_compute")


def window_grid(h: int, w: int, win_h: int, win_w: int, stride: int):
    """(ny, nx) of the window grid ihist_window_search scores."""
    return (h - win_h) // stride + 1, (w - win_w) // stride + 1


def ihist_sequence_host(plan: int, h_frames: int, frame_stride: int, nframes: int, d_slots: int,
                        d_outs: int, nouts: int, d_rects: int, nrects: int, d_query: int,
                        h_query_out: int, stream: int, copy_stream: int) -> None:
    _check(load().ihist_sequence_host(plan, h_frames, frame_stride, nframes, d_slots, d_outs, nouts,
                                      d_rects, nrects, d_query, h_query_out, stream, copy_stream),
           "ihist_sequence_host")


def ihist_compute_noalloc(h: int, w: int, nbins: int, layout: int, d_in: int, in_pitch: int, d_out: int,
                          stream: int = 0, wait: bool = True):
    """Integral histogram with no device allocation (fixed scratch in the
    library); returns the device status when wait is true, else None."""
    st = ctypes.c_int(-1)
    _check(load().ihist_compute_noalloc(h, w, nbins, layout, d_in, in_pitch, d_out, stream,
                                        ctypes.byref(st) if wait else None), "ihist_compute_noalloc")
    return st.value if wait else None


def ihist_status(plan: int, stream: int = 0) -> int:
    st = ctypes.c_int(-1)
    _check(load().ihist_status(plan, stream, ctypes.byref(st)), "ihist_status")
    return st.value


def ihist_destroy(plan: int) -> None:
    if plan:
        load().ihist_destroy(plan)


def _table_ptr(table):
    """A 256-entry value -> bin table as a C int array (None stays NULL)."""
    if table is None:
        return None
    vals = [int(v) for v in table]
    if len(vals) != 256:
        raise ValueError("a bin table has 256 entries, one per intensity")
    return ctypes.cast((ctypes.c_int * 256)(*vals), ctypes.POINTER(ctypes.c_int))


def _frames_array(frames):
    """frames: (h, w, nbins, layout, d_in, in_pitch, d_out[, table[,
    bins_per_channel]]) tuples; bins_per_channel (2..4 entries) makes a
    joint-bin frame of that many interleaved channels."""
    arr = (ihist_frame_t * len(frames))()
    for i, fr in enumerate(frames):
        h, w, nbins, layout, d_in, pitch, d_out = fr[:7]
        table = fr[7] if len(fr) > 7 else None
        joint = list(fr[8]) if len(fr) > 8 and fr[8] is not None else []
        if len(joint) > 4:
            raise ValueError("at most 4 channels")
        arr[i] = ihist_frame_t(h, w, nbins, layout, d_in, pitch, d_out, _table_ptr(table), len(joint),
                               (ctypes.c_int * 4)(*(joint + [0] * (4 - len(joint)))))
    return arr


def edges_table(edges):
    """Value -> bin table of bins by edges (ihist_edges_table): bin k holds
    edges[k] <= v < edges[k + 1]; values outside [edges[0], edges[-1]) are in
    no bin (-1).  ValueError for edges that do not increase within [0, 256]."""
    e = [int(x) for x in edges]
    out = (ctypes.c_int * 256)()
    code = load().ihist_edges_table(len(e) - 1, _ints(e) if e else None, out)
    if code == IHIST_ERR_INVALID_ARG:
        raise ValueError("edges must increase strictly within [0, 256]")
    _check(code, "ihist_edges_table")
    return list(out)


def ihist_batch_plan(frames, tune=None) -> int:
    """frames: sequence of (h, w, nbins, layout, d_in, in_pitch, d_out[, table])."""
    arr = _frames_array(frames)
    out = ctypes.c_void_p()
    t = _tune_struct(tune) if tune else None
    _check(load().ihist_batch_plan(arr, len(frames), ctypes.byref(t) if t else None, ctypes.byref(out)),
           "ihist_batch_plan")
    return out.value


def ihist_batch_get_tune(batch: int) -> dict:
    t = ihist_tune_t()
    _check(load().ihist_batch_get_tune(batch, ctypes.byref(t)), "ihist_batch_get_tune")
    return {k: getattr(t, k) for k in TUNE_FIELDS}


def ihist_batch_set_io(batch: int, frames, stream: int = 0) -> None:
    arr = _frames_array(frames)
    _check(load().ihist_batch_set_io(batch, arr, len(frames), stream), "ihist_batch_set_io")


def ihist_batch_compute(batch: int, stream: int = 0) -> None:
    _check(load().ihist_batch_compute(batch, stream), "ihist_batch_compute")


def ihist_batch_query(batch: int, frame: int, d_hist: int, d_rects: int, n: int, d_hist_out: int,
                      stream: int = 0) -> None:
    _check(load().ihist_batch_query(batch, frame, d_hist, d_rects, n, d_hist_out, stream),
           "ihist_batch_query")


def ihist_batch_query_all(batch: int, d_rects: int, n: int, d_out: int, stream: int = 0) -> None:
    _check(load().ihist_batch_query_all(batch, d_rects, n, d_out, stream), "ihist_batch_query_all")


def ihist_batch_upload_compute(batch: int, h_frames, stream: int = 0, copy_stream: int = 0) -> None:
    """h_frames: host addresses (ints) of the batch's frames, page-locked."""
    arr = (ctypes.c_void_p * len(h_frames))(*h_frames)
    _check(load().ihist_batch_upload_compute(batch, arr, stream, copy_stream), "ihist_batch_upload_compute")


def ihist_batch_status(batch: int, stream: int = 0) -> int:
    st = ctypes.c_int(-1)
    _check(load().ihist_batch_status(batch, stream, ctypes.byref(st)), "ihist_batch_status")
    return st.value


def ihist_batch_workspace_bytes(batch: int) -> int:
    return int(load().ihist_batch_workspace_bytes(batch))


def ihist_batch_items(batch: int) -> int:
    return int(load().ihist_batch_items(batch))


def ihist_batch_destroy(batch: int) -> None:
    if batch:
        load().ihist_batch_destroy(batch)


# --------------------------------------------------------------- torch glue

def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """A plan for (h, w, nbins, layout) frames; torch tensors in and out.

    Output tensors are int32 storage holding uint32 counts (view them as
    uint32 on the host: ``t.cpu().numpy().view(numpy.uint32)``).
    """

    def __init__(self, h: int, w: int, nbins: int = 0, layout: int = IHIST_BIN_MAJOR, tune=None,
                 bin_of_value=None, edges=None, bins_per_channel=None):
        """tune: None (library defaults), a dict of ihist_tune_t fields, or
        "auto" (measured by the autotuner, cached per device and shape).
        Binning: uniform over nbins bins by default; or bin_of_value (256
        ints, -1 = no bin), or edges (nbins + 1 increasing ints in [0, 256]),
        or bins_per_channel for the joint bins of multi-channel frames
        ([h][w][C] uint8 tensors; nbins = the product)."""
        if edges is not None:
            nbins = len(edges) - 1
        if bins_per_channel is not None:
            nbins = 1
            for b in bins_per_channel:
                nbins *= int(b)
        self.h, self.w, self.nbins, self.layout = h, w, nbins, layout
        self.channels = len(bins_per_channel) if bins_per_channel is not None else 1
        if tune == "auto":
            from . import autotune
            tune = autotune.tune_plan(h, w, nbins, layout)
        if bin_of_value is not None:
            self.handle = ihist_plan_lut(h, w, nbins, layout, bin_of_value, tune)
        elif edges is not None:
            self.handle = ihist_plan_edges(h, w, layout, edges, tune)
        elif bins_per_channel is not None:
            self.handle = ihist_plan_joint(h, w, bins_per_channel, layout, tune)
        else:
            self.handle = (ihist_plan_tuned(h, w, nbins, layout, tune) if tune
                           else ihist_plan(h, w, nbins, layout))
        self.tune = ihist_plan_get_tune(self.handle)

    @property
    def out_shape(self):
        return out_shape(self.h, self.w, self.nbins, self.layout)

    def empty_output(self, device=None):
        import torch
        return torch.empty(self.out_shape, dtype=torch.int32, device=device or "cuda")

    def compute(self, frame, out=None, stream=None):
        """Integral histogram of a CUDA uint8 [h][w] tensor (row stride may
        exceed w), or [h][w][C] with interleaved channels for a joint plan."""
        import torch
        if self.channels > 1 or frame.dim() == 3:
            if (frame.dtype != torch.uint8 or frame.dim() != 3 or not frame.is_cuda
                    or tuple(frame.shape) != (self.h, self.w, self.channels)
                    or frame.stride(2) != 1 or frame.stride(1) != self.channels):
                raise ValueError("frame must be a uint8 CUDA [h][w][C] tensor with interleaved channels")
        elif frame.dtype != torch.uint8 or frame.dim() != 2 or not frame.is_cuda:
            raise ValueError("frame must be a 2-D uint8 CUDA tensor")
        elif tuple(frame.shape) != (self.h, self.w) or frame.stride(1) != 1:
            raise ValueError("frame shape/stride mismatch: %s %s" % (tuple(frame.shape), frame.stride()))
        if out is None:
            out = self.empty_output(frame.device)
        if out.dtype not in (torch.int32,) or not out.is_contiguous() or out.numel() != self.h * self.w * self.nbins:
            raise ValueError("out must be a contiguous int32 tensor of %d elements" % (self.h * self.w * self.nbins))
        ihist_compute(self.handle, frame.data_ptr(), frame.stride(0), out.data_ptr(), _stream(stream))
        return out

    def query(self, hist, rects, out=None, stream=None):
        """Region histograms (Eq. 2) of CUDA int32 rects [n][4] -> int32 [n][nbins]."""
        import torch
        if rects.dtype != torch.int32 or not rects.is_contiguous() or rects.dim() != 2 or rects.shape[1] != 4:
            raise ValueError("rects must be a contiguous int32 [n][4] tensor")
        n = rects.shape[0]
        if out is None:
            out = torch.empty((n, self.nbins), dtype=torch.int32, device=rects.device)
        ihist_query(self.handle, hist.data_ptr(), rects.data_ptr(), n, out.data_ptr(), _stream(stream))
        return out

    def query_sorted(self, hist, rects, out=None, work=None, bins_per_pass: int = 0, stream=None):
        """As query, with the corners bucketed by row first (bin-major plans,
        large batches; see ihist_query_sorted).  work: a CUDA uint8 scratch
        tensor of query_work_bytes(n) bytes (allocated here if None)."""
        import torch
        if rects.dtype != torch.int32 or not rects.is_contiguous() or rects.dim() != 2 or rects.shape[1] != 4:
            raise ValueError("rects must be a contiguous int32 [n][4] tensor")
        n = rects.shape[0]
        if out is None:
            out = torch.empty((n, self.nbins), dtype=torch.int32, device=rects.device)
        need = self.query_work_bytes(n, bins_per_pass)
        if work is None:
            work = torch.empty((need,), dtype=torch.uint8, device=rects.device)
        if work.numel() < need or work.data_ptr() % 256:
            raise ValueError("work must be a 256-byte aligned uint8 tensor of %d bytes" % need)
        ihist_query_sorted(self.handle, hist.data_ptr(), rects.data_ptr(), n, out.data_ptr(), bins_per_pass,
                           work.data_ptr(), work.numel(), _stream(stream))
        return out

    def query_work_bytes(self, n: int, bins_per_pass: int = 0) -> int:
        return ihist_query_work_bytes(self.handle, n, bins_per_pass)

    def window_search(self, hist, target, win_h: int, win_w: int, stride: int, out=None, stream=None):
        """Histogram-intersection score of every win_h x win_w window on a
        stride grid against target (CUDA int32 [nbins]) -> int32 [ny][nx]."""
        import torch
        if target.dtype != torch.int32 or not target.is_contiguous() or target.numel() != self.nbins:
            raise ValueError("target must be a contiguous int32 tensor of nbins counts")
        ny, nx = window_grid(self.h, self.w, win_h, win_w, stride) if stride >= 1 else (0, 0)
        if out is None:
            out = torch.empty((max(ny, 0), max(nx, 0)), dtype=torch.int32, device=target.device)
        ihist_window_search(self.handle, hist.data_ptr(), target.data_ptr(), win_h, win_w, stride, out.data_ptr(),
                            0, _stream(stream))
        return out

    def window_best(self, hist, target, win_h: int, win_w: int, stride: int, stream=None):
        """(score, i, j) of the best window of the search (highest score, the
        first in row-major order among ties); no score map is written."""
        import torch
        if target.dtype != torch.int32 or not target.is_contiguous() or target.numel() != self.nbins:
            raise ValueError("target must be a contiguous int32 tensor of nbins counts")
        best = torch.zeros(1, dtype=torch.int64, device=target.device)
        ihist_window_search(self.handle, hist.data_ptr(), target.data_ptr(), win_h, win_w, stride, 0,
                            best.data_ptr(), _stream(stream))
        v = int(best.item()) & 0xffffffffffffffff
        if v == 0:
            return None
        _, nx = window_grid(self.h, self.w, win_h, win_w, stride)
        idx = 0xffffffff - (v & 0xffffffff)
        return v >> 32, idx // nx, idx % nx

    def status(self, stream=None) -> int:
        return ihist_status(self.handle, _stream(stream))

    def workspace_bytes(self) -> int:
        return ihist_workspace_bytes(self.handle)

    def close(self):
        if self.handle:
            ihist_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def out_shape(h: int, w: int, nbins: int, layout: int):
    """Shape of H in a layout: [B][h][w], [h][w][B] or [B/4][h][w][4]."""
    if layout == IHIST_BIN_MAJOR:
        return (nbins, h, w)
    if layout == IHIST_QUAD_MAJOR:
        return (nbins // 4, h, w, 4)
    return (h, w, nbins)


class Batch:
    """Many frames (CUDA uint8 [h][w] tensors, any mix of shapes) in one
    persistent launch; outputs are int32 tensors holding uint32 counts."""

    def __init__(self, frames, nbins, layouts=None, outs=None, tune=None, tables=None, joint=None):
        """tables: None, or one entry per frame, None (uniform bins) or a
        256-entry value -> bin table (see edges_table).  joint: None, or one
        entry per frame, None or the bins of each channel of a joint-bin
        frame ([h][w][C] uint8 tensor, nbins = their product)."""
        import torch
        n = len(frames)
        nb = list(nbins) if hasattr(nbins, "__len__") else [nbins] * n
        ly = list(layouts) if layouts is not None else [IHIST_BIN_MAJOR] * n
        self.frames = list(frames)
        self.nbins, self.layouts = nb, ly
        self.tables = list(tables) if tables is not None else [None] * n
        self.joint = list(joint) if joint is not None else [None] * n
        self.outs = list(outs) if outs is not None else [
            torch.empty(out_shape(f.shape[0], f.shape[1], b, l), dtype=torch.int32, device=f.device)
            for f, b, l in zip(self.frames, nb, ly)]
        if tune == "auto":
            from . import autotune
            tune = autotune.tune_batch([(f.shape[0], f.shape[1], b, l) for f, b, l in zip(self.frames, nb, ly)],
                                       tables=any(t is not None for t in self.tables))
        self.handle = ihist_batch_plan(self._desc(), tune or None)
        self.tune = ihist_batch_get_tune(self.handle)

    def _desc(self):
        d = []
        for f, b, l, o, t, j in zip(self.frames, self.nbins, self.layouts, self.outs, self.tables, self.joint):
            if j is not None:
                if (f.dtype.itemsize != 1 or f.dim() != 3 or f.shape[2] != len(j) or f.stride(2) != 1
                        or f.stride(1) != len(j)):
                    raise ValueError("joint frames must be uint8 [h][w][C] tensors with interleaved channels")
            elif f.dtype.itemsize != 1 or f.dim() != 2 or f.stride(1) != 1:
                raise ValueError("frames must be 2-D uint8 tensors with unit column stride")
            d.append((f.shape[0], f.shape[1], b, l, f.data_ptr(), f.stride(0), o.data_ptr(), t, j))
        return d

    def set_io(self, frames, outs, nbins=None, layouts=None, stream=None, tables=None, joint=None):
        """Bind new frames/outputs (any shapes that fit the planned slots);
        tables and joint as for the constructor (default: uniform bins of
        one-channel frames)."""
        frames, outs = list(frames), list(outs)
        nb = list(nbins) if nbins is not None else self.nbins[:len(frames)]
        ly = list(layouts) if layouts is not None else self.layouts[:len(frames)]
        tb = list(tables) if tables is not None else [None] * len(frames)
        jt = list(joint) if joint is not None else [None] * len(frames)
        old = (self.frames, self.outs, self.nbins, self.layouts, self.tables, self.joint)
        self.frames, self.outs, self.nbins, self.layouts, self.tables, self.joint = frames, outs, nb, ly, tb, jt
        try:
            ihist_batch_set_io(self.handle, self._desc(), _stream(stream))
        except Exception:
            self.frames, self.outs, self.nbins, self.layouts, self.tables, self.joint = old
            raise

    def compute(self, stream=None):
        ihist_batch_compute(self.handle, _stream(stream))
        return self.outs

    def query(self, i, rects, out=None, stream=None):
        import torch
        n = rects.shape[0]
        if out is None:
            out = torch.empty((n, self.nbins[i]), dtype=torch.int32, device=rects.device)
        ihist_batch_query(self.handle, i, self.outs[i].data_ptr(), rects.data_ptr(), n, out.data_ptr(),
                          _stream(stream))
        return out

    def query_all(self, rects, out=None, stream=None):
        """rects: CUDA int32 [nframes][n][4] -> int32 [n * sum(nbins)] (frame-major rows)."""
        import torch
        n = rects.shape[1]
        if out is None:
            out = torch.empty((n * sum(self.nbins),), dtype=torch.int32, device=rects.device)
        ihist_batch_query_all(self.handle, rects.data_ptr(), n, out.data_ptr(), _stream(stream))
        return out

    def upload_compute(self, h_frames, stream=None, copy_stream=None):
        """Copy page-locked host frames (CPU uint8 tensors) in on copy_stream, then compute."""
        ihist_batch_upload_compute(self.handle, [f.data_ptr() for f in h_frames], _stream(stream),
                                   _stream(copy_stream))
        return self.outs

    def status(self, stream=None) -> int:
        return ihist_batch_status(self.handle, _stream(stream))

    def items(self) -> int:
        return ihist_batch_items(self.handle)

    def close(self):
        if self.handle:
            ihist_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
