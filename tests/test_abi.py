"""The C ABI library loads and exports every entry point its header declares
(no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_1711_01919_gb300 import build as cuda_build
from paper_1711_01919_gb300 import ihist

HEADER = os.path.join(cuda_build.ROOT, "include", "ihist.h")


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return ihist.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ihist_[a-z_]+)\s*\(", text)))


def test_header_declares_binding_names():
    assert set(declared_functions()) == set(ihist.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(cuda_build.LIB)
    for name in declared_functions():
        assert hasattr(so, name), name


def test_output_bytes_and_error_strings(lib):
    assert ihist.ihist_output_bytes(1080, 1920, 64) == 530841600
    assert ihist.ihist_output_bytes(8192, 8192, 128) == 34359738368
    assert ihist.ihist_output_bytes(0, 5, 5) == 0
    for code in range(8):
        assert ihist.ihist_error_string(code) and ihist.ihist_error_string(code) != "unknown status"
    assert ihist.ihist_error_string(99) == "unknown status"


@pytest.mark.parametrize("h,w,b,layout", [(0, 10, 4, 0), (10, 0, 4, 0), (65536, 4, 4, 0), (4, 4, 0, 0),
                                          (4, 4, 257, 0), (4, 4, 4, 3), (4, 4, 6, 2), (70000, 70000, 4, 0)])
def test_plan_rejects_bad_shapes_before_touching_cuda(lib, h, w, b, layout):
    with pytest.raises(ihist.IhistError) as e:
        ihist.ihist_plan(h, w, b, layout)
    assert e.value.code == ihist.IHIST_ERR_INVALID_ARG


def test_plan_rejects_bad_tuning(lib):
    for tune in ({"rows_per_band": 256}, {"bins_per_cta": 5}, {"chunks_per_warp": 3}, {"overlap": 2}, {"overlap": -1}):
        with pytest.raises(ihist.IhistError) as e:
            ihist.ihist_plan_tuned(16, 16, 4, 0, tune)
        assert e.value.code == ihist.IHIST_ERR_INVALID_ARG
    for h, w in ((16, 65536), (65536, 16), (0, 16), (16, 0)):  # outside 1 <= h, w <= 65535
        with pytest.raises(ihist.IhistError) as e:
            ihist.ihist_plan(h, w, 4, 0)
        assert e.value.code == ihist.IHIST_ERR_INVALID_ARG


def test_null_plan_calls_are_rejected(lib):
    L = lib
    assert L.ihist_compute(None, None, 0, None, None) == ihist.IHIST_ERR_INVALID_ARG
    assert L.ihist_query(None, None, None, 0, None, None) == ihist.IHIST_ERR_INVALID_ARG
    st = ctypes.c_int()
    assert L.ihist_status(None, None, ctypes.byref(st)) == ihist.IHIST_ERR_INVALID_ARG
    assert L.ihist_workspace_bytes(None) == 0
    L.ihist_destroy(None)


def test_plan_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ihist.IhistError) as e:
        ihist.ihist_plan(64, 64, 8, 0)
    assert e.value.code == ihist.IHIST_ERR_CUDA


def test_other_bin_structures_reject_bad_arguments_before_touching_cuda(lib):
    bad = [
        (lambda: ihist.ihist_plan_edges(8, 8, 0, [10, 10, 20]), ihist.IHIST_ERR_INVALID_ARG),   # not increasing
        (lambda: ihist.ihist_plan_edges(8, 8, 0, [-1, 20]), ihist.IHIST_ERR_INVALID_ARG),        # below 0
        (lambda: ihist.ihist_plan_edges(8, 8, 0, [0, 257]), ihist.IHIST_ERR_INVALID_ARG),        # above 256
        (lambda: ihist.ihist_plan_lut(8, 8, 4, 0, [4] * 256), ihist.IHIST_ERR_INVALID_ARG),      # bin >= nbins
        (lambda: ihist.ihist_plan_lut(8, 8, 4, 0, [-2] * 256), ihist.IHIST_ERR_INVALID_ARG),     # below -1
        (lambda: ihist.ihist_plan_lut(8, 8, 4, 0, [0] * 256, {"bins_per_cta": 16}), ihist.IHIST_ERR_UNSUPPORTED),
        (lambda: ihist.ihist_plan_joint(8, 8, [8, 8, 8]), ihist.IHIST_ERR_UNSUPPORTED),         # 512 joint bins
        (lambda: ihist.ihist_plan_joint(8, 8, [2, 0]), ihist.IHIST_ERR_INVALID_ARG),
        (lambda: ihist.ihist_plan_joint(8, 8, [2] * 5), ihist.IHIST_ERR_INVALID_ARG),           # 5 channels
        (lambda: ihist.ihist_plan_joint(8, 20000, [2, 2, 2, 2]), ihist.IHIST_ERR_UNSUPPORTED),  # w * C too wide
    ]
    for make, code in bad:
        with pytest.raises(ihist.IhistError) as e:
            make()
        assert e.value.code == code
    assert ihist.ihist_plan_channels(None) == 0


def test_window_search_rejects_null_plan(lib):
    assert lib.ihist_window_search(None, None, None, 1, 1, 1, None, None, None) == ihist.IHIST_ERR_INVALID_ARG
    assert ihist.window_grid(1080, 1920, 64, 64, 4) == (255, 465)
    assert ihist.window_grid(10, 10, 10, 10, 3) == (1, 1)


def test_mapping_arguments_checked_before_touching_cuda(lib):
    assert ihist.ihist_mapping_workspace_bytes(ihist.IHIST_MAPPING_CW_STS, 1080, 1920, 64) == 530841600
    assert ihist.ihist_mapping_workspace_bytes(ihist.IHIST_MAPPING_WF_TIS, 1080, 1920, 64) == 0
    for mapping, h, w, b in [(0, 8, 8, 4), (4, 8, 8, 4), (2, 0, 8, 4), (3, 8, 8, 0), (1, 8, 8, 4)]:
        # (the last: CW-STS without its workspace)
        assert lib.ihist_mapping_compute(mapping, h, w, b, ctypes.c_void_p(16), w, ctypes.c_void_p(16), None,
                                         None) == ihist.IHIST_ERR_INVALID_ARG


def test_batch_tables_are_checked_before_touching_cuda(lib):
    # (h, w, nbins, layout, d_in, in_pitch, d_out, table): pointers are never
    # dereferenced because the arguments are refused first
    good = [(v * 8) >> 8 for v in range(256)]
    for table, code in ((good[:255] + [8], ihist.IHIST_ERR_INVALID_ARG),
                        ([-2] + good[1:], ihist.IHIST_ERR_INVALID_ARG)):
        with pytest.raises(ihist.IhistError) as e:
            ihist.ihist_batch_plan([(16, 16, 8, 0, 16, 16, 16, table)])
        assert e.value.code == code
    with pytest.raises(ihist.IhistError) as e:  # tables need 4 or 8 bins per CTA
        ihist.ihist_batch_plan([(16, 16, 8, 0, 16, 16, 16, good)], tune={"bins_per_cta": 16})
    assert e.value.code == ihist.IHIST_ERR_UNSUPPORTED
    with pytest.raises(ValueError):
        ihist.ihist_batch_plan([(16, 16, 8, 0, 16, 16, 16, good[:100])])


def test_edges_table_matches_the_oracle_binning():
    import oracle
    for edges in ([0, 256], [0, 16, 64, 128, 256], [10, 11, 200], [0, 1, 2, 255, 256]):
        table = ihist.edges_table(edges)
        assert table == [int(oracle.bin_of_edges(v, edges)) for v in range(256)]
    for bad in ([0], [5, 5], [0, 300], [-1, 4], [9, 3]):
        with pytest.raises(ValueError):
            ihist.edges_table(bad)


def test_batch_joint_frames_are_checked_before_touching_cuda(lib):
    # (h, w, nbins, layout, d_in, in_pitch, d_out, table, bins_per_channel)
    good = [4, 4]
    for fr, code in (((16, 16, 15, 0, 16, 64, 16, None, good), ihist.IHIST_ERR_INVALID_ARG),   # 4 x 4 != 15
                     ((16, 16, 16, 0, 16, 64, 16, [0] * 256, good), ihist.IHIST_ERR_INVALID_ARG),  # joint + table
                     ((16, 16, 0, 0, 16, 64, 16, None, [0, 4]), ihist.IHIST_ERR_INVALID_ARG),
                     ((16, 16, 256, 0, 16, 64, 16, None, [32, 16]), ihist.IHIST_ERR_UNSUPPORTED)):   # 512 bins
        with pytest.raises(ihist.IhistError) as e:
            ihist.ihist_batch_plan([fr])
        assert e.value.code == code, fr
    with pytest.raises(ValueError):
        ihist.ihist_batch_plan([(16, 16, 32, 0, 16, 64, 16, None, [2, 2, 2, 2, 2])])
