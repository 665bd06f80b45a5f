"""Host-side helpers of the Python binding, on the CPU: output shapes of the
three layouts, the layouts the autotuner may pick, and how frame tuples are
packed into the C frame struct (tables and joint bins included)."""
import ctypes

import pytest

from paper_1711_01919_gb300 import autotune, ihist


def test_out_shape_of_each_layout():
    assert ihist.out_shape(3, 5, 8, ihist.IHIST_BIN_MAJOR) == (8, 3, 5)
    assert ihist.out_shape(3, 5, 8, ihist.IHIST_PIXEL_MAJOR) == (3, 5, 8)
    assert ihist.out_shape(3, 5, 8, ihist.IHIST_QUAD_MAJOR) == (2, 3, 5, 4)
    for layout in (0, 1, 2):
        shape = ihist.out_shape(7, 11, 12, layout)
        n = 1
        for d in shape:
            n *= d
        assert n == 7 * 11 * 12 == ihist.ihist_output_bytes(7, 11, 12) // 4


def test_quad_major_is_offered_only_when_every_bin_count_is_a_multiple_of_4():
    assert autotune.layouts_for([16, 32, 64]) == [0, 1, 2]
    assert autotune.layouts_for([16, 7]) == [0, 1]
    assert autotune.layouts_for([4]) == [0, 1, 2]


def test_frame_tuples_pack_into_the_c_struct():
    table = [v % 3 - 1 for v in range(256)]
    arr = ihist._frames_array([(4, 5, 6, 1, 0x1000, 7, 0x2000),
                               (8, 9, 12, 0, 0x3000, 9, 0x4000, table),
                               (2, 3, 64, 2, 0x5000, 9, 0x6000, None, [4, 4, 4])])
    f0, f1, f2 = arr[0], arr[1], arr[2]
    assert (f0.h, f0.w, f0.nbins, f0.layout, f0.d_in, f0.in_pitch, f0.d_out) == (4, 5, 6, 1, 0x1000, 7, 0x2000)
    assert not f0.bin_of_value and f0.channels == 0
    assert [f1.bin_of_value[v] for v in range(256)] == table and f1.channels == 0
    assert not f2.bin_of_value and f2.channels == 3 and list(f2.bins_per_channel) == [4, 4, 4, 0]
    # the sizes tests/c_client.c asserts for the C declarations
    assert ctypes.sizeof(ihist.ihist_frame_t) == 72
    assert ctypes.sizeof(ihist.ihist_tune_t) == 40


def test_bad_tables_are_refused_before_any_call():
    with pytest.raises(ValueError):
        ihist._frames_array([(4, 5, 6, 0, 0x1000, 7, 0x2000, [0] * 255)])
