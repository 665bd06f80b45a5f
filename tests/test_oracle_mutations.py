"""Plant plausible mistakes in copies of the oracle source and check that the
pins catch every one (CPU only; the committed oracle is never modified)."""
import os

import pytest

import oracle
import oracle_pins as pins

# (name, text in ihist_oracle.c, replacement) -- each a plausible slip.
MUTATIONS = [
    ("dropped_diagonal_term", "above + left - diag + q", "above + left + q"),
    ("diagonal_sign", "above + left - diag + q", "above + left + diag + q"),
    ("exclusive_not_inclusive", "above + left - diag + q", "above + left - diag"),
    ("diagonal_index", "plane[(size_t)(x - 1) * w + (y - 1)] : 0u", "plane[(size_t)(x - 1) * w + y] : 0u"),
    ("left_index", "plane[(size_t)x * w + (y - 1)] : 0u", "plane[(size_t)(x > 1 ? x - 1 : x) * w + (y - 1)] : 0u"),
    ("mirrored_column", "img[(size_t)x * pitch + y]", "img[(size_t)x * pitch + (w - 1 - y)]"),
    ("rounded_bins", "return (v * nbins) / 256;", "return (v * nbins + 128) / 256;"),
    ("bins_over_255", "return (v * nbins) / 256;", "return (v * nbins) / 255 < nbins ? (v * nbins) / 255 : nbins - 1;"),
    ("query_corner_sign", "r = br - tr - bl + tl;", "r = br - tr - bl - tl;"),
    ("query_left_off_by_one", "P[(size_t)y1 * w + (x0 - 1)] : 0u", "P[(size_t)y1 * w + x0] : 0u"),
    ("query_top_off_by_one", "P[(size_t)(y0 - 1) * w + x1] : 0u", "P[(size_t)y0 * w + x1] : 0u"),
    ("query_transposed_corner", "P[(size_t)y1 * w + x1];", "P[(size_t)(y1 < w ? y1 : 0) * w + (x1 < h ? x1 : 0)];"),
    ("brute_region_open_end", "for (int r = y0; r <= y1; ++r)", "for (int r = y0; r < y1; ++r)"),
    ("threads_skip_last_bin", "for (int k = j->first; k < j->nbins; k += j->stride)",
     "for (int k = j->first; k < j->nbins - 1; k += j->stride)"),
    ("edges_closed_upper", "if (edges[k] <= v && v < edges[k + 1]) return k;",
     "if (edges[k] <= v && v <= edges[k + 1]) return k;"),
    ("edges_outside_to_last_bin", "  return -1;\n}\n\n/* Algorithm 1 with Q(k, v)",
     "  return nbins - 1;\n}\n\n/* Algorithm 1 with Q(k, v)"),
    ("mapped_no_bin_counts_in_bin_0", "uint32_t q = (map[img[(size_t)x * pitch + y]] == k) ? 1u : 0u;",
     "uint32_t q = (map[img[(size_t)x * pitch + y]] == k || (k == 0 && map[img[(size_t)x * pitch + y]] < 0)) ? 1u : 0u;"),
    ("joint_channel_order", "k = k * bins[c] + oracle_bin_of(px[c], bins[c]);",
     "k = k * bins[c] + oracle_bin_of(px[channels - 1 - c], bins[c]);"),
    ("joint_radix", "k = k * bins[c] + oracle_bin_of(px[c], bins[c]);",
     "k = k + oracle_bin_of(px[c], bins[c]) * (c ? bins[c - 1] : 1);"),
    ("joint_pixel_stride", "img + (size_t)x * pitch + (size_t)y * channels;", "img + (size_t)x * pitch + (size_t)y;"),
    ("window_short_rows", "for (int r = i * stride; r < i * stride + win_h; ++r)",
     "for (int r = i * stride; r < i * stride + win_h - 1; ++r)"),
    # (each mutant below still reads and writes only inside its buffers)
    ("window_square_assumed", "for (int r = i * stride; r < i * stride + win_h; ++r)",
     "for (int r = i * stride; r < i * stride + (win_w < win_h ? win_w : win_h); ++r)"),
    ("window_max_not_min", "score += count[b] < target[b] ? count[b] : target[b];",
     "score += count[b] > target[b] ? count[b] : target[b];"),
    ("window_row_step", "for (int r = i * stride; r < i * stride + win_h; ++r)",
     "for (int r = i * (stride - (stride > 1)); r < i * (stride - (stride > 1)) + win_h; ++r)"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_reject_mutant(tmp_path, name, old, new):
    src = open(oracle.SOURCE).read()
    assert src.count(old) >= 1, "mutation site not found: %s" % name
    mutated = tmp_path / ("mut_%s.c" % name)
    mutated.write_text(src.replace(old, new, 1))
    lib = oracle.compile_c(str(mutated), str(tmp_path / ("libmut_%s.so" % name)))
    o = oracle.Oracle(lib)
    failed = []
    for check in pins.ALL_CHECKS:
        try:
            check(o)
        except AssertionError:
            failed.append(check.__name__)
    assert failed, "no pin caught mutation %s" % name
