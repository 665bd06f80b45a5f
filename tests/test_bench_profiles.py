"""The bench's reading of the committed ncu summaries (CPU): the traffic of
the bench's kernel and of the 8192x8192 launch shape is taken from
profiles/ only while the summary was captured on the current kernel source,
and inline comments after a value are ignored."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_committed_summaries_match_the_kernel_source():
    for path in (bench.PROFILE, bench.PROFILE_MP64):
        traffic = bench.profiled_traffic(path)
        assert traffic is not None, "%s was not captured on the current kernel source" % path
        # DRAM traffic of a launch is close to its algorithmic bytes (each word written once)
        algo = (64 * bench.algorithmic_bytes_per_frame() if path == bench.PROFILE
                else 8192 * 8192 * 128 * 4 + 8192 * 8192)
        assert 0.99 < traffic / algo < 1.02


def test_stale_or_commented_summaries(tmp_path):
    p = tmp_path / "s.txt"
    p.write_text("# a comment = not a value\nscan_source_sha256_16 = %s\n"
                 "traffic_bytes_per_launch = 123456   # trailing comment\n" % bench.scan_source_hash())
    assert bench.profiled_traffic(str(p)) == 123456
    p.write_text("scan_source_sha256_16 = 0000000000000000\ntraffic_bytes_per_launch = 123456\n")
    assert bench.profiled_traffic(str(p)) is None
    assert bench.profiled_traffic(str(tmp_path / "missing.txt")) is None
