"""The DRAM-traffic records under profiles/ that bench.py puts into its
roofline blocks are of the current kernel sources: each record carries a hash
of the sources it was captured on, and bench.py reports no traffic for a
kernel whose sources have changed since.  This fails as soon as a kernel is
edited without its record being captured again."""
import glob
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_traffic_records_match_the_kernel_sources():
    import bench
    records = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.json")))
    assert records, "no traffic records"
    for path in records:
        name = os.path.splitext(os.path.basename(path))[0]
        rec = json.load(open(path))
        assert name in bench.KERNEL_SOURCES, name
        assert rec["kernel_source_sha"] == bench.kernel_source_sha(name), name
        assert rec["dram_bytes_per_launch"] > 0 and rec["algorithmic_bytes_per_launch"] > 0, name
        # the captured traffic is within a few per cent of the algorithmic bytes (no re-reads)
        assert 0.9 <= rec["dram_bytes_per_launch"] / rec["algorithmic_bytes_per_launch"] <= 1.05, name
