"""Host logic of bench.py that decides which recorded counters it may use.

The roofline line reports a kernel's DRAM traffic from the committed ncu
summary only while that summary was taken on the current kernel source; the
match is by a hash of the sources with comments and blank lines removed.
"""
import os
import re
import shutil

import pytest

import bench

KDIR = os.path.join("paper_2404_16322_gb300", "csrc", "kernels")


def _copy_tree(tmp_path):
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, KDIR), root / KDIR)
    return root


@pytest.mark.parametrize("kernel", sorted(bench.SCAN_SOURCES))
def test_kernel_hash_ignores_comments_and_blank_lines(tmp_path, kernel):
    root = _copy_tree(tmp_path)
    h0 = bench.kernel_hash(kernel, root=str(root))
    assert h0 == bench.kernel_hash(kernel, root=bench.ROOT)
    f = root / KDIR / bench.SCAN_SOURCES[kernel][-1]
    src = f.read_text()
    f.write_text("// a comment line\n\n/* a block\n   comment */\n" + src.replace("\n", "\n\n", 3) + "\n// tail\n")
    assert bench.kernel_hash(kernel, root=str(root)) == h0
    # a change to the code itself changes the hash
    f.write_text(src + "\nstatic const int kHashProbe = 1;\n")
    assert bench.kernel_hash(kernel, root=str(root)) != h0


def test_every_hashed_source_exists():
    for kernel, files in bench.SCAN_SOURCES.items():
        for name in files:
            assert os.path.exists(os.path.join(bench.ROOT, KDIR, name)), (kernel, name)
        assert os.path.exists(os.path.join(bench.ROOT, "profiles", bench.PROFILE_OF[kernel]))


def test_traffic_only_for_the_recorded_source():
    txt = open(os.path.join(bench.ROOT, "profiles", bench.PROFILE_OF["tc_scan_kernel"])).read()
    recorded = re.search(r"kernel source sha256: ([0-9a-f]{12})", txt).group(1)
    t = bench.traffic_from_profiles("tc_scan_kernel", recorded)
    assert t is not None and t > 0
    other = "0" * 12 if recorded != "0" * 12 else "1" * 12
    assert bench.traffic_from_profiles("tc_scan_kernel", other) is None


def test_peak_is_the_measured_copy_bandwidth():
    gbs, kind = bench.peaks()
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and gbs > 1000
    else:
        assert kind == "fallback" and gbs == 6800.0
