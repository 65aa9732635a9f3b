"""Host logic of bench.py that needs no GPU: the stored-traffic lookup (a
capture counts only for the sources and launch it was taken of) and the
per-phase algorithmic byte counts."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def write_capture(path, sha, **kv):
    lines = ["# a capture", f"sources_sha256 = {sha}"] + [f"{k} = {v}" for k, v in kv.items()]
    path.write_text("\n".join(lines) + "\n")


def test_stored_traffic_matches_sources_and_launch(tmp_path):
    sha = bench.sources_sha256(bench.LOB_TRAFFIC_SOURCES)
    f = tmp_path / "cap.txt"
    write_capture(f, sha, n_books=10, cap=64, warps_per_book=2, dram_bytes_read=1000, dram_bytes_write=24)
    assert bench.stored_traffic(str(f), bench.LOB_TRAFFIC_SOURCES, n_books=10, cap=64, warps_per_book=2) == 1024
    # another launch shape or size: not this capture
    assert bench.stored_traffic(str(f), bench.LOB_TRAFFIC_SOURCES, n_books=10, cap=64, warps_per_book=1) is None
    assert bench.stored_traffic(str(f), bench.LOB_TRAFFIC_SOURCES, n_books=11, cap=64, warps_per_book=2) is None
    # sources changed since the capture
    write_capture(f, "0" * 64, n_books=10, cap=64, warps_per_book=2, dram_bytes_read=1000, dram_bytes_write=24)
    assert bench.stored_traffic(str(f), bench.LOB_TRAFFIC_SOURCES, n_books=10, cap=64, warps_per_book=2) is None
    # a key the caller requires is missing, or no file
    write_capture(f, sha, n_books=10, dram_bytes_read=1000, dram_bytes_write=24)
    assert bench.stored_traffic(str(f), bench.LOB_TRAFFIC_SOURCES, n_books=10, cap=64) is None
    assert bench.stored_traffic(str(tmp_path / "none.txt"), bench.LOB_TRAFFIC_SOURCES) is None


def test_sources_hash_covers_every_listed_file(tmp_path):
    a = bench.sources_sha256(("lob.cu",))
    b = bench.sources_sha256(("lob.cu", "common.cuh"))
    assert a != b and len(a) == 64


def test_kernel_bytes_per_phase():
    st = {"n_start": [100, 10], "extent": [200, 50], "grass_eaten": 7, "eaten": 3, "parents": [5, 2],
          "starved": [4, 1], "births": [5, 2]}
    # move: every live flag of the extent, then per agent record + cell accesses
    assert bench.kernel_bytes(0, st) == 4 * 200 + 100 * (16 + 16 + 12)
    assert bench.kernel_bytes(3, st) == 4 * 50 + 10 * (16 + 16 + 8)
    # births: per child index, parent read/write, child write, flag (+ sheep victim key)
    assert bench.kernel_bytes(2, st) == 5 * (4 + 4 + 16 + 4 + 16 + 4 + 8)
    assert bench.kernel_bytes(5, st) == 2 * (4 + 4 + 16 + 4 + 16 + 4)
    # scan: grows with winners, parents and deaths
    base = bench.kernel_bytes(1, st)
    more = dict(st, grass_eaten=8)
    assert bench.kernel_bytes(1, more) - base == 4 + 8 + 4
    more = dict(st, eaten=4)
    assert bench.kernel_bytes(4, more) - bench.kernel_bytes(4, st) == 4 + 8 + 8 + 8 + 4
