"""The values the paper prints for the stages this library covers: the
compressed sizes of §4.2, Tables 1-2 (tests/golden/paper_compression_tables.txt).
The fixture's transcription and its reading of the columns are pinned by the
savings the paper's text quotes beside the tables; the codec bench reports
its ratios against these sizes."""
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_compression_tables.txt")


def paper_tables():
    """{(array, tol): [size / raw, ...]} from the fixture."""
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if not line:
            continue
        arr, tol, raw, size = line[0], float(line[1]), float(line[2]), float(line[3])
        out.setdefault((arr, tol), []).append(size / raw)
    return out


@pytest.mark.parametrize("arr,tol,saving", [
    ("velocity", 1e-1, 51.1), ("velocity", 0.0, 21.6), ("image", 1e-1, 70.0),
    ("image", 0.0, 12.5), ("seismogram", 1e-4, 82.4), ("seismogram", 1e-4, 89.0)])
def test_table_sizes_match_the_quoted_savings(arr, tol, saving):
    fracs = paper_tables()[(arr, tol)]
    assert any(abs(100.0 * (1.0 - f) - saving) < 0.06 for f in fracs), (arr, tol, fracs)


def test_every_table_entry_is_present_and_ordered():
    t = paper_tables()
    assert sorted(t) == sorted([("velocity", 0.0), ("velocity", 1e-4), ("velocity", 1e-1),
                                ("image", 0.0), ("image", 1e-4), ("image", 1e-1),
                                ("seismogram", 0.0), ("seismogram", 1e-4)])
    for arr in ("velocity", "image"):
        # a looser tolerance never gives a larger file
        assert t[(arr, 1e-1)][0] <= t[(arr, 1e-4)][0] <= t[(arr, 0.0)][0] < 1.0
    assert max(t[("seismogram", 1e-4)]) < min(t[("seismogram", 0.0)]) < 1.0


def test_bench_reads_the_fixture():
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import bench

    t = bench.paper_compression_tables()
    assert t[("seismogram", 1e-4)] == (8.38 / 76.20, 13.38 / 76.20)
    assert t[("velocity", 1e-1)] == 2.98 / 6.10 and t[("image", 0.0)] == 5.34 / 6.10
