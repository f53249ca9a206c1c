"""Host-side logic of bench.py that needs no GPU: the MUPS reading of the paper's speed formula,
checked against every row the paper prints in Table 2 (Sec. 4.5)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table2():
    rows = []
    for line in open(os.path.join(GOLDEN, "paper_table2_mups.txt")):
        line = line.split("#")[0].split()
        if len(line) == 3:
            rows.append((int(line[0]), float(line[1]), float(line[2])))
    return rows


def test_mups_reading_reproduces_table2():
    """The speed formula is garbled in the text; read as N k / (10^6 t) with k = 1000 timed steps it
    gives every printed speed of Table 2 to the printed digits."""
    sys.path.insert(0, ROOT)
    import bench
    rows = _table2()
    assert len(rows) == 7
    for n, seconds, printed in rows:
        assert bench.mups(n, 1000, seconds) == pytest.approx(printed, rel=5e-6, abs=5e-4), (n, seconds)
