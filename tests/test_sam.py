"""SAM output and mapping quality (host code of the library; no GPU).

MAPQ is pinned to the closed forms the paper prints (-100 log2 0.9 = 15.2, 2^-0.62 = 0.651)
and to exact powers of two; the SAM lines are checked field by field on hand-made results.
"""
import math

import numpy as np
import pytest

import paper_1403_2136_gb300 as mss
from tests.parity_util import concat_reads


@pytest.fixture(scope="module")
def lib():
    from paper_1403_2136_gb300 import build
    build.build()
    return mss.load_library()


def test_mapq_closed_forms(lib):
    assert mss.mss_mapq(10, 9) == 15          # -100 log2 0.9 = 15.2
    assert mss.mss_mapq(1000, 651) == 62      # p = 0.651 = 2^-0.62
    assert mss.mss_mapq(100, 50) == 100       # p = 1/2
    assert mss.mss_mapq(100, 25) == 200       # p = 1/4
    assert mss.mss_mapq(100, 12) == 254       # above 254: capped
    assert mss.mss_mapq(100, 0) == 254        # no competing fragment
    assert mss.mss_mapq(0, 0) == 0            # nothing mapped
    assert mss.mss_mapq(7, 7) == 0            # tie: certainly ambiguous
    for best in range(1, 60):
        for second in range(1, best):
            want = min(254, int(math.floor(-100 * math.log2(second / best) + 0.5)))
            assert mss.mss_mapq(best, second) == want


def _hits(rows):
    h = np.zeros(len(rows), dtype=mss.HIT_DTYPE)
    for i, (b1, b2, s1, s2, off, strand, flags) in enumerate(rows):
        h[i] = (b1, b2, s1, s2, off, strand, flags)
    return h


def _alns(rows):
    a = np.zeros(len(rows), dtype=mss.ALN_DTYPE)
    for i, r in enumerate(rows):
        a[i] = r
    return a


def test_sam_lines(lib):
    reads = ["ACGTACGTAC", "aacgTTG", "ACGTN", "GGGG", ""]
    seq, off = concat_reads(reads)
    hits = _hits([(3, 7, 50, 10, 1234, 0, 0),      # mapped, forward
                  (0, 1, 35, 20, 99, 1, 0),        # mapped, reverse strand
                  (5, 6, 20, 19, 500, 0, 1),       # repeat: unmapped
                  (2, 4, 20, 5, 700, 0, 0),        # no in-band alignment: unmapped
                  (0, -1, 0, 0, 0, 0, 1)])         # empty read
    cig = ["10M", "3M1I3M", "5M", "", ""]
    alns = _alns([(50, 3, 1234, 1244), (20, 6, 99, 105), (25, 2, 500, 505), (-2147483648, 0, 0, 0), (0, 0, 0, 0)])
    text = mss.format_sam("chr1", 100_000, seq, off, hits, alns, cig)
    lines = text.rstrip("\n").split("\n")
    assert lines[0] == "@HD\tVN:1.6\tSO:unsorted"
    assert lines[1] == "@SQ\tSN:chr1\tLN:100000"
    assert lines[2].startswith("@PG\tID:maxss")
    f = [ln.split("\t") for ln in lines[3:]]
    assert len(f) == 5 and all(len(x) >= 11 for x in f)
    assert f[0][:11] == ["r0", "0", "chr1", "1235", str(mss.mss_mapq(50, 10)), "10M", "*", "0", "0", "ACGTACGTAC", "*"]
    assert "AS:i:50" in f[0] and "ZM:i:50" in f[0] and "XS:i:10" in f[0]
    # reverse strand: SEQ is the reverse complement, upper case
    assert f[1][1] == "16" and f[1][3] == "100" and f[1][5] == "3M1I3M" and f[1][9] == "CAACGTT"
    assert f[2][1] == "4" and f[2][2] == "*" and f[2][3] == "0" and f[2][4] == "0" and f[2][9] == "ACGTN"
    assert f[3][1] == "4" and "AS:i" not in lines[6]
    assert f[4][1] == "4" and f[4][9] == "*"
    # no header, no CIGARs
    t2 = mss.format_sam("chr1", 100_000, seq, off, hits, alns, None, header=False)
    assert not t2.startswith("@") and t2.split("\n")[0].split("\t")[5] == "*"


def test_sam_size_query_and_errors(lib):
    seq, off = concat_reads(["ACGT"])
    hits = _hits([(0, -1, 4, 0, 0, 0, 0)])
    alns = _alns([(4, 2, 0, 4)])
    cbuf = np.frombuffer(b"4M\x00\x00", dtype=np.uint8).copy()
    import ctypes
    n = lib.mss_format_sam(b"g", 10, seq.ctypes.data, off.ctypes.data, 1, hits.ctypes.data, alns.ctypes.data,
                           cbuf.ctypes.data, 4, 0, None, 0)
    assert n > 0
    small = ctypes.create_string_buffer(int(n))          # one byte short of the NUL: nothing written
    assert lib.mss_format_sam(b"g", 10, seq.ctypes.data, off.ctypes.data, 1, hits.ctypes.data, alns.ctypes.data,
                              cbuf.ctypes.data, 4, 0, small, n) == n and small.value == b""
    assert lib.mss_format_sam(b"bad name", 10, seq.ctypes.data, off.ctypes.data, 1, hits.ctypes.data,
                              alns.ctypes.data, None, 0, 0, None, 0) < 0
    assert lib.mss_format_sam(b"g", 0, seq.ctypes.data, off.ctypes.data, 1, hits.ctypes.data, alns.ctypes.data,
                              None, 0, 0, None, 0) < 0
