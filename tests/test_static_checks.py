"""Static checks of the CUDA sources (no GPU): every device-side wait goes through the one
time-bounded mbarrier wait, no kernel traps on purpose, and every unbounded loop header is a
work-queue loop that ends when the queue runs dry."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = sorted(glob.glob(os.path.join(ROOT, "paper_1403_2136_gb300", "csrc", "*.cu")) +
             glob.glob(os.path.join(ROOT, "paper_1403_2136_gb300", "csrc", "*.cuh")) +
             glob.glob(os.path.join(ROOT, "paper_1403_2136_gb300", "csrc", "*.h")))


def _text(path):
    with open(path) as fh:
        return fh.read()


def test_sources_found():
    names = {os.path.basename(p) for p in SRC}
    assert {"scan.cu", "common.cuh", "conv_tc.cu", "score_tc.cu"} <= names


def test_mbarrier_waits_are_bounded():
    """The only mbarrier try_wait is inside mss::mbar_wait, which gives up after a time limit."""
    sites = [(os.path.basename(p), m.start()) for p in SRC for m in re.finditer(r"mbarrier\.try_wait", _text(p))]
    assert [s[0] for s in sites] == ["common.cuh"], sites
    body = _text(os.path.join(ROOT, "paper_1403_2136_gb300", "csrc", "common.cuh"))
    fn = body[body.index("bool mbar_wait("):]
    fn = fn[:fn.index("\n}\n")]
    assert "limit_ns" in fn and "return false" in fn and "globaltimer" in body


def test_no_deliberate_traps():
    for p in SRC:
        t = _text(p)
        assert "__trap" not in t and not re.search(r"\btrap;", t), p
        assert not re.search(r"\bassert\s*\(", t), p      # no device asserts that could fault


def test_unbounded_loops_are_work_queues():
    """`for (;;)` / `while (true)` appear only where a CTA pulls work items from a counter and
    leaves when the items run out."""
    for p in SRC:
        t = _text(p)
        for m in re.finditer(r"for \(;;\)|while \(true\)|while \(1\)", t):
            window = t[m.start():m.start() + 600]
            assert "n_items" in window and "break" in window, (os.path.basename(p), t[m.start():m.start() + 200])
