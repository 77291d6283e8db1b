"""The compiler's resource report of every kernel in libpic.so (written by
the build beside each object): no kernel may keep a large stack frame.  A
frame of kilobytes means that the compiler copied a whole parameter block
(the 2.5 KB particle launch block) to local memory -- once it doubled the
boundary-variant particle kernel's time without changing a result.  Runs on
the CPU; skips when the build has not written its reports."""
import glob
import os
import re

import pytest

BUILD = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                     "paper_2501_07465_gb300", "_build")
LIMIT = 512  # bytes of stack a thread; the kernels keep 0-120


def _reports():
    return sorted(glob.glob(os.path.join(BUILD, "*.ptxas.txt")))


def _frames(text):
    """(kernel, stack frame bytes) for every entry function of a report."""
    out = []
    name = None
    for line in text.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            name = m.group(1)
            continue
        m = re.search(r"(\d+) bytes stack frame", line)
        if m and name:
            out.append((name, int(m.group(1))))
            name = None
    return out


def test_no_kernel_keeps_a_large_stack_frame():
    reports = _reports()
    if not reports:
        pytest.skip("no resource reports (the library was not built here)")
    frames = [f for r in reports for f in _frames(open(r).read())]
    assert frames, "reports without entry functions"
    big = [(k, b) for k, b in frames if b > LIMIT]
    assert not big, big


def test_the_report_parser_reads_entries_and_frames():
    text = ("ptxas info    : Compiling entry function '_Z1kv' for 'sm_103a'\n"
            "ptxas info    : Function properties for _Z1kv\n"
            "    2488 bytes stack frame, 12 bytes spill stores, 8 bytes spill loads\n"
            "ptxas info    : Used 64 registers\n")
    assert _frames(text) == [("_Z1kv", 2488)]
