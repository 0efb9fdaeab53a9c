"""The benchmark's source hash (which decides whether a stored ncu capture
still describes a kernel): it follows the code and ignores comments and
blank lines. Host logic only."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _reader(files):
    return lambda f: files[f]


def _sources():
    return {f: open(os.path.join(ROOT, f), encoding="utf-8").read() for f in bench.KERNEL_SOURCES["k_trace_q"]}


def test_code_text_drops_comments_and_blank_lines():
    src = "int a; // one\n\n/* two\n   lines */ int b;\n  \nint c;  /* three */\n"
    assert bench.code_text(src) == "int a;\n int b;\nint c;"


def test_hash_ignores_comment_edits_and_follows_code():
    files = _sources()
    h = bench.src_sha("k_trace_q", _reader(files))
    assert h == bench.src_sha("k_trace_q")  # the working tree through the default reader
    f = "include/dcem.h"
    doc = dict(files)
    doc[f] = files[f].replace("/*", "/* edited:", 1) + "\n// a trailing note\n\n"
    assert bench.src_sha("k_trace_q", _reader(doc)) == h
    code = dict(files)
    code[f] = files[f] + "\nint dcem_extra_symbol;\n"
    assert bench.src_sha("k_trace_q", _reader(code)) != h

