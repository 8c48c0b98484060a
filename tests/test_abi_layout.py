"""Every struct the Python binding mirrors has the C header's layout: a small C
program compiled against include/difuser_im.h prints each struct's size and
each field's offset, which must equal the ctypes ones (CPU only)."""
import ctypes
import os
import subprocess

import pytest

import paper_2410_14047_gb300 as im

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["im_model", "im_allocator", "im_stats", "im_tuning", "im_trace_rec", "im_server_config",
           "im_query", "im_query_result", "im_server_stats"]


def test_struct_layouts_match_the_header(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "difuser_im.h"', "int main(void) {"]
    expect = []
    for name in STRUCTS:
        cls = getattr(im, name)
        lines.append(f'printf("%zu\\n", sizeof({name}));')
        expect.append((name, "sizeof", ctypes.sizeof(cls)))
        for field, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({name}, {field}));')
            expect.append((name, field, getattr(cls, field).offset))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0 and "not found" in r.stderr:
        pytest.skip("no C compiler")
    assert r.returncode == 0, r.stderr[-2000:]
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert len(got) == len(expect)
    for (name, field, want), have in zip(expect, got):
        assert have == want, (name, field, have, want)
