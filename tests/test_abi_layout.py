"""The ctypes mirrors of the C ABI's structs (paper_1802_09277_gb300/st.py)
have the same size and field offsets as the structs in include/st_iga.h, as
laid out by the host C compiler (no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_layout(tmp_path, structs):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "st_iga.h"', "int main(void) {"]
    for cname, fields in structs:
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in fields:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        cname, key, val = line.split()
        res[(cname, key)] = int(val)
    return res


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_struct_layouts_match(tmp_path):
    from paper_1802_09277_gb300 import st
    pairs = [("st_options", st.StOptions), ("st_solve_info", st.StSolveInfo),
             ("st_server_opts", st.StServerOpts), ("st_request", st.StRequest),
             ("st_result", st.StResult)]
    structs = [(c, [f for f, _ in py._fields_]) for c, py in pairs]
    lay = _c_layout(tmp_path, structs)
    for cname, py in pairs:
        assert lay[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert lay[(cname, f)] == getattr(py, f).offset, (cname, f)
