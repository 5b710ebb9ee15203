"""The binding's mirrors of the C ABI's structs have the header's layout: a
small C program built with the host compiler against include/tfg.h prints
every struct's size and each field's offset, which must equal the ctypes
structures' and numpy dtypes' (a field added on one side only would shift
every later field the kernels read)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2511_20317_gb300 import tfg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CTYPES = [tfg.tfg_format, tfg.tfg_params, tfg.tfg_resize_args, tfg.tfg_stats, tfg.tfg_log_spec]
DTYPES = {"tfg_log_entry": tfg.LOG_ENTRY_DTYPE, "tfg_walker_info": tfg.WALKER_INFO_DTYPE}


def c_layout(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tfg.h"', "int main(void) {"]
    for st in CTYPES:
        n = st.__name__
        lines.append(f'printf("{n} size %zu\\n", sizeof({n}));')
        for f in st._fields_:
            lines.append(f'printf("{n} {f[0]} %zu\\n", offsetof({n}, {f[0]}));')
    for n, dt in DTYPES.items():
        lines.append(f'printf("{n} size %zu\\n", sizeof({n}));')
        for f in dt.names:
            lines.append(f'printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no host C compiler")
def test_binding_structs_match_the_header(tmp_path):
    lay = c_layout(tmp_path)
    for st in CTYPES:
        n = st.__name__
        assert lay[(n, "size")] == ctypes.sizeof(st), n
        for f in st._fields_:
            assert lay[(n, f[0])] == getattr(st, f[0]).offset, (n, f[0])
    for n, dt in DTYPES.items():
        assert lay[(n, "size")] == dt.itemsize, n
        for f in dt.names:
            assert lay[(n, f)] == dt.fields[f][1], (n, f)
