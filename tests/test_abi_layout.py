"""The Python binding agrees with include/rasp.h: every struct mirrored in
ctypes has the C compiler's size and field offsets, and every bound function
takes as many arguments as its declaration (no compute calls, no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _structs():
    from paper_2604_12902_gb300 import rasp as R, serving as S
    return {"rasp_config": R.rasp_config, "rasp_state_view": R.rasp_state_view, "rasp_stats": R.rasp_stats,
            "rasp_static_run": R.rasp_static_run, "rasp_request": S.rasp_request,
            "rasp_pool_counters": S.rasp_pool_counters}


def _c_layout(tmp_path, structs):
    """sizeof and offsetof of every mirrored field, as gcc lays them out."""
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rasp.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (ln.split() for ln in out.splitlines())}


def test_struct_layouts_match_the_header(tmp_path):
    structs = _structs()
    c = _c_layout(tmp_path, structs)
    for name, cls in structs.items():
        assert ctypes.sizeof(cls) == c[name], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == c["%s.%s" % (name, field)], (name, field)


def _declared_arity():
    """{function: (return type, number of parameters)} from the header."""
    src = open(os.path.join(ROOT, "include", "rasp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"^\s*(int|void|const char\s*\*)\s+(rasp_\w+)\s*\(([^)]*)\)\s*;", src, flags=re.M):
        params = m.group(3).strip()
        out[m.group(2)] = (m.group(1).replace(" ", ""), 0 if params in ("", "void") else params.count(",") + 1)
    return out


def test_bound_functions_take_the_declared_arguments():
    from paper_2604_12902_gb300 import build, rasp as R, serving as S
    build.build()
    L = R.lib()
    S._lib()
    run = R.rasp_static_run()
    run.word_bits = 0
    buf = ctypes.create_string_buffer(256)
    run.err_buf = ctypes.cast(buf, ctypes.c_char_p)
    run.err_buf_size = 256
    assert R.rasp_run_static(run) == R.RASP_EINVAL       # argument check only: no device call
    assert b"word_bits" in buf.value
    arity = _declared_arity()
    assert len(arity) >= 20, sorted(arity)
    checked = 0
    restypes = {"int": ctypes.c_int, "void": None, "constchar*": ctypes.c_char_p}
    for name, (ret, n) in arity.items():
        fn = getattr(L, name)
        assert fn.restype is restypes[ret], (name, fn.restype, ret)
        argtypes = fn.argtypes
        if argtypes is None:
            assert n == 0, "%s takes %d arguments but has no argtypes" % (name, n)
            continue
        assert len(argtypes) == n, (name, len(argtypes), n)
        checked += 1
    assert checked >= 20
