"""The Python binding mirrors the C ABI by hand: its constants must equal the header's enums
and defines, and its ctypes structures must list the header's struct fields in the same
order (a missing or reordered field shifts every later one)."""
import os
import re

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "include", "sisso.h")


def _header():
    return open(HEADER).read()


def _no_comments(text):
    return re.sub(r"/\*.*?\*/", "", text, flags=re.S)


def _struct_fields(text, name):
    text = _no_comments(text)
    end = re.search(r"\}\s*" + name + r"\s*;", text)
    assert end, name
    start = text.rfind("typedef struct {", 0, end.start())
    body = text[start + len("typedef struct {"):end.start()]
    fields = []
    for decl in body.split(";"):
        decl = re.sub(r"\[[^\]]*\]", "", decl).strip()
        if not decl:
            continue
        first, *rest = decl.split(",")
        fields.append(first.split()[-1].lstrip("*"))
        fields += [r.strip().lstrip("*") for r in rest]
    return fields


@pytest.mark.parametrize("prefix,names", [
    ("PREC", ["FP64", "FP32", "MIXED_BF16", "MIXED_FP16"]),
    ("GRAMMAR", ["EQ2", "NEW_X_PREV"]),
    ("PRESCREEN", ["NONE", "MI", "SPEARMAN"]),
    ("SCREEN", ["AUTO", "CORES", "TENSOR"]),
    ("GRAM", ["AUTO", "FP64", "TF32X3"]),
])
def test_enum_values_match_header(prefix, names):
    from paper_2410_01752_gb300 import sisso
    text = _header()
    for n in names:
        m = re.search(r"SISSO_%s_%s\s*=\s*(-?\d+)" % (prefix, n), text)
        assert m, f"SISSO_{prefix}_{n} not in the header"
        assert getattr(sisso, f"{prefix}_{n}") == int(m.group(1)), f"{prefix}_{n}"


def test_defines_match_header():
    from paper_2410_01752_gb300 import sisso
    text = _header()
    for c_name, py_name in [("SISSO_MAX_DIM", "MAX_DIM"), ("SISSO_MAX_SIS", "MAX_SIS"), ("SISSO_MAX_RUNG", "MAX_RUNG"),
                            ("SISSO_NOALLOC_MAX_N", "NOALLOC_MAX_N"), ("SISSO_NOALLOC_MAX_BAND", "NOALLOC_MAX_BAND")]:
        m = re.search(r"#define %s\s+(\d+)" % c_name, text)
        assert m, c_name
        assert getattr(sisso, py_name) == int(m.group(1)), c_name


@pytest.mark.parametrize("c_struct,py_struct", [("sisso_opts", "Opts"), ("sisso_stats", "Stats"), ("sisso_task", "Task"),
                                               ("sisso_task_result", "TaskResult"), ("sisso_batch_tune", "BatchTune"),
                                               ("sisso_batch_stats", "BatchStats")])
def test_struct_fields_match_header(c_struct, py_struct):
    from paper_2410_01752_gb300 import sisso
    assert [f for f, _ in getattr(sisso, py_struct)._fields_] == _struct_fields(_header(), c_struct)


def test_struct_layout_matches_the_c_compiler(tmp_path):
    """sizeof and every field's offsetof, as gcc lays the header's structs out, equal the
    ctypes mirrors' (a field of the wrong width moves every later offset)."""
    import ctypes
    import shutil
    import subprocess
    from paper_2410_01752_gb300 import sisso
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    pairs = [("sisso_opts", sisso.Opts), ("sisso_stats", sisso.Stats), ("sisso_task", sisso.Task),
             ("sisso_task_result", sisso.TaskResult), ("sisso_batch_tune", sisso.BatchTune),
             ("sisso_batch_stats", sisso.BatchStats)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sisso.h"', "int main(void) {"]
    for c_name, py in pairs:
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (c_name, c_name))
        for f, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (c_name, f, c_name, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict((" ".join(l.split()[:2]), int(l.split()[2])) for l in out if l.strip())
    for c_name, py in pairs:
        assert got[f"{c_name} size"] == ctypes.sizeof(py), c_name
        for f, _ in py._fields_:
            assert got[f"{c_name} {f}"] == getattr(py, f).offset, (c_name, f)
