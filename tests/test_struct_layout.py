"""The ctypes mirrors of the C structs (the library's include/slidemesh.h and the oracle's
dg_oracle.h) have the C compiler's sizes and field offsets, so that the binding and the
library read the same bytes.  Compiles a small C program with the host compiler (no GPU)."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def c_layout(header_dir, header, structs):
    """{struct: (sizeof, {field: offsetof})} as the C compiler lays them out."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "%s"' % header, "int main(void) {"]
    for name, fields in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f in fields:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([cc, "-I", header_dir, src, "-o", exe], check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        name, key, val = line.split()
        entry = res.setdefault(name, [0, {}])
        if key == "size":
            entry[0] = int(val)
        else:
            entry[1][key] = int(val)
    return res


def check(cstruct, name, layout):
    size, offs = layout[name]
    assert C.sizeof(cstruct) == size, (name, C.sizeof(cstruct), size)
    for f, off in offs.items():
        assert getattr(cstruct, f).offset == off, (name, f, getattr(cstruct, f).offset, off)


def fields(cstruct):
    return [f[0] for f in cstruct._fields_]


def test_library_structs_match_the_header():
    from paper_2008_04356_gb300 import slidemesh as S
    mirrors = {"sm_mesh_desc": S.SmMeshDesc, "sm_motion": S.SmMotion, "sm_diag_out": S.SmDiag,
               "sm_request": S.SmRequest, "sm_result": S.SmResult, "sm_server_stats_out": S.SmServerStats}
    layout = c_layout(os.path.join(ROOT, "include"), "slidemesh.h", {k: fields(v) for k, v in mirrors.items()})
    for name, cs in mirrors.items():
        check(cs, name, layout)


def test_oracle_problem_matches_its_header():
    from oracle import oracle as O
    layout = c_layout(os.path.join(ROOT, "oracle"), "dg_oracle.h", {"orc_problem": fields(O.OrcProblem)})
    check(O.OrcProblem, "orc_problem", layout)
