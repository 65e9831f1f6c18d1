"""The ctypes mirrors of the C structs have the C layout.

The binding (dg.py) and the oracle's wrapper (oracle/__init__.py) pass their
parameter structs by pointer, so every field must sit at the offset the C
compiler gives it.  A C program built here with gcc prints sizeof and
offsetof for every field the mirrors name (a field the header lacks fails the
compile); the test compares them.  No GPU needed.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
from paper_1805_01443_gb300 import dg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    "dg": (os.path.join(ROOT, "include"), "dg.h",
           [("dg_mesh", dg.DgMesh), ("dg_eos", dg.DgEos), ("dg_planet", dg.DgPlanet),
            ("dg_disc", dg.DgDisc)]),
    "oracle": (os.path.join(ROOT, "oracle"), "dg_oracle.h",
               [("ref_mesh", oracle.RefMesh), ("ref_eos", oracle.RefEos),
                ("ref_planet", oracle.RefPlanet), ("ref_disc", oracle.RefDisc)]),
}


def c_layout(tmp_path, incdir, header, structs):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "%s"' % header, "int main(void) {"]
    for cname, cls in structs:
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", incdir, str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True)
    return {k: int(v) for k, v in (ln.split() for ln in out.splitlines())}


@pytest.mark.parametrize("which", sorted(CASES))
def test_ctypes_structs_have_the_c_layout(tmp_path, which):
    incdir, header, structs = CASES[which]
    got = c_layout(tmp_path, incdir, header, structs)
    for cname, cls in structs:
        assert got[cname] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got["%s.%s" % (cname, f)] == getattr(cls, f).offset, (cname, f)
