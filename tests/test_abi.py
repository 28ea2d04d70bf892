"""The C-ABI library loads and exports every entry point include/raftgp.h declares, and the
Python mirror of its structs has the C layout (no GPU needed: no compute call is made)."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        names += re.findall(r"^[A-Za-z_][\w \t\*]*?\b(raftgp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def library():
    from paper_2312_01560_gb300 import _abi, build
    if not build.up_to_date():
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc unavailable and libraftgp.so not built")
        build.build()
    return C.CDLL(_abi.LIB_PATH)


def test_every_declared_symbol_is_exported(library):
    names = declared_functions()
    assert len(names) >= 9
    missing = [n for n in names if not hasattr(library, n)]
    assert not missing, missing


def test_python_mirror_lists_every_declared_symbol():
    from paper_2312_01560_gb300 import _abi
    assert sorted(_abi.EXPORTS) == declared_functions()


def test_version_string(library):
    library.raftgp_version.restype = C.c_char_p
    assert b"sm_103a" in library.raftgp_version()


def test_struct_layouts_match_header(tmp_path):
    from paper_2312_01560_gb300 import _abi
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc unavailable")
    structs = {"raftgp_csr": _abi.Csr, "raftgp_embed_opts": _abi.EmbedOpts, "raftgp_select_opts": _abi.SelectOpts,
               "raftgp_select_result": _abi.SelectResult}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "raftgp.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        cname, field, val = line.split()
        py = structs[cname]
        want = C.sizeof(py) if field == "size" else getattr(py, field).offset
        assert int(val) == want, (cname, field, val, want)


def test_missing_library_fails_loudly(monkeypatch):
    from paper_2312_01560_gb300 import _abi
    monkeypatch.setattr(_abi, "_lib", None)
    monkeypatch.setattr(_abi, "LIB_PATH", "/nonexistent/libraftgp.so")
    with pytest.raises(RuntimeError, match="not built"):
        _abi.lib()
