"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads without a GPU and
exports every entry point that include/sptrsv.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_2206_05843_gb300 import binding
from paper_2206_05843_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "sptrsv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(sptrsv_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 25
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(names) == sorted(binding.EXPORTED)


def test_binding_loads_signatures():
    lib = binding.load()
    for n in binding.EXPORTED:
        assert getattr(lib, n).restype is not None or n.endswith("destroy")


def test_strategy_struct_layout_matches_header():
    # the binding mirrors the header's struct field order
    src = open(os.path.join(ROOT, "include", "sptrsv.h")).read()
    body = src[src.index("typedef struct {\n    int32_t kind;"):src.index("} sptrsv_strategy;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\*?\s*([a-z_0-9]+);", body)
    assert fields == [f for f, _ in binding.Strategy._fields_]


def test_struct_sizes_and_offsets_match_the_compiled_header(tmp_path):
    """The ctypes mirrors of the ABI structs have the sizes and field offsets that a C compiler
    gives the header's declarations."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    structs = {"sptrsv_system_info": binding.SystemInfo, "sptrsv_strategy": binding.Strategy,
               "sptrsv_level_stats": binding.LevelStats, "sptrsv_batch_info": binding.BatchInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sptrsv.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            a, b, c = ln.split()
            got[(a, b)] = int(c)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
