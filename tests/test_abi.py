"""The C-ABI library loads and exports every entry point that include/kdss.h
declares, and the ctypes structures match the C layouts.  No GPU needed: no
compute call is made."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2403_05775_gb300 as K
from paper_2403_05775_gb300 import build_ext

HEADERS = sorted(os.path.join(build_ext.INCLUDE, f) for f in os.listdir(build_ext.INCLUDE)
                 if f.endswith(".h"))


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kdss_[a-z_0-9]+)\s*\(", text)) - {"kdss_alloc_fn", "kdss_free_fn"})


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return ctypes.CDLL(build_ext.LIB)


def test_library_exports_every_declared_entry_point(lib):
    names = declared_functions()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", build_ext.LIB], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (kdss_\w+)", out))
    assert exported == set(names), exported ^ set(names)


def test_binding_loads_and_reports_version():
    assert "sm_103a" in K.kdss_version()


def test_struct_layouts_match_the_header(tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "kdss_server.h"\n'
                   "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
                   "sizeof(kdss_opts), sizeof(kdss_graph_desc), sizeof(kdss_sct_stats),"
                   "sizeof(kdss_result), sizeof(kdss_timing), sizeof(kdss_query),"
                   "offsetof(kdss_result, status), offsetof(kdss_opts, stream),"
                   "sizeof(kdss_server_opts), sizeof(kdss_query_timing),"
                   "sizeof(kdss_server_stats), sizeof(kdss_sct_count_stats),"
                   "offsetof(kdss_sct_count_stats, seconds));return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", build_ext.INCLUDE, "-o", str(exe), str(src)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(K.kdss_opts), ctypes.sizeof(K.kdss_graph_desc),
            ctypes.sizeof(K.kdss_sct_stats), ctypes.sizeof(K.kdss_result),
            ctypes.sizeof(K.kdss_timing), ctypes.sizeof(K.kdss_query),
            K.kdss_result.status.offset, K.kdss_opts.stream.offset,
            ctypes.sizeof(K.kdss_server_opts), ctypes.sizeof(K.kdss_query_timing),
            ctypes.sizeof(K.kdss_server_stats), ctypes.sizeof(K.kdss_sct_count_stats),
            K.kdss_sct_count_stats.seconds.offset]
    assert got == want


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: a missing library is an error, not a slow path."""
    monkeypatch.setattr(build_ext, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(K, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        K.load()
