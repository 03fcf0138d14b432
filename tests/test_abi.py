"""The C ABI library builds, loads without a GPU, and exports every function
the public header declares; the binding's structs match the header's sizes."""
import ctypes as C
import os
import re
import subprocess

import paper_1906_12211_gb300 as pf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_header_symbols():
    pf.build()
    lib = pf.lib()
    names = pf.header_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", pf.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pf_\w+)", out))
    assert set(names) <= exported


def test_status_strings_without_gpu():
    lib = pf.lib()
    assert lib.pf_status_string(0) == b"ok"
    assert lib.pf_status_string(-2).startswith(b"memory budget")
    opts = pf.SearchOpts()
    lib.pf_search_opts_default(C.byref(opts))
    assert opts.filter == 1 and opts.scoring == 0 and opts.start_depth is None


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "puffinn_gb300.h"\n'
                   "int main(void){printf(\"%zu %zu %zu %zu\\n\", sizeof(pf_build_params),"
                   " sizeof(pf_search_opts), sizeof(pf_query_stats), sizeof(pf_index_info_t));return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    sizes = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert sizes == [C.sizeof(pf.BuildParams), C.sizeof(pf.SearchOpts), C.sizeof(pf.QueryStats),
                     C.sizeof(pf.IndexInfo)]
    assert C.sizeof(pf.QueryStats) == pf.STATS_DTYPE.itemsize


def test_null_arguments_are_rejected_without_gpu():
    lib = pf.lib()
    assert lib.pf_index_build(None, None, None, None) == -1
    assert lib.pf_index_set_shape(None, 8, 4, 0, 0) == -1
    assert lib.pf_index_info(None, None) == -1
    lib.pf_index_free(None)
