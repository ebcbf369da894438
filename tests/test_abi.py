"""CPU checks of the C ABI: the library builds and loads, exports every entry
point the header declares, and its structs match the ctypes mirrors.  No
compute call runs here (no GPU)."""

import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kkspgemm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1801_03065_gb300 import build
    build.build()
    from paper_1801_03065_gb300 import _binding
    return _binding.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spgemm_[a-z_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("spgemm_handle_create", "spgemm_symbolic", "spgemm_numeric", "spgemm_handle_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1801_03065_gb300 import _binding
    names = declared_functions()
    for n in names:
        assert hasattr(lib, n), "missing export %s" % n
    assert set(names) == set(_binding.SIGNATURES), "binding and header disagree"


def test_status_strings_and_version(lib):
    assert lib.spgemm_status_string(0) == b"SPGEMM_OK"
    assert lib.spgemm_status_string(7) == b"SPGEMM_ERR_PATTERN_MISMATCH"
    assert lib.spgemm_status_string(99) == b"SPGEMM_ERR_UNKNOWN"
    assert lib.spgemm_version() >= 100


def test_options_defaults(lib):
    from paper_1801_03065_gb300 import _binding as B
    o = B.OptionsT()
    assert lib.spgemm_options_default(C.byref(o)) == 0
    assert o.compression == -1 and abs(o.compress_threshold - 0.85) < 1e-15
    assert abs(o.l1_max_occupancy - 0.5) < 1e-15 and o.dense == -1
    assert o.hash_function == 1 and o.numeric_positions == 1 and o.window_positions == 1
    assert o.sym_merge == 1 and o.stage_b == 0 and o.tune == 0
    assert lib.spgemm_options_default(None) == 1


def test_null_arguments_rejected(lib):
    assert lib.spgemm_handle_create(None, None) == 1
    assert lib.spgemm_handle_destroy(None) == 1
    assert lib.spgemm_symbolic(None, None, None, None, None, None) == 1
    assert lib.spgemm_get_stats(None, None) == 1


def test_handle_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = lib.spgemm_handle_create(C.byref(h), None)
    assert rc == 6 and not h.value   # SPGEMM_ERR_CUDA, no handle


def test_struct_layout_matches_header(tmp_path):
    """sizeof / offsetof of the header's structs from gcc equal the ctypes mirrors."""
    from paper_1801_03065_gb300 import _binding as B
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "kkspgemm.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(spgemm_csr_t), offsetof(spgemm_csr_t, rowptr),
         offsetof(spgemm_csr_t, values), offsetof(spgemm_csr_t, dtype));
  printf("%zu %zu %zu %zu\n", sizeof(spgemm_options_t), offsetof(spgemm_options_t, workspace_limit_bytes),
         offsetof(spgemm_options_t, device), offsetof(spgemm_options_t, compress_threshold));
  printf("%zu %zu %zu %zu\n", sizeof(spgemm_stats_t), offsetof(spgemm_stats_t, CF),
         offsetof(spgemm_stats_t, nnzC), offsetof(spgemm_stats_t, bin_rows_numeric));
  return 0;
}
"""
    src = tmp_path / "layout.c"
    src.write_text(prog)
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    got = [int(x) for x in out]
    exp = [C.sizeof(B.CsrT), B.CsrT.rowptr.offset, B.CsrT.values.offset, B.CsrT.dtype.offset,
           C.sizeof(B.OptionsT), B.OptionsT.workspace_limit_bytes.offset, B.OptionsT.device.offset,
           B.OptionsT.compress_threshold.offset,
           C.sizeof(B.StatsT), B.StatsT.CF.offset, B.StatsT.nnzC.offset, B.StatsT.bin_rows_numeric.offset]
    assert got == exp


def test_header_compiles_as_cplusplus(tmp_path):
    src = tmp_path / "h.cpp"
    src.write_text('#include "kkspgemm.h"\nint main() { spgemm_options_t o; return spgemm_options_default(&o) == SPGEMM_OK ? 0 : 1; }\n')
    subprocess.check_call(["g++", "-fsyntax-only", "-I", os.path.join(ROOT, "include"), str(src)])


def test_no_oracle_import_in_product():
    """The product package never imports the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_1801_03065_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f), encoding="utf-8", errors="ignore").read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "oracle.h" not in text and "liboracle" not in text, f
