"""The C-ABI library loads and exports every entry point include/jacpcg.h
declares; the ctypes structures match the C layout.  CPU only: no compute
call is made (none can run without a GPU)."""
import ctypes
import pathlib
import re
import subprocess

import pytest

from paper_2305_13925_gb300 import binding, build

ROOT = pathlib.Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "jacpcg.h"


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(jacpcg_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(str(build.LIB))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "jacpcg_create" in names and "jacpcg_precode" in names and "jacpcg_destroy" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(binding.EXPORTS)


def test_version_and_strerror_without_gpu(lib):
    lib.jacpcg_version.restype = ctypes.c_char_p
    lib.jacpcg_strerror.restype = ctypes.c_char_p
    assert lib.jacpcg_version().decode().count(".") == 2
    assert lib.jacpcg_strerror(0) == b"ok"
    assert b"invalid" in lib.jacpcg_strerror(1)


def test_null_arguments_rejected_without_gpu(lib):
    lib.jacpcg_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.jacpcg_create(None, None) == binding.JACPCG_EINVAL
    lib.jacpcg_destroy.argtypes = [ctypes.c_void_p]
    assert lib.jacpcg_destroy(None) == binding.JACPCG_EINVAL
    lib.jacpcg_launch_count.restype = ctypes.c_int64
    lib.jacpcg_launch_count.argtypes = [ctypes.c_void_p]
    assert lib.jacpcg_launch_count(None) == -1


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(f"""
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(jacpcg_config),
         offsetof(jacpcg_config, arena_bytes), offsetof(jacpcg_config, flags), sizeof(jacpcg_instance),
         offsetof(jacpcg_instance, W), offsetof(jacpcg_instance, tol), offsetof(jacpcg_instance, B),
         offsetof(jacpcg_instance, ldb), offsetof(jacpcg_instance, n_rhs), offsetof(jacpcg_instance, X0));
  return 0;
}}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-o", str(exe), str(src)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    C, I = binding.jacpcg_config, binding.jacpcg_instance
    assert got == [ctypes.sizeof(C), C.arena_bytes.offset, C.flags.offset, ctypes.sizeof(I),
                   I.W.offset, I.tol.offset, I.B.offset, I.ldb.offset, I.n_rhs.offset, I.X0.offset]
