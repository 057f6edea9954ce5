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
    return sorted(set(re.findall(r"\b(jacpcg_[a-z0-9_]+)\s*\(", text)))


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
    """Every field offset and every size of the structs the binding mirrors
    (config, instance, server config, block) equals the C header's."""
    structs = [("jacpcg_config", binding.jacpcg_config), ("jacpcg_instance", binding.jacpcg_instance),
               ("jacpcg_server_config", binding.jacpcg_server_config), ("jacpcg_block", binding.jacpcg_block)]
    lines, want = [], []
    for cname, py in structs:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(py))
        for fname, _ in py._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {fname}));')
            want.append(getattr(py, fname).offset)
    src = tmp_path / "layout.c"
    body = "\n".join(lines)
    src.write_text(f"""
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
{body}
  return 0;
}}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-o", str(exe), str(src)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == want


def test_blocks_helper_points_into_the_full_channel():
    """jacpcg_blocks is host-only arithmetic: sub-instance pointers, shapes and
    scalars, and its EINVAL rules (no GPU, fake device addresses)."""
    I = binding.jacpcg_instance
    full = I(M=1024, K=64, ldh=1030, H=0x100000, xi=0.5, power=2.0, W=0x900000, ldw=1026,
             max_iter=6, tol=1e-5, h_dtype=binding.JACPCG_H_C64)
    blocks = [(0, 384, 0, 32), (384, 256, 0, 64), (640, 384, 32, 32)]
    out = binding.jacpcg_blocks(full, blocks)
    for q, (r0, nr, c0, nc) in zip(out, blocks):
        assert (q.M, q.K, q.ldh, q.ldw) == (nr, nc, 1030, 1026)
        assert q.H == 0x100000 + (c0 * 1030 + r0) * 8
        assert q.W == 0x900000 + (c0 * 1026 + r0) * 8
        assert (q.xi, q.power, q.max_iter) == (0.5, 2.0, 6) and abs(q.tol - 1e-5) < 1e-12
        assert not q.X and not q.A and not q.B and not q.X0
    bf = I(M=64, K=8, ldh=64, H=0x100000, xi=0.5, W=0x900000, ldw=64, h_dtype=binding.JACPCG_H_BF16)
    assert binding.jacpcg_blocks(bf, [(4, 8, 1, 2)])[0].H == 0x100000 + (64 + 4) * 4
    bad = [(0, 1025, 0, 8), (2, 8, 60, 8), (1, 8, 0, 2), (0, 0, 0, 2), (-2, 8, 0, 2)]
    for b in bad:
        with pytest.raises(binding.JacpcgError) as e:
            binding.jacpcg_blocks(full, [b])
        assert e.value.status == binding.JACPCG_EINVAL, b
    with pytest.raises(binding.JacpcgError):                 # bfloat16 rows need row0 % 4 == 0
        binding.jacpcg_blocks(bf, [(2, 8, 0, 2)])
    nreg = I(M=64, K=8, ldh=64, H=0x100000, xi=0.0, W=0x900000, ldw=64)
    with pytest.raises(binding.JacpcgError):                 # more users than antennas, xi = 0
        binding.jacpcg_blocks(nreg, [(0, 4, 0, 6)])
