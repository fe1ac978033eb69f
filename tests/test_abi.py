"""The C-ABI library: it loads without a GPU, exports every function the header
declares, and its host-only entry points behave as documented.  No compute
call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "paam_rta.h")


def _declared() -> list:
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)  # drop comments
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(paam_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_06452_gb300 import _binding

    return _binding.lib()


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "paam_rta.h"\nint main(void) { return PAAM_OK; }\n')
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c",
                           str(src), "-o", str(tmp_path / "t.o")])


def test_every_declared_function_is_exported(lib):
    names = _declared()
    assert len(names) >= 25, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2404_06452_gb300 import _binding

    assert sorted(_binding.exported_symbols()) == _declared()


def test_host_only_entry_points(lib):
    lib.paam_strerror.restype = ctypes.c_char_p
    lib.paam_strerror.argtypes = [ctypes.c_int]
    assert lib.paam_strerror(0)
    assert lib.paam_strerror(-1) != lib.paam_strerror(0)
    assert lib.paam_strerror(-12345)  # unknown codes still give a string
    lib.paam_rta_num_launch_configs.restype = ctypes.c_int
    assert lib.paam_rta_num_launch_configs() >= 1
    lib.paam_model_num_params.restype = ctypes.c_int64
    p = 1024 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 64 + 64
    assert lib.paam_model_num_params() == p
    # argument checks come before any device work
    lib.paam_rta_load_systems.argtypes = [ctypes.c_void_p] * 4
    assert lib.paam_rta_load_systems(None, None, None, None) < 0
    lib.paam_rta_set_launch_config.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.paam_rta_set_launch_config(None, 0) < 0


def _define(name):
    m = re.search(r"#define\s+" + name + r"\s+\(?(\d+)(?:\s*<<\s*(\d+))?\)?", open(HEADER).read())
    assert m, name
    return int(m.group(1)) << int(m.group(2) or 0)


def test_binding_constants_match_the_header():
    import paper_2404_06452_gb300 as pkg

    assert pkg.PAAM_NOALLOC_MAX_SYS == _define("PAAM_NOALLOC_MAX_SYS")
    assert pkg.PAAM_MAX_CHAINS == _define("PAAM_MAX_CHAINS")
    assert _define("PAAM_MAX_ITER") == 1 << 20
