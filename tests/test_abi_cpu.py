"""The C ABI library builds, loads without a GPU and exports every symbol
include/*.h declares (no compute calls: this runs on CPU-only machines)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(prcg_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1905_01549_gb300 import binding
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"prcg_create_csr", "prcg_create_stencil", "prcg_solve", "prcg_destroy",
            "prcg_last_error"} <= names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_names_match_header(lib):
    from paper_1905_01549_gb300 import binding
    assert set(binding.EXPORTS) <= _declared()
    for name in binding.EXPORTS:
        assert callable(getattr(binding, name))


def test_host_side_argument_checks_need_no_gpu(lib):
    """Argument validation happens before any CUDA call."""
    from paper_1905_01549_gb300 import binding
    out = ctypes.c_void_p()
    assert lib.prcg_create_stencil(ctypes.byref(out), 4, 8, 8, 8, None, 0.0, 0, None) == -1
    assert b"dim" in lib.prcg_last_error(None)
    assert lib.prcg_create_stencil(ctypes.byref(out), 3, 0, 8, 8, None, 0.0, 0, None) == -1
    assert lib.prcg_create_stencil(ctypes.byref(out), 3, 8, 8, 8, None, -1.0, 0, None) == -1
    assert lib.prcg_create_stencil(ctypes.byref(out), 3, 8, 8, 8, None, 0.0, 7, None) == -1
    assert lib.prcg_create_csr(ctypes.byref(out), 0, 0, None, None, None, 0, None) == -1
    assert lib.prcg_solve(None, 1, None, None, 1e-8, 10, None, None, None) == -1
    assert lib.prcg_destroy(None) == 0
    assert lib.prcg_n(None) == -1
    assert lib.prcg_jacobi_form(None) == -1
    assert lib.prcg_int_diagonal(None) == -1
    with pytest.raises(binding.PrcgError):
        binding.prcg_create_stencil(5, 4, 4, 4)


def test_no_cpu_fallback_in_product_path():
    """The package must not import the oracle (test infrastructure) anywhere."""
    pkg = os.path.join(ROOT, "paper_1905_01549_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(f).read()
        assert "import oracle" not in src and "from oracle" not in src, f


def _header_enum(name):
    src = open(os.path.join(ROOT, "include", "prcg.h")).read()
    body = re.search(r"enum\s+" + name + r"\s*\{(.*?)\}", src, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return {k: int(v) for k, v in re.findall(r"\b(PRCG_[A-Z_]+)\s*=\s*(-?\d+)", body)}


def test_binding_variant_ids_match_header():
    """Every variant the header declares is reachable from Python by name,
    with the header's value."""
    from paper_1905_01549_gb300 import binding
    enum = _header_enum("prcg_variant")
    assert len(enum) == 9
    for k, v in enum.items():
        assert getattr(binding, k) == v, k
    assert sorted(binding.VARIANT_IDS.values()) == sorted(enum.values())


@pytest.mark.parametrize("lang", ["c", "c++"])
def test_header_compiles_for_c_and_cpp_callers(lib, tmp_path, lang):
    """include/prcg.h is a plain C header (C99, pedantic, no warnings) that
    C++ callers can include too; a call through it links against the
    library."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "prcg.h"\n'
                   'int main(void) { return prcg_int_diagonal(0) == -1 ? 0 : 1; }\n')
    std = ["-std=c99", "-pedantic"] if lang == "c" else ["-std=c++17", "-x", "c++"]
    lib_dir = os.path.join(ROOT, "paper_1905_01549_gb300")
    exe = tmp_path / "use_header"
    r = subprocess.run([cc, *std, "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", lib_dir, "-lprcg",
                        f"-Wl,-rpath,{lib_dir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert subprocess.run([str(exe)]).returncode == 0
