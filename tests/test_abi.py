"""The C ABI library builds, loads and exports every entry point declared in include/*.h, and the
ctypes struct layouts match the C header (CPU only: no compute calls)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(tbk_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1812_05264_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib):
    from paper_1812_05264_gb300 import _lib
    bound = set(_lib.SIGNATURES) | set(_lib.OTHER)
    assert _declared() <= bound


def test_struct_layouts_match_header(tmp_path):
    from paper_1812_05264_gb300 import _lib
    c = tmp_path / "layout.c"
    c.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "tbk.h"\n'
        "int main(void){\n"
        'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(tbk_model), offsetof(tbk_model, n_disp),'
        " offsetof(tbk_model, disp), offsetof(tbk_model, onsite_site), sizeof(tbk_bsr),"
        " offsetof(tbk_bsr, val));\nreturn 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    M, B = _lib.tbk_model, _lib.tbk_bsr
    assert vals == [ctypes.sizeof(M), M.n_disp.offset, M.disp.offset, M.onsite_site.offset,
                    ctypes.sizeof(B), B.val.offset]


def test_errors_without_a_device_are_reported_not_raised(lib):
    """A call with a NULL context returns TBK_ERR_ARG and a message; nothing crosses the ABI."""
    from paper_1812_05264_gb300 import _lib
    rc = lib.tbk_chebyshev_moments(None, None, 0.0, 1.0, 0, 8, 10, 0, None)
    assert rc == _lib.TBK_ERR_ARG
    assert b"NULL" in lib.tbk_last_error()


def test_missing_library_fails_loudly(tmp_path):
    """No fallback: without the built library the binding raises instead of computing anything."""
    code = ("from paper_1812_05264_gb300 import _lib\n"
            f"_lib.load({str(tmp_path / 'libtbk.so')!r})\n")
    r = subprocess.run(["python", "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert r.returncode != 0
    assert "libtbk.so not found" in r.stderr


def test_no_device_means_an_error_not_a_fallback(lib):
    """On a machine without a usable GPU the context cannot be made: the ABI returns an error code
    with a message (no handle), and the Python layer raises before any work."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1812_05264_gb300 import _lib, api
    h = ctypes.c_void_p()
    rc = lib.tbk_create(ctypes.byref(h), 0, None)
    assert rc in (_lib.TBK_ERR_CUDA, _lib.TBK_ERR_ARG) and h.value is None
    assert lib.tbk_last_error()
    with pytest.raises(RuntimeError, match="CUDA device"):
        api.Context()
