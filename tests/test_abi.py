"""The C-ABI library loads and exports every entry point include/lnr.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lnr_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def liblnr():
    from paper_2502_11618_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["lnr_load_cloud", "lnr_build_grid", "lnr_set_unet", "lnr_render", "lnr_render_batch",
              "lnr_submit", "lnr_poll"]:
        assert n in names


def test_library_exports_every_declared_symbol(liblnr):
    missing = [n for n in sorted(_declared()) if not hasattr(liblnr, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_2502_11618_gb300 as p
    assert set(p.SYMBOLS) == _declared()


def test_null_context_is_an_argument_error(liblnr):
    liblnr.lnr_build_grid.argtypes = [ctypes.c_void_p, ctypes.c_double]
    assert liblnr.lnr_build_grid(None, 0.5) == -1
    liblnr.lnr_destroy.argtypes = [ctypes.c_void_p]
    assert liblnr.lnr_destroy(None) == -1


def test_product_path_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2502_11618_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "lnr_oracle" not in src, f
