"""CPU-side checks of the C ABI: the library builds, loads without a GPU and exports every
function include/ntf.h declares; the Python binding refuses to run without it."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+(ntf_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location("_ntf_build", os.path.join(ROOT, "paper_2602_14683_gb300", "build.py"))
    build = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(build)
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_boundary():
    names = declared_functions()
    for n in ["ntf_cp_mu_sweep", "ntf_tucker_mu_sweep", "ntf_jcomm_outer", "ntf_beta_div",
              "ntf_ctx_create", "ntf_ctx_destroy", "ntf_last_error", "ntf_opts_default"]:
        assert n in names, n


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_package_import_requires_library(lib):
    # the binding loads the in-tree library; it has no fallback path
    import paper_2602_14683_gb300 as ntf
    assert os.path.samefile(ntf.LIB_PATH, os.path.join(ROOT, "paper_2602_14683_gb300", "_build", "libntf.so"))


def test_opts_default_without_gpu(lib):
    from paper_2602_14683_gb300 import _lib
    o = _lib.Opts()
    lib.ntf_opts_default(ctypes.byref(o))
    assert o.eps == 1e-12 and o.eps_x == 1e-12 and o.inner_L == 1 and o.precision == 0
    assert o.autotune == 0 and o.merge == 0


def test_ctx_create_rejects_bad_device(lib):
    h = ctypes.c_void_p()
    rc = lib.ntf_ctx_create(ctypes.byref(h), ctypes.c_int(-1))
    assert rc == -7 and not h.value
    assert lib.ntf_ctx_create(None, 0) == -1


def test_binding_exports_match_header():
    import paper_2602_14683_gb300 as ntf
    assert set(ntf.EXPORTED) == set(declared_functions())
