"""The C-ABI library loads and exports every entry point include/tagi.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "tagi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tagi_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_01833_gb300 import build as B

    B.build()
    return ctypes.CDLL(B.LIB)


def test_header_declares_the_boundary():
    names = declared()
    for n in ("tagi_tree_build", "tagi_anterpolate", "tagi_yukawa_conv", "tagi_coulomb_conv", "tagi_green_step"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared():
        assert hasattr(lib, n), n


def test_version_and_error_without_gpu(lib):
    lib.tagi_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.tagi_version()
    lib.tagi_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.tagi_last_error(), bytes)


def test_argument_validation_needs_no_gpu(lib):
    """Bad arguments are rejected before any device work."""
    import paper_2003_01833_gb300.tagi as T

    h = ctypes.c_void_p()
    p = T.make_params(theta=1.5)
    st = lib.tagi_tree_build(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_int64(10), ctypes.byref(p), None,
                             ctypes.byref(h))
    assert st == T.TAGI_ERR_INVALID_ARG
    p = T.make_params(degree=12)
    assert lib.tagi_tree_build(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_int64(10), ctypes.byref(p), None,
                               ctypes.byref(h)) == T.TAGI_ERR_INVALID_ARG
    for seg in (512, 100000):
        p = T.make_params(segment=seg)
        assert lib.tagi_tree_build(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_int64(10), ctypes.byref(p),
                                   None, ctypes.byref(h)) == T.TAGI_ERR_INVALID_ARG
        assert "segment" in lib.tagi_last_error().decode()
    assert lib.tagi_tree_destroy(None) == T.TAGI_OK
    lib.tagi_yukawa_conv.argtypes = [ctypes.c_void_p] * 6
    assert lib.tagi_yukawa_conv(None, None, None, 1, None, None) == T.TAGI_ERR_INVALID_ARG


def test_green_iterate_validation_needs_no_gpu(lib):
    import paper_2003_01833_gb300.tagi as T

    L = T.lib()
    gp = T.tagi_gi_params(1e-6, 10, 0.5, 5, float("inf"))
    eps = (ctypes.c_double * 1)(-0.5)
    # no tree
    assert L.tagi_green_iterate(None, None, 0.0, None, eps, 1, ctypes.byref(gp), None, None, None,
                                None) == T.TAGI_ERR_INVALID_ARG
    assert "NULL" in T.lib().tagi_last_error().decode()


def test_new_entry_points_validate_without_gpu(lib):
    import paper_2003_01833_gb300.tagi as T

    L = T.lib()
    k = (ctypes.c_double * 1)(1.0)
    assert L.tagi_fields_conv(None, None, k, 1, None, None, None, None) == T.TAGI_ERR_INVALID_ARG
    p = T.tagi_scf_params(3.0, 6.3e-4, 0.0, 0.5, 5, 3e-3, 1e-5, 4, 100, 0.5, 5, float("inf"))
    h = ctypes.c_void_p()
    assert L.tagi_scf_create(None, ctypes.byref(p), ctypes.byref(h)) == T.TAGI_ERR_INVALID_ARG
    eps = (ctypes.c_double * 1)(-0.5)
    assert L.tagi_scf_step(None, None, 0.0, None, None, eps, 1, None, None, None, None) == T.TAGI_ERR_INVALID_ARG
    assert L.tagi_scf_destroy(None) == T.TAGI_OK


def test_warm_start_entry_points_validate_without_gpu(lib):
    """The MLP calls reject bad arguments before touching a device."""
    import numpy as np

    import paper_2003_01833_gb300.tagi as T

    L = T.lib()
    h = ctypes.c_void_p()
    p = np.zeros(T.MLP_PARAMS)
    D = ctypes.POINTER(ctypes.c_double)
    assert L.tagi_mlp_create(7, 32, p.ctypes.data_as(D), p.size, ctypes.byref(h)) == T.TAGI_ERR_INVALID_ARG
    assert L.tagi_mlp_create(8, 64, p.ctypes.data_as(D), p.size, ctypes.byref(h)) == T.TAGI_ERR_INVALID_ARG
    p64 = np.zeros(T.mlp_params(64))
    assert L.tagi_mlp_create(8, 48, p64.ctypes.data_as(D), p64.size, ctypes.byref(h)) == T.TAGI_ERR_INVALID_ARG
    assert L.tagi_mlp_create(8, 64, p64.ctypes.data_as(D), p64.size - 1, ctypes.byref(h)) == T.TAGI_ERR_INVALID_ARG
    assert L.tagi_mlp_create(8, 32, p.ctypes.data_as(D), p.size - 1, ctypes.byref(h)) == T.TAGI_ERR_INVALID_ARG
    q = p.copy()
    q[5] = np.nan
    assert L.tagi_mlp_create(8, 32, q.ctypes.data_as(D), q.size, ctypes.byref(h)) == T.TAGI_ERR_INVALID_ARG
    assert "finite" in L.tagi_last_error().decode()
    nuc = np.array([[0.0, 0, 0], [1.0, 0, 0]])
    fake = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    assert L.tagi_mlp_features(fake, 10, nuc.ctypes.data_as(D), 1, fake, None) == T.TAGI_ERR_INVALID_ARG
    same = np.zeros((2, 3))
    assert L.tagi_mlp_features(fake, 10, same.ctypes.data_as(D), 2, fake, None) == T.TAGI_ERR_INVALID_ARG
    assert L.tagi_mlp_features(fake, 10, nuc.ctypes.data_as(D), 2, ctypes.c_void_p(18), None) \
        == T.TAGI_ERR_INVALID_ARG  # feat not 16-byte aligned
    assert L.tagi_mlp_features(fake, 0, nuc.ctypes.data_as(D), 2, fake, None) == T.TAGI_ERR_INVALID_ARG
    zs = np.array([5.7, 0.0])
    assert L.tagi_mlp_features_scaled(fake, 10, nuc.ctypes.data_as(D), zs.ctypes.data_as(D), 2, 1, fake, None) \
        == T.TAGI_ERR_INVALID_ARG  # a rate must be positive
    assert L.tagi_mlp_features_scaled(fake, 10, nuc.ctypes.data_as(D), None, 2, 1, fake, None) \
        == T.TAGI_ERR_INVALID_ARG
    assert L.tagi_mlp_forward(None, fake, 10, fake, None) == T.TAGI_ERR_INVALID_ARG
    a = T.tagi_adam_params(1e-3, 0.9, 0.999, 1e-8)
    assert L.tagi_mlp_train_step(None, fake, fake, fake, 10, ctypes.byref(a), None, None) == T.TAGI_ERR_INVALID_ARG
    assert L.tagi_mlp_warm_start(None, fake, fake, fake, 10, fake, None) == T.TAGI_ERR_INVALID_ARG
    assert L.tagi_mlp_destroy(None) == T.TAGI_OK


def test_header_is_plain_c(tmp_path):
    """include/tagi.h compiles as pedantic C99: the boundary needs no C++."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "include/tagi.h"\n'
                   "int main(void) {\n"
                   "    tagi_gi_params g = {1e-5, 10, 0.5, 5, 1.0, 0};\n"
                   "    tagi_adam_params a = {1e-3, 0.9, 0.999, 1e-8};\n"
                   "    (void)g; (void)a;\n"
                   "    return tagi_version() == 0;\n"
                   "}\n")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-I", ROOT,
                        str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
