"""The C ABI library loads on a machine without a GPU and exports every entry
point that include/glint.h declares; argument checks that need no device
answer with GLINT_ERR_INVALID_ARG and a message.  CPU only."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "glint.h")


def declared_functions(path=HEADER):
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(glint_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_02674_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("glint_ctx_create", "glint_env_create", "glint_env_update", "glint_shade", "glint_lut_export",
                 "glint_env_levels", "glint_env_export", "glint_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_argument_checks_without_gpu(lib):
    lib.glint_last_error.restype = ctypes.c_char_p
    lib.glint_abi_version.restype = ctypes.c_int
    assert lib.glint_abi_version() == 8
    assert lib.glint_ctx_create(0, 0, 0, None) == 1
    assert b"NULL" in lib.glint_last_error()
    assert lib.glint_env_create(None, None, None) == 1
    assert lib.glint_shade(None, None, None, None, None, None, None) == 1
    assert lib.glint_env_update(None, None, None) == 1
    assert lib.glint_reflect_probs(None, None, None, None, None, None) == 1
    assert lib.glint_mlp_create(None, 8, ctypes.c_long(1024), 0, None) == 1
    assert lib.glint_mlp_train_step(None, None, None, ctypes.c_long(0), ctypes.c_long(1), ctypes.c_float(0.0),
                                    None, None) == 1
    assert lib.glint_mlp_infer(None, None, None, None) == 1
    assert lib.glint_mlp_param_count() == 64 * 64 + 64 + 64 * 64 + 64 + 64 * 16 + 16
    lib.glint_hostpipe_create.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_int, ctypes.c_void_p]
    assert lib.glint_hostpipe_create(None, ctypes.c_long(1024), 2, None) == 1
    lib.glint_shade_host.argtypes = [ctypes.c_void_p] * 5 + [ctypes.c_int, ctypes.c_uint, ctypes.c_void_p]
    assert lib.glint_shade_host(None, None, None, None, None, 0, 0, None) == 1
    assert b"NULL" in lib.glint_last_error()
    lib.glint_ctx_destroy(None)
    lib.glint_env_destroy(None)
    lib.glint_mlp_destroy(None)
    lib.glint_hostpipe_destroy(None)
