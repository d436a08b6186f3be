"""CPU checks of the C ABI: the library builds, loads without a GPU, and
exports every function include/*.h declares; the binding covers them all."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(nb_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2405_01420_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("nb_pairlist_create", "nb_search", "nb_prune", "nb_forces", "nb_status",
                     "nb_pairlist_destroy", "nb_pairlist_export", "nb_pairlist_stats"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_every_declared_symbol():
    from paper_2405_01420_gb300 import nb
    assert sorted(nb.SIGNATURES) == declared_functions()


def test_version_and_error_without_gpu(lib):
    lib.nb_version.restype = ctypes.c_char_p
    assert lib.nb_version().decode().startswith("nb ")
    lib.nb_last_error.restype = ctypes.c_char_p
    # argument checks run on the host and need no GPU
    lib.nb_pairlist_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.nb_pairlist_create(ctypes.byref(h), 0, None) == 1  # NB_ERR_ARG
    assert "n_atoms" in lib.nb_last_error().decode()


def test_kernels_built_for_sm_103a_only():
    from paper_2405_01420_gb300 import build
    flags = " ".join(build.NVCC_FLAGS)
    assert "arch=compute_103a,code=sm_103a" in flags
    assert flags.count("-gencode") == 1
