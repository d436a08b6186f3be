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


def header_defines():
    text = open(os.path.join(ROOT, "include", "nb.h")).read()
    return {m.group(1): int(m.group(2), 0)
            for m in re.finditer(r"^#define (NB_\w+) (0x[0-9a-fA-F]+|\d+)u?\b", text, flags=re.M)}


def header_struct_fields(name):
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "nb.h")).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", text).group(1)
    return [m.group(2) for m in re.finditer(r"^\s*(int|unsigned|float|long long|size_t)\s+(\w+);", body, flags=re.M)]


def test_binding_constants_match_the_header():
    from paper_2405_01420_gb300 import nb
    defs = header_defines()
    shared = [k for k in defs if hasattr(nb, k)]
    assert len(shared) >= 25, shared
    wrong = {k: (defs[k], getattr(nb, k)) for k in shared if defs[k] != getattr(nb, k)}
    assert not wrong, wrong


def test_binding_structs_match_the_header():
    from paper_2405_01420_gb300 import nb
    assert [f for f, _ in nb.nb_stats._fields_] == header_struct_fields("nb_stats")
    assert [f for f, _ in nb.nb_config._fields_] == header_struct_fields("nb_config")
    assert header_struct_fields("nb_tracker") == ["error_word", "max_disp2_search", "max_disp2_prune"]
    # the tracker copy is three 4-byte words, decoded in this order
    words = __import__("numpy").array([5, 0x3F800000, 0x40000000], dtype="int32")
    t = nb.decode_tracker(words)
    assert t["error_word"] == 5 and t["max_disp_search"] == 1.0 and abs(t["max_disp_prune"] - 2 ** 0.5) < 1e-6


# Host-side argument checks of every entry point that takes a pair list: a NULL list (or NULL
# arguments) returns NB_ERR_ARG with a message naming the function, before any CUDA call.
NULL_CALLS = [
    ("nb_search", [None, None, None, 1.0, None, None, None]),
    ("nb_prune", [None, None, 1.0, None]),
    ("nb_forces", [None, None, None, None, 1, None, 1.0, 1.0, None, None, None]),
    ("nb_forces_part", [None, 0, None, None, None, 1, None, 1.0, 1.0, None, None, None]),
    ("nb_backward", [None, None, None, None, 1, None, 1.0, 1.0, None, None, None, None, None]),
    ("nb_status", [None, None, 0, None]),
    ("nb_pairlist_stats", [None, None, None]),
    ("nb_tracker_enqueue", [None, None, None]),
    ("nb_pairlist_export", [None, 0, None, None, None, None, 0, None, None, 0, None, None]),
    ("nb_pairlist_export_tiles", [None, None, None, None, 0, None, None]),
    ("nb_set_timing_events", [None, None, None]),
    ("nb_set_force_shape", [None, 0, 0, 0]),
    ("nb_set_coulomb", [None, 0, 0.0, 0]),
    ("nb_set_flags", [None, 0]),
    ("nb_set_home", [None, 1]),
]


@pytest.mark.parametrize("name, args", NULL_CALLS, ids=[c[0] for c in NULL_CALLS])
def test_null_pair_list_is_an_argument_error(lib, name, args):
    from paper_2405_01420_gb300 import nb
    restype, argtypes = nb.SIGNATURES[name]
    fn = getattr(lib, name)
    fn.restype, fn.argtypes = restype, argtypes
    lib.nb_last_error.restype = ctypes.c_char_p
    assert fn(*args) == nb.NB_ERR_ARG
    assert lib.nb_last_error().decode().startswith(name)


def test_destroy_of_null_is_a_no_op(lib):
    lib.nb_pairlist_destroy.argtypes = [ctypes.c_void_p]
    assert lib.nb_pairlist_destroy(None) == 0


def test_batch_create_argument_errors(lib):
    from paper_2405_01420_gb300 import nb
    restype, argtypes = nb.SIGNATURES["nb_batch_create"]
    lib.nb_batch_create.restype, lib.nb_batch_create.argtypes = restype, argtypes
    h = ctypes.c_void_p()
    assert lib.nb_batch_create(ctypes.byref(h), 0, None, None, None) == nb.NB_ERR_ARG
    assert h.value is None


def test_noalloc_argument_checks_run_on_the_host(lib):
    """nb_forces_noalloc rejects bad sizes, pointers and radii before any CUDA call."""
    import numpy as np
    from paper_2405_01420_gb300 import nb
    restype, argtypes = nb.SIGNATURES["nb_forces_noalloc"]
    f = lib.nb_forces_noalloc
    f.restype, f.argtypes = restype, argtypes
    lib.nb_last_error.restype = ctypes.c_char_p
    box = np.array([3.0, 3.0, 3.0], np.float32)
    small_box = np.array([1.5, 3.0, 3.0], np.float32)
    dummy = ctypes.c_void_p(16)  # never dereferenced: every case fails on the host first
    word = ctypes.c_uint(0)

    def call(n, b, ntype=1, rc=0.9, beta=3.0, eo=None, ei=None, forces=dummy):
        return f(n, dummy, b.ctypes.data_as(ctypes.c_void_p), dummy, dummy, ntype, dummy, rc, beta, eo, ei, forces,
                 None, ctypes.byref(word), None)

    assert call(0, box) == nb.NB_ERR_ARG
    assert call(nb.NB_NOALLOC_MAX_ATOMS + 1, box) == nb.NB_ERR_CAPACITY
    assert call(10, box, forces=None) == nb.NB_ERR_ARG
    assert call(10, box, eo=dummy) == nb.NB_ERR_ARG  # one exclusion array without the other
    assert call(10, box, ntype=0) == nb.NB_ERR_ARG
    assert call(10, box, ntype=33) == nb.NB_ERR_ARG
    assert call(10, box, rc=0.0) == nb.NB_ERR_ARG
    assert call(10, box, beta=4.0) == nb.NB_ERR_ARG  # beta * rc > 3.2
    assert call(10, small_box) == nb.NB_ERR_ARG      # an edge not above 2 rc
    assert lib.nb_last_error().decode().startswith("nb_forces_noalloc")


def test_pme_argument_checks_run_on_the_host(lib):
    """nb_pme_spread / nb_pme_gather reject bad orders, mesh sizes, boxes and
    pointers before any CUDA call."""
    import numpy as np
    from paper_2405_01420_gb300 import nb
    lib.nb_last_error.restype = ctypes.c_char_p
    sp, ga = lib.nb_pme_spread, lib.nb_pme_gather
    sp.restype, sp.argtypes = nb.SIGNATURES["nb_pme_spread"]
    ga.restype, ga.argtypes = nb.SIGNATURES["nb_pme_gather"]
    box = np.array([3.0, 3.0, 3.0], np.float32)
    bad_box = np.array([3.0, 0.0, 3.0], np.float32)
    dummy = ctypes.c_void_p(16)  # never dereferenced: every case fails on the host first

    def spread(n=10, b=box, K=(16, 16, 16), order=4, grid=dummy, x=dummy):
        return sp(n, x, dummy, b.ctypes.data_as(ctypes.c_void_p), *K, order, grid, None)

    def gather(n=10, b=box, K=(16, 16, 16), order=4, phi=dummy, forces=dummy):
        return ga(n, dummy, dummy, b.ctypes.data_as(ctypes.c_void_p), *K, order, phi, forces, 0, None, None)

    for call, name in ((spread, "nb_pme_spread"), (gather, "nb_pme_gather")):
        assert call(n=-1) == nb.NB_ERR_ARG
        assert call(order=5) == nb.NB_ERR_ARG
        assert "order 4" in lib.nb_last_error().decode()
        assert call(K=(3, 16, 16)) == nb.NB_ERR_ARG
        assert call(K=(16, 16, 4097)) == nb.NB_ERR_ARG
        assert call(b=bad_box) == nb.NB_ERR_ARG
        assert lib.nb_last_error().decode().startswith(name)
    assert spread(grid=None) == nb.NB_ERR_ARG
    assert spread(x=None) == nb.NB_ERR_ARG
    assert gather(phi=None) == nb.NB_ERR_ARG
    assert gather(forces=None) == nb.NB_ERR_ARG


def test_peak_probe_argument_checks_run_on_the_host(lib):
    """nb_fp32_peak_probe rejects NULL pointers and bad launch sizes before any CUDA call."""
    from paper_2405_01420_gb300 import nb
    f = lib.nb_fp32_peak_probe
    f.restype, f.argtypes = nb.SIGNATURES["nb_fp32_peak_probe"]
    lib.nb_last_error.restype = ctypes.c_char_p
    flops = ctypes.c_double(0.0)
    dummy = ctypes.c_void_p(16)  # never dereferenced
    assert f(1, 8, 16, None, 1 << 20, ctypes.byref(flops), None) == nb.NB_ERR_ARG
    assert f(1, 8, 16, dummy, 1 << 20, None, None) == nb.NB_ERR_ARG
    assert f(1, 0, 16, dummy, 1 << 20, ctypes.byref(flops), None) == nb.NB_ERR_ARG
    assert f(1, 9, 16, dummy, 1 << 20, ctypes.byref(flops), None) == nb.NB_ERR_ARG
    assert f(1, 8, 0, dummy, 1 << 20, ctypes.byref(flops), None) == nb.NB_ERR_ARG
    assert lib.nb_last_error().decode().startswith("nb_fp32_peak_probe")
