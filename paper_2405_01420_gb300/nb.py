"""Python binding of libnb.so (include/nb.h).

Argument marshalling only: each function checks tensor dtype, device and
size, passes raw device pointers and a CUDA stream to the C entry point of
the same name, and raises ``NBError`` on a non-zero status. Every step of
the computation runs in the CUDA kernels of libnb.so; there is no CPU or
PyTorch fallback, and using the binding without the built library raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libnb.so")

NB_OK = 0
NB_ERR_ARG = 1
NB_ERR_CUDA = 2
NB_ERR_CAPACITY = 3
NB_ERR_NONFINITE = 4
NB_ERR_TIMEOUT = 5
NB_ERR_STATE = 6
NB_ERR_NOMEM = 7

NB_DEV_LIST_OVERFLOW = 0x01
NB_DEV_COLUMN_OVERFLOW = 0x02
NB_DEV_NONFINITE = 0x04
NB_DEV_STALE_SEARCH = 0x08
NB_DEV_STALE_PRUNE = 0x10
NB_DEV_EXCL_OVERFLOW = 0x20
NB_DEV_CLUSTER_OVERFLOW = 0x40
NB_DEV_BAD_TYPE = 0x80

NB_LIST_OUTER = 0
NB_LIST_INNER = 1

NB_FLAG_COUNT_PAIRS = 0x1
NB_FLAG_NO_LIST_SORT = 0x2
NB_FLAG_CLUSTER_TILES = 0x4
NB_PART_ALL = 0
NB_PART_LOCAL = 1
NB_PART_NONLOCAL = 2
NB_COUL_EWALD = 0
NB_COUL_RF = 1
NB_COUL_SHIFT = 0x1
NB_COUL_EXCL_CORR = 0x2


class NBError(RuntimeError):
    """A libnb call returned a non-zero status."""

    def __init__(self, code: int, message: str):
        super().__init__(f"libnb error {code}: {message}")
        self.code = code


class nb_config(ctypes.Structure):
    _fields_ = [("capacity_entries", ctypes.c_size_t), ("flags", ctypes.c_uint)]


class nb_stats(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int),
        ("n_clusters", ctypes.c_int),
        ("n_columns", ctypes.c_int),
        ("has_inner", ctypes.c_int),
        ("outer_entries", ctypes.c_longlong),
        ("inner_entries", ctypes.c_longlong),
        ("capacity_entries", ctypes.c_longlong),
        ("pairs_last", ctypes.c_longlong),
        ("rlist", ctypes.c_float),
        ("r_inner", ctypes.c_float),
        ("max_disp_search", ctypes.c_float),
        ("max_disp_prune", ctypes.c_float),
        ("error_word", ctypes.c_uint),
        ("gathered_tiles", ctypes.c_longlong),
    ]


_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_SZ = ctypes.c_size_t

# name -> (restype, argtypes); mirrors include/nb.h
SIGNATURES = {
    "nb_version": (ctypes.c_char_p, []),
    "nb_last_error": (ctypes.c_char_p, []),
    "nb_pairlist_create": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(nb_config)]),
    "nb_pairlist_destroy": (_I, [_P]),
    "nb_batch_create": (_I, [ctypes.POINTER(_P), _I, _P, _P, ctypes.POINTER(nb_config)]),
    "nb_search": (_I, [_P, _P, _P, _F, _P, _P, _P]),
    "nb_prune": (_I, [_P, _P, _F, _P]),
    "nb_forces": (_I, [_P, _P, _P, _P, _I, _P, _F, _F, _P, _P, _P]),
    "nb_status": (_I, [_P, ctypes.POINTER(ctypes.c_uint), _I, _P]),
    "nb_pairlist_stats": (_I, [_P, ctypes.POINTER(nb_stats), _P]),
    "nb_tracker_enqueue": (_I, [_P, _P, _P]),
    "nb_pairlist_export": (_I, [_P, _I, _P, _P, _P, _P, _SZ, ctypes.POINTER(_SZ), _P, _SZ,
                                ctypes.POINTER(_SZ), _P]),
    "nb_set_timing_events": (_I, [_P, _P, _P]),
    "nb_set_force_shape": (_I, [_P, _I, _I, _I]),
    "nb_pairlist_export_tiles": (_I, [_P, _P, _P, _P, _SZ, ctypes.POINTER(_SZ), _P]),
    "nb_set_coulomb": (_I, [_P, _I, ctypes.c_float, ctypes.c_uint]),
    "nb_set_flags": (_I, [_P, ctypes.c_uint]),
    "nb_set_home": (_I, [_P, _I]),
    "nb_forces_part": (_I, [_P, _I, _P, _P, _P, _I, _P, ctypes.c_float, ctypes.c_float, _P, _P, _P]),
    "nb_backward": (_I, [_P, _P, _P, _P, _I, _P, _F, _F, _P, _P, _P, _P, _P]),
    "nb_forces_noalloc": (_I, [_I, _P, _P, _P, _P, _I, _P, _F, _F, _P, _P, _P, _P,
                               ctypes.POINTER(ctypes.c_uint), _P]),
    "nb_fp32_peak_probe": (_I, [_I, _I, _I, _P, _SZ, ctypes.POINTER(ctypes.c_double), _P]),
    "nb_pme_spread": (_I, [_I, _P, _P, _P, _I, _I, _I, _I, _P, _P]),
    "nb_pme_gather": (_I, [_I, _P, _P, _P, _I, _I, _I, _I, _P, _P, _I, _P, _P]),
}

NB_NOALLOC_MAX_ATOMS = 4096


def load_library(path: str = LIB_PATH):
    """Load libnb.so and declare its signatures. Raises if it is not built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(
                    f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`. "
                    "The nonbonded path runs only in its CUDA kernels; there is no fallback.")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(code: int):
    if code != NB_OK:
        raise NBError(code, load_library().nb_last_error().decode())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev(t, dtype, numel=None, name="tensor", allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def nb_version() -> str:
    return load_library().nb_version().decode()


def nb_last_error() -> str:
    return load_library().nb_last_error().decode()


def nb_pairlist_create(n_atoms: int, capacity_entries: int = 0, flags: int = 0) -> ctypes.c_void_p:
    handle = ctypes.c_void_p()
    cfg = nb_config(capacity_entries, flags)
    _check(load_library().nb_pairlist_create(ctypes.byref(handle), int(n_atoms), ctypes.byref(cfg)))
    return handle


def nb_batch_create(atom_off, boxes, capacity_entries: int = 0, flags: int = 0) -> ctypes.c_void_p:
    """Pair list over independent systems: atom_off [B+1] and boxes [B, 3] on the host."""
    off = np.ascontiguousarray(np.asarray(atom_off, dtype=np.int32))
    bx = np.ascontiguousarray(np.asarray(boxes, dtype=np.float32).reshape(-1))
    handle = ctypes.c_void_p()
    cfg = nb_config(capacity_entries, flags)
    _check(load_library().nb_batch_create(ctypes.byref(handle), int(off.size - 1), off.ctypes.data_as(_P),
                                          bx.ctypes.data_as(_P), ctypes.byref(cfg)))
    return handle


def nb_pairlist_destroy(pl) -> None:
    if pl is not None:
        _check(load_library().nb_pairlist_destroy(pl))


def nb_search(pl, coords, box, rlist, excl_off=None, excl_idx=None, stream=None) -> None:
    n = coords.numel() // 3
    box_h = None if box is None else (ctypes.c_float * 3)(*[float(v) for v in box])
    _check(load_library().nb_search(pl, _dev(coords, torch.float32, 3 * n, "coords"), box_h, float(rlist),
                                    _dev(excl_off, torch.int32, n + 1, "excl_off", True),
                                    _dev(excl_idx, torch.int32, None, "excl_idx", True), _stream(stream)))


def nb_prune(pl, coords, r_inner, stream=None) -> None:
    _check(load_library().nb_prune(pl, _dev(coords, torch.float32, None, "coords"), float(r_inner),
                                   _stream(stream)))


def nb_forces(pl, coords, q, type_, ljparams, rc, beta, forces, energies=None, stream=None, n_systems=1) -> None:
    n = coords.numel() // 3
    ntype = int(ljparams.shape[0])
    _check(load_library().nb_forces(pl, _dev(coords, torch.float32, 3 * n, "coords"),
                                    _dev(q, torch.float32, n, "q"), _dev(type_, torch.int32, n, "type"), ntype,
                                    _dev(ljparams, torch.float32, 2 * ntype * ntype, "ljparams"), float(rc),
                                    float(beta), _dev(forces, torch.float32, 3 * n, "forces"),
                                    _dev(energies, torch.float64, 2 * n_systems, "energies", True),
                                    _stream(stream)))


def nb_forces_part(pl, part, coords, q, type_, ljparams, rc, beta, forces=None, energies=None, stream=None,
                   n_systems=1) -> None:
    """One part (NB_PART_ALL / NB_PART_LOCAL / NB_PART_NONLOCAL) of nb_forces; see nb.h."""
    n = coords.numel() // 3
    ntype = int(ljparams.shape[0])
    _check(load_library().nb_forces_part(pl, int(part), _dev(coords, torch.float32, 3 * n, "coords"),
                                         _dev(q, torch.float32, n, "q"), _dev(type_, torch.int32, n, "type"), ntype,
                                         _dev(ljparams, torch.float32, 2 * ntype * ntype, "ljparams"), float(rc),
                                         float(beta), _dev(forces, torch.float32, 3 * n, "forces", True),
                                         _dev(energies, torch.float64, 2 * n_systems, "energies", True),
                                         _stream(stream)))


def nb_set_home(pl, n_home: int) -> None:
    """Atoms [0, n_home) are home atoms, the rest halo atoms (see nb.h)."""
    _check(load_library().nb_set_home(pl, int(n_home)))


def nb_backward(pl, coords, q, type_, ljparams, rc, beta, g, grad_x, grad_q, grad_lj, stream=None) -> None:
    n = coords.numel() // 3
    ntype = int(ljparams.shape[0])
    _check(load_library().nb_backward(pl, _dev(coords, torch.float32, 3 * n, "coords"),
                                      _dev(q, torch.float32, n, "q"), _dev(type_, torch.int32, n, "type"), ntype,
                                      _dev(ljparams, torch.float32, 2 * ntype * ntype, "ljparams"), float(rc),
                                      float(beta), _dev(g, torch.float32, 3 * n, "g"),
                                      _dev(grad_x, torch.float32, 3 * n, "grad_x"),
                                      _dev(grad_q, torch.float32, n, "grad_q"),
                                      _dev(grad_lj, torch.float64, 2 * ntype * ntype, "grad_lj"), _stream(stream)))


def nb_status(pl, clear: bool = False, stream=None) -> int:
    w = ctypes.c_uint(0)
    _check(load_library().nb_status(pl, ctypes.byref(w), 1 if clear else 0, _stream(stream)))
    return int(w.value)


def nb_pairlist_stats(pl, stream=None) -> dict:
    s = nb_stats()
    _check(load_library().nb_pairlist_stats(pl, ctypes.byref(s), _stream(stream)))
    return {name: getattr(s, name) for name, _ in nb_stats._fields_}


def nb_tracker_enqueue(pl, host_ptr: int, stream=None) -> None:
    """Enqueue the 12-byte tracker copy (error word, squared displacement
    maxima since the search and the prune) to host address host_ptr."""
    _check(load_library().nb_tracker_enqueue(pl, ctypes.c_void_p(host_ptr), _stream(stream)))


def decode_tracker(words) -> dict:
    """The three 32-bit words of an nb_tracker (e.g. an int32 tensor or
    array of 3) as error_word, max_disp_search, max_disp_prune (nm)."""
    w = np.asarray(words, dtype=np.int32)[:3].copy()
    d2 = w[1:3].view(np.float32).astype(np.float64)
    return {"error_word": int(np.uint32(w[0])), "max_disp_search": float(np.sqrt(d2[0])),
            "max_disp_prune": float(np.sqrt(d2[1]))}


def nb_pairlist_export(pl, which: int = NB_LIST_OUTER, stream=None) -> dict:
    """Copy a list to host numpy arrays: ci, cj, shift, mask (uint64), perm."""
    st = nb_pairlist_stats(pl, stream)
    cap = int(st["outer_entries"]) + 1
    nslot = 8 * int(st["n_clusters"])
    ci = np.empty(cap, np.int32)
    cj = np.empty(cap, np.int32)
    sh = np.empty(cap, np.int32)
    mk = np.empty(cap, np.uint64)
    perm = np.empty(max(nslot, 1), np.int32)
    n_out = ctypes.c_size_t(0)
    n_slots = ctypes.c_size_t(0)
    _check(load_library().nb_pairlist_export(
        pl, int(which), ci.ctypes.data_as(_P), cj.ctypes.data_as(_P), sh.ctypes.data_as(_P),
        mk.ctypes.data_as(_P), cap, ctypes.byref(n_out), perm.ctypes.data_as(_P), perm.size,
        ctypes.byref(n_slots), _stream(stream)))
    k = n_out.value
    return {"ci": ci[:k], "cj": cj[:k], "shift": sh[:k], "mask": mk[:k], "perm": perm[:n_slots.value]}


def nb_set_timing_events(pl, start=None, stop=None) -> None:
    """Record torch.cuda.Event ``start``/``stop`` around the force kernel of later nb_forces calls."""
    sp = None if start is None else ctypes.c_void_p(start.cuda_event)
    ep = None if stop is None else ctypes.c_void_p(stop.cuda_event)
    _check(load_library().nb_set_timing_events(pl, sp, ep))


def nb_forces_noalloc(coords, box, q, type_, ljparams, rc, beta, forces, energies=None, excl_off=None,
                      excl_idx=None, read_error_word=True, stream=None):
    """Search + forces for up to 4,096 atoms with no device allocation.

    For callers that cannot allocate device memory: all scratch lives in a
    static device array inside libnb.so. Returns the device error word when
    ``read_error_word`` (the call then synchronises the stream), else None.
    """
    n = coords.numel() // 3
    ntype = int(ljparams.shape[0])
    box_h = (ctypes.c_float * 3)(*[float(v) for v in box])
    word = ctypes.c_uint(0)
    _check(load_library().nb_forces_noalloc(
        n, _dev(coords, torch.float32, 3 * n, "coords"), box_h, _dev(q, torch.float32, n, "q"),
        _dev(type_, torch.int32, n, "type"), ntype, _dev(ljparams, torch.float32, 2 * ntype * ntype, "ljparams"),
        float(rc), float(beta), _dev(excl_off, torch.int32, n + 1, "excl_off", True),
        _dev(excl_idx, torch.int32, None, "excl_idx", True), _dev(forces, torch.float32, 3 * n, "forces"),
        _dev(energies, torch.float64, 2, "energies", True), ctypes.byref(word) if read_error_word else None,
        _stream(stream)))
    return int(word.value) if read_error_word else None


def nb_fp32_peak_probe(out, packed: bool = True, blocks_per_sm: int = 8, iters: int = 4096, stream=None) -> float:
    """Queue the FP32 fused multiply-add probe on ``stream``; returns the FP32
    operations it performs (a fused multiply-add counted as 2). ``out`` is a
    float32 device tensor with at least SMs x blocks_per_sm x 256 elements."""
    flops = ctypes.c_double(0.0)
    _check(load_library().nb_fp32_peak_probe(int(bool(packed)), int(blocks_per_sm), int(iters),
                                             _dev(out, torch.float32, None, "out"), out.numel(),
                                             ctypes.byref(flops), _stream(stream)))
    return float(flops.value)


def _mesh(K):
    K = tuple(int(k) for k in K)
    if len(K) != 3:
        raise ValueError("K must give three mesh dimensions")
    return K


def nb_pme_spread(coords, q, box, K, grid, order: int = 4, stream=None) -> None:
    """Smooth-PME charge spreading: ``grid`` (float32 [K0, K1, K2], device) is
    overwritten with Q(k) = sum_i q_i prod_a M4(u_ia - k_a)."""
    n = coords.numel() // 3
    K = _mesh(K)
    box_h = (ctypes.c_float * 3)(*[float(v) for v in box])
    _check(load_library().nb_pme_spread(
        n, _dev(coords, torch.float32, 3 * n, "coords"), _dev(q, torch.float32, n, "q"), box_h, *K, int(order),
        _dev(grid, torch.float32, K[0] * K[1] * K[2], "grid"), _stream(stream)))


def nb_pme_gather(coords, q, box, K, phi, forces, order: int = 4, accumulate: bool = False, energy=None,
                  stream=None) -> None:
    """Smooth-PME force gathering from the mesh potential ``phi``: forces
    (float32 [N, 3], device) set to, or with ``accumulate`` added to,
    -q grad psi; ``energy`` (float64 [1], device, optional) set to
    (1/2) sum_i q_i psi_i."""
    n = coords.numel() // 3
    K = _mesh(K)
    box_h = (ctypes.c_float * 3)(*[float(v) for v in box])
    _check(load_library().nb_pme_gather(
        n, _dev(coords, torch.float32, 3 * n, "coords"), _dev(q, torch.float32, n, "q"), box_h, *K, int(order),
        _dev(phi, torch.float32, K[0] * K[1] * K[2], "phi"), _dev(forces, torch.float32, 3 * n, "forces"),
        int(bool(accumulate)), _dev(energy, torch.float64, 1, "energy", True), _stream(stream)))


def nb_pairlist_export_tiles(pl, stream=None) -> dict:
    """Gathered 4x8 tiles of the last prune: half_id [T], slots [T, 8] (slot | shift << 27), masks [T]."""
    st = nb_pairlist_stats(pl, stream)
    cap = 2 * int(st["outer_entries"]) + 1
    hid = np.empty(cap, np.int32)
    slots = np.empty((cap, 8), np.int32)
    masks = np.empty(cap, np.uint32)
    n = ctypes.c_size_t(0)
    _check(load_library().nb_pairlist_export_tiles(pl, hid.ctypes.data_as(_P), slots.ctypes.data_as(_P),
                                                   masks.ctypes.data_as(_P), cap, ctypes.byref(n), _stream(stream)))
    k = n.value
    return {"half_id": hid[:k], "slots": slots[:k], "masks": masks[:k]}


def nb_set_coulomb(pl, kind: int = NB_COUL_EWALD, eps_rf: float = 0.0, flags: int = 0) -> None:
    """Coulomb flavour of later nb_forces / nb_backward calls (NB_COUL_EWALD or NB_COUL_RF)."""
    _check(load_library().nb_set_coulomb(pl, int(kind), float(eps_rf), int(flags)))


def nb_set_flags(pl, flags: int) -> None:
    """Replace the pair list's NB_FLAG_* flags (see nb.h)."""
    _check(load_library().nb_set_flags(pl, int(flags)))


def nb_set_force_shape(pl, threads: int = 0, chunk: int = 0, blocks_per_sm: int = 0) -> None:
    _check(load_library().nb_set_force_shape(pl, int(threads), int(chunk), int(blocks_per_sm)))


class Pairlist:
    """Owns one nb_pairlist handle (destroyed on close / garbage collection)."""

    def __init__(self, n_atoms: int, capacity_entries: int = 0, count_pairs: bool = False, sort_lists: bool = True,
                 cluster_tiles: bool = False, _handle=None, _n_systems: int = 1):
        self.n_atoms = int(n_atoms)
        self.n_systems = int(_n_systems)
        self.handle = _handle if _handle is not None else nb_pairlist_create(
            self.n_atoms, capacity_entries, self._flags(count_pairs, sort_lists, cluster_tiles))

    @staticmethod
    def _flags(count_pairs: bool, sort_lists: bool, cluster_tiles: bool = False) -> int:
        return ((NB_FLAG_COUNT_PAIRS if count_pairs else 0) | (0 if sort_lists else NB_FLAG_NO_LIST_SORT)
                | (NB_FLAG_CLUSTER_TILES if cluster_tiles else 0))

    @classmethod
    def batch(cls, atom_off, boxes, capacity_entries: int = 0, count_pairs: bool = False, sort_lists: bool = True):
        """A pair list over independent systems (see nb_batch_create)."""
        h = nb_batch_create(atom_off, boxes, capacity_entries, cls._flags(count_pairs, sort_lists))
        return cls(int(atom_off[-1]), _handle=h, _n_systems=len(atom_off) - 1)

    def search(self, coords, box, rlist, excl_off=None, excl_idx=None, stream=None):
        nb_search(self.handle, coords, box, rlist, excl_off, excl_idx, stream)

    def prune(self, coords, r_inner, stream=None):
        nb_prune(self.handle, coords, r_inner, stream)

    def forces(self, coords, q, type_, ljparams, rc, beta, forces=None, energies=None, want_energy=True,
               stream=None):
        if forces is None:
            forces = torch.empty((self.n_atoms, 3), dtype=torch.float32, device=coords.device)
        if energies is None and want_energy:
            energies = torch.empty(2 * self.n_systems, dtype=torch.float64, device=coords.device)
        nb_forces(self.handle, coords, q, type_, ljparams, rc, beta, forces, energies, stream, self.n_systems)
        return forces, energies

    def set_home(self, n_home: int) -> None:
        nb_set_home(self.handle, n_home)

    def forces_part(self, part, coords, q, type_, ljparams, rc, beta, forces=None, energies=None, stream=None):
        """nb_forces_part; returns (forces, energies) (forces is not written by the local part)."""
        if forces is None and part != NB_PART_LOCAL:
            forces = torch.empty((self.n_atoms, 3), dtype=torch.float32, device=coords.device)
        nb_forces_part(self.handle, part, coords, q, type_, ljparams, rc, beta, forces, energies, stream,
                       self.n_systems)
        return forces, energies

    def backward(self, coords, q, type_, ljparams, rc, beta, g, stream=None):
        """dL/dx [N,3], dL/dq [N], dL/dC [nt,nt,2] (FP64) for g = dL/dF."""
        nt = int(ljparams.shape[0])
        gx = torch.empty((self.n_atoms, 3), dtype=torch.float32, device=coords.device)
        gq = torch.empty(self.n_atoms, dtype=torch.float32, device=coords.device)
        glj = torch.empty((nt, nt, 2), dtype=torch.float64, device=coords.device)
        nb_backward(self.handle, coords, q, type_, ljparams, rc, beta, g, gx, gq, glj, stream)
        return gx, gq, glj

    def status(self, clear=False, stream=None) -> int:
        return nb_status(self.handle, clear, stream)

    def stats(self, stream=None) -> dict:
        return nb_pairlist_stats(self.handle, stream)

    def tracker_enqueue(self, host_words, stream=None) -> None:
        """Enqueue the tracker copy into host_words, a page-locked int32
        tensor of 3 or more elements; decode_tracker reads it once the
        stream has passed this point."""
        if host_words.dtype != torch.int32 or host_words.numel() < 3 or host_words.device.type != "cpu":
            raise ValueError("host_words: a host int32 tensor of at least 3 elements")
        nb_tracker_enqueue(self.handle, host_words.data_ptr(), stream)

    def export(self, which=NB_LIST_OUTER, stream=None) -> dict:
        return nb_pairlist_export(self.handle, which, stream)

    def export_tiles(self, stream=None) -> dict:
        return nb_pairlist_export_tiles(self.handle, stream)

    def set_flags(self, count_pairs: bool = False, sort_lists: bool = True, cluster_tiles: bool = False) -> None:
        nb_set_flags(self.handle, self._flags(count_pairs, sort_lists, cluster_tiles))

    def set_coulomb(self, kind: str = "ewald", eps_rf: float = 0.0, shift: bool = False,
                    excl_corr: bool = False) -> None:
        """kind "ewald" or "rf" (reaction field, eps_rf = 0 meaning infinity);
        shift (Ewald) and excl_corr (excluded-pair correction) as in nb.h."""
        flags = (NB_COUL_SHIFT if shift else 0) | (NB_COUL_EXCL_CORR if excl_corr else 0)
        nb_set_coulomb(self.handle, {"ewald": NB_COUL_EWALD, "rf": NB_COUL_RF}[kind], eps_rf, flags)

    def close(self):
        if getattr(self, "handle", None) is not None:
            nb_pairlist_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
