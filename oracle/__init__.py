"""CPU FP64 oracle for the short-range nonbonded path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package. The CUDA library never loads it and
shares no code with it. The arithmetic lives in ``oracle.c`` (plain C,
FP64, OpenMP); this module compiles it with gcc on first use and marshals
numpy arrays.

Functions:

* ``energy_forces`` - E_LJ, E_C and F for every atom (O(N^2) or cell list).
* ``forces_subset`` - F on chosen atoms only, each summed over all partners.
* ``pairs_f64`` - brute-force set of pairs with r < r_cut in FP64.
* ``pairs_f32`` - the set of pairs within rc under the FP32 contract that the
  GPU pair list must reproduce bit for bit.
* ``image_f32`` - the FP32 positions that contract uses.
* ``energy_f32`` - E_LJ and E_C at the distances that contract fixes.
* ``force_vjp`` - adjoint of the forces: dL/dx, dL/dq, dL/dC given dL/dF.
* ``force_matching`` - loss (1/3N) sum |F - T|^2 and its gradients.
* ``bspline``, ``pme_spread``, ``pme_gather`` - smooth-PME cardinal
  B-splines, charge spreading onto the mesh and force gathering from a mesh
  potential (Essmann et al. 1995).

Parity: pinned by the CPU tests in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.environ.get("NB_ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

COULOMB_F = 138.935458


def build(force: bool = False, src: str = _SRC, out: str | None = None) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, OpenMP, no FP contraction).

    ``src``/``out`` let the mutation tests compile a deliberately broken copy
    elsewhere; ``NB_ORACLE_LIB`` then points the loader at it.
    """
    out = out or _LIB_PATH
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", tmp, src, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.environ.get("NB_ORACLE_LIB"):
                build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            F = ctypes.c_float
            LL = ctypes.c_longlong
            lib.oracle_threads.restype = I
            lib.oracle_energy_forces.argtypes = [I, P, P, P, I, P, P, D, D, P, P, I, P, P, P, P]
            lib.oracle_energy_forces.restype = I
            lib.oracle_forces_subset.argtypes = [I, P, P, P, I, P, P, D, D, P, P, I, P, P]
            lib.oracle_forces_subset.restype = I
            lib.oracle_pairs_f64.argtypes = [I, P, P, D, P, P, P, P, LL, P]
            lib.oracle_pairs_f64.restype = I
            lib.oracle_pairs_f32.argtypes = [I, P, P, P, F, P, P, P, P, LL, P]
            lib.oracle_pairs_f32.restype = I
            lib.oracle_image_f32.argtypes = [I, P, P, P, P]
            lib.oracle_image_f32.restype = None
            lib.oracle_energy_f32.argtypes = [I, P, P, P, P, I, P, P, D, D, P, P, P, P]
            lib.oracle_energy_f32.restype = I
            lib.oracle_force_vjp.argtypes = [I, P, P, P, I, P, P, D, D, P, P, P, P, P, P]
            lib.oracle_force_vjp.restype = I
            lib.oracle_energy_forces_coul.argtypes = [I, P, P, P, I, P, P, D, D, P, P, I, D, I, P, P, P]
            lib.oracle_energy_forces_coul.restype = I
            lib.oracle_force_vjp_coul.argtypes = [I, P, P, P, I, P, P, D, D, P, P, I, D, I, P, P, P, P]
            lib.oracle_force_vjp_coul.restype = I
            lib.oracle_energy_forces_coul_list.argtypes = [I, P, P, P, I, P, P, D, D, P, P, I, D, I, P, LL, P, P]
            lib.oracle_energy_forces_coul_list.restype = I
            lib.oracle_bspline.argtypes = [I, D]
            lib.oracle_bspline.restype = D
            lib.oracle_bspline_deriv.argtypes = [I, D]
            lib.oracle_bspline_deriv.restype = D
            lib.oracle_pme_spread.argtypes = [I, P, P, P, P, I, P, P]
            lib.oracle_pme_spread.restype = I
            lib.oracle_pme_gather.argtypes = [I, P, P, P, P, I, P, P, P, P]
            lib.oracle_pme_gather.restype = I
            _lib = lib
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _i32(a) -> np.ndarray | None:
    return None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_threads())


def energy_forces(x, q, type_, lj, box, rc, beta, excl_off=None, excl_idx=None, method="auto",
                  abs_sums=False):
    """FP64 energies and forces.

    Returns ``(F [N,3], E_lj, E_coul, npairs)``; with ``abs_sums`` also
    ``(sum |e_lj|, sum |e_coul|)`` over the pairs as a fifth item. ``lj`` is
    [ntype, ntype, 2] holding (C6, C12). ``method`` is "auto", "n2" or "cell".
    """
    lib = _load()
    x = _f64(x).reshape(-1, 3)
    n = x.shape[0]
    lj = _f64(lj)
    ntype = lj.shape[0]
    F = np.zeros((n, 3), dtype=np.float64)
    E = np.zeros(2, dtype=np.float64)
    A = np.zeros(2, dtype=np.float64)
    npairs = ctypes.c_longlong(0)
    m = {"auto": 0, "n2": 1, "cell": 2}[method]
    rcode = lib.oracle_energy_forces(n, _p(x), _p(_f64(q)), _p(_i32(type_)), ntype, _p(lj),
                                     _p(_f64(box)), float(rc), float(beta), _p(_i32(excl_off)),
                                     _p(_i32(excl_idx)), m, _p(F), _p(E), ctypes.byref(npairs), _p(A))
    if rcode != 0:
        raise ValueError(f"oracle_energy_forces failed with code {rcode}")
    if abs_sums:
        return F, float(E[0]), float(E[1]), int(npairs.value), (float(A[0]), float(A[1]))
    return F, float(E[0]), float(E[1]), int(npairs.value)


def forces_subset(x, q, type_, lj, box, rc, beta, atoms, excl_off=None, excl_idx=None):
    """FP64 forces on the atoms listed in ``atoms`` ([m, 3])."""
    lib = _load()
    x = _f64(x).reshape(-1, 3)
    lj = _f64(lj)
    atoms = _i32(atoms)
    out = np.zeros((atoms.size, 3), dtype=np.float64)
    rcode = lib.oracle_forces_subset(x.shape[0], _p(x), _p(_f64(q)), _p(_i32(type_)), lj.shape[0],
                                     _p(lj), _p(_f64(box)), float(rc), float(beta),
                                     _p(_i32(excl_off)), _p(_i32(excl_idx)), atoms.size, _p(atoms),
                                     _p(out))
    if rcode != 0:
        raise ValueError(f"oracle_forces_subset failed with code {rcode}")
    return out


def pairs_f64(x, box, r_cut, excl_off=None, excl_idx=None):
    """Brute-force FP64 set of pairs (i < j) within r_cut, as an int64 array [P, 2]."""
    lib = _load()
    x = _f64(x).reshape(-1, 3)
    n = x.shape[0]
    cap = max(16, n * 512)
    while True:
        pi = np.empty(cap, dtype=np.int32)
        pj = np.empty(cap, dtype=np.int32)
        cnt = ctypes.c_longlong(0)
        lib.oracle_pairs_f64(n, _p(x), _p(_f64(box)), float(r_cut), _p(_i32(excl_off)),
                             _p(_i32(excl_idx)), _p(pi), _p(pj), cap, ctypes.byref(cnt))
        if cnt.value <= cap:
            return np.stack([pi[:cnt.value], pj[:cnt.value]], axis=1).astype(np.int64)
        cap = int(cnt.value)


def pairs_f32(x0, x, box, rc, excl_off=None, excl_idx=None, count_only=False):
    """Pairs within rc under the FP32 contract (see ``oracle.c``).

    ``x0`` is the frame the list was searched on, ``x`` the current frame
    (pass the same array twice for the search frame). Returns an int64 array
    [P, 2] with i < j, or the count if ``count_only``.
    """
    lib = _load()
    x0 = _f32(x0).reshape(-1, 3)
    x = _f32(x).reshape(-1, 3)
    n = x.shape[0]
    box = _f32(box)
    cnt = ctypes.c_longlong(0)
    if count_only:
        rc_ = lib.oracle_pairs_f32(n, _p(x0), _p(x), _p(box), float(rc), _p(_i32(excl_off)),
                                   _p(_i32(excl_idx)), None, None, 0, ctypes.byref(cnt))
        if rc_ < 0:
            raise ValueError(f"oracle_pairs_f32 failed with code {rc_}")
        return int(cnt.value)
    cap = max(16, n * 400)
    while True:
        pi = np.empty(cap, dtype=np.int32)
        pj = np.empty(cap, dtype=np.int32)
        rc_ = lib.oracle_pairs_f32(n, _p(x0), _p(x), _p(box), float(rc), _p(_i32(excl_off)),
                                   _p(_i32(excl_idx)), _p(pi), _p(pj), cap, ctypes.byref(cnt))
        if rc_ < 0:
            raise ValueError(f"oracle_pairs_f32 failed with code {rc_}")
        if cnt.value <= cap:
            return np.stack([pi[:cnt.value], pj[:cnt.value]], axis=1).astype(np.int64)
        cap = int(cnt.value)


def energy_f32(x0, x, q, type_, lj, box, rc, beta, excl_off=None, excl_idx=None, abs_sums=False):
    """FP64 pair energies of the FP32 contract: ``(E_lj, E_coul, npairs)``, with ``abs_sums``
    also ``(sum |e_lj|, sum |e_coul|)`` over the pairs as a fourth item.

    The plain definitions of ``energy_forces``, summed over the ``pairs_f32``
    set, each pair at its FP32-contract r^2, with the cutoff the C ABI
    receives (``float32(rc)``) for the set and the LJ shift. The difference
    from ``energy_forces(..., rc)`` is what rounding the displacements and
    the cutoff to FP32 does to the energies by itself.
    """
    lib = _load()
    x0 = _f32(x0).reshape(-1, 3)
    x = _f32(x).reshape(-1, 3)
    lj = _f64(lj)
    E = np.zeros(4, dtype=np.float64)
    npairs = ctypes.c_longlong(0)
    rcode = lib.oracle_energy_f32(x.shape[0], _p(x0), _p(x), _p(_f64(q)), _p(_i32(type_)), lj.shape[0], _p(lj),
                                  _p(_f32(box)), float(rc), float(beta), _p(_i32(excl_off)), _p(_i32(excl_idx)),
                                  _p(E), ctypes.byref(npairs))
    if rcode != 0:
        raise ValueError(f"oracle_energy_f32 failed with code {rcode}")
    if abs_sums:
        return float(E[0]), float(E[1]), int(npairs.value), (float(E[2]), float(E[3]))
    return float(E[0]), float(E[1]), int(npairs.value)


def image_f32(x0, x, box):
    """FP32 positions of the contract: image of ``x`` nearest wrap(``x0``)."""
    lib = _load()
    x0 = _f32(x0).reshape(-1, 3)
    x = _f32(x).reshape(-1, 3)
    y = np.empty_like(x)
    lib.oracle_image_f32(x.shape[0], _p(x0), _p(x), _p(_f32(box)), _p(y))
    return y


def force_vjp(x, q, type_, lj, box, rc, beta, g, excl_off=None, excl_idx=None):
    """Adjoint of the forces: given g = dL/dF [N, 3], returns (gx [N,3], gq [N], glj [nt,nt,2])."""
    lib = _load()
    x = _f64(x).reshape(-1, 3)
    n = x.shape[0]
    lj = _f64(lj)
    nt = lj.shape[0]
    g = _f64(g).reshape(-1, 3)
    gx = np.zeros((n, 3))
    gq = np.zeros(n)
    glj = np.zeros((nt, nt, 2))
    rcode = lib.oracle_force_vjp(n, _p(x), _p(_f64(q)), _p(_i32(type_)), nt, _p(lj), _p(_f64(box)), float(rc),
                                 float(beta), _p(_i32(excl_off)), _p(_i32(excl_idx)), _p(g), _p(gx), _p(gq), _p(glj))
    if rcode != 0:
        raise ValueError(f"oracle_force_vjp failed with code {rcode}")
    return gx, gq, glj


def force_matching(x, q, type_, lj, box, rc, beta, target, excl_off=None, excl_idx=None):
    """Loss L = (1/3N) sum_i |F_i - T_i|^2 and (dL/dx, dL/dq, dL/dC, F)."""
    F, _, _, _ = energy_forces(x, q, type_, lj, box, rc, beta, excl_off, excl_idx)
    n = F.shape[0]
    diff = F - np.asarray(target, np.float64).reshape(-1, 3)
    L = float((diff ** 2).sum() / (3 * n))
    g = 2.0 * diff / (3 * n)
    gx, gq, glj = force_vjp(x, q, type_, lj, box, rc, beta, g, excl_off, excl_idx)
    return L, gx, gq, glj, F


COUL_KINDS = {"ewald": 0, "rf": 1}
COUL_SHIFT = 0x1
COUL_EXCL_CORR = 0x2


def _coul_flags(shift: bool, excl_corr: bool) -> int:
    return (COUL_SHIFT if shift else 0) | (COUL_EXCL_CORR if excl_corr else 0)


def energy_forces_coul(x, q, type_, lj, box, rc, beta, excl_off=None, excl_idx=None, kind="ewald",
                       eps_rf=0.0, shift=False, excl_corr=False):
    """FP64 energies and forces with the Coulomb options (reaction field,
    Ewald potential shift, excluded-pair correction).

    Returns ``(F [N,3], E_lj, E_coul, npairs)``; E_coul includes the
    excluded-pair corrections, npairs counts non-excluded pairs within rc.
    ``eps_rf`` = 0 means an infinite reaction-field permittivity.
    """
    lib = _load()
    x = _f64(x).reshape(-1, 3)
    n = x.shape[0]
    lj = _f64(lj)
    F = np.zeros((n, 3))
    E = np.zeros(2)
    npairs = ctypes.c_longlong(0)
    rcode = lib.oracle_energy_forces_coul(n, _p(x), _p(_f64(q)), _p(_i32(type_)), lj.shape[0], _p(lj),
                                          _p(_f64(box)), float(rc), float(beta), _p(_i32(excl_off)),
                                          _p(_i32(excl_idx)), COUL_KINDS[kind], float(eps_rf),
                                          _coul_flags(shift, excl_corr), _p(F), _p(E), ctypes.byref(npairs))
    if rcode != 0:
        raise ValueError(f"oracle_energy_forces_coul failed with code {rcode}")
    return F, float(E[0]), float(E[1]), int(npairs.value)


def force_vjp_coul(x, q, type_, lj, box, rc, beta, g, excl_off=None, excl_idx=None, kind="ewald", eps_rf=0.0,
                   excl_corr=False):
    """Adjoint of energy_forces_coul's forces for g = dL/dF: (gx [N,3], gq [N], glj [nt,nt,2]).
    O(N^2); for small systems."""
    lib = _load()
    x = _f64(x).reshape(-1, 3)
    n = x.shape[0]
    lj = _f64(lj)
    nt = lj.shape[0]
    g = _f64(g).reshape(-1, 3)
    gx = np.zeros((n, 3))
    gq = np.zeros(n)
    glj = np.zeros((nt, nt, 2))
    rcode = lib.oracle_force_vjp_coul(n, _p(x), _p(_f64(q)), _p(_i32(type_)), nt, _p(lj), _p(_f64(box)), float(rc),
                                      float(beta), _p(_i32(excl_off)), _p(_i32(excl_idx)), COUL_KINDS[kind],
                                      float(eps_rf), _coul_flags(False, excl_corr), _p(g), _p(gx), _p(gq), _p(glj))
    if rcode != 0:
        raise ValueError(f"oracle_force_vjp_coul failed with code {rcode}")
    return gx, gq, glj


def rf_constants(rc: float, eps_rf: float) -> tuple[float, float]:
    """(k_rf, c_rf) of the reaction field; eps_rf = 0 means infinity."""
    k = 1.0 / (2.0 * rc ** 3) if eps_rf == 0.0 else (eps_rf - 1.0) / ((2.0 * eps_rf + 1.0) * rc ** 3)
    return k, 1.0 / rc + k * rc * rc


def energy_forces_coul_pairs(x, q, type_, lj, box, rc, beta, pairs, excl_off=None, excl_idx=None, kind="ewald",
                             eps_rf=0.0, shift=False, excl_corr=False):
    """energy_forces_coul over an explicit set of non-excluded pairs ``pairs``
    [P, 2] (i < j), e.g. the FP32-contract set of ``pairs_f32``; returns
    ``(F [N,3], E_lj, E_coul)``."""
    lib = _load()
    x = _f64(x).reshape(-1, 3)
    n = x.shape[0]
    lj = _f64(lj)
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
    F = np.zeros((n, 3))
    E = np.zeros(2)
    rcode = lib.oracle_energy_forces_coul_list(n, _p(x), _p(_f64(q)), _p(_i32(type_)), lj.shape[0], _p(lj),
                                               _p(_f64(box)), float(rc), float(beta), _p(_i32(excl_off)),
                                               _p(_i32(excl_idx)), COUL_KINDS[kind], float(eps_rf),
                                               _coul_flags(shift, excl_corr), _p(pr), pr.shape[0], _p(F), _p(E))
    if rcode != 0:
        raise ValueError(f"oracle_energy_forces_coul_list failed with code {rcode}")
    return F, float(E[0]), float(E[1])


def bspline(order: int, u: float, deriv: bool = False) -> float:
    """Cardinal B-spline M_order(u), or its derivative dM/du."""
    lib = _load()
    return float((lib.oracle_bspline_deriv if deriv else lib.oracle_bspline)(int(order), float(u)))


def pme_spread(x, q, box, K, order=4, abs_sums=False):
    """Charge grid Q [K0, K1, K2] of smooth PME; with ``abs_sums`` also the spread of |q|."""
    lib = _load()
    x = _f64(x).reshape(-1, 3)
    K = np.ascontiguousarray(np.asarray(K, dtype=np.int32))
    Q = np.empty(tuple(int(k) for k in K), dtype=np.float64)
    Qa = np.empty_like(Q) if abs_sums else None
    rcode = lib.oracle_pme_spread(x.shape[0], _p(x), _p(_f64(q)), _p(_f64(box)), _p(K), int(order), _p(Q), _p(Qa))
    if rcode != 0:
        raise ValueError(f"oracle_pme_spread failed with code {rcode}")
    return (Q, Qa) if abs_sums else Q


def pme_gather(x, q, box, K, phi, order=4, abs_sums=False):
    """Forces F [N, 3] = -q grad psi and potentials psi [N] interpolated from the
    mesh potential ``phi`` [K0, K1, K2]; with ``abs_sums`` also the per-component
    sums of |terms| [N, 3]."""
    lib = _load()
    x = _f64(x).reshape(-1, 3)
    K = np.ascontiguousarray(np.asarray(K, dtype=np.int32))
    phi = _f64(phi)
    assert phi.shape == tuple(int(k) for k in K)
    n = x.shape[0]
    F = np.empty((n, 3), dtype=np.float64)
    psi = np.empty(n, dtype=np.float64)
    Fa = np.empty((n, 3), dtype=np.float64) if abs_sums else None
    rcode = lib.oracle_pme_gather(n, _p(x), _p(_f64(q)), _p(_f64(box)), _p(K), int(order), _p(phi), _p(F), _p(psi),
                                  _p(Fa))
    if rcode != 0:
        raise ValueError(f"oracle_pme_gather failed with code {rcode}")
    return (F, psi, Fa) if abs_sums else (F, psi)
