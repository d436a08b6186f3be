"""Shared helpers of the GPU parity tests: run the CUDA path, expand its list."""
import numpy as np
import torch

import oracle
from fp32util import r2_contract

F_TOL = 1e-4   # per-atom |dF| <= F_TOL * rms(F_oracle)
E_TOL = 1e-6   # relative energy error


def to_dev(box, dev="cuda"):
    """Device tensors of a synth.WaterBox."""
    return {
        "coords": torch.from_numpy(np.ascontiguousarray(box.coords)).to(dev),
        "q": torch.from_numpy(np.ascontiguousarray(box.q)).to(dev),
        "type": torch.from_numpy(np.ascontiguousarray(box.type)).to(dev),
        "lj": torch.from_numpy(np.ascontiguousarray(box.ljparams)).to(dev),
        "excl_off": torch.from_numpy(np.ascontiguousarray(box.excl_off)).to(dev),
        "excl_idx": torch.from_numpy(np.ascontiguousarray(box.excl_idx)).to(dev),
    }


def expand_counted_pairs(exp, y, box, r_cut):
    """Atom pairs of an exported list whose mask bit is set and whose FP32
    distance under the kernels' contract is below r_cut.

    ``y`` are the contract positions (oracle.image_f32). Returns an int64 [P, 2]
    array with i < j, one row per (entry, bit) that passes (duplicates kept).
    """
    ci, cj, sh, mk, perm = exp["ci"], exp["cj"], exp["shift"], exp["mask"], exp["perm"]
    if ci.size == 0:
        return np.zeros((0, 2), np.int64)
    bits = ((mk[:, None] >> np.arange(64, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(bool)
    e_idx, bit = np.nonzero(bits)
    a = bit // 8
    b = bit % 8
    p = perm[ci[e_idx] * 8 + a]
    q = perm[cj[e_idx] * 8 + b]
    assert (p >= 0).all() and (q >= 0).all(), "mask bit set on a padding slot"
    s = sh[e_idx]
    S = np.stack([(s // 9 - 1), ((s // 3) % 3 - 1), (s % 3 - 1)], axis=1).astype(np.float32) * box.astype(np.float32)
    d = (y[p] - y[q]).astype(np.float32)
    d = (d + S).astype(np.float32)
    r2 = r2_contract(d[:, 0], d[:, 1], d[:, 2])
    rc2 = np.float32(r_cut) * np.float32(r_cut)
    keep = r2 < rc2
    i = np.minimum(p[keep], q[keep])
    j = np.maximum(p[keep], q[keep])
    return np.stack([i, j], axis=1).astype(np.int64)


def expand_tile_pairs(tiles, perm, y, box, r_cut):
    """Atom pairs of the gathered 4 x 8 tiles whose mask bit is set and whose
    FP32 contract distance is below r_cut (int64 [P, 2], i < j, duplicates kept).

    Tile k covers rows 4h..4h+3 of i-cluster ci (half_id = 2 ci + h) and the
    8 j atoms slots[k] (cluster slot in the low 27 bits, shift index above).
    """
    hid, slots, masks = tiles["half_id"], tiles["slots"], tiles["masks"]
    if hid.size == 0:
        return np.zeros((0, 2), np.int64)
    bits = ((masks[:, None].astype(np.uint64) >> np.arange(32, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(bool)
    t_idx, bit = np.nonzero(bits)
    a = bit // 8
    col = bit % 8
    v = slots[t_idx, col].view(np.uint32)
    jslot = (v & np.uint32(0x07FFFFFF)).astype(np.int64)
    s = (v >> np.uint32(27)).astype(np.int64)
    assert (jslot < perm.size).all(), "mask bit set on the pad slot"
    islot = (hid[t_idx] // 2).astype(np.int64) * 8 + 4 * (hid[t_idx] % 2) + a
    p = perm[islot]
    q = perm[jslot]
    assert (p >= 0).all() and (q >= 0).all(), "mask bit set on a padding slot"
    assert (s < 27).all()
    S = np.stack([(s // 9 - 1), ((s // 3) % 3 - 1), (s % 3 - 1)], axis=1).astype(np.float32) * box.astype(np.float32)
    d = (y[p] - y[q]).astype(np.float32)
    d = (d + S).astype(np.float32)
    r2 = r2_contract(d[:, 0], d[:, 1], d[:, 2])
    keep = r2 < np.float32(r_cut) * np.float32(r_cut)
    i = np.minimum(p[keep], q[keep])
    j = np.maximum(p[keep], q[keep])
    return np.stack([i, j], axis=1).astype(np.int64)


def assert_same_pairs(got, ref, n_atoms):
    """Two [P, 2] (i < j) pair arrays hold the same pairs, and ``got`` none twice.

    Compares sorted int64 keys i * n + j, which scales to tens of millions
    of pairs where Python sets do not.
    """
    kg = np.sort(np.asarray(got, np.int64)[:, 0] * n_atoms + np.asarray(got, np.int64)[:, 1])
    kr = np.sort(np.asarray(ref, np.int64)[:, 0] * n_atoms + np.asarray(ref, np.int64)[:, 1])
    assert kg.size == 0 or (np.diff(kg) > 0).all(), "an atom pair is listed twice"
    if not np.array_equal(kg, kr):
        extra = np.setdiff1d(kg, kr)[:5]
        missing = np.setdiff1d(kr, kg)[:5]
        raise AssertionError(f"pair sets differ ({kg.size} vs {kr.size}): extra {[(k // n_atoms, k % n_atoms) for k in extra]}"
                             f", missing {[(k // n_atoms, k % n_atoms) for k in missing]}")


def pair_set(arr):
    return set(map(tuple, np.asarray(arr).tolist()))


def compare_forces(F_gpu, F_ref, tol=F_TOL):
    """max_i |F_gpu_i - F_ref_i| / rms(F_ref); asserts <= tol."""
    F_gpu = np.asarray(F_gpu, np.float64)
    rms = np.sqrt((F_ref ** 2).sum(1).mean())
    err = np.sqrt(((F_gpu - F_ref) ** 2).sum(1))
    worst = float(err.max() / rms)
    assert worst <= tol, f"max per-atom |dF| = {err.max():.3e} = {worst:.2e} rms(F) (rms {rms:.3e})"
    return worst


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def oracle_ref(box, rc, beta, coords=None):
    x = box.coords if coords is None else coords
    return oracle.energy_forces(x, box.q, box.type, box.ljparams, box.box, rc, beta, box.excl_off,
                                box.excl_idx)


def tiled_along_z(b, reps):
    """The cubic box b repeated reps times along z: an orthorhombic L x L x reps L box of whole
    molecules (each water made whole by the minimum image before it is copied and rewrapped)."""
    L = b.box.astype(np.float64)
    x = b.coords.astype(np.float64).reshape(-1, 3, 3)  # [molecule, atom (O, H, H), xyz]
    d = x[:, 1:, :] - x[:, :1, :]
    x[:, 1:, :] = x[:, :1, :] + d - L * np.rint(d / L)
    box = np.array([L[0], L[1], reps * L[2]])
    y = np.concatenate([x + np.array([0.0, 0.0, k * L[2]]) for k in range(reps)]).reshape(-1, 3)
    y -= box * np.floor(y / box)

    class Tiled:
        pass

    t = Tiled()
    n = b.n_atoms
    t.coords = y.astype(np.float32)
    t.box = box.astype(np.float32)
    t.n_atoms = reps * n
    t.q = np.tile(b.q, reps)
    t.type = np.tile(b.type, reps)
    t.ljparams = b.ljparams
    t.excl_off = np.concatenate([[0]] + [b.excl_off[1:] + k * b.excl_off[-1] for k in range(reps)]).astype(np.int32)
    t.excl_idx = np.concatenate([b.excl_idx + k * n for k in range(reps)]).astype(np.int32)
    return t
