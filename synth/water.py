"""Synthetic water boxes for the short-range nonbonded path.

The benchmark systems of the paper (Grappa, STMV, ADH, RNAse; §II
"Benchmark systems") are not available, and the paper describes Grappa as a
uniform-density water/ethanol mix. Uniform rigid 3-site water boxes stand in
for them. Recipe:

* ``n_w`` waters in a cubic box of edge ``L = (n_w / 33.4)^(1/3)`` nm
  (33.4 molecules per nm^3, i.e. about 100 atoms per nm^3).
* Oxygen sites on an ``n^3`` lattice, ``n = ceil(n_w^(1/3))``, spacing
  ``a = L / n``. When ``n^3 > n_w`` a seeded random subset of sites is
  occupied (sites kept in lattice order).
* Each oxygen is jittered uniformly by up to ``0.05 a`` per axis; each
  molecule gets a uniformly random orientation (Shoemake quaternion).
* A molecule whose atoms come closer than 0.15 nm to an atom of another
  molecule gets a fresh orientation, up to 100 rounds; generation fails
  otherwise.
* Geometry: O-H 0.1 nm, H-O-H 109.47 deg. Charges O -0.8476 e, H +0.4238 e.
  LJ on O only, sigma 0.3166 nm, epsilon 0.650 kJ/mol, stored as
  C6 = 4 eps sigma^6 and C12 = 4 eps sigma^12. Type 0 = O, type 1 = H.
* Exclusions: the three intra-molecular pairs, stored as a symmetric CSR
  (each atom lists the other two atoms of its molecule).
* Coordinates are FP32 and lie in ``[0, L)``.

Everything is drawn from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DENSITY_WATERS_PER_NM3 = 33.4
WATER_Q_O = -0.8476
WATER_Q_H = 0.4238
_SIGMA_O = 0.3166
_EPS_O = 0.650
WATER_C6 = 4.0 * _EPS_O * _SIGMA_O ** 6
WATER_C12 = 4.0 * _EPS_O * _SIGMA_O ** 12
_R_OH = 0.1
_THETA_HOH = math.radians(109.47)
_MIN_CONTACT = 0.15


@dataclass
class WaterBox:
    """One synthetic system. Arrays are host numpy arrays in original atom order."""

    coords: np.ndarray        # float32 [N, 3], each component in [0, L)
    q: np.ndarray             # float32 [N]
    type: np.ndarray          # int32 [N]
    box: np.ndarray           # float32 [3]
    ljparams: np.ndarray      # float32 [ntype, ntype, 2] = (C6, C12), symmetric
    excl_off: np.ndarray      # int32 [N + 1]
    excl_idx: np.ndarray      # int32 [excl_off[N]]
    n_waters: int
    seed: int
    extra: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.coords.shape[0])

    @property
    def ntype(self) -> int:
        return int(self.ljparams.shape[0])


def box_edge(n_waters: int, density: float = DENSITY_WATERS_PER_NM3) -> float:
    """Cubic box edge (nm) holding ``n_waters`` at ``density`` molecules/nm^3."""
    return (n_waters / density) ** (1.0 / 3.0)


def ewald_beta(rc: float, tol: float = 1e-5) -> float:
    """Ewald splitting parameter with erfc(beta * rc) = tol, by FP64 bisection."""
    lo, hi = 0.0, 10.0
    while math.erfc(hi * rc) > tol:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if math.erfc(mid * rc) > tol:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _random_rotations(rng: np.random.Generator, m: int) -> np.ndarray:
    """m uniformly random rotation matrices [m, 3, 3] (Shoemake 1992)."""
    u1, u2, u3 = rng.random(m), rng.random(m), rng.random(m)
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    w = b * np.cos(2 * np.pi * u3)
    x = a * np.sin(2 * np.pi * u2)
    y = a * np.cos(2 * np.pi * u2)
    z = b * np.sin(2 * np.pi * u3)
    r = np.empty((m, 3, 3))
    r[:, 0, 0] = 1 - 2 * (y * y + z * z)
    r[:, 0, 1] = 2 * (x * y - z * w)
    r[:, 0, 2] = 2 * (x * z + y * w)
    r[:, 1, 0] = 2 * (x * y + z * w)
    r[:, 1, 1] = 1 - 2 * (x * x + z * z)
    r[:, 1, 2] = 2 * (y * z - x * w)
    r[:, 2, 0] = 2 * (x * z - y * w)
    r[:, 2, 1] = 2 * (y * z + x * w)
    r[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return r


def _body_frame() -> np.ndarray:
    """Rigid water in its body frame [3 atoms, 3]: O at the origin."""
    s, c = math.sin(_THETA_HOH / 2), math.cos(_THETA_HOH / 2)
    return np.array([[0.0, 0.0, 0.0], [_R_OH * s, 0.0, _R_OH * c], [-_R_OH * s, 0.0, _R_OH * c]])


def _wrap_f32(x64: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Wrap FP64 positions into [0, L) and round to FP32, keeping x < L after rounding."""
    w = x64 - L * np.floor(x64 / L)
    xf = w.astype(np.float32)
    Lf = L.astype(np.float32)
    xf = np.where(xf >= Lf, np.float32(0.0), xf)
    xf = np.where(xf < 0, np.float32(0.0), xf)
    return xf.astype(np.float32)


def _close_contacts(pos: np.ndarray, site_of_mol: np.ndarray, grid: np.ndarray, n: int,
                    L: float, moved: np.ndarray | None = None) -> np.ndarray:
    """Flag molecules with an atom closer than 0.15 nm to an atom of another molecule.

    Only molecules on neighbouring lattice sites can come that close (two sites
    apart the gap is at least 1.8 a - 0.2 nm > 0.15 nm), so each molecule is
    compared with the molecules on the 26 sites around it. With ``moved`` given,
    only neighbour pairs that include a moved molecule are checked.
    """
    m = pos.shape[0]
    bad = np.zeros(m, dtype=bool)
    sx, sy, sz = site_of_mol[:, 0], site_of_mol[:, 1], site_of_mol[:, 2]
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                if (dx, dy, dz) <= (0, 0, 0):
                    continue  # each unordered neighbour pair once
                other = grid[(sx + dx) % n, (sy + dy) % n, (sz + dz) % n]
                ok = (other >= 0) & (other != np.arange(m))
                if moved is not None:
                    ok &= moved | moved[np.maximum(other, 0)]
                if not ok.any():
                    continue
                a = np.nonzero(ok)[0]
                b = other[a]
                d = pos[a][:, :, None, :] - pos[b][:, None, :, :]
                d -= L * np.rint(d / L)
                close = (np.einsum("kijx,kijx->kij", d, d) < _MIN_CONTACT ** 2).any(axis=(1, 2))
                bad[a[close]] = True
                bad[b[close]] = True
    return bad


def water_box(n_waters: int, seed: int, density: float = DENSITY_WATERS_PER_NM3,
              jitter: float = 0.05, max_tries: int = 100) -> WaterBox:
    """Seeded box of ``n_waters`` rigid 3-site waters (see the module docstring)."""
    if n_waters < 1:
        raise ValueError("n_waters must be >= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    L = box_edge(n_waters, density)
    n = int(math.ceil(n_waters ** (1.0 / 3.0) - 1e-12))
    while n ** 3 < n_waters:
        n += 1
    a = L / n
    n_sites = n ** 3
    if n_sites > n_waters:
        sites = np.sort(rng.permutation(n_sites)[:n_waters])
    else:
        sites = np.arange(n_sites)
    site_xyz = np.stack([sites // (n * n), (sites // n) % n, sites % n], axis=1)
    grid = -np.ones((n, n, n), dtype=np.int64)
    grid[site_xyz[:, 0], site_xyz[:, 1], site_xyz[:, 2]] = np.arange(n_waters)
    oxy = (site_xyz + 0.5) * a + rng.uniform(-jitter * a, jitter * a, size=(n_waters, 3))
    body = _body_frame()
    rot = _random_rotations(rng, n_waters)
    pos = oxy[:, None, :] + np.einsum("mij,aj->mai", rot, body)
    moved = None
    for _ in range(max_tries):
        bad = _close_contacts(pos, site_xyz, grid, n, L, moved)
        if not bad.any():
            break
        moved = bad
        k = np.nonzero(bad)[0]
        rot_k = _random_rotations(rng, k.size)
        pos[k] = oxy[k][:, None, :] + np.einsum("mij,aj->mai", rot_k, body)
    else:
        raise RuntimeError("water_box: could not remove close contacts")

    Lv = np.array([L, L, L])
    coords = _wrap_f32(pos.reshape(-1, 3), Lv)
    N = 3 * n_waters
    q = np.tile(np.array([WATER_Q_O, WATER_Q_H, WATER_Q_H], dtype=np.float32), n_waters)
    typ = np.tile(np.array([0, 1, 1], dtype=np.int32), n_waters)
    lj = np.zeros((2, 2, 2), dtype=np.float32)
    lj[0, 0] = (WATER_C6, WATER_C12)
    excl_off = (2 * np.arange(N + 1)).astype(np.int32)
    base = 3 * (np.arange(N) // 3)
    k = np.arange(N) % 3
    partners = np.stack([base + (k + 1) % 3, base + (k + 2) % 3], axis=1)
    partners.sort(axis=1)
    return WaterBox(coords=coords, q=q, type=typ, box=Lv.astype(np.float32), ljparams=lj,
                    excl_off=excl_off, excl_idx=partners.reshape(-1).astype(np.int32),
                    n_waters=n_waters, seed=seed)


def water_box_for_atoms(n_atoms: int, seed: int, **kw) -> WaterBox:
    """Water box with ``n_atoms`` rounded down to whole waters (at least one)."""
    return water_box(max(1, n_atoms // 3), seed, **kw)


def random_walk_frames(box: WaterBox, n_frames: int, sigma: float, seed: int) -> np.ndarray:
    """Frames of a cumulative Gaussian random walk, wrapped to [0, L) in FP32.

    Frame k (k = 1..n_frames) is frame k-1 plus N(0, sigma^2) per component,
    accumulated in FP64 from the FP32 starting coordinates. Returns float32
    [n_frames, N, 3].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x = box.coords.astype(np.float64)
    L = box.box.astype(np.float64)
    out = np.empty((n_frames,) + box.coords.shape, dtype=np.float32)
    for f in range(n_frames):
        x = x + rng.normal(0.0, sigma, size=x.shape)
        out[f] = _wrap_f32(x, L)
    return out


def combine_geometric(c6_t: np.ndarray, c12_t: np.ndarray) -> np.ndarray:
    """Per-type (c6, c12) -> pair matrix [ntype, ntype, 2] with C_ij = sqrt(c_i c_j)."""
    c6 = np.sqrt(np.outer(c6_t, c6_t))
    c12 = np.sqrt(np.outer(c12_t, c12_t))
    return np.stack([c6, c12], axis=-1)


def diff_params(box: WaterBox, seed: int, ntype: int = 4, q_sigma: float = 0.4,
                perturb: float = 0.05) -> dict:
    """Parameters for the force-matching workload.

    Charges are redrawn per atom as N(0, q_sigma^2) and net-neutralised by
    subtracting their mean; each atom gets a type uniform in {0..ntype-1};
    each type gets c6 ~ U[1e-3, 3e-3] and c12 ~ U[1e-6, 3e-6]. The target
    parameters are p' = p (1 + perturb * xi), xi ~ N(0, 1), per atom for q
    (then re-neutralised) and per type for c6 and c12. All arrays FP64.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    N = box.n_atoms
    q = rng.normal(0.0, q_sigma, size=N)
    q -= q.mean()
    typ = rng.integers(0, ntype, size=N).astype(np.int32)
    c6 = rng.uniform(1e-3, 3e-3, size=ntype)
    c12 = rng.uniform(1e-6, 3e-6, size=ntype)
    q_t = q * (1.0 + perturb * rng.normal(size=N))
    q_t -= q_t.mean()
    c6_t = c6 * (1.0 + perturb * rng.normal(size=ntype))
    c12_t = c12 * (1.0 + perturb * rng.normal(size=ntype))
    return {"q": q, "type": typ, "c6": c6, "c12": c12,
            "q_target": q_t, "c6_target": c6_t, "c12_target": c12_t}


def batch_boxes(n_boxes: int = 256, lo: int = 1536, hi: int = 24000, seed: int = 5):
    """Independent water boxes with atom counts uniform in [lo, hi], whole waters.

    Box b uses generator seed ``seed + b``; its size is drawn from a generator
    seeded with ``seed``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = rng.integers(lo, hi + 1, size=n_boxes)
    return [water_box(max(1, int(s) // 3), seed + b) for b, s in enumerate(sizes)]
