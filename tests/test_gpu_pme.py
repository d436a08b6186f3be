"""Parity of the PME spread and gather kernels (through the C ABI) with the FP64 oracle.

Tolerances come from the FP32 arithmetic of the kernels:

* the fractional part w of each scaled coordinate is exact to about 2^-23
  (it is formed as a two-float product), and |dM/du| <= 1/2, |d2M/du2| <= 1
  for the cubic B-spline, so a weight product M M M moves by at most
  3 * 0.5 * (2/3)^2 * 2^-23 < 1e-7 and a derivative product M' M M by at
  most 0.8 * 2^-23 < 1e-7;
* the weights take about 10 rounded operations (relative 10 * 2^-24 each
  factor, 2e-6 for a product of three and the charge);
* every FP32 addition into a mesh point rounds by 2^-24 of the running sum,
  so m additions cost at most m * 2^-24 * sum |terms|.

Per mesh point:  |dQ_k| <= 2e-7 T_k + (2e-6 + m_k 6e-8) A_k + 1e-9 max|q|
                 (T_k = sum of |q_i| over the atoms whose support holds k,
                  m_k = their number, A_k = sum |q_i M M M|)
Per force component: |dF_ia| <= 2e-7 |q_i| (K_a/L_a) P_i + 6e-6 S_ia
                 (P_i = sum of |phi| over the atom's 64 support points,
                  S_ia = sum of |terms| of F_ia from the oracle)
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    from paper_2405_01420_gb300 import nb as nbmod
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    nbmod.load_library()
    return nbmod


def support(x, box, K):
    """Flat mesh indices [N, 64] of each atom's order-4 support (FP64 floor)."""
    x = np.asarray(x, np.float64)
    box = np.asarray(box, np.float64)
    s = x / box
    u = (s - np.floor(s)) * np.asarray(K)
    base = np.floor(u).astype(np.int64)
    j = np.arange(4)
    i0 = (base[:, 0, None] - j) % K[0]
    i1 = (base[:, 1, None] - j) % K[1]
    i2 = (base[:, 2, None] - j) % K[2]
    flat = (i0[:, :, None, None] * K[1] + i1[:, None, :, None]) * K[2] + i2[:, None, None, :]
    return flat.reshape(len(x), 64)


def spread_tol(x, q, box, K, Qabs):
    sup = support(x, box, K)
    n = np.prod(K)
    T = np.bincount(sup.ravel(), weights=np.repeat(np.abs(q).astype(np.float64), 64), minlength=n)
    m = np.bincount(sup.ravel(), minlength=n)
    return (2e-7 * T + (2e-6 + 6e-8 * m) * Qabs.ravel() + 1e-9 * np.abs(q).max()).reshape(K)


def gather_tol(x, q, box, K, phi, Fabs):
    sup = support(x, box, K)
    P = np.abs(phi.ravel()[sup]).sum(1)
    s = np.asarray(K, np.float64) / np.asarray(box, np.float64)
    return 2e-7 * np.abs(q)[:, None] * s[None, :] * P[:, None] + 6e-6 * Fabs


def run_spread(nb, x, q, box, K):
    grid = torch.full(tuple(K), float("nan"), dtype=torch.float32, device="cuda")
    nb.nb_pme_spread(torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda(),
                     torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda(), box, K, grid)
    torch.cuda.synchronize()
    return grid.cpu().numpy().astype(np.float64)


def run_gather(nb, x, q, box, K, phi, accumulate=False, forces=None):
    n = len(q)
    F = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda") if forces is None else forces
    E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    nb.nb_pme_gather(torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda(),
                     torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda(), box, K,
                     torch.from_numpy(np.ascontiguousarray(phi, np.float32)).cuda(), F, accumulate=accumulate,
                     energy=E)
    torch.cuda.synchronize()
    return F.cpu().numpy().astype(np.float64), float(E.item())


def check_spread(nb, x, q, box, K):
    x32 = np.asarray(x, np.float32)
    q32 = np.asarray(q, np.float32)
    Q = run_spread(nb, x32, q32, box, K)
    Qo, Qa = oracle.pme_spread(x32, q32, np.asarray(box, np.float32), K, 4, abs_sums=True)
    tol = spread_tol(x32, q32, np.asarray(box, np.float32), K, Qa)
    bad = np.abs(Q - Qo) > tol
    assert not bad.any(), f"{bad.sum()} mesh points off; worst excess {np.max(np.abs(Q - Qo) - tol):.3e}"
    return Q, Qo


def check_gather(nb, x, q, box, K, phi):
    x32 = np.asarray(x, np.float32)
    q32 = np.asarray(q, np.float32)
    phi32 = np.asarray(phi, np.float32)
    F, E = run_gather(nb, x32, q32, box, K, phi32)
    Fo, psi, Fa = oracle.pme_gather(x32, q32, np.asarray(box, np.float32), K, phi32, 4, abs_sums=True)
    tol = gather_tol(x32, q32, np.asarray(box, np.float32), K, phi32, Fa)
    bad = np.abs(F - Fo) > tol
    assert not bad.any(), f"{bad.sum()} force components off; worst excess {np.max(np.abs(F - Fo) - tol):.3e}"
    Eo = 0.5 * (q32.astype(np.float64) * psi).sum()
    P = np.abs(phi32.ravel()[support(x32, np.asarray(box, np.float32), K)]).sum(1)
    assert abs(E - Eo) <= 1e-6 * 0.5 * (np.abs(q32) * P).sum(), (E, Eo)
    return F, E


def water(nw, seed):
    b = synth.water_box(nw, seed)
    return b.coords, b.q, b.box


def fft_size(n):
    """Smallest size >= n with no prime factor above 7 (what an FFT library handles fast)."""
    while True:
        m = n
        for p in (2, 3, 5, 7):
            while m % p == 0:
                m //= p
        if m == 1:
            return n
        n += 1


def mesh_for(box, spacing=0.12):
    """Mesh with at most ``spacing`` nm between points, FFT-friendly sizes."""
    return tuple(fft_size(int(np.ceil(float(L) / spacing))) for L in box)


# ------------------------------------------------------------------ spread

def test_spread_small_water_box(nb):
    x, q, box = water(512, 1)
    check_spread(nb, x, q, box, mesh_for(box))


def test_spread_orthorhombic_mesh_and_unwrapped_coordinates(nb):
    rng = np.random.default_rng(3)
    box = np.array([2.1, 2.6, 3.3], np.float32)
    K = (20, 24, 28)
    x = (rng.uniform(0, 1, (3000, 3)) * box + rng.integers(-2, 3, (3000, 3)) * box).astype(np.float32)
    q = rng.normal(0, 0.5, 3000).astype(np.float32)
    check_spread(nb, x, q, box, K)


def test_spread_edges(nb):
    box = np.array([2.0, 2.0, 2.0], np.float32)
    K = (16, 16, 16)
    # atoms exactly at 0, at L (wraps to 0), on mesh planes and just below them
    x = np.array([[0, 0, 0], [2.0, 2.0, 2.0], [0.125, 0.25, 0.375], [np.nextafter(np.float32(0.125), 0), 1.0, 1.5],
                  [1.999999, 0.5, 1.0]], np.float32)
    q = np.array([1.0, -0.5, 0.25, 2.0, -1.0], np.float32)
    check_spread(nb, x, q, box, K)
    # the smallest mesh the order allows: every atom reaches every point of each axis
    check_spread(nb, x, q, box, (4, 4, 4))
    # one atom; no atoms (the mesh is cleared)
    check_spread(nb, x[:1], q[:1], box, K)
    Q = run_spread(nb, np.zeros((0, 3), np.float32), np.zeros(0, np.float32), box, K)
    assert not Q.any()


def test_spread_production_box_96k(nb):
    """96,000 atoms on an 84^3 mesh (0.117 nm spacing), as the benchmark launches it."""
    x, q, box = water(32000, 2)
    K = mesh_for(box)
    assert K == (84, 84, 84)
    Q, Qo = check_spread(nb, x, q, box, K)
    assert abs(Q.sum() - float(np.asarray(q, np.float64).sum())) <= 1e-3


# ------------------------------------------------------------------ gather

def test_gather_small_water_box(nb):
    x, q, box = water(512, 1)
    K = mesh_for(box)
    phi = np.random.default_rng(4).normal(size=K)
    check_gather(nb, x, q, box, K, phi)


def test_gather_orthorhombic_unwrapped_and_edges(nb):
    rng = np.random.default_rng(5)
    box = np.array([2.1, 2.6, 3.3], np.float32)
    K = (20, 24, 28)
    x = (rng.uniform(0, 1, (2999, 3)) * box + rng.integers(-2, 3, (2999, 3)) * box).astype(np.float32)
    x[0] = 0.0
    x[1] = box
    q = rng.normal(0, 0.5, 2999).astype(np.float32)
    phi = rng.normal(size=K)
    check_gather(nb, x, q, box, K, phi)
    check_gather(nb, x[:7], q[:7], box, (4, 4, 4), rng.normal(size=(4, 4, 4)))


def test_gather_accumulates_and_handles_no_atoms(nb):
    x, q, box = water(100, 6)
    K = mesh_for(box)
    phi = np.random.default_rng(6).normal(size=K).astype(np.float32)
    F1, _ = run_gather(nb, x, q, box, K, phi)
    base = torch.from_numpy(np.random.default_rng(7).normal(size=(len(q), 3)).astype(np.float32)).cuda()
    F2, _ = run_gather(nb, x, q, box, K, phi, accumulate=True, forces=base.clone())
    np.testing.assert_allclose(F2, base.cpu().numpy().astype(np.float64) + F1, rtol=0, atol=1e-6 * np.abs(F1).max())
    F0, E0 = run_gather(nb, np.zeros((0, 3), np.float32), np.zeros(0, np.float32), box, K, phi)
    assert F0.shape == (0, 3) and E0 == 0.0


def test_smooth_pme_chain_96k(nb):
    """96,000 atoms: the GPU spread, a mesh potential solved from it (numpy FFT
    with the smooth-PME influence function, beta for rc = 1.0 nm), the GPU
    gather; each kernel against the oracle, and the energy from the gather
    equal to (1/2) sum Q phi over the GPU's own mesh."""
    x, q, box = water(32000, 2)
    K = mesh_for(box)
    Q, _ = check_spread(nb, x, q, box, K)
    phi = solve(Q, box, K, synth.ewald_beta(1.0))
    F, E = check_gather(nb, x, q, box, K, phi)
    assert E == pytest.approx(0.5 * (Q * phi.astype(np.float32).astype(np.float64)).sum(), rel=1e-5)


def _bspline_moduli(K):
    """|b(m)|^2 of order-4 smooth PME: 1 / |sum_k M4(k + 1) exp(2 pi i m k / K)|^2."""
    m = np.arange(K)
    den = (1 / 6) + (2 / 3) * np.exp(2j * np.pi * m / K) + (1 / 6) * np.exp(4j * np.pi * m / K)
    return 1.0 / np.abs(den) ** 2


def solve(Q, box, K, beta):
    """Mesh potential phi = theta_rec * Q of smooth PME (Essmann et al. 1995)."""
    box = np.asarray(box, np.float64)
    V = float(np.prod(box))
    mh = [np.where(np.arange(K[a]) <= K[a] // 2, np.arange(K[a]), np.arange(K[a]) - K[a]) / box[a] for a in range(3)]
    m2 = mh[0][:, None, None] ** 2 + mh[1][None, :, None] ** 2 + mh[2][None, None, :] ** 2
    B = _bspline_moduli(K[0])[:, None, None] * _bspline_moduli(K[1])[None, :, None] * _bspline_moduli(K[2])[None, None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        C = 138.935458 * np.exp(-np.pi ** 2 * m2 / beta ** 2) / (np.pi * V * m2)
    C[0, 0, 0] = 0.0
    return np.fft.fftn(C * B * np.fft.ifftn(Q) * Q.size).real


def test_pme_argument_errors(nb):
    x, q, box = water(100, 6)
    grid = torch.empty((16, 16, 16), dtype=torch.float32, device="cuda")
    xd = torch.from_numpy(x).cuda()
    qd = torch.from_numpy(q).cuda()
    with pytest.raises(nb.NBError):
        nb.nb_pme_spread(xd, qd, box, (16, 16, 16), grid, order=5)
    with pytest.raises(nb.NBError):
        nb.nb_pme_spread(xd, qd, box, (3, 16, 16), torch.empty(3 * 16 * 16, device="cuda"))
    with pytest.raises(ValueError):
        nb.nb_pme_spread(xd, qd, box, (16, 16, 17), grid)  # grid of the wrong size


def test_pme_million_atoms(nb):
    """1,000,002 atoms on a 180^3 mesh: the spread conserves the charge and is the
    gather's adjoint (sum Q phi = 2 E over the GPU's own outputs), and the gathered
    forces of 3,000 sampled atoms match the oracle (the gather is per atom, so the
    oracle needs only those atoms)."""
    b = synth.water_box(333334, 3)
    K = mesh_for(b.box)
    assert K == (180, 180, 180)
    x = torch.from_numpy(b.coords).cuda()
    q = torch.from_numpy(b.q).cuda()
    grid = torch.empty(K, dtype=torch.float32, device="cuda")
    nb.nb_pme_spread(x, q, b.box, K, grid)
    Q = grid.double()
    qsum = float(np.abs(b.q.astype(np.float64)).sum())
    assert abs(float(Q.sum()) - float(b.q.astype(np.float64).sum())) <= 1e-6 * qsum
    phi = torch.randn(K, generator=torch.Generator(device="cuda").manual_seed(3), device="cuda")
    F = torch.empty((b.n_atoms, 3), dtype=torch.float32, device="cuda")
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    nb.nb_pme_gather(x, q, b.box, K, phi, F, energy=E)
    torch.cuda.synchronize()
    qphi = float((Q * phi.double()).sum())
    # both sides sum 64 M terms of size ~|q| |phi|; FP32 weights and atomics: 1e-5 of sum |q| |phi|
    scale = float((torch.from_numpy(np.abs(b.q)).cuda().double().sum()) * phi.abs().max().double())
    assert abs(2.0 * float(E.item()) - qphi) <= 1e-5 * scale
    rng = np.random.default_rng(6)
    atoms = np.sort(rng.choice(b.n_atoms, 3000, replace=False))
    phi_h = phi.cpu().numpy().astype(np.float32)
    Fo, _, Fa = oracle.pme_gather(b.coords[atoms], b.q[atoms], b.box, K, phi_h, 4, abs_sums=True)
    tol = gather_tol(b.coords[atoms], b.q[atoms], b.box, K, phi_h, Fa)
    Fg = F.cpu().numpy()[atoms].astype(np.float64)
    assert (np.abs(Fg - Fo) <= tol).all(), np.max(np.abs(Fg - Fo) - tol)
