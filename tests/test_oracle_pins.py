"""Pins for the CPU oracle: closed forms, tabulated values, invariants, brute force.

None of these re-types the oracle's own pair formula. Each checks the oracle
against a fact the mathematics or a textbook fixes (Coulomb's law, the LJ
well depth and zero crossing, tabulated erfc, Newton's third law,
translation / permutation invariance, scaling laws, F = -dE/dx), or against
an independent brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

F_COUL = 138.935458
SIGMA, EPS = 0.3166, 0.650
C6_O, C12_O = 4 * EPS * SIGMA ** 6, 4 * EPS * SIGMA ** 12


def two_atoms(r, q1=0.0, q2=0.0, lj=True, L=10.0, direction=(1.0, 2.0, -0.5)):
    u = np.asarray(direction, dtype=np.float64)
    u /= np.linalg.norm(u)
    c = np.array([L / 2, L / 2, L / 2])
    x = np.stack([c + 0.5 * r * u, c - 0.5 * r * u])
    q = np.array([q1, q2])
    typ = np.zeros(2, dtype=np.int32)
    ljp = np.zeros((1, 1, 2))
    if lj:
        ljp[0, 0] = (C6_O, C12_O)
    return x, q, typ, ljp, np.array([L, L, L]), u


def lj_textbook(r):
    """Lennard-Jones in sigma-epsilon form: 4 eps [(s/r)^12 - (s/r)^6]."""
    return 4 * EPS * ((SIGMA / r) ** 12 - (SIGMA / r) ** 6)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("r", [0.15, 0.31, 0.5, 0.89])
@pytest.mark.parametrize("q1,q2", [(1.0, 1.0), (-0.8476, 0.4238), (0.5, -2.0)])
def test_coulomb_law_at_beta_zero(r, q1, q2):
    """beta = 0 turns erfc(beta r) into 1: plain Coulomb's law."""
    x, q, t, lj, box, u = two_atoms(r, q1, q2, lj=False)
    F, elj, ec, npairs = oracle.energy_forces(x, q, t, lj, box, 0.9, 0.0, method="n2")
    assert npairs == 1
    assert elj == 0.0
    assert ec == pytest.approx(F_COUL * q1 * q2 / r, rel=1e-14)
    # like charges repel: the force on atom 0 points away from atom 1 (along +u)
    mag = F_COUL * q1 * q2 / r ** 2
    np.testing.assert_allclose(F[0], mag * u, rtol=1e-13, atol=1e-12 * abs(mag))
    np.testing.assert_allclose(F[1], -mag * u, rtol=1e-13, atol=1e-12 * abs(mag))


def test_erfc_against_table(golden_dir):
    """E_C for two unit charges with beta r = x equals f erfc(x) / r (A&S Table 7.1)."""
    rows = np.loadtxt(os.path.join(golden_dir, "erfc_table.txt"))
    r = 0.4
    for xval, erfc_tab in rows:
        beta = xval / r
        x, q, t, lj, box, _ = two_atoms(r, 1.0, 1.0, lj=False)
        _, _, ec, _ = oracle.energy_forces(x, q, t, lj, box, 0.9, beta, method="n2")
        assert ec == pytest.approx(F_COUL * erfc_tab / r, rel=2e-14), xval


def test_lj_well_depth_and_zero_crossing():
    """LJ: force zero and depth -eps at r = 2^(1/6) sigma; zero crossing at sigma."""
    rc = 0.9
    shift = lj_textbook(rc)  # potential-shifted: E(r) = V(r) - V(rc)
    rmin = 2 ** (1 / 6) * SIGMA
    x, q, t, lj, box, _ = two_atoms(rmin)
    F, elj, ec, _ = oracle.energy_forces(x, q, t, lj, box, rc, 3.0, method="n2")
    assert ec == 0.0
    assert elj == pytest.approx(-EPS - shift, rel=1e-12)
    assert np.abs(F).max() < 1e-10
    x, q, t, lj, box, _ = two_atoms(SIGMA)
    F, elj, _, _ = oracle.energy_forces(x, q, t, lj, box, rc, 3.0, method="n2")
    assert elj == pytest.approx(-shift, rel=1e-12)
    # repulsive inside sigma: the force on atom 0 points away from atom 1
    x, q, t, lj, box, u = two_atoms(0.3)
    F, _, _, _ = oracle.energy_forces(x, q, t, lj, box, rc, 3.0, method="n2")
    assert np.dot(F[0], u) > 0


def test_cutoff_continuity_and_strictness():
    """Potential-shifted LJ vanishes at rc; the Coulomb term there is f q q 1e-5 / rc."""
    rc = 0.9
    beta = synth.ewald_beta(rc)
    x, q, t, lj, box, _ = two_atoms(rc * (1 - 1e-12), 1.0, -1.0)
    _, elj, ec, n = oracle.energy_forces(x, q, t, lj, box, rc, beta, method="n2")
    assert n == 1
    assert abs(elj) < 1e-12
    assert ec == pytest.approx(-F_COUL * 1e-5 / rc, rel=1e-9)
    x, q, t, lj, box, _ = two_atoms(rc * (1 + 1e-12), 1.0, -1.0)
    _, elj, ec, n = oracle.energy_forces(x, q, t, lj, box, rc, beta, method="n2")
    assert n == 0 and elj == 0.0 and ec == 0.0


# ------------------------------------------------------------------- invariants

@pytest.fixture(scope="module")
def box512():
    return synth.water_box(512, 1)


def run(b, x=None, rc=0.9, beta=None, method="auto", q=None, lj=None):
    beta = synth.ewald_beta(rc) if beta is None else beta
    return oracle.energy_forces(b.coords if x is None else x, b.q if q is None else q, b.type,
                                b.ljparams if lj is None else lj, b.box, rc, beta,
                                b.excl_off, b.excl_idx, method)


def test_newton_third_law(box512):
    F, elj, ec, _ = run(box512)
    rms = np.sqrt((F ** 2).sum(1).mean())
    assert np.abs(F.sum(0)).max() <= 1e-10 * len(F) * rms


def test_translation_invariance(box512):
    F, elj, ec, n = run(box512)
    rng = np.random.default_rng(7)
    t = rng.uniform(-3, 3, size=3)
    L = box512.box.astype(np.float64)
    x2 = box512.coords.astype(np.float64) + t
    x2 -= L * np.floor(x2 / L)
    F2, elj2, ec2, n2 = run(box512, x=x2)
    assert n2 == n
    assert elj2 == pytest.approx(elj, rel=1e-12)
    assert ec2 == pytest.approx(ec, rel=1e-11)
    np.testing.assert_allclose(F2, F, atol=1e-9 * np.abs(F).max())


def test_permutation_invariance(box512):
    b = box512
    F, elj, ec, n = run(b)
    rng = np.random.default_rng(3)
    p = rng.permutation(b.n_atoms)  # new atom k is old atom p[k]
    inv = np.empty_like(p)
    inv[p] = np.arange(len(p))
    offs = [0]
    idx = []
    for k in range(len(p)):
        old = p[k]
        partners = b.excl_idx[b.excl_off[old]:b.excl_off[old + 1]]
        idx.extend(inv[partners])
        offs.append(len(idx))
    F2, elj2, ec2, n2 = oracle.energy_forces(b.coords[p], b.q[p], b.type[p], b.ljparams, b.box, 0.9,
                                             synth.ewald_beta(0.9), np.array(offs), np.array(idx), "n2")
    assert n2 == n
    assert elj2 == pytest.approx(elj, rel=1e-12)
    assert ec2 == pytest.approx(ec, rel=1e-11)
    np.testing.assert_allclose(F2, F[p], atol=1e-9 * np.abs(F).max())


def test_scaling_laws(box512):
    """x, L, rc -> lam x, lam L, lam rc; beta -> beta/lam; C6 -> lam^6 C6; C12 -> lam^12 C12.

    Then E_LJ is unchanged, E_C scales by 1/lam, and the LJ and Coulomb forces
    by 1/lam (LJ) and 1/lam^2 (Coulomb). Catches a wrong power anywhere.
    """
    b = box512
    lam = 1.7
    beta = synth.ewald_beta(0.9)
    q0 = np.zeros(b.n_atoms)
    F_lj, elj, _, _ = oracle.energy_forces(b.coords, q0, b.type, b.ljparams, b.box, 0.9, beta,
                                           b.excl_off, b.excl_idx, "n2")
    F_c, _, ec, _ = oracle.energy_forces(b.coords, b.q, b.type, 0 * b.ljparams, b.box, 0.9, beta,
                                         b.excl_off, b.excl_idx, "n2")
    lj2 = b.ljparams.astype(np.float64).copy()
    lj2[..., 0] *= lam ** 6
    lj2[..., 1] *= lam ** 12
    x2 = b.coords.astype(np.float64) * lam
    box2 = b.box.astype(np.float64) * lam
    F_lj2, elj2, _, _ = oracle.energy_forces(x2, q0, b.type, lj2, box2, 0.9 * lam, beta / lam,
                                             b.excl_off, b.excl_idx, "n2")
    F_c2, _, ec2, _ = oracle.energy_forces(x2, b.q, b.type, 0 * lj2, box2, 0.9 * lam, beta / lam,
                                           b.excl_off, b.excl_idx, "n2")
    assert elj2 == pytest.approx(elj, rel=1e-11)
    assert ec2 == pytest.approx(ec / lam, rel=1e-10)
    np.testing.assert_allclose(F_lj2, F_lj / lam, atol=1e-9 * np.abs(F_lj).max())
    np.testing.assert_allclose(F_c2, F_c / lam ** 2, atol=1e-9 * np.abs(F_c).max())


def test_charge_scaling(box512):
    """E_C is quadratic in the charges: q -> 2q multiplies E_C and F_C by 4."""
    b = box512
    F, _, ec, _ = run(b, lj=0 * b.ljparams)
    F2, _, ec2, _ = run(b, lj=0 * b.ljparams, q=2 * b.q.astype(np.float64))
    assert ec2 == pytest.approx(4 * ec, rel=1e-13)
    np.testing.assert_allclose(F2, 4 * F, rtol=1e-12, atol=1e-10)


def test_force_is_minus_energy_gradient(box512):
    """Central finite differences of E (pair set frozen) equal -F."""
    b = box512
    rc = 0.9
    beta = synth.ewald_beta(rc)
    x = b.coords.astype(np.float64)
    F, _, _, n = run(b, x=x)
    rng = np.random.default_rng(11)
    h = 1e-6
    checked = 0
    for atom in rng.choice(b.n_atoms, 12, replace=False):
        for k in range(3):
            xp = x.copy()
            xm = x.copy()
            xp[atom, k] += h
            xm[atom, k] -= h
            _, elp, ecp, np_ = run(b, x=xp)
            _, elm, ecm, nm = run(b, x=xm)
            if np_ != n or nm != n:
                continue  # a pair crossed rc; the energy is discontinuous there
            fd = -((elp + ecp) - (elm + ecm)) / (2 * h)
            assert fd == pytest.approx(F[atom, k], rel=1e-6, abs=1e-4), (atom, k)
            checked += 1
    assert checked >= 30


def test_n2_equals_cell_list():
    b = synth.water_box(4096, 5)  # L = 4.97 nm: 5 cells of >= 0.9 nm per axis
    F1, elj1, ec1, n1 = run(b, method="n2")
    F2, elj2, ec2, n2 = run(b, method="cell")
    assert n1 == n2
    assert elj2 == pytest.approx(elj1, rel=1e-12)
    assert ec2 == pytest.approx(ec1, rel=1e-12)
    np.testing.assert_allclose(F2, F1, atol=1e-10 * np.abs(F1).max())


def test_forces_subset_matches_full():
    b = synth.water_box(4096, 5)
    beta = synth.ewald_beta(0.9)
    F, _, _, _ = run(b)
    atoms = np.array([0, 1, 2, 100, 5000, b.n_atoms - 1])
    Fs = oracle.forces_subset(b.coords, b.q, b.type, b.ljparams, b.box, 0.9, beta, atoms,
                              b.excl_off, b.excl_idx)
    np.testing.assert_allclose(Fs, F[atoms], atol=1e-10 * np.abs(F).max())


# --------------------------------------------------------------- special cases

def test_single_water_is_fully_excluded():
    b = synth.water_box(1, 1)
    F, elj, ec, n = oracle.energy_forces(b.coords, b.q, b.type, b.ljparams, 10 * b.box, 0.9,
                                         3.0, b.excl_off, b.excl_idx)
    assert n == 0 and elj == 0.0 and ec == 0.0 and np.all(F == 0)


def test_superposition_of_separated_groups():
    """Two groups more than rc apart: E(A u B) = E(A) + E(B)."""
    a = synth.water_box(27, 1)
    L = 8.0
    xa = a.coords.astype(np.float64) + 0.5
    xb = a.coords.astype(np.float64) + 4.5  # gap > 0.9 nm in every direction
    x = np.concatenate([xa, xb])
    q = np.concatenate([a.q, a.q]).astype(np.float64)
    t = np.concatenate([a.type, a.type])
    off = np.concatenate([a.excl_off, a.excl_off[1:] + a.excl_off[-1]])
    idx = np.concatenate([a.excl_idx, a.excl_idx + a.n_atoms])
    box = np.array([L, L, L])
    beta = synth.ewald_beta(0.9)
    _, elj, ec, n = oracle.energy_forces(x, q, t, a.ljparams, box, 0.9, beta, off, idx, "n2")
    _, elj1, ec1, n1 = oracle.energy_forces(xa, a.q, a.type, a.ljparams, box, 0.9, beta,
                                            a.excl_off, a.excl_idx, "n2")
    assert n == 2 * n1
    assert elj == pytest.approx(2 * elj1, rel=1e-13)
    assert ec == pytest.approx(2 * ec1, rel=1e-13)


def test_pairs_f64_against_numpy_brute_force():
    b = synth.water_box(8, 4)
    L = b.box.astype(np.float64)
    x = b.coords.astype(np.float64)
    n = b.n_atoms
    rc = 0.3
    want = set()
    for i in range(n):
        for j in range(i + 1, n):
            if i // 3 == j // 3:
                continue
            d = x[i] - x[j]
            d -= L * np.round(d / L)
            if math.sqrt((d * d).sum()) < rc:
                want.add((i, j))
    got = oracle.pairs_f64(x, b.box, rc, b.excl_off, b.excl_idx)
    assert set(map(tuple, got.tolist())) == want
    assert len(want) > 0


def test_pairs_f32_differs_from_f64_only_at_the_cutoff(box512):
    b = box512
    rc = 0.9
    p32 = set(map(tuple, oracle.pairs_f32(b.coords, b.coords, b.box, rc, b.excl_off, b.excl_idx).tolist()))
    p64 = set(map(tuple, oracle.pairs_f64(b.coords, b.box, rc, b.excl_off, b.excl_idx).tolist()))
    x = b.coords.astype(np.float64)
    L = b.box.astype(np.float64)
    for (i, j) in p32 ^ p64:
        d = x[i] - x[j]
        d -= L * np.round(d / L)
        assert abs(math.sqrt((d * d).sum()) - rc) < 1e-5
    assert len(p32 ^ p64) <= 5


def _walk_across_faces(b, n_frames=12, sigma=0.02, seed=11):
    """A random walk fast enough that a few percent of the atoms cross a box face per frame."""
    return synth.random_walk_frames(b, n_frames, sigma, seed)


def _unwrap_randomly(x, L, seed):
    """Add a random whole number of box edges (-2..2) to every coordinate of x."""
    m = np.random.default_rng(seed).integers(-2, 3, size=x.shape)
    return (x.astype(np.float64) + m * L).astype(np.float32), m


def test_image_f32_is_the_image_nearest_the_search_position(box512):
    """Brute force over whole box shifts: y is the image of x nearest to x0 wrapped into [0, L).

    For each coordinate the periodic images x - k L (k = -6..6) are formed in
    FP64 and the one nearest to the search frame's position, wrapped into
    [0, L) in FP64, is taken; the FP32 image must equal it to a few ulp of the
    largest magnitude involved. Frames of a walk whose atoms cross the faces
    and the same frames shifted by random whole box edges make x - x0 reach
    every case: no shift, a face crossing either way, and unwrapped input.
    """
    b = box512
    L32 = b.box.astype(np.float32)
    L = L32.astype(np.float64)
    frames = _walk_across_faces(b)
    x0 = b.coords
    crossings = 0
    for t, xt in enumerate(frames[[0, 5, 11]]):
        for x0_in, x_in in ((x0, xt), (_unwrap_randomly(x0, L, 100 + t)[0], _unwrap_randomly(xt, L, 200 + t)[0])):
            y = oracle.image_f32(x0_in, x_in, L32).astype(np.float64)
            w0 = x0_in.astype(np.float64)
            w0 = w0 - L * np.floor(w0 / L)
            k = np.arange(-6, 7, dtype=np.float64)
            cand = x_in.astype(np.float64)[..., None] - k * L[None, :, None]
            best = np.take_along_axis(cand, np.abs(cand - w0[..., None]).argmin(-1)[..., None], -1)[..., 0]
            scale = np.maximum(np.abs(x_in.astype(np.float64)), L)
            assert np.all(np.abs(y - best) <= 4 * np.spacing(scale.astype(np.float32)).astype(np.float64))
            assert np.all(np.abs(y - w0) <= 0.5 * L + 1e-5)
        crossings += int((np.abs(xt.astype(np.float64) - x0) > 0.5 * L).sum())
    assert crossings > 20, "the walk should carry atoms across the faces"


def test_pairs_f32_on_a_walk_across_the_faces(box512):
    """Displaced frames: the FP32 set relative to the search frame is the current frame's FP64 set.

    Pairs are within rc at the current frame whatever image the positions
    are given in, so the contract's set, taken against the search frame x0,
    may differ from the FP64 minimum-image set of the current frame only for
    pairs whose FP64 distance is within 1e-5 nm of rc. That holds for wrapped
    frames of a walk whose atoms cross the faces, and for the same frames
    (and search frame) shifted by random whole box edges.
    """
    b = box512
    rc = 0.9
    L = b.box.astype(np.float64)
    frames = _walk_across_faces(b)
    for t in (3, 11):
        xt = frames[t]
        p64 = set(map(tuple, oracle.pairs_f64(xt, b.box, rc, b.excl_off, b.excl_idx).tolist()))
        x64 = xt.astype(np.float64)
        for x0_in, x_in in ((b.coords, xt), (_unwrap_randomly(b.coords, L, 300 + t)[0],
                                             _unwrap_randomly(xt, L, 400 + t)[0])):
            p32 = set(map(tuple, oracle.pairs_f32(x0_in, x_in, b.box, rc, b.excl_off, b.excl_idx).tolist()))
            assert len(p32) > 100000
            for (i, j) in p32 ^ p64:
                d = x64[i] - x64[j]
                d -= L * np.round(d / L)
                assert abs(math.sqrt((d * d).sum()) - rc) < 1e-5, (t, i, j)
            assert len(p32 ^ p64) <= 5


def test_pairs_f32_invariant_under_whole_box_shifts(box512):
    """Exact invariance: adding k L to any input coordinate changes neither the images nor the set.

    Coordinates and the box edge are rounded to multiples of 2^-16 nm, so
    that every x + k L (|k| <= 2) and every image is exactly representable in
    FP32; the contract's images of the shifted inputs must then equal those
    of the original inputs bit for bit, for the search frame and a displaced
    frame alike, and so must the pair set.
    """
    b = box512
    q = 2.0 ** -16
    L32 = (np.round(b.box.astype(np.float64) / q) * q).astype(np.float32)
    L = L32.astype(np.float64)

    def grid(x):
        return np.clip(np.round(x.astype(np.float64) / q) * q, 0.0, L - q).astype(np.float32)

    x0 = grid(b.coords)
    xt = grid(_walk_across_faces(b)[7])
    y = oracle.image_f32(x0, xt, L32)
    p = oracle.pairs_f32(x0, xt, L32, 0.9, b.excl_off, b.excl_idx)
    for s in range(3):
        x0s, m0 = _unwrap_randomly(x0, L, 500 + s)
        xts, m = _unwrap_randomly(xt, L, 600 + s)
        assert np.array_equal(x0s.astype(np.float64), x0 + m0 * L)  # the shifts are exact
        assert np.array_equal(xts.astype(np.float64), xt + m * L)
        assert np.array_equal(oracle.image_f32(x0s, xts, L32), y)
        assert np.array_equal(oracle.pairs_f32(x0s, xts, L32, 0.9, b.excl_off, b.excl_idx), p)


def _grid_system(seed, n=128, L=4.0, step=1.0 / 16.0, dmin=0.3):
    """n atoms at distinct points of a 1/16 nm grid in an L = 4 nm box, at least dmin apart (minimum
    image), two LJ types. Every FP32 displacement of the contract (|d| < 2 nm, a multiple of 1/16),
    its square and the sum of three squares (multiples of 1/256 below 12) are exact in FP32."""
    rng = np.random.default_rng(seed)
    m = int(round(L / step))
    pts = []
    while len(pts) < n:
        p = rng.integers(0, m, 3) * step
        if all(np.linalg.norm((p - o) - L * np.rint((p - o) / L)) >= dmin for o in pts):
            pts.append(p)
    x = np.array(pts, dtype=np.float32)
    q = rng.normal(0.0, 0.5, n)
    typ = rng.integers(0, 2, n).astype(np.int32)
    lj = np.zeros((2, 2, 2))
    c6, c12 = np.array([2e-3, 1e-3]), np.array([2e-6, 1e-6])
    for a in range(2):
        for b in range(2):
            lj[a, b] = (math.sqrt(c6[a] * c6[b]), math.sqrt(c12[a] * c12[b]))
    return x, q, typ, lj, np.array([L, L, L], dtype=np.float32)


def test_energy_f32_equals_fp64_where_fp32_distances_are_exact():
    """Where every FP32 displacement and r^2 of the contract is exact (grid coordinates), the energies
    at the contract's distances are the FP64 energies at the same (FP32) cutoff: same pair count,
    E_LJ and E_C to rounding."""
    for seed in range(3):
        x, q, typ, lj, box = _grid_system(seed)
        beta = synth.ewald_beta(0.9)
        rc32 = float(np.float32(0.9))  # the cutoff the contract uses
        _, elj, ec, npairs, (alj, ac) = oracle.energy_forces(x, q, typ, lj, box, rc32, beta, method="n2",
                                                             abs_sums=True)
        e32_lj, e32_c, n32, (a32_lj, a32_c) = oracle.energy_f32(x, x, q, typ, lj, box, 0.9, beta, abs_sums=True)
        assert n32 == npairs > 200
        assert abs(e32_lj - elj) <= 1e-12 * abs(elj) and abs(e32_c - ec) <= 1e-12 * abs(ec)
        assert abs(a32_lj - alj) <= 1e-12 * alj and abs(a32_c - ac) <= 1e-12 * ac


def test_energy_f32_unchanged_by_whole_box_shifts():
    """Adding whole box vectors to the inputs (exact on the grid) changes no contract distance, so the
    energies at those distances are unchanged bit for bit; a displaced frame too."""
    x, q, typ, lj, box = _grid_system(7)
    beta = synth.ewald_beta(0.9)
    L = box.astype(np.float64)
    rng = np.random.default_rng(8)
    xt = (x + rng.integers(-1, 2, x.shape) / 16.0 * (rng.random(x.shape) < 0.3)).astype(np.float32)
    xt = (xt - L * np.floor(xt.astype(np.float64) / L)).astype(np.float32)
    ref = oracle.energy_f32(x, xt, q, typ, lj, box, 0.9, beta)
    for s in range(3):
        k0 = rng.integers(-2, 3, x.shape)
        k = rng.integers(-2, 3, x.shape)
        got = oracle.energy_f32((x + k0 * L).astype(np.float32), (xt + k * L).astype(np.float32), q, typ, lj, box,
                                0.9, beta)
        assert got == ref


def test_energy_f32_close_to_fp64_on_water(box512):
    """On water the two differ only by FP32 rounding of the displacements: within 2e-6 of each energy
    (the Coulomb pair energies cancel to ~1/300 of their absolute sum, which amplifies that rounding)."""
    b = box512
    beta = synth.ewald_beta(0.9)
    _, elj, ec, npairs = oracle.energy_forces(b.coords, b.q, b.type, b.ljparams, b.box, 0.9, beta, b.excl_off,
                                              b.excl_idx)
    e32_lj, e32_c, n32 = oracle.energy_f32(b.coords, b.coords, b.q, b.type, b.ljparams, b.box, 0.9, beta,
                                           b.excl_off, b.excl_idx)
    assert n32 == oracle.pairs_f32(b.coords, b.coords, b.box, 0.9, b.excl_off, b.excl_idx, count_only=True)
    assert abs(n32 - npairs) <= 2
    assert abs(e32_lj - elj) <= 2e-6 * abs(elj) and abs(e32_c - ec) <= 2e-6 * abs(ec)
    assert e32_c != ec  # the rounding is there


def test_pair_count_matches_density(box512):
    """Half-pairs per atom within rc ~ rho (2/3) pi rc^3, minus one excluded pair per atom."""
    b = synth.water_box(32000, 2)
    _, _, _, n = oracle.energy_forces(b.coords, b.q, b.type, b.ljparams, b.box, 1.0, 3.1234,
                                      b.excl_off, b.excl_idx)
    rho = b.n_atoms / float(b.box[0]) ** 3
    expect = rho * (2.0 / 3.0) * math.pi * 1.0 ** 3 - 1.0
    assert n / b.n_atoms == pytest.approx(expect, rel=0.02)
