"""Pins for the smooth-PME spread and gather of the CPU oracle.

None of these re-types the oracle's recursion. The B-spline is checked
against the textbook closed form of the uniform cubic B-spline and its
known values, partition of unity and symmetry; the spread against a brute
force over every grid point and periodic image with that closed form, the
total charge and a cyclic shift under translation by one grid spacing; the
gather against central finite differences of the interpolated potential and
against the spread (they are adjoint); and the whole smooth-PME chain
(spread, an FFT solve written here with numpy, gather) against the direct
Ewald reciprocal-space sum, which it must approach as the mesh is refined.
"""
import math

import numpy as np
import pytest

import oracle

F_COUL = 138.935458


def cubic_bspline(u):
    """Uniform cubic B-spline on [0, 4] in closed form (piecewise cubic)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    a = (u >= 0) & (u < 1)
    b = (u >= 1) & (u < 2)
    c = (u >= 2) & (u < 3)
    d = (u >= 3) & (u < 4)
    out[a] = u[a] ** 3 / 6
    out[b] = (-3 * u[b] ** 3 + 12 * u[b] ** 2 - 12 * u[b] + 4) / 6
    out[c] = (3 * u[c] ** 3 - 24 * u[c] ** 2 + 60 * u[c] - 44) / 6
    out[d] = (4 - u[d]) ** 3 / 6
    return out


def random_system(n, box, seed, unwrap=False):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (n, 3)) * box
    if unwrap:
        x += rng.integers(-2, 3, (n, 3)) * box
    q = rng.normal(0, 0.5, n)
    q -= q.mean()
    return x, q


# ------------------------------------------------------------------ B-splines

def test_bspline_matches_the_cubic_closed_form():
    u = np.linspace(-0.5, 4.5, 1001)
    got = np.array([oracle.bspline(4, v) for v in u])
    np.testing.assert_allclose(got, cubic_bspline(u), rtol=0, atol=1e-13)  # the closed form cancels near u = 2
    assert [oracle.bspline(4, k) for k in range(5)] == pytest.approx([0, 1 / 6, 2 / 3, 1 / 6, 0], abs=1e-16)
    # quadratic B-spline at its knot midpoints: 1/8, 3/4, 1/8
    assert [oracle.bspline(3, k + 0.5) for k in range(3)] == pytest.approx([1 / 8, 3 / 4, 1 / 8], abs=1e-16)


@pytest.mark.parametrize("order", [3, 4, 5, 6, 8])
def test_bspline_partition_of_unity_symmetry_and_derivative(order):
    rng = np.random.default_rng(order)
    for w in rng.uniform(0, 1, 20):
        assert sum(oracle.bspline(order, w + j) for j in range(order)) == pytest.approx(1.0, abs=1e-14)
        assert sum(oracle.bspline(order, w + j, deriv=True) for j in range(order)) == pytest.approx(0.0, abs=1e-13)
    h = 1e-6
    for u in rng.uniform(0.05, order - 0.05, 20):
        assert oracle.bspline(order, u) == pytest.approx(oracle.bspline(order, order - u), abs=1e-14)
        fd = (oracle.bspline(order, u + h) - oracle.bspline(order, u - h)) / (2 * h)
        assert oracle.bspline(order, u, deriv=True) == pytest.approx(fd, abs=1e-8)
    assert oracle.bspline(order, -0.1) == 0.0 and oracle.bspline(order, order + 0.1) == 0.0


# ------------------------------------------------------------------ spread

def test_spread_against_brute_force_over_every_point_and_image():
    box = np.array([1.3, 1.7, 2.1])
    K = (6, 7, 8)
    x, q = random_system(5, box, 1, unwrap=True)
    got = oracle.pme_spread(x, q, box, K, 4)
    want = np.zeros(K)
    s = x / box
    u = (s - np.floor(s)) * np.array(K)
    k = [np.arange(K[a]) for a in range(3)]
    for i in range(len(q)):
        w = []
        for a in range(3):
            # every periodic image of every grid point: sum_m M(u - k - m K)
            w.append(sum(cubic_bspline(u[i, a] - k[a] - m * K[a]) for m in (-1, 0, 1)))
        want += q[i] * w[0][:, None, None] * w[1][None, :, None] * w[2][None, None, :]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("order", [3, 4, 6])
def test_spread_conserves_charge(order):
    box = np.array([2.0, 2.2, 2.4])
    x, q = random_system(200, box, 2, unwrap=True)
    q = q + 0.3  # not neutral, so the total is a real check
    Q, Qa = oracle.pme_spread(x, q, box, (16, 18, 20), order, abs_sums=True)
    assert Q.sum() == pytest.approx(q.sum(), abs=1e-12)
    assert Qa.sum() == pytest.approx(np.abs(q).sum(), rel=1e-13)
    assert (Qa >= np.abs(Q) - 1e-15).all()


def test_spread_translation_by_one_grid_spacing_is_a_cyclic_shift():
    box = np.array([2.0, 2.25, 2.5])
    K = (16, 18, 20)  # spacings 0.125 exactly
    x, q = random_system(50, box, 3)
    Q = oracle.pme_spread(x, q, box, K, 4)
    for a in range(3):
        x2 = x.copy()
        x2[:, a] += box[a] / K[a]
        np.testing.assert_allclose(oracle.pme_spread(x2, q, box, K, 4), np.roll(Q, 1, axis=a), atol=1e-13)
    # a whole box vector changes nothing
    np.testing.assert_allclose(oracle.pme_spread(x + box * np.array([1, -2, 3]), q, box, K, 4), Q, atol=1e-13)


# ------------------------------------------------------------------ gather

def test_gather_is_minus_charge_times_gradient_of_the_interpolated_potential():
    box = np.array([2.0, 2.2, 2.4])
    K = (12, 13, 14)
    x, q = random_system(30, box, 4)
    phi = np.random.default_rng(5).normal(size=K)
    F, psi = oracle.pme_gather(x, q, box, K, phi, 4)
    h = 1e-6
    for a in range(3):
        xp, xm = x.copy(), x.copy()
        xp[:, a] += h
        xm[:, a] -= h
        fd = -q * (oracle.pme_gather(xp, q, box, K, phi, 4)[1] - oracle.pme_gather(xm, q, box, K, phi, 4)[1]) / (2 * h)
        np.testing.assert_allclose(F[:, a], fd, rtol=0, atol=1e-6 * np.abs(F).max())


def test_gather_is_the_adjoint_of_spread():
    """sum_k Q(k) phi(k) = sum_i q_i psi_i for any mesh potential phi."""
    box = np.array([2.0, 2.2, 2.4])
    K = (10, 12, 14)
    x, q = random_system(40, box, 6, unwrap=True)
    phi = np.random.default_rng(7).normal(size=K)
    Q = oracle.pme_spread(x, q, box, K, 5)
    _, psi = oracle.pme_gather(x, q, box, K, phi, 5)
    assert (Q * phi).sum() == pytest.approx((q * psi).sum(), rel=1e-12)


def test_gather_of_a_constant_potential():
    box = np.array([2.0, 2.2, 2.4])
    K = (10, 12, 14)
    x, q = random_system(20, box, 8)
    F, psi = oracle.pme_gather(x, q, box, K, np.full(K, 3.25), 4)
    np.testing.assert_allclose(psi, 3.25, rtol=1e-14)
    assert np.abs(F).max() < 1e-12


# ------------------------------------------------------------------ smooth PME vs direct Ewald

def _signed(K):
    m = np.arange(K)
    return np.where(m <= K // 2, m, m - K)


def smooth_pme(x, q, box, K, beta, order=4):
    """Smooth PME reciprocal energy and forces: the oracle's spread, a numpy
    FFT solve with the Euler exponential-spline factors B(m), the oracle's
    gather. Only order 4 (the factors use the cubic closed form)."""
    assert order == 4
    Q = oracle.pme_spread(x, q, box, K, order)
    V = float(np.prod(box))
    mh = [(_signed(K[a]) / box[a]) for a in range(3)]
    m2 = mh[0][:, None, None] ** 2 + mh[1][None, :, None] ** 2 + mh[2][None, None, :] ** 2
    B = np.ones(K)
    for a in range(3):
        mk = np.arange(K[a])
        den = sum(cubic_bspline(k + 1.0) * np.exp(2j * np.pi * mk * k / K[a]) for k in range(order - 1))
        b2 = 1.0 / np.abs(den) ** 2  # |b(m)|^2; the numerator has modulus 1
        shape = [1, 1, 1]
        shape[a] = K[a]
        B = B * b2.reshape(shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        C = F_COUL * np.exp(-np.pi ** 2 * m2 / beta ** 2) / (np.pi * V * m2)
    C[0, 0, 0] = 0.0
    FQ = np.fft.ifftn(Q) * Q.size  # sum_k Q(k) exp(+2 pi i m.k/K)
    phi = np.fft.fftn(C * B * FQ).real  # sum_m ... exp(-2 pi i m.k/K)
    F, psi = oracle.pme_gather(x, q, box, K, phi, order)
    return 0.5 * (q * psi).sum(), F, 0.5 * (Q * phi).sum()


def direct_reciprocal(x, q, box, beta, kmax):
    """Ewald reciprocal-space energy and forces by the direct sum over m != 0."""
    V = float(np.prod(box))
    r = np.arange(-kmax, kmax + 1)
    M = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    M = M[(M != 0).any(1)] / box
    m2 = (M ** 2).sum(1)
    g = np.exp(-np.pi ** 2 * m2 / beta ** 2) / m2
    ph = np.exp(2j * np.pi * x @ M.T)  # [N, nm]
    S = (q[:, None] * ph).sum(0)
    E = F_COUL / (2 * np.pi * V) * (g * np.abs(S) ** 2).sum()
    F = 2 * F_COUL * q[:, None] / V * ((g * np.imag(np.conj(S)[None, :] * ph)) @ M)
    return E, F


def test_direct_reciprocal_sum_forces_are_minus_its_gradient():
    box = np.array([2.0, 2.2, 2.4])
    x, q = random_system(8, box, 9)
    E, F = direct_reciprocal(x, q, box, 3.0, 8)
    h = 1e-6
    for i in range(3):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = -(direct_reciprocal(xp, q, box, 3.0, 8)[0] - direct_reciprocal(xm, q, box, 3.0, 8)[0]) / (2 * h)
            assert F[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(F).max())


def test_smooth_pme_converges_to_the_direct_ewald_reciprocal_sum():
    """Spread + solve + gather approaches the exact reciprocal sum as the mesh
    is refined: within 1e-4 (energy) and 1e-3 rms (forces) at about 0.06 nm
    spacing, and closer on a finer mesh, the interpolation error of order-4
    smooth PME. A wrong sign, index or scale in the spread or the gather
    breaks the agreement by far more."""
    box = np.array([2.0, 2.2, 2.4])
    beta = 3.0
    x, q = random_system(60, box, 10)
    E_ref, F_ref = direct_reciprocal(x, q, box, beta, 14)
    rms = np.sqrt((F_ref ** 2).sum(1).mean())
    errs = []
    for K in ((32, 36, 40), (48, 54, 60)):
        E, F, E_mesh = smooth_pme(x, q, box, K, beta)
        assert E == pytest.approx(E_mesh, rel=1e-12)  # 1/2 sum q psi = 1/2 sum Q phi
        errs.append((abs(E - E_ref) / abs(E_ref), np.sqrt(((F - F_ref) ** 2).sum(1).mean()) / rms))
    assert errs[0][0] < 1e-4 and errs[0][1] < 1e-3, errs
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1], errs
